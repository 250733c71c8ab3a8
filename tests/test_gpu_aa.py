"""In-place (AA) storage pattern on the GPU.

The AA pattern keeps one population buffer and alternates two step kinds
(even: read and write the node's own slots; odd: read and write the
neighbours' slots). It computes the same update as the two-buffer pull
scheme: same collision (Eqs. 5, 7, 9), same streaming with halfway
bounce-back (Eq. 8), same stochastic-rounding dither per (step, node,
direction). The tests require bit-identical states against the A/B
pattern after even and odd step counts, for every storage format, both
lattices, periodic and walled boxes, and check the AA path against the FP64
oracle directly.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_common import F32_REL_TOL, W, dev, report, s2_of, t
from paper_1801_04586_gb300 import Lattice, _capi, synthetic

pytestmark = pytest.mark.gpu

W27 = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8).reshape(27, 1, 1, 1)
RATES19 = dict(s2b=1.2, s3=1.1, s4=0.9)
RATES27 = dict(s2b=1.2, s3=1.1, s4=0.9, s3b=1.3, s4b=0.8, s5=1.15, s6=0.95)


def lattices(shape_xyz, nu, walls, storage, q):
    nx, ny, nz = shape_xyz
    rates = RATES27 if q == 27 else RATES19
    ab = Lattice(nx, ny, nz, nu, walls=walls, storage=storage, device=dev(), lattice=q, **rates)
    aa = Lattice(nx, ny, nz, nu, walls=walls, storage=storage, device=dev(), lattice=q, pattern="aa", **rates)
    return ab, aa


def start(lats, shape, seed, force="field"):
    rho = synthetic.density_perturbation(shape, 0.01, seed=seed)
    u = synthetic.divfree_velocity(shape, seed=seed + 1, umax=0.04)
    F = synthetic.gaussian_force(shape, 1e-4, seed=seed + 2)
    Ft = t(F)
    for g in lats:
        if force == "field":
            g.set_force_field(Ft)
        else:
            g.set_force_uniform(2e-5, -1e-5, 3e-5)
        g.init_equilibrium(t(rho), t(u))
    return F


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "f16sr", "bf16sr"])
@pytest.mark.parametrize("shape_walls", [((40, 12, 9), 0), ((37, 11, 13), 7), ((150, 6, 5), 6), ((1, 9, 13), 4)])
def test_aa_bitwise_equals_ab(q, storage, shape_walls):
    (nx, ny, nz), walls = shape_walls
    shape = (nz, ny, nx)
    ab, aa = lattices((nx, ny, nz), 0.02, walls, storage, q)
    assert aa.info()["buffers"] == 1 and ab.info()["buffers"] == 2
    assert aa.info()["pattern"] == 1 and aa.state_bytes() == ab.state_bytes()
    start((ab, aa), shape, seed=301 + q, force="field" if walls else "uniform")
    done = 0
    for n in (1, 1, 5, 8):  # state checked at step counts 1, 2, 7, 15 (odd and even)
        ab.step(n)
        aa.step(n)
        done += n
        assert aa.steps_done == done
        pa, pb = aa.populations(deviation=True), ab.populations(deviation=True)
        assert torch.equal(pa, pb), f"populations differ after {done} steps"
        ra, ua = aa.macros()
        rb, ub = ab.macros()
        assert torch.equal(ra, rb) and torch.equal(ua, ub)
        ma, mb = aa.reduce_moments(), ab.reduce_moments()
        assert torch.equal(ma, mb)
    aa.check()


@pytest.mark.parametrize("q", [19, 27])
def test_aa_oracle_parity_100_steps(q):
    nx, ny, nz, walls, nu = 29, 14, 11, 5, 0.03
    shape = (nz, ny, nx)
    rates = RATES27 if q == 27 else RATES19
    g = Lattice(nx, ny, nz, nu, walls=walls, device=dev(), lattice=q, pattern="aa", **rates)
    o = oracle.Lattice(nx, ny, nz, walls=walls, q=q, s2=s2_of(nu), **rates)
    w = W27 if q == 27 else W
    h0 = synthetic.rng(321).uniform(-2e-3, 2e-3, (q,) + shape).astype(np.float32)
    F = synthetic.gaussian_force(shape, 1e-4, seed=322)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    fo = h0.astype(np.float64) + w
    for n in (37, 63):  # odd, then even total
        g.step(n)
        fo = oracle.step(o, fo, F, n)
        fg = g.populations(deviation=True).double().cpu().numpy() + w
        rel = float(np.max(np.abs(fg - fo) / np.abs(fo)))
        report("aa_parity", q=q, steps=g.steps_done, rel=rel)
        assert rel < F32_REL_TOL


def test_aa_save_load_resume_and_pattern_check():
    nx, ny, nz = 33, 10, 7
    shape = (nz, ny, nx)
    a1 = Lattice(nx, ny, nz, 0.05, walls=4, device=dev(), pattern="aa")
    a2 = Lattice(nx, ny, nz, 0.05, walls=4, device=dev(), pattern="aa")
    ab = Lattice(nx, ny, nz, 0.05, walls=4, device=dev())
    start((a1, a2, ab), shape, seed=331)
    a1.step(5)  # odd parity
    blob = a1.save_state()
    a1.step(6)
    a2.load_state(blob)
    assert a2.steps_done == 5
    a2.step(6)
    assert torch.equal(a1.populations(deviation=True), a2.populations(deviation=True))
    with pytest.raises(_capi.CLBMError):
        ab.load_state(blob)
    # raw export / import at the same parity
    raw = a1.export_state()
    a2.step(2)  # a2 now at 13, same parity as a1 (11)
    a2.import_state(raw, set_steps=11)
    assert torch.equal(a1.populations(deviation=True), a2.populations(deviation=True))


def test_aa_run_host_matches_ab():
    nx, ny, nz = 48, 20, 12
    shape = (nz, ny, nx)
    rho = torch.from_numpy(synthetic.density_perturbation(shape, 0.01, seed=341)).contiguous()
    u = torch.from_numpy(synthetic.divfree_velocity(shape, seed=342, umax=0.03)).contiguous()
    out = {}
    for pat in ("ab", "aa"):
        g = Lattice(nx, ny, nz, 0.04, walls=2, device=dev(), pattern=pat)
        g.set_force_uniform(1e-5)
        r_out, u_out = torch.empty_like(rho), torch.empty_like(u)
        mom = torch.empty(4 * 10, dtype=torch.float64)
        g.run_host(rho, u, 9, r_out, u_out, mom)
        out[pat] = (r_out, u_out, mom)
        # a second job starts after an odd step count: it initialises in the even state's slots again
        r2, u2, mom2 = torch.empty_like(rho), torch.empty_like(u), torch.empty_like(mom)
        g.run_host(rho, u, 9, r2, u2, mom2)
        assert torch.equal(r2, r_out) and torch.equal(u2, u_out) and torch.equal(mom2, mom)
    for a, b in zip(out["ab"], out["aa"]):
        assert torch.equal(a, b)


def test_aa_rejects_adjoint_and_raw_step():
    g = Lattice(16, 8, 8, 0.05, device=dev(), pattern="aa")
    buf = g.export_state()
    with pytest.raises(_capi.CLBMError):
        g.step_raw(buf, torch.empty_like(buf))
    lam = torch.zeros(19, 8, 8, 16, device=dev())
    gF = torch.zeros(3, 8, 8, 16, device=dev())
    with pytest.raises(_capi.CLBMError):
        g.adjoint_step(buf, lam, torch.empty_like(lam), gF)
    code = g.lib.clbm_adjoint_segment(g.h, ctypes.c_void_p(buf.data_ptr()), None, 1,
                                      ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(torch.empty_like(lam).data_ptr()),
                                      ctypes.c_void_p(gF.data_ptr()))
    assert code == _capi.CLBM_ERR_ARG
