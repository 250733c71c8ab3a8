"""The comparison collision models on the GPU versus the FP64 oracle: the
SRT-LBM (discrete equilibrium of Sec. II.B, Guo's forcing) and the
non-orthogonal raw-moment MRT of Appendix B, on D3Q19 and D3Q27, run by the
same step kernels (layout, streaming, bounce-back, storage formats, in-place
pattern) as the cascaded collision."""
import numpy as np
import pytest
import torch

import analytic as an
import oracle
from gpu_common import F32_REL_TOL, W, dev, report, s2_of, t
from paper_1801_04586_gb300 import Lattice, synthetic

pytestmark = pytest.mark.gpu

RATES = {19: dict(s2b=1.2, s3=1.1, s4=0.9),
         27: dict(s2b=1.2, s3=1.1, s4=0.9, s3b=1.3, s4b=0.8, s5=1.15, s6=0.95)}
W27 = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8).reshape(27, 1, 1, 1)
MODEL_ID = {"srt": 1, "mrt": 2}


def pair(nx, ny, nz, nu, model, walls=0, pattern="ab", storage="f32", q=19):
    g = Lattice(nx, ny, nz, nu, walls=walls, device=dev(), model=model, pattern=pattern, storage=storage, lattice=q,
                **RATES[q])
    o = oracle.Lattice(nx, ny, nz, walls=walls, s2=s2_of(nu), model=MODEL_ID[model], q=q, **RATES[q])
    return g, o


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", ["srt", "mrt"])
@pytest.mark.parametrize("shape_walls", [((40, 20, 16), 0), ((37, 19, 11), 7), ((150, 6, 5), 6), ((1, 9, 13), 4)])
def test_models_100_steps_parity(q, model, shape_walls):
    (nx, ny, nz), walls = shape_walls
    shape = (nz, ny, nx)
    w = W27 if q == 27 else W
    g, o = pair(nx, ny, nz, 0.03, model, walls, q=q)
    assert g.info()["model"] == MODEL_ID[model]
    h0 = synthetic.rng(401).uniform(-2e-3, 2e-3, (q,) + shape).astype(np.float32)
    F = synthetic.gaussian_force(shape, 1e-4, seed=402)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    g.step(100)
    fo = oracle.step(o, h0.astype(np.float64) + w, F, 100)
    fg = g.populations(deviation=True).double().cpu().numpy() + w
    rel = float(np.max(np.abs(fg - fo) / np.abs(fo)))
    report("model_parity_100_steps", q=q, model=model, shape=str(shape), walls=walls, rel=rel)
    assert rel < F32_REL_TOL
    g.check()


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", ["srt", "mrt"])
@pytest.mark.parametrize("storage", ["f32", "f16sr"])
def test_models_in_place_bitwise(q, model, storage):
    nx, ny, nz = 45, 13, 10
    shape = (nz, ny, nx)
    ab, _ = pair(nx, ny, nz, 0.02, model, walls=5, storage=storage, q=q)
    aa, _ = pair(nx, ny, nz, 0.02, model, walls=5, pattern="aa", storage=storage, q=q)
    rho = synthetic.density_perturbation(shape, 0.01, seed=411)
    u = synthetic.divfree_velocity(shape, seed=412, umax=0.04)
    F = t(synthetic.gaussian_force(shape, 1e-4, seed=413))
    for g in (ab, aa):
        g.set_force_field(F)
        g.init_equilibrium(t(rho), t(u))
    for n in (3, 4):
        ab.step(n)
        aa.step(n)
        assert torch.equal(ab.populations(deviation=True), aa.populations(deviation=True))


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", ["srt", "mrt"])
def test_models_poiseuille_slip(q, model):
    """Steady channel flow on the GPU: the closed-form bounce-back slip
    u_s = F (16 Lambda - 3) / (24 nu) of two-rate schemes (zero for MRT at the
    paper's no-slip s3)."""
    n, F, nu = 24, 1e-6, 0.1
    s2 = s2_of(nu)
    s3 = an.noslip_s3(s2) if model == "mrt" else s2
    g = Lattice(1, 1, n, nu, walls=4, device=dev(), model=model, s2b=s2, s3=s3, lattice=q)
    g.set_force_uniform(F)
    g.init_equilibrium()
    g.step(int(40 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu)))
    ux = g.macros()[1][0, :, 0, 0].double().cpu().numpy()
    ua = an.poiseuille_steady(n, F, nu)
    lam = (1 / s2 - 0.5) * (1 / s3 - 0.5)
    slip = F * (16 * lam - 3) / (24 * nu)
    err = float(np.max(np.abs(ux - ua - slip)) / ua.max())
    report("model_poiseuille", q=q, model=model, err=err, slip_rel=slip / ua.max())
    assert err < 1e-4


@pytest.mark.parametrize("q", [19, 27])
def test_shear_wave_moving_frame_gpu(q):
    """Sec. III.A on the GPU: shear wave of Eq. 17 on a frame moving at
    Ma = B/c_s = 0.3. The cascaded collision keeps the imposed viscosity
    (paper: 0.08 % error); the SRT-LBM loses 8.91 % (paper), nu (1 - 3 B^2).
    The wave amplitude is 1e-2 of the 0.17 background so that FP32 rounding
    over 5000 steps stays far below the measured effect (at 1e-3 it moved
    the D3Q27 SRT value by 0.1 percentage point)."""
    L, nu, A, t1, t2 = 101, 0.05, 1e-2, 200, 5200
    B = 0.3 * np.sqrt(1.0 / 3.0)
    phi = 2 * np.pi / L
    y = np.arange(L)
    u = np.zeros((3, 1, L, 1), dtype=np.float32)
    u[0, 0, :, 0] = A * np.sin(phi * y)
    u[1] = B
    errs = {}
    for model in ("cascaded", "srt"):
        g = Lattice(1, L, 1, nu, device=dev(), model=model, lattice=q)
        g.init_equilibrium(None, t(u))
        g.step(t1)
        a1 = abs(np.fft.fft(g.macros()[1][0, 0, :, 0].double().cpu().numpy())[1])
        g.step(t2 - t1)
        a2 = abs(np.fft.fft(g.macros()[1][0, 0, :, 0].double().cpu().numpy())[1])
        errs[model] = 100 * (np.log(a1 / a2) / (phi ** 2 * (t2 - t1)) - nu) / nu
    report("shear_wave_moving_frame", q=q, clbm_err_pct=errs["cascaded"], srt_err_pct=errs["srt"])
    assert abs(errs["cascaded"]) < 0.08
    assert errs["srt"] == pytest.approx(-8.91, abs=0.15)
