"""D3Q27 (Sec. II) on the GPU versus the FP64 oracle's D3Q27 build."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import F32_REL_TOL, dev, report, t
from paper_1801_04586_gb300 import Lattice, synthetic

pytestmark = pytest.mark.gpu

W27 = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8).reshape(27, 1, 1, 1)
RATES = dict(s2b=1.2, s3=1.1, s4=0.9, s3b=1.3, s4b=0.8, s5=1.15, s6=0.95)


def pair(nx, ny, nz, nu, walls=0, rates=RATES, storage="f32"):
    g = Lattice(nx, ny, nz, nu, walls=walls, device=dev(), lattice=27, storage=storage, **rates)
    o = oracle.Lattice(nx, ny, nz, walls=walls, q=27, s2=1.0 / (3 * nu + 0.5), **rates)
    return g, o


def rel(fg, fo):
    return float(np.max(np.abs(fg - fo) / np.abs(fo)))


def test_d3q27_init_parity():
    nx, ny, nz = 21, 14, 9
    shape = (nz, ny, nx)
    g, o = pair(nx, ny, nz, 0.05, walls=7)
    assert g.info()["q"] == 27
    rho = synthetic.density_perturbation(shape, 0.01, seed=201)
    u = synthetic.divfree_velocity(shape, seed=202, umax=0.05)
    F = synthetic.gaussian_force(shape, 1e-4, seed=203)
    g.set_force_field(t(F))
    g.init_equilibrium(t(rho), t(u))
    fg = g.populations(deviation=True).double().cpu().numpy() + W27
    assert rel(fg, oracle.init(o, rho, u, F)) < 1e-6
    r2, u2 = g.macros()
    np.testing.assert_allclose(u2.cpu().numpy(), u, rtol=0, atol=3e-8)


@pytest.mark.parametrize("shape_walls", [((24, 20, 16), 0), ((37, 19, 11), 7), ((150, 6, 5), 6), ((1, 9, 13), 4)])
def test_d3q27_100_steps_parity(shape_walls):
    (nx, ny, nz), walls = shape_walls
    shape = (nz, ny, nx)
    g, o = pair(nx, ny, nz, 0.03, walls=walls)
    h0 = synthetic.rng(211).uniform(-2e-3, 2e-3, (27,) + shape).astype(np.float32)
    F = synthetic.gaussian_force(shape, 1e-4, seed=212)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    np.testing.assert_array_equal(g.populations(deviation=True).cpu().numpy(), h0)
    g.step(100)
    fo = oracle.step(o, h0.astype(np.float64) + W27, F, 100)
    fg = g.populations(deviation=True).double().cpu().numpy() + W27
    report("d3q27_parity_100_steps", shape=str(shape), walls=walls, rel=rel(fg, fo))
    assert rel(fg, fo) < F32_REL_TOL
    g.check()


def test_d3q27_conservation():
    nx, ny, nz = 40, 24, 16
    shape = (nz, ny, nx)
    g, _ = pair(nx, ny, nz, 0.05)
    F = synthetic.gaussian_force(shape, 1e-4, seed=221) + np.float32(2e-5)
    g.set_force_field(t(F))
    g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=222, umax=0.02)))
    m0 = g.reduce_moments().cpu().numpy()
    g.step(50)
    m1 = g.reduce_moments().cpu().numpy()
    np.testing.assert_allclose(m1[1:] - m0[1:], 50 * F.astype(np.float64).sum(axis=(1, 2, 3)), rtol=1e-5)
    assert abs(m1[0] - m0[0]) < 1e-6


@pytest.mark.parametrize("storage", ["f32", "bf16sr"])
def test_d3q27_checkpoint_resume_bit_exact(storage):
    """save_state / load_state and export / import on the D3Q27 lattice:
    resuming reproduces the uninterrupted run bit for bit (the stochastic
    dither depends on the step count, which the state carries)."""
    nx, ny, nz = 24, 10, 8
    shape = (nz, ny, nx)
    a, _ = pair(nx, ny, nz, 0.04, walls=2, storage=storage)
    b, _ = pair(nx, ny, nz, 0.04, walls=2, storage=storage)
    F = t(synthetic.gaussian_force(shape, 1e-4, seed=221))
    for g in (a, b):
        g.set_force_field(F)
        g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=222, umax=0.03)))
    a.step(7)
    blob = a.save_state()
    raw = a.export_state()
    a.step(9)
    b.load_state(blob)
    assert b.steps_done == 7
    b.step(9)
    assert torch.equal(a.populations(deviation=True), b.populations(deviation=True))
    b.import_state(raw, set_steps=7)
    b.step(9)
    assert torch.equal(a.populations(deviation=True), b.populations(deviation=True))
