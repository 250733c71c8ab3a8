"""GPU (libclbm.so through the C ABI) versus the FP64 oracle, element by
element, on seeded synthetic inputs: initial state, 100-step runs on periodic
and walled boxes with every force mode, ragged sizes spanning several blocks,
degenerate lattices, the Poiseuille channel against the oracle and the
start-up series, and sampled nodes of the full 256^3 workload in the launch
configuration the benchmark times.
"""
import numpy as np
import pytest
import torch

import analytic as an
import oracle
from gpu_common import F32_REL_TOL, W, dev, dev_err, gpu_f, make_pair, rel_err, report, t
from paper_1801_04586_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("walls", [0, 7])
def test_init_equilibrium_parity(walls):
    nx, ny, nz = 37, 24, 20
    g, o = make_pair(nx, ny, nz, 0.05, walls=walls)
    shape = (nz, ny, nx)
    rho = synthetic.density_perturbation(shape, 0.01, seed=11)
    u = synthetic.divfree_velocity(shape, seed=12, umax=0.05)
    F = synthetic.gaussian_force(shape, 1e-4, seed=13)
    g.set_force_field(t(F))
    g.init_equilibrium(t(rho), t(u))
    fo = oracle.init(o, rho, u, F)
    assert rel_err(gpu_f(g), fo) < 1e-6
    r2, u2 = g.macros()
    np.testing.assert_allclose(r2.cpu().numpy(), rho, rtol=0, atol=2e-7)
    np.testing.assert_allclose(u2.cpu().numpy(), u, rtol=0, atol=2e-8)


CASES = [
    # (nx, ny, nz, walls, force, nu, s2b, s3, s4)
    (32, 32, 32, 0, "field", 0.02, 1.2, 1.1, 0.9),
    (150, 20, 12, 0, "uniform", 0.05, 1.0, 1.0, 1.0),      # two x blocks, ragged tail
    (150, 20, 12, 7, "field", 0.05, 1.3, 0.8, 1.2),
    (37, 19, 23, 6, "profile", 0.1, 1.0, an.noslip_s3(1.25), 1.0),
    (33, 7, 5, 1, "uniform", 0.03, 0.7, 1.5, 1.1),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}w{c[3]}{c[4]}")
def test_100_steps_parity(case):
    nx, ny, nz, walls, fmode, nu, s2b, s3, s4 = case
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, nu, walls=walls, s2b=s2b, s3=s3, s4=s4)
    u0 = synthetic.divfree_velocity(shape, seed=21, umax=0.03)
    if fmode == "field":
        F = synthetic.gaussian_force(shape, 1e-4, seed=22)
        g.set_force_field(t(F))
    elif fmode == "profile":
        prof = synthetic.kolmogorov_profile(nz, 1e-4)
        F = synthetic.profile_to_field(prof, shape)
        g.set_force_profile_z(t(prof))
    else:
        F = synthetic.uniform_field(shape, (2e-5, -1e-5, 5e-6))
        g.set_force_uniform(2e-5, -1e-5, 5e-6)
    g.init_equilibrium(None, t(u0))
    g.step(100)
    fo = oracle.step(o, oracle.init(o, None, u0, F), F, 100)
    fg = gpu_f(g)
    report("parity_100_steps", case=str(case[:5]), rel=rel_err(fg, fo), dev=dev_err(fg, fo))
    assert rel_err(fg, fo) < F32_REL_TOL
    assert dev_err(fg, fo) < 1e-4
    g.check()
    rg, ug = g.macros()
    ro, uo = oracle.macros(o, fo, F)
    np.testing.assert_allclose(ug.double().cpu().numpy(), uo, rtol=0, atol=1e-7)
    np.testing.assert_allclose(rg.double().cpu().numpy(), ro, rtol=0, atol=1e-6)


@pytest.mark.parametrize("shape_walls", [((150, 20, 12), 7), ((37, 19, 23), 0), ((1, 5, 9), 4), ((300, 3, 2), 2)])
def test_two_nodes_per_thread_parity(shape_walls):
    """The packed step (two nodes per thread, FP32x2 arithmetic) on FP32
    storage, including row tails where the second lane has no node."""
    (nx, ny, nz), walls = shape_walls
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.03, walls=walls, s2b=1.2, s3=1.1, s4=0.9, variant=2)
    assert g.info()["nodes_per_thread"] == 2
    h0 = synthetic.random_deviations(shape, 2e-3, seed=33)
    F = synthetic.gaussian_force(shape, 1e-4, seed=34)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    g.step(100)
    fo = oracle.step(o, h0.astype(np.float64) + W, F, 100)
    report("parity_packed", shape=str(shape), rel=rel_err(gpu_f(g), fo))
    assert rel_err(gpu_f(g), fo) < F32_REL_TOL
    g.check()


def test_random_state_parity():
    """An arbitrary non-equilibrium state (random deviations) set through the ABI."""
    nx, ny, nz = 32, 32, 32
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.02, walls=0, s2b=1.2, s3=1.1, s4=0.9)
    h0 = synthetic.random_deviations(shape, 2e-3, seed=31)
    F = synthetic.gaussian_force(shape, 1e-5, seed=32)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    np.testing.assert_array_equal(g.populations(deviation=True).cpu().numpy(), h0)
    g.step(100)
    fo = oracle.step(o, h0.astype(np.float64) + W, F, 100)
    report("parity_random_state", rel=rel_err(gpu_f(g), fo), dev=dev_err(gpu_f(g), fo))
    assert rel_err(gpu_f(g), fo) < F32_REL_TOL


@pytest.mark.parametrize("shape_walls", [((1, 1, 1), 0), ((1, 1, 1), 7), ((1, 1, 40), 4), ((5, 1, 1), 0),
                                         ((2, 3, 2), 7), ((64, 1, 3), 2), ((65535, 1, 1), 1), ((1, 65535, 1), 0),
                                         ((1, 1, 65535), 4)])
def test_degenerate_lattices(shape_walls):
    """Single nodes, single rows and the longest extents the ABI accepts
    (65535 along one axis: the grid's z limit, and ny / block_y rows)."""
    (nx, ny, nz), walls = shape_walls
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.1, walls=walls, s2b=0.9, s3=1.2)
    h0 = synthetic.random_deviations(shape, 1e-3, seed=41)
    F = synthetic.gaussian_force(shape, 1e-5, seed=42)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    g.step(30)
    fo = oracle.step(o, h0.astype(np.float64) + W, F, 30)
    assert rel_err(gpu_f(g), fo) < F32_REL_TOL


def test_block_shape_does_not_change_results():
    """Each node's arithmetic is independent of the launch shape: bit-identical."""
    nx, ny, nz = 96, 20, 6
    shape = (nz, ny, nx)
    u0 = synthetic.divfree_velocity(shape, seed=51, umax=0.02)
    outs = []
    for block in [(32, 1), (64, 4), (128, 2), (96, 5)]:
        g, _ = make_pair(nx, ny, nz, 0.05, walls=4, block=block)
        g.set_force_uniform(1e-5)
        g.init_equilibrium(None, t(u0))
        g.step(10)
        outs.append(g.populations(deviation=True).cpu().numpy())
    for o2 in outs[1:]:
        np.testing.assert_array_equal(outs[0], o2)


def test_poiseuille_channel_2000_steps():
    """16 x 32 x 32 channel, walls at z, F_x = 1e-6, nu = 0.1, other rates 1,
    rho = 1 and u = U(+-1e-8) at t = 0, 2000 steps: against the oracle and the
    start-up series of the Sec. III.B profile."""
    nx, ny, nz, nu, F, steps = 16, 32, 32, 0.1, 1e-6, 2000
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, nu, walls=4)
    u0 = synthetic.uniform_perturbation(shape, 1e-8, seed=0)
    Ff = synthetic.uniform_field(shape, (F, 0, 0))
    g.set_force_uniform(F)
    g.init_equilibrium(None, t(u0))
    g.step(steps)
    fo = oracle.step(o, oracle.init(o, None, u0, Ff), Ff, steps, nthreads=0)
    report("parity_poiseuille_2000", rel=rel_err(gpu_f(g), fo), dev=dev_err(gpu_f(g), fo))
    assert rel_err(gpu_f(g), fo) < F32_REL_TOL
    ux = g.macros()[1][0].double().cpu().numpy()
    uo = oracle.macros(o, fo, Ff)[1][0]
    assert np.max(np.abs(ux - uo)) < 1e-4 * np.max(np.abs(uo))
    ua = an.poiseuille_startup(nz, F, nu, steps)[:, None, None] * np.ones(shape)
    e2 = np.sqrt(((ux - ua) ** 2).sum() / (ua ** 2).sum())
    report("poiseuille_vs_series", e2=e2)
    assert e2 < 5e-4


def test_duct_parity():
    nx, ny, nz, nu, F = 24, 20, 18, 0.05, 2e-5
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, nu, walls=6, s2b=an.s2_from_nu(nu), s3=an.noslip_s3(an.s2_from_nu(nu)))
    Ff = synthetic.uniform_field(shape, (F, 0, 0))
    g.set_force_uniform(F)
    g.init_equilibrium()
    g.step(300)
    fo = oracle.step(o, oracle.init(o, None, None, Ff), Ff, 300)
    assert rel_err(gpu_f(g), fo) < F32_REL_TOL


def test_kolmogorov_64cube_100_steps_on_the_benchmark_kernel():
    """A 64^3 copy of the benchmark workload on the kernel the benchmark times:
    FP32 A/B populations, periodic faces, z-profile force F_x = 1e-5
    sin(2 pi z/64), nu = 0.01 (other rates 1), divergence-free u0 with
    max |u| = 0.02 on wavenumbers 1-4 (seed 1), default launch shape, one
    launch per step as the timed loop issues them. After 100 steps every
    population matches the oracle within the 1e-5 relative tolerance (the
    algorithm of Sec. II.B, Steps 1-4, iterated)."""
    n, nu, steps = 64, 0.01, 100
    shape = (n, n, n)
    g, o = make_pair(n, n, n, nu)
    info = g.info()
    assert (info["staged"], info["nodes_per_thread"], info["pattern"], info["model"], info["q"]) == (0, 1, 0, 0, 19)
    prof = synthetic.kolmogorov_profile(n, 1e-5)
    u0 = synthetic.divfree_velocity(shape, seed=1, umax=0.02)
    g.set_force_profile_z(t(prof))
    g.init_equilibrium(None, t(u0))
    for _ in range(steps):
        g.step(1)
    F = synthetic.profile_to_field(prof, shape)
    fo = oracle.step(o, oracle.init(o, None, u0, F), F, steps)
    fg = gpu_f(g)
    report("kolmogorov_64cube_100_steps", rel=rel_err(fg, fo), dev=dev_err(fg, fo))
    assert rel_err(fg, fo) < F32_REL_TOL
    g.check()
    rg, ug = g.macros()
    ro, uo = oracle.macros(o, fo, F)
    np.testing.assert_allclose(ug.double().cpu().numpy(), uo, rtol=0, atol=1e-7)
    g.close()


def test_full_size_kolmogorov_sampled_first_step():
    """The 256^3 periodic Kolmogorov workload (F_x = 1e-5 sin(2 pi z/256),
    nu = 0.01, divergence-free u0 with max |u| = 0.02), default launch shape:
    one step on the GPU against the oracle at 2048 sampled nodes."""
    n, nu = 256, 0.01
    shape = (n, n, n)
    g, o = make_pair(n, n, n, nu)
    prof = synthetic.kolmogorov_profile(n, 1e-5)
    u0 = synthetic.divfree_velocity(shape, seed=1, umax=0.02)
    g.set_force_profile_z(t(prof))
    g.init_equilibrium(None, t(u0))
    g.step(1)
    fg = g.populations(deviation=True)
    nodes = np.random.default_rng(7).choice(n ** 3, 2048, replace=False)
    hg = fg.reshape(19, -1)[:, torch.from_numpy(nodes).to(dev())].double().cpu().numpy().T
    F = synthetic.profile_to_field(prof, shape)
    fo = oracle.first_step_nodes(o, nodes, None, u0, F)
    err = np.max(np.abs(hg + W.reshape(1, 19) - fo) / np.abs(fo))
    report("full_size_sampled_first_step", rel=float(err))
    assert err < 1e-6
    g.close()


def _rounding_bounds(n_nodes, steps, h_max, j_max, f_abs_sum, k=8.0):
    """Bounds on the drift of the FP64 totals of Eq. 9 mass and momentum over
    `steps` FP32 steps, from rounding alone (the exact update conserves mass
    and adds sum F to the momentum, Eqs. 5 and 8).
    - Each step stores the Q = 19 post-collision deviations of every node; each
      carries at most 4 round-to-nearest errors of at most half a unit in the
      last place of |h| <= h_max, i.e. zero-mean errors of standard deviation
      at most 2^-24 h_max / sqrt(3). The node's mass and momentum are +-1
      combinations of the 19 values.
    - The momentum moment itself (rho u + F/2, then + F/2 again) is rounded
      twice at its own magnitude |rho u| <= j_max.
    - Independent errors over n_nodes * steps node updates add as a random
      walk; the bound takes k = 8 standard deviations of it.
    - The force increment may carry one more rounding of relative size 2^-24
      per node and step, bounded without cancellation by steps 2^-24 sum |F|.
    - The fixed-point totals quantise each node's value to 2^-36 (error at
      most 2^-37), once for each of the two totals compared."""
    s_h = np.sqrt(19 * 4 / 3.0) * 2.0 ** -24 * h_max
    s_j = np.sqrt(2 / 3.0) * 2.0 ** -24 * j_max
    walk = np.sqrt(float(n_nodes) * steps)
    quant = 2 * n_nodes * 2.0 ** -37
    mass = k * s_h * walk + quant
    momentum = k * np.hypot(s_h, s_j) * walk + steps * 2.0 ** -24 * f_abs_sum + quant
    return mass, momentum


def test_full_size_conservation_and_determinism():
    """Properties that hold at any size, at 256^3 over 100 steps: total mass is
    constant and total momentum grows by the total force (sum F = 0 up to the
    FP32 rounding of the profile) in FP64 sums, within the bounds that FP32
    rounding allows (_rounding_bounds); two runs are bit-identical."""
    n, nu, steps = 256, 0.01, 100
    shape = (n, n, n)
    prof = synthetic.kolmogorov_profile(n, 1e-5)
    u0 = t(synthetic.divfree_velocity(shape, seed=1, umax=0.02))
    gain = steps * n * n * prof.astype(np.float64).sum(axis=1)
    f_abs_sum = n * n * float(np.abs(prof.astype(np.float64)).sum())
    states = []
    for _ in range(2):
        g, _ = make_pair(n, n, n, nu)
        tp = t(prof)
        g.set_force_profile_z(tp)
        g.init_equilibrium(None, u0)
        m0 = g.reduce_moments().cpu().numpy()
        g.step(steps)
        m1 = g.reduce_moments().cpu().numpy()
        g.check()
        h_max = float(g.populations(deviation=True).abs().max().item())
        rho, u = g.macros()
        j_max = 1.05 * float((rho * u).abs().max().item())
        b_mass, b_mom = _rounding_bounds(n ** 3, steps, h_max, j_max, f_abs_sum)
        report("full_size_conservation", mass_drift=float(m1[0] - m0[0]),
               momentum_drift=[float(v) for v in (m1[1:] - m0[1:] - gain)], bound_mass=b_mass,
               bound_momentum=b_mom, h_max=h_max, j_max=j_max)
        assert abs(m1[0] - m0[0]) < b_mass
        np.testing.assert_allclose(m1[1:] - m0[1:], gain, rtol=0, atol=b_mom)
        states.append(g.export_state().cpu())
        g.close()
    assert torch.equal(states[0], states[1])


def test_momentum_grows_by_total_force():
    nx, ny, nz = 40, 24, 16
    shape = (nz, ny, nx)
    g, _ = make_pair(nx, ny, nz, 0.05)
    F = synthetic.gaussian_force(shape, 1e-4, seed=61) + np.float32(2e-5)
    g.set_force_field(t(F))
    g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=62, umax=0.02)))
    m0 = g.reduce_moments().cpu().numpy()
    g.step(50)
    m1 = g.reduce_moments().cpu().numpy()
    gain = 50 * F.astype(np.float64).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(m1[1:] - m0[1:], gain, rtol=1e-5, atol=1e-9)
    # FP32 rounding of the stored deviations is not exactly mass-conserving: a
    # random walk of ~1e-10 per node and step (15360 nodes x 50 steps here)
    assert abs(m1[0] - m0[0]) < 1e-6
