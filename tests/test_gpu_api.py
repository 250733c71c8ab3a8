"""GPU checks of the rest of the C ABI: reductions, state round trips,
checkpoint/resume, the host-buffer job and the instability flag."""
import numpy as np
import pytest
import torch

from gpu_common import dev, make_pair, t
from paper_1801_04586_gb300 import UnstableError, synthetic

pytestmark = pytest.mark.gpu


def test_reduce_pair_matches_numpy():
    g, _ = make_pair(8, 8, 8, 0.1)
    rng = np.random.default_rng(3)
    for n in (1, 257, 100_003, 3 * 64 ** 3):
        a = rng.normal(size=n).astype(np.float32)
        b = rng.normal(size=n).astype(np.float32)
        out = g.reduce_pair(t(a), t(b)).cpu().numpy()
        a64, b64 = a.astype(np.float64), b.astype(np.float64)
        np.testing.assert_allclose(out, [((a64 - b64) ** 2).sum(), (b64 ** 2).sum(), (a64 * b64).sum()],
                                   rtol=1e-12)
        out0 = g.reduce_pair(t(a)).cpu().numpy()
        np.testing.assert_allclose(out0[0], (a64 ** 2).sum(), rtol=1e-12)
    empty = torch.empty(0, device=dev())
    np.testing.assert_array_equal(g.reduce_pair(empty).cpu().numpy(), [0.0, 0.0, 0.0])


def test_reduce_moments_matches_macros():
    nx, ny, nz = 33, 17, 9
    shape = (nz, ny, nx)
    g, _ = make_pair(nx, ny, nz, 0.05, walls=2)
    F = synthetic.gaussian_force(shape, 1e-4, seed=5)
    g.set_force_field(t(F))
    g.init_equilibrium(t(synthetic.density_perturbation(shape, 0.01, 6)),
                       t(synthetic.divfree_velocity(shape, seed=7, umax=0.03)))
    g.step(7)
    rho, u = g.macros()
    m = g.reduce_moments().cpu().numpy()
    r64, u64 = rho.double().cpu().numpy(), u.double().cpu().numpy()
    assert m[0] == pytest.approx(r64.sum(), rel=1e-7)
    np.testing.assert_allclose(m[1:], (r64[None] * u64).sum(axis=(1, 2, 3)), rtol=1e-4, atol=1e-8)


@pytest.mark.parametrize("walls", [0, 5])
def test_set_get_populations_roundtrip(walls):
    nx, ny, nz = 21, 10, 7
    g, _ = make_pair(nx, ny, nz, 0.05, walls=walls)
    h = synthetic.random_deviations((nz, ny, nx), 1e-2, seed=9)
    g.set_populations(t(h), deviation=True)
    np.testing.assert_array_equal(g.populations(deviation=True).cpu().numpy(), h)
    f = h.astype(np.float32) + np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, np.float32).reshape(19, 1, 1, 1)
    g.set_populations(t(f), deviation=False)
    np.testing.assert_allclose(g.populations(deviation=False).cpu().numpy(), f, rtol=0, atol=1e-7)


def test_checkpoint_resume_bit_exact():
    nx, ny, nz = 40, 30, 20
    shape = (nz, ny, nx)
    g, _ = make_pair(nx, ny, nz, 0.02, walls=4, s3=1.2)
    g.set_force_uniform(1e-5, 2e-6)
    g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=3, umax=0.02)))
    g.step(60)
    blob = g.save_state()
    g.step(40)
    a = g.populations(deviation=True).cpu()
    assert g.steps_done == 100
    g2, _ = make_pair(nx, ny, nz, 0.02, walls=4, s3=1.2)
    g2.set_force_uniform(1e-5, 2e-6)
    g2.load_state(blob)
    assert g2.steps_done == 60
    g2.step(40)
    assert torch.equal(a, g2.populations(deviation=True).cpu())
    # device-side export/import
    snap = g.export_state()
    g.step(5)
    g.import_state(snap, set_steps=100)
    assert torch.equal(a, g.populations(deviation=True).cpu())
    with pytest.raises(Exception):
        g3, _ = make_pair(nx, ny, nz + 1, 0.02, walls=4)
        g3.load_state(blob)


def test_run_host_job_matches_device_path():
    # 150 steps wrap the 64-slot ring of per-step totals twice; nz = 23 leaves a
    # ragged group of z-planes for the kernels that take four planes per thread
    nx, ny, nz, steps = 48, 32, 23, 150
    shape = (nz, ny, nx)
    rho = synthetic.density_perturbation(shape, 1e-3, 1)
    u = synthetic.divfree_velocity(shape, seed=2, umax=0.02)
    g, _ = make_pair(nx, ny, nz, 0.05, walls=4)
    g.set_force_uniform(1e-5)
    g.init_equilibrium(t(rho), t(u))
    g.step(steps)
    r_ref, u_ref = g.macros()
    m_ref = g.reduce_moments().cpu()
    g2, _ = make_pair(nx, ny, nz, 0.05, walls=4)
    g2.set_force_uniform(1e-5)
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    r_out = torch.empty(shape).pin_memory()
    u_out = torch.empty((3,) + shape).pin_memory()
    mom = torch.empty(4 * (steps + 1), dtype=torch.float64).pin_memory()
    g2.run_host(rho_h, u_h, steps, r_out, u_out, mom)
    assert torch.equal(r_out, r_ref.cpu())
    assert torch.equal(u_out, u_ref.cpu())
    assert torch.equal(mom[-4:], m_ref)
    # a second job on the same context (its host copies and read-out run in plane chunks on a second stream)
    r_out2, u_out2 = torch.zeros(shape).pin_memory(), torch.zeros((3,) + shape).pin_memory()
    mom_b = torch.empty_like(mom).pin_memory()
    g2.run_host(rho_h, u_h, steps, r_out2, u_out2, mom_b)
    assert torch.equal(r_out2, r_out) and torch.equal(u_out2, u_out) and torch.equal(mom_b, mom)
    # per-step sums formed inside the step kernels are exact fixed-point sums of
    # the same per-node values as clbm_reduce_moments: equal bit for bit
    g3, _ = make_pair(nx, ny, nz, 0.05, walls=4)
    g3.set_force_uniform(1e-5)
    g3.init_equilibrium(t(rho), t(u))
    m = mom.numpy().reshape(steps + 1, 4)
    m0 = g3.reduce_moments().cpu().numpy()
    assert np.all(np.abs(m[:, 0] - m0[0]) < 1e-6)
    for k in range(steps + 1):  # every step's sums, written by the next launch
        np.testing.assert_array_equal(m[k], g3.reduce_moments().cpu().numpy())
        g3.step(1)
    # pageable host buffers take the copy path: same values
    g4, _ = make_pair(nx, ny, nz, 0.05, walls=4)
    g4.set_force_uniform(1e-5)
    mom2 = torch.empty(4 * (steps + 1), dtype=torch.float64)
    g4.run_host(torch.from_numpy(rho), torch.from_numpy(u), steps, None, None, mom2)
    assert torch.equal(mom2, mom)
    # one step and no steps
    for n in (1, 0):
        g5, _ = make_pair(nx, ny, nz, 0.05, walls=4)
        g5.set_force_uniform(1e-5)
        m5 = torch.empty(4 * (n + 1), dtype=torch.float64).pin_memory()
        g5.run_host(rho_h, u_h, n, None, None, m5)
        assert torch.equal(m5, mom[: 4 * (n + 1)])


@pytest.mark.parametrize("nz,walls,steps", [(1, 0, 2), (2, 0, 1), (3, 0, 2), (3, 0, 4), (9, 0, 5), (40, 0, 2),
                                             (17, 4, 3), (8, 0, 1), (26, 0, 7)])
def test_run_host_split_steps(nz, walls, steps):
    """With per-step sums, a host job runs its first two steps plane chunk by
    plane chunk as the input lands, and its last step chunk by chunk, each chunk read
    out as soon as it and its two neighbouring chunks are stepped. Periodic z
    makes the two end chunks neighbours; 1-3 planes give 1-3 chunks; a decaying
    z-profile force makes the read-out take the force of the final step.
    Everything equals the device path bit for bit."""
    nx, ny = 32, 12
    shape = (nz, ny, nx)
    rho = synthetic.density_perturbation(shape, 1e-3, 60 + nz)
    u = synthetic.divfree_velocity(shape, seed=61 + nz, umax=0.02)
    prof = torch.zeros(3, nz)
    prof[0] = 1e-5 * torch.cos(2 * np.pi * torch.arange(nz) / nz)
    prof[2] = 3e-6

    def lattice():
        g, _ = make_pair(nx, ny, nz, 0.04, walls=walls, s3=1.1)
        g.set_force_profile_z(prof.to(dev()))
        g.set_force_decay(0.05)
        return g

    g = lattice()
    g.init_equilibrium(t(rho), t(u))
    sums = []
    for _ in range(steps):
        sums.append(g.reduce_moments().cpu())
        g.step(1)
    sums.append(g.reduce_moments().cpu())
    r_ref, u_ref = g.macros()
    h = lattice()
    r_out = torch.empty(shape).pin_memory()
    u_out = torch.empty((3,) + shape).pin_memory()
    mom = torch.empty(4 * (steps + 1), dtype=torch.float64).pin_memory()
    h.run_host(torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(), steps, r_out, u_out, mom)
    assert torch.equal(r_out, r_ref.cpu()) and torch.equal(u_out, u_ref.cpu())
    assert torch.equal(mom, torch.cat(sums))
    assert torch.equal(h.populations(deviation=True), g.populations(deviation=True))
    # only rho read back, then no output at all: the same state and sums
    r_only = torch.empty(shape).pin_memory()
    h.run_host(torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(), steps, r_only, None, mom)
    assert torch.equal(r_only, r_out) and torch.equal(mom, torch.cat(sums))
    h.run_host(torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(), steps, None, None, mom)
    assert torch.equal(mom, torch.cat(sums))
    assert torch.equal(h.populations(deviation=True), g.populations(deviation=True))


def test_instability_flag():
    g, _ = make_pair(16, 8, 8, 0.05)
    g.init_equilibrium()
    g.step(3)
    g.check()
    h = torch.zeros(19, 8, 8, 16, device=dev())
    h[0, 3, 4, 5] = float("nan")
    g.set_populations(h, deviation=True)
    g.step(2)
    with pytest.raises(UnstableError):
        g.check(clear=True)
    g.init_equilibrium()
    g.step(2)
    g.check()


def test_bulk_rate_instability_is_flagged():
    """A physical blow-up, not an injected NaN: at nu = 0.1 with the bulk rate
    at 1.9 the rest state is linearly unstable (von Neumann spectral radius
    1.11, tests/test_oracle_collision.py); a small perturbation grows until a
    density leaves (0.1, 1.9) and the step kernel raises the flag. With the
    bulk rate at 1.2 the same perturbation decays."""
    shape = (16, 16, 16)
    h0 = synthetic.rng(71).uniform(-1e-5, 1e-5, (19,) + shape).astype(np.float32)
    for s2b, unstable in ((1.2, False), (1.9, True)):
        g, _ = make_pair(16, 16, 16, 0.1, s2b=s2b)
        g.set_populations(t(h0), deviation=True)
        g.step(400)
        if unstable:
            with pytest.raises(UnstableError):
                g.check()
        else:
            g.check()
            assert float(g.populations(deviation=True).abs().max()) < 1e-4  # no growth


@pytest.mark.parametrize("kw", [dict(), dict(pattern="aa"), dict(lattice=27), dict(model="mrt"),
                                dict(storage="f16sr")])
def test_long_steps_replay_graph_bit_identical(kw):
    """step(n) for n >= 32 replays a captured 16-step graph when the launch
    arguments are static (not for stochastic rounding or a decaying force):
    bit-identical to single steps, from either phase, and rebuilt when the
    force changes."""
    from paper_1801_04586_gb300 import Lattice
    nx, ny, nz = 40, 12, 10
    shape = (nz, ny, nx)
    u0 = t(synthetic.divfree_velocity(shape, seed=81, umax=0.03))
    a = Lattice(nx, ny, nz, 0.05, walls=4, device=dev(), **kw)
    b = Lattice(nx, ny, nz, 0.05, walls=4, device=dev(), **kw)
    for g in (a, b):
        g.set_force_uniform(1e-5)
        g.init_equilibrium(None, u0)
    a.step(1)  # odd phase: the next long run first takes one plain step
    b.step(1)
    a.step(53)
    for _ in range(53):
        b.step(1)
    assert a.steps_done == b.steps_done == 54
    assert torch.equal(a.populations(deviation=True), b.populations(deviation=True))
    for g in (a, b):
        g.set_force_uniform(-2e-5, 1e-5)
    a.step(40)
    for _ in range(40):
        b.step(1)
    assert torch.equal(a.populations(deviation=True), b.populations(deviation=True))


def test_allocation_failure_is_reported():
    """A real allocation failure, not a GPU fault: 2047 x 2047 x 512 nodes
    (within the ABI's 2^31 - 1 limit) need 326 GB for the FP32 A/B pair, more
    than the device holds. clbm_create returns CLBM_ERR_OOM, leaves nothing
    allocated, and the next lattice works."""
    from paper_1801_04586_gb300 import CLBMError, Lattice
    with pytest.raises(CLBMError) as exc:
        Lattice(2047, 2047, 512, 0.05, device=dev())
    assert "status -2" in str(exc.value)
    g, _ = make_pair(8, 8, 8, 0.05)
    g.init_equilibrium()
    g.step(3)
    g.check()
