"""The shared-memory staged A/B step for 16-bit storage (step_tma.cuh)
against the one-node-per-thread step (k_step), and against the FP64 oracle.

The staged kernel copies the pulled rows into shared memory with bulk
asynchronous copies and reads them back shifted along x; it performs the same
collision on the same values (the cascaded collision on two adjacent nodes at
once, with FP32x2 instructions that round like the one-node form, and pair
conversions), so its populations must equal k_step's bit for bit, for every
16-bit format, collision model, wall set and tile shape: tiles
of several rows with a partial last tile, one row per tile (nx = 1024), a
single row (ny = 1), a single plane (nz = 1), and x walls, whose nodes read
their bounce-back partners from global memory.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import W, dev, report, s2_of, t
from paper_1801_04586_gb300 import Lattice, synthetic

pytestmark = pytest.mark.gpu

RATES = dict(s2b=1.2, s3=1.1, s4=0.9)

CASES = [
    # (nx, ny, nz), walls, storage, model
    ((64, 20, 9), 0, "f16", "cascaded"),     # 16 rows per tile, partial last tile, y wrap runs
    ((40, 33, 7), 6, "bf16", "cascaded"),    # y and z walls, 25 rows per tile
    ((40, 33, 7), 6, "f16", "srt"),
    ((40, 33, 7), 6, "f16sr", "mrt"),
    ((8, 70, 5), 7, "f16", "cascaded"),      # walls on every axis, one tile per plane
    ((1024, 3, 4), 2, "f16", "cascaded"),    # one row per tile
    ((512, 5, 3), 0, "bf16", "mrt"),         # two rows per tile, partial last tile
    ((256, 1, 3), 0, "bf16sr", "cascaded"),  # ny = 1: the y shift maps a row onto itself
    ((24, 50, 1), 4, "f16", "cascaded"),     # nz = 1 between two z walls
    ((48, 16, 16), 1, "f16sr", "srt"),       # x walls
    ((32, 32, 32), 0, "bf16", "mrt"),
    ((48, 16, 16), 1, "bf16sr", "cascaded"),  # x walls, node pairs (both lanes bounce at the two x faces)
    ((16, 9, 5), 5, "f16", "cascaded"),       # x and z walls, node pairs
    ((8, 3, 2), 7, "f16sr", "cascaded"),      # a single node pair between x walls
]


def pair(shape_xyz, walls, storage, model, lattice=19):
    nx, ny, nz = shape_xyz
    kw = dict(walls=walls, storage=storage, model=model, device=dev(), lattice=lattice, **RATES)
    if lattice == 27:
        kw.update(s3b=1.3, s4b=0.8, s5=1.15, s6=0.95)
    return Lattice(nx, ny, nz, 0.02, variant=0, **kw), Lattice(nx, ny, nz, 0.02, variant=1, **kw)


@pytest.mark.parametrize("shape_xyz,walls,storage,model", CASES)
def test_staged_step_equals_plain_step(shape_xyz, walls, storage, model):
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    staged, plain = pair(shape_xyz, walls, storage, model)
    assert staged.info()["staged"] == 1 and plain.info()["staged"] == 0
    rho = synthetic.density_perturbation(shape, 0.01, seed=501)
    u = synthetic.divfree_velocity(shape, seed=502, umax=0.04)
    F = t(synthetic.gaussian_force(shape, 1e-4, seed=503))
    for g in (staged, plain):
        g.set_force_field(F)
        g.init_equilibrium(t(rho), t(u))
    for n in (1, 6):
        staged.step(n)
        plain.step(n)
        assert torch.equal(staged.populations(deviation=True), plain.populations(deviation=True))
    staged.check()


CASES27 = [
    ((64, 20, 9), 0, "f16", "cascaded"),
    ((40, 33, 7), 6, "bf16sr", "cascaded"),
    ((8, 70, 5), 7, "f16sr", "mrt"),
    ((24, 50, 1), 4, "bf16", "srt"),
    ((1024, 3, 4), 1, "f16", "cascaded"),
]


@pytest.mark.parametrize("shape_xyz,walls,storage,model", CASES27)
@pytest.mark.parametrize("force", ["field", "profile"])
def test_staged_d3q27_equals_plain_step(shape_xyz, walls, storage, model, force):
    """D3Q27 (Sec. II) through the same staged pipeline, 27 populations per
    tile. A force field does not fit two blocks' buffers per SM and runs the
    one-node-per-thread step, so it is checked as a fallback."""
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    staged, plain = pair(shape_xyz, walls, storage, model, lattice=27)
    rho = synthetic.density_perturbation(shape, 0.01, seed=521)
    u = synthetic.divfree_velocity(shape, seed=522, umax=0.04)
    for g in (staged, plain):
        if force == "field":
            g.set_force_field(t(synthetic.gaussian_force(shape, 1e-4, seed=523)))
        else:
            prof = torch.zeros(3, nz, device=dev())
            prof[0] = torch.linspace(-1e-4, 1e-4, nz, device=dev())
            prof[2] = 3e-5
            g.set_force_profile_z(prof)
        g.init_equilibrium(t(rho), t(u))
    assert staged.info()["staged"] == (0 if force == "field" else 1) and plain.info()["staged"] == 0
    for n in (1, 6):
        staged.step(n)
        plain.step(n)
        assert torch.equal(staged.populations(deviation=True), plain.populations(deviation=True))
    staged.check()


@pytest.mark.parametrize("storage", ["f16", "f16sr"])
def test_run_host_16bit_matches_staged_steps(storage):
    """A host job with 16-bit storage runs the fused step with in-kernel sums
    (one node per thread); its final state and per-step sums equal those of
    staged steps on the device, bit for bit."""
    nx, ny, nz, steps = 64, 24, 13, 40
    shape = (nz, ny, nx)
    rho = synthetic.density_perturbation(shape, 1e-3, 541)
    u = synthetic.divfree_velocity(shape, seed=542, umax=0.02)
    kw = dict(walls=4, storage=storage, device=dev(), **RATES)
    g = Lattice(nx, ny, nz, 0.05, **kw)
    assert g.info()["staged"] == 1
    g.set_force_uniform(1e-5)
    g.init_equilibrium(t(rho), t(u))
    sums = [g.reduce_moments().cpu()]
    for _ in range(steps):
        g.step(1)
        sums.append(g.reduce_moments().cpu())
    r_ref, u_ref = g.macros()
    h = Lattice(nx, ny, nz, 0.05, **kw)
    h.set_force_uniform(1e-5)
    r_out = torch.empty(shape).pin_memory()
    u_out = torch.empty((3,) + shape).pin_memory()
    mom = torch.empty(4 * (steps + 1), dtype=torch.float64).pin_memory()
    h.run_host(torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(), steps, r_out, u_out, mom)
    assert torch.equal(r_out, r_ref.cpu()) and torch.equal(u_out, u_ref.cpu())
    assert torch.equal(mom, torch.cat(sums))


@pytest.mark.parametrize("storage", ["f16", "bf16sr"])
def test_staged_step_full_size(storage):
    """The 256^3 Kolmogorov workload of the benchmark, in its launch
    configuration (persistent grid, 4-row tiles): two staged steps equal two
    one-node-per-thread steps bit for bit."""
    n = 256
    staged, plain = pair((n, n, n), 0, storage, "cascaded")
    prof = torch.zeros(3, n, device=dev())
    prof[0] = 1e-5 * torch.sin(2 * np.pi * torch.arange(n, device=dev()) / n)
    u = t(synthetic.divfree_velocity((n, n, n), seed=1, umax=0.02))
    for g in (staged, plain):
        g.set_force_profile_z(prof)
        g.init_equilibrium(None, u)
        g.step(2)
    assert torch.equal(staged.populations(deviation=True), plain.populations(deviation=True))
    staged.close()
    plain.close()


@pytest.mark.parametrize("force", ["uniform", "profile"])
def test_staged_step_force_modes(force):
    nx, ny, nz = 96, 24, 12
    staged, plain = pair((nx, ny, nz), 4, "f16", "cascaded")
    prof = torch.zeros(3, nz, device=dev())
    prof[0] = torch.linspace(-1e-4, 1e-4, nz, device=dev())
    for g in (staged, plain):
        if force == "uniform":
            g.set_force_uniform(1e-5, -2e-5, 3e-6)
        else:
            g.set_force_profile_z(prof)
        g.init_equilibrium()
    staged.step(9)
    plain.step(9)
    assert torch.equal(staged.populations(deviation=True), plain.populations(deviation=True))


@pytest.mark.parametrize("shape_xyz,storage", [((64, 16, 8), "f32"), ((36, 19, 11), "f16"), ((1040, 4, 4), "f16"),
                                               ((12, 9, 5), "bf16")])
def test_geometries_without_staging_fall_back(shape_xyz, storage):
    """FP32 storage, rows that are not a multiple of 16 bytes, and rows longer
    than a tile run the one-node-per-thread step."""
    g = Lattice(*shape_xyz, 0.02, storage=storage, device=dev())
    assert g.info()["staged"] == 0


def test_staged_full_size_sampled_against_oracle():
    """The FP16 256^3 Kolmogorov workload of the benchmark, in the launch
    configuration it times: for 2048 sampled nodes x, the oracle collides the
    node's (FP16) state; the staged step's result, read at x + e_i where
    population i streams to, equals it rounded to FP16, within half a unit in
    the last place plus the FP32 arithmetic's error."""
    n = 256
    g = Lattice(n, n, n, 0.01, storage="f16", device=dev())
    assert g.info()["staged"] == 1
    o = oracle.Lattice(1, 1, 1, s2=s2_of(0.01))
    prof = synthetic.kolmogorov_profile(n, 1e-5)
    g.set_force_profile_z(t(prof))
    g.init_equilibrium(None, t(synthetic.divfree_velocity((n, n, n), seed=1, umax=0.02)))
    nodes = np.random.default_rng(551).choice(n ** 3, 2048, replace=False)
    z, y, x = nodes // (n * n), (nodes // n) % n, nodes % n
    E = oracle.velocities(19).astype(np.int64)
    # the state read out is post-streaming: population i of node x at t = 1 is
    # the post-collision value of node x - e_i, so node x's result sits at x + e_i
    dst = np.stack([(((z + E[i, 2]) % n) * n + (y + E[i, 1]) % n) * n + (x + E[i, 0]) % n + i * n ** 3
                    for i in range(19)], axis=1)
    h0 = g.populations(deviation=True).reshape(19, -1)[:, torch.from_numpy(nodes).to(dev())]
    h0 = h0.double().cpu().numpy().T
    g.step(1)
    hg = g.populations(deviation=True).reshape(-1)[torch.from_numpy(dst.reshape(-1)).to(dev())]
    hg = hg.double().cpu().numpy().reshape(-1, 19)
    w = W.reshape(19)
    ho = np.stack([oracle.collide(o, h0[k] + w, (prof[0, z[k]], prof[1, z[k]], prof[2, z[k]])) - w
                   for k in range(len(nodes))])
    err = np.abs(hg - ho) / ulp16(np.maximum(np.abs(hg), np.abs(ho)))
    report("staged_f16_full_size_sampled_ulp", max_ulp=float(err.max()))
    assert err.max() <= 0.55
    g.close()


def ulp16(v):
    """Spacing of FP16 numbers at |v| (subnormal spacing below 2^-14)."""
    e = np.floor(np.log2(np.maximum(np.abs(v), 2.0 ** -14)))
    return 2.0 ** (e - 10)


def test_staged_step_against_oracle():
    """One staged FP16 step from an FP16-representable state against the
    FP64 oracle's step: each stored deviation is the oracle's rounded to
    FP16, within half a unit in the last place plus the FP32 arithmetic's
    error (about 1e-9 absolute, at most a few hundredths of an FP16 unit in
    the subnormal range)."""
    nx, ny, nz, walls = 64, 24, 18, 6
    shape = (nz, ny, nx)
    g = Lattice(nx, ny, nz, 0.03, walls=walls, storage="f16", device=dev(), **RATES)
    assert g.info()["staged"] == 1
    o = oracle.Lattice(nx, ny, nz, walls=walls, s2=s2_of(0.03), **RATES)
    h0 = torch.from_numpy(synthetic.rng(511).uniform(-2e-3, 2e-3, (19,) + shape)).half().float().numpy()
    F = synthetic.gaussian_force(shape, 1e-4, seed=512)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    g.step(1)
    ho = oracle.step(o, h0.astype(np.float64) + W, F, 1) - W
    hg = g.populations(deviation=True).double().cpu().numpy()
    err = np.abs(hg - ho) / ulp16(np.maximum(np.abs(hg), np.abs(ho)))
    report("staged_f16_one_step_ulp", shape=str(shape), walls=walls, max_ulp=float(err.max()))
    assert err.max() <= 0.55


# ---- the in-place (AA) pattern, staged in node pairs
AA_CASES = [
    # (nx, ny, nz), walls, storage, force
    ((48, 30, 10), 7, "f16", "field"),       # walls on every axis, 21 rows per tile, ragged second tile
    ((48, 30, 10), 7, "bf16sr", "field"),
    ((64, 40, 6), 2, "f16sr", "profile"),    # y walls only: pushes across the y faces bounce
    ((32, 20, 12), 1, "bf16", "uniform"),    # x walls only: both lanes of a pair at the two x faces
    ((256, 8, 5), 4, "f16sr", "field"),      # 4 rows per tile, z walls
    ((8, 130, 3), 0, "bf16sr", "uniform"),   # nx = 8: pushes wrap in x inside one pair row, two tiles per plane
    ((40, 12, 9), 0, "f16", "profile"),      # periodic: every push wraps somewhere
    ((16, 9, 1), 3, "f16sr", "field"),       # nz = 1, periodic z: z pushes land in the same plane
]


@pytest.mark.parametrize("shape_xyz,walls,storage,force", AA_CASES)
def test_staged_in_place_equals_one_node_in_place_and_ab(shape_xyz, walls, storage, force):
    """The staged node-pair in-place step (even kind: own rows, stores to the
    opposite slots; odd kind: opposite rows shifted as the pull, pushes with
    16-bit stores where a pair's targets straddle) stores the same bits as the
    one-node in-place kernel and as the A/B step, after odd and even step
    counts."""
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    mk = lambda **kw: Lattice(nx, ny, nz, 0.03, walls=walls, storage=storage, device=dev(), **RATES, **kw)
    staged, plain, ab = mk(pattern="aa"), mk(pattern="aa", variant=1), mk()
    assert staged.info()["staged"] == 1 and plain.info()["staged"] == 0
    rho = synthetic.density_perturbation(shape, 0.01, seed=41)
    u = synthetic.divfree_velocity(shape, seed=42, umax=0.04)
    F = t(synthetic.gaussian_force(shape, 1e-4, seed=43))
    prof = t(synthetic.kolmogorov_profile(nz, 1e-4))
    for g in (staged, plain, ab):
        if force == "field":
            g.set_force_field(F)
        elif force == "profile":
            g.set_force_profile_z(prof)
        else:
            g.set_force_uniform(2e-5, -1e-5, 3e-5)
        g.init_equilibrium(t(rho), t(u))
    done = 0
    for n in (1, 1, 5, 9):  # compared after 1, 2, 7 and 16 steps
        for g in (staged, plain, ab):
            g.step(n)
        done += n
        ps = staged.populations(deviation=True)
        assert torch.equal(ps, plain.populations(deviation=True)), f"staged vs one-node in place after {done}"
        assert torch.equal(ps, ab.populations(deviation=True)), f"staged in place vs A/B after {done}"
    for g in (staged, plain, ab):
        g.check()
        g.close()
