"""The z-slab decomposition of the library's step (Eq. 8 across the slab
faces) against one undivided lattice, through the C ABI: slabs that exchange
their faces after every step reproduce the undivided state bit for bit, for
periodic and walled z axes, x/y walls, every storage format (stochastic
rounding included: its dither takes the global node index), a one-plane
slab, the split step (faces, then interior, with the exchange between), and
two ranks in separate processes on the one GPU exchanging through host
memory (gloo). Plus the calls a slab context refuses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from gpu_common import dev, t
from paper_1801_04586_gb300 import Lattice, _capi, slabs, synthetic

pytestmark = pytest.mark.gpu

RATES = dict(s2b=1.2, s3=1.1, s4=0.9)


def _inputs(shape, seed):
    u0 = synthetic.divfree_velocity(shape, seed=seed, umax=0.03)
    F = synthetic.gaussian_force(shape, 1e-4, seed=seed + 1)
    return u0, F


def _undivided(nx, ny, nz, walls, storage, u0, F, steps, nu=0.04):
    g = Lattice(nx, ny, nz, nu, walls=walls, storage=storage, device=dev(), **RATES)
    g.set_force_field(t(F))
    g.init_equilibrium(None, t(u0))
    for _ in range(steps):
        g.step(1)
    out = g.populations(deviation=True).cpu()
    g.close()
    return out


def _make_slabs(nx, ny, nz, walls, storage, u0, F, ranges, periodic, nu=0.04):
    lats, keep = [], []
    world = len(ranges)
    for r, (z0, z1) in enumerate(ranges):
        if periodic:
            bits = 3
        else:
            bits = (1 if r > 0 else 0) | (2 if r < world - 1 else 0)
        lat = Lattice(nx, ny, z1 - z0, nu, walls=walls, storage=storage, device=dev(), slab=bits, z0=z0, **RATES)
        Fs = t(np.ascontiguousarray(F[:, z0:z1]))
        lat.set_force_field(Fs)
        lat.init_equilibrium(None, t(np.ascontiguousarray(u0[:, z0:z1])))
        lats.append(lat)
        keep.append(Fs)
    return lats, keep


def _exchange_all(lats, faces=None):
    """Every face to its neighbour (one process; the lattices share a stream).
    faces: (send, recv) views per slab (default: the newest states')."""
    world = len(lats)
    faces = [lat.faces() for lat in lats] if faces is None else faces
    for r, lat in enumerate(lats):
        send = faces[r][0]
        half = send.numel() // 2
        lo, hi = (r - 1) % world, (r + 1) % world
        if lat.slab & 2:
            faces[hi][1][:half].copy_(send[half:])
        if lat.slab & 1:
            faces[lo][1][half:].copy_(send[:half])


def _gather(lats):
    return torch.cat([lat.populations(deviation=True).cpu() for lat in lats], dim=1)


CASES = [
    # (nx, ny, nz, walls, storage, ranges, periodic)
    (24, 20, 16, 0, "f32", [(0, 8), (8, 16)], True),
    (24, 20, 16, 4, "f32", [(0, 8), (8, 16)], False),
    (33, 17, 12, 7, "f32", [(0, 5), (5, 6), (6, 12)], False),
    (24, 20, 15, 3, "f32", [(0, 4), (4, 5), (5, 15)], True),
    (32, 16, 16, 6, "f16", [(0, 7), (7, 16)], False),
    (32, 16, 16, 0, "bf16", [(0, 9), (9, 16)], True),
    (32, 16, 16, 4, "f16sr", [(0, 8), (8, 16)], False),
    (32, 16, 16, 0, "bf16sr", [(0, 3), (3, 11), (11, 16)], True),
    (40, 12, 10, 0, "f32", [(0, 10)], True),
    (32, 16, 10, 2, "f16", [(0, 4), (4, 5), (5, 10)], True),   # staged 16-bit, a one-plane slab
    (40, 12, 9, 5, "f16sr", [(0, 3), (3, 9)], False),          # staged, x walls and z walls at the ends
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}w{c[3]}{c[4]}s{len(c[5])}")
def test_slabs_reproduce_the_undivided_lattice(case):
    nx, ny, nz, walls, storage, ranges, periodic = case
    if not periodic:
        walls |= 4
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 5)
    steps = 40
    ref = _undivided(nx, ny, nz, walls, storage, u0, F, steps)
    lats, keep = _make_slabs(nx, ny, nz, walls, storage, u0, F, ranges, periodic)
    if storage != "f32":  # 16-bit slabs run the staged step, reading the halo planes in its copies
        assert all(lat.info()["staged"] == 1 for lat in lats)
    assert torch.equal(_gather(lats), _undivided(nx, ny, nz, walls, storage, u0, F, 0))
    for _ in range(steps):
        for lat in lats:
            lat.slab_step()
        _exchange_all(lats)
    got = _gather(lats)
    assert torch.equal(got, ref)
    mom = sum(lat.reduce_moments().cpu().numpy() for lat in lats)
    g = Lattice(nx, ny, nz, 0.04, walls=walls, storage=storage, device=dev(), **RATES)
    g.set_force_field(t(F))
    g.set_populations(ref.to(dev()), deviation=True)
    np.testing.assert_allclose(mom, g.reduce_moments().cpu().numpy(), rtol=1e-13, atol=1e-13)
    g.close()
    for lat in lats:
        lat.check()
        lat.close()


def test_split_step_with_overlapped_exchange_equals_whole_step():
    """SLAB_FACES, the exchange, then SLAB_INTERIOR: the receive planes of the
    new state are written while the interior part is still to run."""
    nx, ny, nz = 48, 24, 20
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 9)
    ref = _undivided(nx, ny, nz, 0, "f32", u0, F, 30)
    lats, keep = _make_slabs(nx, ny, nz, 0, "f32", u0, F, [(0, 10), (10, 20)], True)
    for _ in range(30):
        for lat in lats:
            lat.slab_step(_capi.SLAB_FACES)
        _exchange_all(lats)
        for lat in lats:
            lat.slab_step(_capi.SLAB_INTERIOR)
    assert torch.equal(_gather(lats), ref)
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("storage", ["f32", "f16sr"])
def test_self_neighbour_with_unwaited_side_stream_exchange(storage):
    """One periodic slab that is its own neighbour, its face copies left
    unwaited on the side stream while the interior part runs (the benchmark's
    single-GPU slab line): equal to the undivided lattice after 60 steps."""
    nx, ny, nz = 32, 16, 14
    u0, F = _inputs((nz, ny, nx), 21)
    ref = _undivided(nx, ny, nz, 0, storage, u0, F, 60)
    lats, keep = _make_slabs(nx, ny, nz, 0, storage, u0, F, [(0, nz)], True)
    lat = lats[0]
    with torch.cuda.stream(lat.stream):
        for _ in range(60):
            lat.slab_step(_capi.SLAB_FACES)
            reqs = slabs.exchange_faces(lat, 0, 1, wait=False)
            assert len(reqs) == 1
            lat.slab_step(_capi.SLAB_INTERIOR)
            for r in reqs:
                r.wait()
    torch.cuda.synchronize()
    assert torch.equal(_gather(lats), ref)
    lat.check()
    lat.close()


def test_kolmogorov_slabs_with_profile_force_and_split_steps():
    """The configuration the benchmark runs on several GPUs, on one: z-slabs of
    a periodic Kolmogorov box (z-profile force F_x = F0 sin(2 pi z/nz), each
    slab given its own planes of the profile), FP32 and stochastic FP16,
    stepped in faces and interior parts with the exchange between them."""
    nx, ny, nz, F0 = 32, 24, 24, 1e-4
    shape = (nz, ny, nx)
    prof = synthetic.kolmogorov_profile(nz, F0)
    u0 = synthetic.divfree_velocity(shape, seed=1, umax=0.02)
    for storage in ("f32", "f16sr"):
        g = Lattice(nx, ny, nz, 0.01, storage=storage, device=dev())
        gp = t(prof)
        g.set_force_profile_z(gp)
        g.init_equilibrium(None, t(u0))
        for _ in range(25):
            g.step(1)
        ref = g.populations(deviation=True).cpu()
        g.close()
        lats, keep = [], []
        for z0, z1 in [(0, 8), (8, 16), (16, 24)]:
            lat = Lattice(nx, ny, z1 - z0, 0.01, storage=storage, device=dev(), slab=3, z0=z0)
            p = t(np.ascontiguousarray(prof[:, z0:z1]))
            lat.set_force_profile_z(p)
            lat.init_equilibrium(None, t(np.ascontiguousarray(u0[:, z0:z1])))
            lats.append(lat)
            keep.append(p)
        for _ in range(25):
            for lat in lats:
                lat.slab_step(_capi.SLAB_FACES)
            _exchange_all(lats)
            for lat in lats:
                lat.slab_step(_capi.SLAB_INTERIOR)
        assert torch.equal(_gather(lats), ref), storage
        for lat in lats:
            lat.check()
            lat.close()


def test_slab_checkpoint_round_trip_continues_bit_identically():
    """A slab's saved state holds its halo planes: restoring it into fresh
    contexts, after the exchange that followed the last step, continues the
    decomposed run exactly as the uninterrupted one."""
    nx, ny, nz = 24, 16, 12
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 31)
    ranges = [(0, 5), (5, 12)]
    lats, keep = _make_slabs(nx, ny, nz, 2, "f16sr", u0, F, ranges, True)
    for _ in range(7):
        for lat in lats:
            lat.slab_step()
        _exchange_all(lats)
    saved = [lat.save_state() for lat in lats]
    for _ in range(9):
        for lat in lats:
            lat.slab_step()
        _exchange_all(lats)
    ref = _gather(lats)
    fresh, keep2 = _make_slabs(nx, ny, nz, 2, "f16sr", u0, F, ranges, True)
    for lat, data in zip(fresh, saved):
        lat.load_state(data)
        assert lat.steps_done == 7
    for _ in range(9):
        for lat in fresh:
            lat.slab_step()
        _exchange_all(fresh)
    assert torch.equal(_gather(fresh), ref)
    for lat in lats + fresh:
        lat.close()


def test_slab_context_refuses_what_needs_no_exchange():
    lat = Lattice(16, 8, 6, 0.05, device=dev(), slab=3, z0=4)
    info = lat.info()
    assert info["slab"] == 3 and info["face_bytes"] == 5 * 16 * 8 * 4
    assert info["state_bytes"] == (19 * info["pop_stride"] + 20 * 16 * 8) * 4
    lib = lat.lib
    assert lib.clbm_step(lat.h, 2) == _capi.CLBM_ERR_STATE
    assert lib.clbm_slab_step(lat.h, _capi.SLAB_INTERIOR) == _capi.CLBM_ERR_STATE
    assert lib.clbm_slab_step(lat.h, 7) == _capi.CLBM_ERR_ARG
    assert lib.clbm_slab_step(lat.h, _capi.SLAB_FACES) == _capi.CLBM_OK
    assert lib.clbm_slab_step(lat.h, _capi.SLAB_FACES) == _capi.CLBM_ERR_STATE
    assert lib.clbm_slab_step(lat.h, _capi.SLAB_INTERIOR) == _capi.CLBM_OK
    assert lib.clbm_run_host(lat.h, None, None, 1, None, None, None) == _capi.CLBM_ERR_STATE
    st = lat.export_state()
    la, lb = lat.empty_lam(), lat.empty_lam()
    assert la.numel() == 19 * 16 * 8 * 6 + 20 * 16 * 8
    gf = torch.zeros(3 * 16 * 8 * 6, device=dev())
    assert lib.clbm_adjoint_segment(lat.h, st.data_ptr(), None, 1, la.data_ptr(), lb.data_ptr(),
                                    gf.data_ptr()) == _capi.CLBM_ERR_STATE
    plain = Lattice(16, 8, 6, 0.05, device=dev())
    assert plain.lib.clbm_slab_step(plain.h, 0) == _capi.CLBM_ERR_ARG
    lat.close()
    plain.close()


# ---- two ranks in separate processes on the one GPU (gloo, faces through host memory)
NX, NY, NZ, STEPS = 40, 24, 18, 100
RANK_CASES = [  # (walls, storage, periodic z)
    (2, "f32", True),
    (2 | 4, "f16sr", False),  # z walls at the box ends, the staged 16-bit step
]


def _rank_worker(rank, world, port, out_path, walls, storage, periodic):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    shape = (NZ, NY, NX)
    u0, F = _inputs(shape, 13)
    z0, nzl, bits = slabs.slab_of(NZ, rank, world, periodic_z=periodic)
    lat = Lattice(NX, NY, nzl, 0.04, walls=walls, storage=storage, device=dev(), slab=bits, z0=z0, **RATES)
    Fs = t(np.ascontiguousarray(F[:, z0:z0 + nzl]))
    lat.set_force_field(Fs)
    lat.init_equilibrium(None, t(np.ascontiguousarray(u0[:, z0:z0 + nzl])))
    for _ in range(STEPS):
        lat.slab_step()
        slabs.exchange_faces(lat, rank, world, dist, host=True)
    torch.save(lat.populations(deviation=True).cpu(), f"{out_path}.{rank}")
    # whole-lattice FP64 totals and an L2 error of the velocity, summed over the ranks
    target = t(np.ascontiguousarray(synthetic.divfree_velocity(shape, seed=14, umax=0.01)[:, z0:z0 + nzl]))
    _, u = lat.macros()
    torch.save((slabs.global_moments(lat, dist).cpu(), slabs.global_pair(lat, u, target, dist).cpu()),
               f"{out_path}.sums.{rank}")
    lat.check()
    lat.close()
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", RANK_CASES, ids=lambda c: f"w{c[0]}{c[1]}{'p' if c[2] else ''}")
def test_two_rank_processes_match_the_undivided_lattice(tmp_path, case):
    walls, storage, periodic = case
    out = str(tmp_path / "slab")
    mp.start_processes(_rank_worker, args=(2, _free_port(), out, walls, storage, periodic), nprocs=2,
                       start_method="spawn", join=True)
    got = torch.cat([torch.load(f"{out}.{r}") for r in range(2)], dim=1)
    u0, F = _inputs((NZ, NY, NX), 13)
    ref = _undivided(NX, NY, NZ, walls, storage, u0, F, STEPS)
    assert torch.equal(got, ref)
    g = Lattice(NX, NY, NZ, 0.04, walls=walls, storage=storage, device=dev(), **RATES)
    g.set_force_field(t(F))
    g.set_populations(ref.to(dev()), deviation=True)
    _, u = g.macros()
    target = t(synthetic.divfree_velocity((NZ, NY, NX), seed=14, umax=0.01))
    m_ref, p_ref = g.reduce_moments().cpu(), g.reduce_pair(u, target).cpu()
    g.close()
    for r in range(2):
        m, pr = torch.load(f"{out}.sums.{r}")
        np.testing.assert_allclose(m.numpy(), m_ref.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(pr.numpy(), p_ref.numpy(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("scaling", ["weak", "strong"])
def test_benchmark_slab_mode_runs_two_ranks_on_one_gpu(scaling):
    """bench.py --gpus 2 under torchrun, its z-slab mode: two ranks sharing the
    one GPU (gloo, faces through host memory; the NCCL exchange needs one GPU
    per rank) print one contract line with two launches per step, for the
    256 x 256 x 512 box (weak scaling) or one 128^3 box split in two (strong
    scaling, a small copy of the 512^3 mode)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2", "--steps", "4",
           "--warmup", "2", "--dist-backend", "gloo", "--no-variants", "--no-cpu-baseline"]
    if scaling == "strong":
        cmd += ["--scaling", "strong", "--size", "64", "--strong-side", "128"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["steps"] == 4 and d["scaling"] == scaling and d["value"] > 0
    assert d["gpu_launches"] == 8
    assert "z-slab" in d["config"]["parallelism"]
    if scaling == "weak":
        assert "256x256x512" in d["config"]["workload"]
    else:
        assert "128^3" in d["config"]["workload"] and d["config"]["nz"] == 128
    assert d["e2e"]["value"] > 0


@pytest.mark.parametrize("storage", ["f32", "f16sr"])
def test_full_size_slab_rank_sampled_first_step(storage):
    """A rank of the multi-GPU benchmark at full size: one 256^3 z-slab of the
    periodic Kolmogorov box (F_x = 1e-5 sin(2 pi z/256), nu = 0.01, u0 of max
    |u| = 0.02), its own neighbour, stepped as the benchmark does (faces part,
    face copies on the side stream, interior part). Bit-identical to the
    unsplit lattice, and (FP32) within 1e-6 of the oracle's first step at 2048
    sampled nodes."""
    import oracle
    from gpu_common import W as W19
    n, nu = 256, 0.01
    shape = (n, n, n)
    prof = synthetic.kolmogorov_profile(n, 1e-5)
    u0 = synthetic.divfree_velocity(shape, seed=1, umax=0.02)
    lat = Lattice(n, n, n, nu, storage=storage, device=dev(), slab=3, z0=0)
    lat.set_force_profile_z(t(prof))
    lat.init_equilibrium(None, t(u0))
    with torch.cuda.stream(lat.stream):
        lat.slab_step(_capi.SLAB_FACES)
        reqs = slabs.exchange_faces(lat, 0, 1, wait=False)
        lat.slab_step(_capi.SLAB_INTERIOR)
        for r in reqs:
            r.wait()
    torch.cuda.synchronize()
    lat.check()
    fs = lat.populations(deviation=True)
    lat.close()
    g = Lattice(n, n, n, nu, storage=storage, device=dev())
    g.set_force_profile_z(t(prof))
    g.init_equilibrium(None, t(u0))
    g.step(1)
    assert torch.equal(fs, g.populations(deviation=True))
    g.close()
    if storage == "f32":
        o = oracle.Lattice(n, n, n, s2=1.0 / (3 * nu + 0.5))
        nodes = np.random.default_rng(9).choice(n ** 3, 2048, replace=False)
        hg = fs.reshape(19, -1)[:, torch.from_numpy(nodes).to(dev())].double().cpu().numpy().T
        fo = oracle.first_step_nodes(o, nodes, None, u0, synthetic.profile_to_field(prof, shape))
        assert np.max(np.abs(hg + W19.reshape(1, 19) - fo) / np.abs(fo)) < 1e-6


ADJ_CASES = [
    # (nx, ny, nz, walls, ranges, periodic z)
    (24, 16, 12, 0, [(0, 5), (5, 6), (6, 12)], True),  # a one-plane slab
    (20, 12, 10, 3, [(0, 4), (4, 10)], False),         # x and y walls, z walls at the ends
]


@pytest.mark.parametrize("case", ADJ_CASES, ids=lambda c: f"w{c[3]}s{len(c[4])}{'p' if c[5] else ''}")
def test_slab_adjoint_equals_undivided(case):
    """The adjoint across slabs (the reverse-direction halo): slabs stepped
    forward with face exchanges, then seeded from a cotangent on the final
    velocity and stepped back with the adjoint faces exchanged after every
    adjoint step, give bit for bit the undivided lattice's lambda^0 and dL/dF.
    The same holds with the slab states recomputed from state 0 by step_raw
    and the state-face exchange."""
    nx, ny, nz, walls, ranges, periodic = case
    if not periodic:
        walls |= 4
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 31)
    gu = synthetic.gaussian_force(shape, 1e-2, seed=33)
    K = 6
    g = Lattice(nx, ny, nz, 0.04, walls=walls, device=dev(), **RATES)
    g.set_force_field(t(F))
    g.init_equilibrium(None, t(u0))
    states = [g.export_state().clone()]
    for _ in range(K):
        g.step(1)
        states.append(g.export_state().clone())
    lam, lam2 = g.empty_lam(), g.empty_lam()
    gF = torch.zeros((3,) + shape, device=dev())
    g.adjoint_seed(t(gu), lam, gF, state=states[K])
    for k in range(K - 1, -1, -1):
        g.adjoint_step(states[k], lam, lam2, gF)
        lam, lam2 = lam2, lam
    ref_lam, ref_gF = lam.view(19, nz, ny, nx).cpu(), gF.cpu()
    g.close()

    lats, keep = _make_slabs(nx, ny, nz, walls, "f32", u0, F, ranges, periodic)
    saved = [[lat.export_state().clone()] for lat in lats]
    for _ in range(K):
        for lat in lats:
            lat.slab_step()
        _exchange_all(lats)
        for r, lat in enumerate(lats):
            saved[r].append(lat.export_state().clone())
    # the same states recomputed from state 0
    recomputed = [[st[0]] for st in saved]
    for _ in range(K):
        outs = [torch.empty_like(st[0]) for st in saved]
        for r, lat in enumerate(lats):
            lat.step_raw(recomputed[r][-1], outs[r])
        _exchange_all(lats, [slabs.state_faces(lat, o) for lat, o in zip(lats, outs)])
        for r in range(len(lats)):
            recomputed[r].append(outs[r])

    for tape in (saved, recomputed):
        lam_s = [lat.empty_lam() for lat in lats]
        lam2_s = [lat.empty_lam() for lat in lats]
        gF_s = [torch.zeros((3, z1 - z0, ny, nx), device=dev()) for z0, z1 in ranges]
        for r, (lat, (z0, z1)) in enumerate(zip(lats, ranges)):
            lat.adjoint_seed(t(np.ascontiguousarray(gu[:, z0:z1])), lam_s[r], gF_s[r], state=tape[r][K])
        _exchange_all(lats, [slabs.lam_faces(lat, a) for lat, a in zip(lats, lam_s)])
        for k in range(K - 1, -1, -1):
            for r, lat in enumerate(lats):
                lat.adjoint_step(tape[r][k], lam_s[r], lam2_s[r], gF_s[r])
            _exchange_all(lats, [slabs.lam_faces(lat, a) for lat, a in zip(lats, lam2_s)])
            lam_s, lam2_s = lam2_s, lam_s
        got_lam = torch.cat([a[:19 * (z1 - z0) * ny * nx].view(19, z1 - z0, ny, nx).cpu()
                             for a, (z0, z1) in zip(lam_s, ranges)], dim=1)
        got_gF = torch.cat([a.cpu() for a in gF_s], dim=1)
        assert torch.equal(got_lam, ref_lam)
        assert torch.equal(got_gF, ref_gF)
    for lat in lats:
        lat.check()
        lat.close()


def _adjoint_rank_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    nx, ny, nz, K = 20, 12, 10, 5
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 41)
    gu = synthetic.gaussian_force(shape, 1e-2, seed=43)
    z0, nzl, bits = slabs.slab_of(nz, rank, world, periodic_z=True)
    lat = Lattice(nx, ny, nzl, 0.04, walls=2, device=dev(), slab=bits, z0=z0, **RATES)
    Fs = t(np.ascontiguousarray(F[:, z0:z0 + nzl]))
    lat.set_force_field(Fs)
    lat.init_equilibrium(None, t(np.ascontiguousarray(u0[:, z0:z0 + nzl])))
    states = [lat.export_state().clone()]
    for _ in range(K):
        lat.slab_step()
        slabs.exchange_faces(lat, rank, world, dist, host=True)
        states.append(lat.export_state().clone())
    lam, lam2 = lat.empty_lam(), lat.empty_lam()
    gF = torch.zeros((3, nzl, ny, nx), device=dev())
    lat.adjoint_seed(t(np.ascontiguousarray(gu[:, z0:z0 + nzl])), lam, gF, state=states[K])
    slabs.exchange_adjoint_faces(lat, lam, rank, world, dist, host=True)
    for k in range(K - 1, -1, -1):
        lat.adjoint_step(states[k], lam, lam2, gF)
        slabs.exchange_adjoint_faces(lat, lam2, rank, world, dist, host=True)
        lam, lam2 = lam2, lam
    torch.save((lam[:19 * nzl * ny * nx].view(19, nzl, ny, nx).cpu(), gF.cpu()), f"{out_path}.{rank}")
    lat.check()
    lat.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_processes_adjoint_matches_the_undivided_lattice(tmp_path):
    """The slab adjoint across two rank processes on the one GPU, forward and
    adjoint faces exchanged over gloo through host memory: lambda^0 and dL/dF
    equal the undivided lattice's bit for bit."""
    out = str(tmp_path / "adj")
    mp.start_processes(_adjoint_rank_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn",
                       join=True)
    parts = [torch.load(f"{out}.{r}") for r in range(2)]
    got_lam = torch.cat([p[0] for p in parts], dim=1)
    got_gF = torch.cat([p[1] for p in parts], dim=1)
    nx, ny, nz, K = 20, 12, 10, 5
    shape = (nz, ny, nx)
    u0, F = _inputs(shape, 41)
    gu = synthetic.gaussian_force(shape, 1e-2, seed=43)
    g = Lattice(nx, ny, nz, 0.04, walls=2, device=dev(), **RATES)
    g.set_force_field(t(F))
    g.init_equilibrium(None, t(u0))
    states = [g.export_state().clone()]
    for _ in range(K):
        g.step(1)
        states.append(g.export_state().clone())
    lam, lam2 = g.empty_lam(), g.empty_lam()
    gF = torch.zeros((3,) + shape, device=dev())
    g.adjoint_seed(t(gu), lam, gF, state=states[K])
    for k in range(K - 1, -1, -1):
        g.adjoint_step(states[k], lam, lam2, gF)
        lam, lam2 = lam2, lam
    assert torch.equal(got_lam, lam.view(19, nz, ny, nx).cpu())
    assert torch.equal(got_gF, gF.cpu())
    g.close()
