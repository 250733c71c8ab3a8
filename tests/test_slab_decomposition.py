"""The z-slab decomposition's host side on CPU ranks (gloo): the partition and
neighbour bookkeeping; the face exchange that the library's slab lattices use
(slabs.exchange_faces) routing every face to the right neighbour and slot, for
2 and 3 ranks, periodic and walled z, over host-staged and batched
point-to-point calls; and one periodic-in-z lattice stepped on 2 ranks, each
its slab extended by ghost planes from its neighbours, with the FP64 oracle
as the local solver, equal to the undivided oracle run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1801_04586_gb300 import slabs, synthetic

NX, NY, NZ, STEPS, WALLS = 6, 5, 9, 6, 3


def _lattice(nz):
    return oracle.Lattice(NX, NY, nz, walls=WALLS, s2=1.6, s2b=1.1, s3=1.2, s4=0.9)


def _inputs():
    shape = (NZ, NY, NX)
    rho = synthetic.density_perturbation(shape, 0.01, seed=101)
    u = synthetic.uniform_perturbation(shape, 0.03, seed=102)
    F = synthetic.gaussian_force(shape, 1e-4, seed=103)
    return rho, u, F


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rho, u, F = _inputs()
    f_global = oracle.init(_lattice(NZ), rho, u, F)
    z0, z1 = slabs.partition(NZ, world)[rank]
    local = torch.from_numpy(np.ascontiguousarray(f_global[:, z0:z1]))
    F_ext = np.concatenate([F[:, [(z0 - 1) % NZ]], F[:, z0:z1], F[:, [z1 % NZ]]], axis=1)
    ext_lat = _lattice(z1 - z0 + 2)
    for _ in range(STEPS):
        below, above = slabs.exchange_planes(local, rank, world, dist)
        ext = torch.cat([below[:, None], local, above[:, None]], dim=1).numpy()
        ext = oracle.step(ext_lat, ext, F_ext, 1)
        local = torch.from_numpy(np.ascontiguousarray(ext[:, 1:-1]))
    parts = [torch.empty(19, b - a, NY, NX, dtype=torch.float64) for a, b in slabs.partition(NZ, world)]
    if rank == 0:
        parts[0] = local
        for r in range(1, world):
            dist.recv(parts[r], r)
        np.save(out_path, torch.cat(parts, dim=1).numpy())
    else:
        dist.send(local, 0)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_and_neighbours():
    assert slabs.partition(9, 2) == [(0, 5), (5, 9)]
    assert slabs.partition(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    assert slabs.neighbours(0, 3) == (2, 1)
    with pytest.raises(ValueError):
        slabs.partition(2, 3)
    assert len(slabs.Z_PLUS) == len(slabs.Z_MINUS) == 5


def test_two_rank_slabs_match_single_domain(tmp_path):
    out = str(tmp_path / "slabs.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    rho, u, F = _inputs()
    lat = _lattice(NZ)
    ref = oracle.step(lat, oracle.init(lat, rho, u, F), F, STEPS)
    np.testing.assert_array_equal(np.load(out), ref)


class _FakeSlab:
    """Stands in for a library slab lattice: send planes filled with a
    pattern naming (rank, half, byte), receive planes zeroed."""

    def __init__(self, rank, bits, half):
        self.slab = bits
        self.stream = None
        i = torch.arange(half, dtype=torch.int64)
        self.send = torch.cat([(rank * 40 + 7 + i * 3) % 251, (rank * 40 + 19 + i * 5) % 251]).to(torch.uint8)
        self.recv = torch.zeros(2 * half, dtype=torch.uint8)

    def faces(self):
        return self.send, self.recv


def _exchange_worker(rank, world, port, periodic, host, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    half = 37
    _, _, bits = slabs.slab_of(3 * world, rank, world, periodic_z=periodic)
    lat = _FakeSlab(rank, bits, half)
    slabs.exchange_faces(lat, rank, world, dist, host=host)
    torch.save({"send": lat.send, "recv": lat.recv, "bits": bits}, f"{out_path}.{rank}")
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic,host", [(2, True, True), (3, True, True), (3, False, True),
                                                 (2, True, False), (3, False, False)])
def test_face_exchange_routes_every_face(tmp_path, world, periodic, host):
    """After exchange_faces, each rank's first receive half holds its lower
    neighbour's upper send half and its second receive half its upper
    neighbour's lower send half; receive halves at wall faces stay untouched."""
    out = str(tmp_path / "faces")
    mp.start_processes(_exchange_worker, args=(world, _free_port(), periodic, host, out), nprocs=world,
                       start_method="spawn", join=True)
    got = [torch.load(f"{out}.{r}") for r in range(world)]
    for r in range(world):
        lo, hi = slabs.neighbours(r, world)
        half = got[r]["send"].numel() // 2
        bits = got[r]["bits"]
        if bits & slabs.SLAB_LO:
            assert torch.equal(got[r]["recv"][:half], got[lo]["send"][half:])
        else:
            assert not periodic and r == 0 and torch.count_nonzero(got[r]["recv"][:half]) == 0
        if bits & slabs.SLAB_HI:
            assert torch.equal(got[r]["recv"][half:], got[hi]["send"][:half])
        else:
            assert not periodic and r == world - 1 and torch.count_nonzero(got[r]["recv"][half:]) == 0


def test_single_slab_is_its_own_neighbour():
    lat = _FakeSlab(0, slabs.SLAB_LO | slabs.SLAB_HI, 5)
    slabs.exchange_faces(lat, 0, 1)
    assert torch.equal(lat.recv[:5], lat.send[5:]) and torch.equal(lat.recv[5:], lat.send[:5])


def test_slab_of_partitions_and_flags_faces():
    assert slabs.slab_of(10, 0, 3) == (0, 4, 3)
    assert slabs.slab_of(10, 1, 3, periodic_z=False) == (4, 3, 3)
    assert slabs.slab_of(10, 2, 3, periodic_z=False) == (7, 3, 1)
    assert slabs.slab_of(10, 0, 3, periodic_z=False) == (0, 4, 2)
    assert slabs.slab_of(5, 0, 1, periodic_z=False) == (0, 5, 0)


class _FakeSums:
    """Stands in for a slab lattice's FP64 reductions (rank-dependent values)."""

    def __init__(self, rank):
        self.rank = rank

    def reduce_moments(self):
        return torch.tensor([1.0 + self.rank, 0.5 * self.rank, -2.0 ** -40 * self.rank, 3.0], dtype=torch.float64)

    def reduce_pair(self, a, b=None):
        d = (a - b) if b is not None else a
        return torch.stack([(d.double() ** 2).sum(), (b.double() ** 2).sum() if b is not None else
                            torch.zeros((), dtype=torch.float64), (a.double() * b.double()).sum()
                            if b is not None else torch.zeros((), dtype=torch.float64)])


def _sums_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lat = _FakeSums(rank)
    a = torch.arange(6, dtype=torch.float32) + rank
    b = torch.ones(6, dtype=torch.float32) * (rank - 1)
    torch.save((slabs.global_moments(lat, dist), slabs.global_pair(lat, a, b, dist)), f"{out_path}.{rank}")
    dist.barrier()
    dist.destroy_process_group()


def test_global_sums_add_every_rank(tmp_path):
    """The FP64 all-reduce behind the global mass/momentum and error norms of
    a slab decomposition (gloo, 3 ranks): every rank ends with the sum of all
    ranks' values; without a process group the slab's own values come back."""
    world = 3
    out = str(tmp_path / "sums")
    mp.start_processes(_sums_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                       join=True)
    want_m = sum(_FakeSums(r).reduce_moments() for r in range(world))
    want_p = sum(_FakeSums(r).reduce_pair(torch.arange(6, dtype=torch.float32) + r,
                                         torch.ones(6, dtype=torch.float32) * (r - 1)) for r in range(world))
    for r in range(world):
        m, pr = torch.load(f"{out}.{r}")
        assert torch.equal(m, want_m)
        assert torch.allclose(pr, want_p, rtol=0, atol=0)
    assert torch.equal(slabs.global_moments(_FakeSums(2)), _FakeSums(2).reduce_moments())
