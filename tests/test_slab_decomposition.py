"""A z-slab decomposition of one periodic-in-z lattice over 2 CPU ranks (gloo):
each rank steps its slab extended by ghost planes received from its
neighbours, with the FP64 oracle as the local solver; the gathered result must
equal the undivided oracle run bit for bit."""
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
