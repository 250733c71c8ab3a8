"""Batched multi-domain stepping: each domain of a batch must evolve exactly as
the same lattice stepped alone (same per-node arithmetic), in every step mode
and block shape, and match the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import F32_REL_TOL, W, dev, make_pair, rel_err
from paper_1801_04586_gb300 import Batch, synthetic

pytestmark = pytest.mark.gpu

DOMAINS = [
    dict(nx=40, ny=20, nz=12, walls=4, nu=0.05, fx=1e-5),
    dict(nx=33, ny=17, nz=9, walls=6, nu=0.02, s2b=1.2, s3=1.1, fx=3e-6, fy=1e-6),
    dict(nx=150, ny=5, nz=4, walls=0, nu=0.1, s4=0.8, fx=-2e-6, fz=4e-6),
    dict(nx=20, ny=24, nz=31, walls=6, nu=0.008, fx=5e-6),
    dict(nx=1, ny=7, nz=40, walls=4, nu=0.03, fx=2e-6),
]


def _single(d, steps, storage="f32"):
    g, _ = make_pair(d["nx"], d["ny"], d["nz"], d["nu"], walls=d.get("walls", 0), s2b=d.get("s2b", 1.0),
                     s3=d.get("s3", 1.0), s4=d.get("s4", 1.0), storage=storage)
    g.set_force_uniform(d.get("fx", 0.0), d.get("fy", 0.0), d.get("fz", 0.0))
    g.init_equilibrium()
    g.step(steps)
    out = g.populations(deviation=True).cpu()
    g.close()
    return out


@pytest.mark.parametrize("mode", [Batch.GRAPH, Batch.DIRECT, Batch.PER_DOMAIN])
def test_batch_domains_match_single_lattices(mode):
    steps = 37  # two graph replays of 16 steps plus 5 direct launches in graph mode
    b = Batch(DOMAINS, device=dev())
    b.init_equilibrium()
    b.step(steps, mode)
    b.check()
    assert b.info()["steps_done"] == steps
    for k, d in enumerate(DOMAINS):
        assert torch.equal(b.populations(k, deviation=True).cpu(), _single(d, steps)), f"domain {k}"
    b.close()


@pytest.mark.parametrize("threads", [32, 96, 256, 512])
def test_batch_tile_size_bit_identical(threads):
    b = Batch(DOMAINS, device=dev())
    b.set_tile(threads)
    b.init_equilibrium()
    b.step(20, Batch.GRAPH)
    for k, d in enumerate(DOMAINS):
        assert torch.equal(b.populations(k, deviation=True).cpu(), _single(d, 20)), f"domain {k}"
    b.close()


def test_autotune_keeps_state_and_picks_a_candidate():
    b = Batch(DOMAINS, device=dev())
    b.init_equilibrium()
    b.step(7, Batch.DIRECT)
    before = [b.populations(k, deviation=True).cpu() for k in range(len(DOMAINS))]
    threads = b.autotune(trial_steps=3)
    assert threads in {64, 128, 192, 256, 384, 512}
    assert b.info()["threads"] == threads
    for k in range(len(DOMAINS)):
        assert torch.equal(b.populations(k, deviation=True).cpu(), before[k])
    b.step(30, Batch.GRAPH)
    for k, d in enumerate(DOMAINS):
        assert torch.equal(b.populations(k, deviation=True).cpu(), _single(d, 37)), f"domain {k}"
    b.close()


def test_batch_against_oracle():
    doms = DOMAINS[:2]
    b = Batch(doms, device=dev())
    b.init_equilibrium()
    b.step(50, Batch.GRAPH)
    for k, d in enumerate(doms):
        shape = (d["nz"], d["ny"], d["nx"])
        o = oracle.Lattice(d["nx"], d["ny"], d["nz"], walls=d["walls"], s2=1.0 / (3 * d["nu"] + 0.5),
                           s2b=d.get("s2b", 1.0), s3=d.get("s3", 1.0), s4=d.get("s4", 1.0))
        F = np.zeros((3,) + shape)
        F[0], F[1], F[2] = d.get("fx", 0.0), d.get("fy", 0.0), d.get("fz", 0.0)
        F = F.astype(np.float32).astype(np.float64)
        fo = oracle.step(o, oracle.init(o, None, None, F), F, 50)
        fg = b.populations(k, deviation=True).double().cpu().numpy() + W
        assert rel_err(fg, fo) < F32_REL_TOL
    b.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_batch_16bit_storage_matches_single_lattices(storage):
    """FP16/BF16 deviation storage in a batch: the same stored bits as each
    lattice stepped alone in that format."""
    b = Batch(DOMAINS, storage=storage, device=dev())
    b.init_equilibrium()
    b.step(21, Batch.GRAPH)
    b.check()
    for k, d in enumerate(DOMAINS):
        assert torch.equal(b.populations(k, deviation=True).cpu(), _single(d, 21, storage)), f"domain {k}"
    b.close()


def test_batch_64_domains_full_size_sampled():
    """The benchmark's batch at full size (64 channels/ducts, sides U{32..128},
    seed 6: 32.4M nodes), autotuned as the benchmark does, one step through
    the graph-mode call: in six domains (the largest, the smallest, the first
    duct and channel, two more), 512 sampled nodes against the FP64 oracle's
    first step, and the whole domain bit-identical to the lattice stepped
    alone."""
    doms = synthetic.batch_domains(64, seed=6)
    b = Batch(doms, device=dev())
    b.init_equilibrium()
    b.autotune(trial_steps=3)
    b.step(1, Batch.GRAPH)
    b.check()
    sizes = [d["nx"] * d["ny"] * d["nz"] for d in doms]
    pick = [int(np.argmax(sizes)), int(np.argmin(sizes)), next(k for k, d in enumerate(doms) if d["walls"] == 6),
            next(k for k, d in enumerate(doms) if d["walls"] == 4), 17, 42]
    rng = np.random.default_rng(11)
    for k in dict.fromkeys(pick):
        d = doms[k]
        shape = (d["nz"], d["ny"], d["nx"])
        n = sizes[k]
        fg = b.populations(k, deviation=True)
        assert torch.equal(fg.cpu(), _single(d, 1)), f"domain {k}"
        o = oracle.Lattice(d["nx"], d["ny"], d["nz"], walls=d["walls"], s2=1.0 / (3 * d["nu"] + 0.5))
        F = np.zeros((3,) + shape)
        F[0] = np.float32(d["fx"])
        nodes = rng.choice(n, min(512, n), replace=False)
        fo = oracle.first_step_nodes(o, nodes, None, None, F)
        hg = fg.reshape(19, -1)[:, torch.from_numpy(nodes).to(dev())].double().cpu().numpy().T
        err = np.max(np.abs(hg + W.reshape(1, 19) - fo) / np.abs(fo))
        assert err < 1e-6, (k, err)
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", [Batch.GRAPH, Batch.DIRECT, Batch.PER_DOMAIN])
def test_batch_in_place_matches_ab(storage, mode):
    """The in-place (AA) pattern over a batch: one buffer instead of two, and
    after odd and even step counts (graph replays starting at either parity)
    every domain's state, velocity and density equal the A/B batch's bit for
    bit."""
    ab = Batch(DOMAINS, storage=storage, device=dev())
    aa = Batch(DOMAINS, storage=storage, device=dev(), pattern="aa")
    ia, ib = aa.info(), ab.info()
    assert (ia["pattern"], ia["buffers"], ib["pattern"], ib["buffers"]) == (1, 1, 0, 2)
    assert ia["state_bytes"] == ib["state_bytes"]
    for g in (ab, aa):
        g.init_equilibrium()
    done = 0
    for n in (1, 1, 17, 18):  # odd and even counts; 17 and 18 steps start graph replays at both parities
        for g in (ab, aa):
            g.step(n, mode)
        done += n
        for k in range(len(DOMAINS)):
            assert torch.equal(aa.populations(k, deviation=True), ab.populations(k, deviation=True)), (done, k)
            ra, ua = aa.macros(k)
            rb, ub = ab.macros(k)
            assert torch.equal(ra, rb) and torch.equal(ua, ub)
    aa.check()
    ab.close()
    aa.close()


def test_batch_in_place_autotune_keeps_state():
    """Autotuning an in-place batch steps a copy of its state: the state and
    the step count are unchanged, and later steps still equal the A/B batch."""
    ab = Batch(DOMAINS, device=dev())
    aa = Batch(DOMAINS, device=dev(), pattern="aa")
    for g in (ab, aa):
        g.init_equilibrium()
        g.step(7, Batch.DIRECT)
    before = [aa.populations(k, deviation=True).cpu() for k in range(len(DOMAINS))]
    threads = aa.autotune(trial_steps=3)
    assert aa.info()["threads"] == threads and aa.info()["steps_done"] == 7
    for k in range(len(DOMAINS)):
        assert torch.equal(aa.populations(k, deviation=True).cpu(), before[k])
    for g in (ab, aa):
        g.step(30, Batch.GRAPH)
    for k in range(len(DOMAINS)):
        assert torch.equal(aa.populations(k, deviation=True), ab.populations(k, deviation=True))
    aa.check()
    ab.close()
    aa.close()
