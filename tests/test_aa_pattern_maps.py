"""Host-side check of the in-place (AA) pattern's slot maps.

The AA kernels (step.cu, step27.cu) read and write one population buffer:
  even step: read (i, x), write post-collision i to (ibar, x);
  odd step:  read (ibar, x - e_i) [or (i, x) if x - e_i is beyond a wall],
             write post-collision i to (i, x + e_i) [or (ibar, x) if x + e_i is
             beyond a wall].
This test restates those maps in numpy and checks, on small walled and
periodic boxes of both lattices, that (1) each node writes exactly the slots
it reads, (2) the read slots of all nodes cover the buffer once (no two
nodes touch a slot), and (3) with an arbitrary per-node collision the AA
sequence reproduces the two-buffer pull scheme of Eq. 8 (halfway
bounce-back) step for step. No GPU is used.
"""
import itertools

import numpy as np
import pytest

import oracle


def velocity_set(q):
    return oracle.velocities(q).astype(int)  # (q, 3) in the paper's order


def opposite(E):
    return np.array([int(np.where((E == -E[i]).all(axis=1))[0][0]) for i in range(len(E))])


def beyond(c, e, n, walls):
    """Is c - e beyond a wall face on any wall axis? c, e, n in (x, y, z)."""
    return any((walls >> a) & 1 and not (0 <= c[a] - e[a] < n[a]) for a in range(3))


def wrap(c, n):
    return tuple(int(v) % int(m) for v, m in zip(c, n))


def slots(q, n, walls, odd, E, opp):
    """Per node: list of read slots and list of write slots (population order)."""
    reads, writes = {}, {}
    for c in itertools.product(*(range(m) for m in n)):
        r, w = [], []
        for i in range(q):
            if not odd:
                r.append((i, c))
                w.append((opp[i], c))
            else:
                r.append((i, c) if beyond(c, E[i], n, walls) else (opp[i], wrap(np.subtract(c, E[i]), n)))
                w.append((opp[i], c) if beyond(c, -E[i], n, walls) else (i, wrap(np.add(c, E[i]), n)))
        reads[c], writes[c] = r, w
    return reads, writes


CASES = [(19, (3, 4, 2), 0), (19, (4, 3, 3), 7), (19, (1, 3, 4), 4), (19, (5, 1, 2), 3),
         (27, (3, 3, 2), 0), (27, (3, 4, 3), 7), (27, (2, 3, 1), 6)]


@pytest.mark.parametrize("q,n,walls", CASES)
def test_each_node_writes_what_it_reads_and_slots_partition(q, n, walls):
    E = velocity_set(q)
    opp = opposite(E)
    total = q * int(np.prod(n))
    for odd in (False, True):
        reads, writes = slots(q, n, walls, odd, E, opp)
        allr = [s for c in reads for s in reads[c]]
        assert len(set(allr)) == total == len(allr)
        for c in reads:
            assert sorted(reads[c]) == sorted(writes[c])


@pytest.mark.parametrize("q,n,walls", CASES)
def test_aa_sequence_reproduces_pull_streaming(q, n, walls):
    """Any per-node map C (here a random linear mix plus a node-dependent
    offset) applied through the AA slots equals the pull scheme."""
    E = velocity_set(q)
    opp = opposite(E)
    rng = np.random.default_rng(5)
    A = rng.normal(size=(q, q)) / q
    nodes = list(itertools.product(*(range(m) for m in n)))
    bias = {c: rng.normal(size=q) for c in nodes}

    def collide(fv, c):
        return A @ fv + bias[c]

    f0 = {c: rng.normal(size=q) for c in nodes}  # post-streaming state at step 0

    # two-buffer pull: state f(n) -> post-collision g -> f(n+1)_i(x) = g_i(x - e_i) or g_ibar(x)
    f = dict(f0)
    pull_states = []
    for _ in range(5):
        g = {c: collide(f[c], c) for c in nodes}
        f = {c: np.array([g[c][opp[i]] if beyond(c, E[i], n, walls) else g[wrap(np.subtract(c, E[i]), n)][i]
                          for i in range(q)]) for c in nodes}
        pull_states.append(f)

    # AA: one buffer, natural order at step 0
    buf = {(i, c): f0[c][i] for c in nodes for i in range(q)}
    for s in range(5):
        odd = s % 2 == 1
        reads, writes = slots(q, n, walls, odd, E, opp)
        new = dict(buf)
        for c in nodes:
            fv = np.array([buf[sl] for sl in reads[c]])
            post = collide(fv, c)
            for i, sl in enumerate(writes[c]):
                new[sl] = post[i]
        buf = new
        # the state after s+1 steps read back through the map of that parity
        read_odd = (s + 1) % 2 == 1
        rmap, _ = slots(q, n, walls, read_odd, E, opp)
        for c in nodes:
            got = np.array([buf[sl] for sl in rmap[c]])
            np.testing.assert_allclose(got, pull_states[s][c], rtol=0, atol=1e-12)

