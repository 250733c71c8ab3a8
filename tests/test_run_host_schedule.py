"""The launch order of a D3Q19 host job with per-step sums (clbm_run_host in
csrc/capi.cu), replayed on the host.

The job uploads rho and u in up to 8 chunks of z-planes, initialises each
chunk as it lands, runs step 0 of each chunk right after its initialisation,
step 1 of chunk k after step 0 of chunk k + 1 (the two end chunks after the
last), whole steps in between, and the last step chunk by chunk, reading out
chunk k after the last step of chunk k + 1 (the end chunks last). The model
below issues the same order on a one-dimensional periodic lattice whose
populations move by e_z in {-1, 0, +1}, with the A/B buffer pair and the
slot conventions of the library:

- initialisation of node x writes slot (i, x - e_i) of the first buffer,
- a step at node x pulls slot (i, x - e_i) of its source buffer and writes
  slots (i, x) of the other buffer (Eq. 8 streaming as a pull),
- the read-out of node x pulls like a step.

Every pull must see the value its node needs: the initialisation of x for
step 0, step t - 1 of node x - e_i otherwise. A write-after-read hazard shows
up as a pull that sees a newer value. The order is kept in step with capi.cu
by hand; planted mistakes in the model (an early read-out, an early step 1)
must fail."""
import pytest

EZ = (-1, 0, 1)
IO_CHUNKS = 8


def job_order(nz, nsteps, outputs, early_readout=False, early_step1=False):
    """The kernels of one job in stream order: ("init", k), ("step", t, k), ("read", k)."""
    nch = min(nz, IO_CHUNKS)
    first_split = nsteps > 0
    second_split = first_split and nsteps >= 3 and nch >= 3
    last_split = nsteps > 1 and outputs
    ops = []
    for k in range(nch):
        ops.append(("init", k))
        if first_split:
            ops.append(("step", 0, k))
        if second_split and k >= (1 if early_step1 else 2):
            ops.append(("step", 1, k - 1))
    if second_split:
        ops += [("step", 1, 0), ("step", 1, nch - 1)]
    for t in range(nsteps):
        if t == nsteps - 1 and last_split:
            for k in range(nch):
                ops.append(("step", t, k))
                if early_readout:
                    ops.append(("read", k))
                elif nch >= 3 and k >= 2:
                    ops.append(("read", k - 1))
            if not early_readout:
                ops += [("read", k) for k in range(nch) if nch < 3 or k in (0, nch - 1)]
        elif not (t == 0 and first_split) and not (t == 1 and second_split):
            ops += [("step", t, k) for k in range(nch)]
    if outputs and not last_split:
        ops += [("read", k) for k in range(nch)]
    return ops


def replay(nz, nsteps, ops):
    nch = min(nz, IO_CHUNKS)
    chunks = [range(nz * k // nch, nz * (k + 1) // nch) for k in range(nch)]
    buf = [dict(), dict()]

    def pull(b, x, t):
        for e in EZ:
            want = ("init", x) if t == 0 else (t - 1, (x - e) % nz)
            got = b.get((e, (x - e) % nz))
            if got != want:
                raise AssertionError(f"node {x}, e_z {e}: saw {got}, needs {want}")

    stepped = set()
    for op in ops:
        if op[0] == "init":
            for x in chunks[op[1]]:
                for e in EZ:
                    buf[0][(e, (x - e) % nz)] = ("init", x)
        elif op[0] == "step":
            t, k = op[1], op[2]
            for x in chunks[k]:
                pull(buf[t & 1], x, t)
            for x in chunks[k]:
                for e in EZ:
                    buf[(t & 1) ^ 1][(e, x)] = (t, x)
            stepped.add((t, k))
        else:
            for x in chunks[op[1]]:
                pull(buf[nsteps & 1], x, nsteps)
    assert stepped == {(t, k) for t in range(nsteps) for k in range(nch)}
    reads = [op[1] for op in ops if op[0] == "read"]
    assert sorted(reads) == (list(range(nch)) if any(op[0] == "read" for op in ops) else [])


@pytest.mark.parametrize("nz", list(range(1, 30)) + [40, 256])
def test_job_order_pulls_the_right_values(nz):
    for nsteps in range(8):
        for outputs in (True, False):
            replay(nz, nsteps, job_order(nz, nsteps, outputs))


@pytest.mark.parametrize("plant", ["early_readout", "early_step1"])
def test_planted_order_mistakes_fail(plant):
    with pytest.raises(AssertionError):
        for nz in (2, 3, 9, 23):
            for nsteps in (2, 3, 5):
                replay(nz, nsteps, job_order(nz, nsteps, True, **{plant: True}))
