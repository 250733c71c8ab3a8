"""Failure detection of the staged step without a GPU fault. The host withholds
the bulk copies of the first tile (clbm_params.inject = CLBM_INJECT_DROP_COPY):
its barrier is armed with the tile's byte count but no copy is issued, so the
waits on it cannot complete and run out after wait_cycles (about 1 ms here).
The kernel must give up and return on its own (each block first waiting,
bounded, for the copies it did issue), clbm_check must report
CLBM_ERR_TIMEOUT, and the device must go on working: the same process then
runs a normal staged step that matches the one-node-per-thread step bit for
bit. No copy fails, nothing faults and no wait is endless."""
import pytest
import torch

from gpu_common import dev, t
from paper_1801_04586_gb300 import CLBMError, Lattice, _capi, synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,pattern,steps", [("f16", "ab", 1), ("bf16sr", "ab", 1), ("f16", "aa", 1),
                                                    ("f16sr", "aa", 2)])
def test_wait_that_runs_out_reports_timeout_and_the_device_recovers(storage, pattern, steps):
    """A/B and both in-place kinds (steps = 2: the even then the odd kind,
    each with its first tile's copies withheld)."""
    nx, ny, nz = 64, 48, 24
    u0 = t(synthetic.divfree_velocity((nz, ny, nx), seed=17, umax=0.02))
    lat = Lattice(nx, ny, nz, 0.05, storage=storage, pattern=pattern, device=dev(), wait_cycles=2_000_000,
                  inject=_capi.INJECT_DROP_COPY)
    assert lat.info()["staged"] == 1
    lat.init_equilibrium(None, u0)
    for _ in range(steps):
        lat.step(1)
    torch.cuda.synchronize()  # the kernel returned by itself
    with pytest.raises(CLBMError) as err:
        lat.check(clear=True)
    assert err.value.code == _capi.CLBM_ERR_TIMEOUT
    lat.check()  # cleared
    lat.close()
    outs = []
    for variant in (0, 1):
        g = Lattice(nx, ny, nz, 0.05, storage=storage, device=dev(), variant=variant)
        assert g.info()["staged"] == (1 if variant == 0 else 0)
        g.init_equilibrium(None, u0)
        g.step(5)
        g.check()
        outs.append(g.populations(deviation=True).cpu())
        g.close()
    assert torch.equal(outs[0], outs[1])
