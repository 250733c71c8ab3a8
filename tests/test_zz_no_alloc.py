"""clbm_reduce_pair_noalloc, the allocation-free FP64 pair reduction for
callers that cannot call cudaMalloc (allocation can synchronise the device
and can fail with out-of-memory): called through the C ABI, it must give
clbm_reduce_pair's sums, twice in a row on the shared static scratch, and
reject sizes beyond its fixed scratch with a clear error. Kept in its own
file, collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1801_04586_gb300 import Lattice, _capi

pytestmark = pytest.mark.gpu

MAX_N = 8192 * 16384


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_context_reduction_twice():
    lib = _capi.lib()
    dev = torch.device("cuda", 0)
    lat = Lattice(8, 8, 8, 0.1, device=dev)
    stream = ctypes.c_void_p(lat.stream.cuda_stream)
    rng = np.random.default_rng(2026)
    # a large call, then a smaller one: the second must not see the first's partials
    for n in (3 * 96 ** 3 + 5, 70_001):
        a = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
        b = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
        ref = lat.reduce_pair(a, b)
        out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.clbm_reduce_pair_noalloc(_p(a), _p(b), n, _p(out), stream)
        assert rc == _capi.CLBM_OK, lib.clbm_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12)
    out0 = torch.empty(3, dtype=torch.float64, device=dev)
    assert lib.clbm_reduce_pair_noalloc(_p(a), None, n, _p(out0), stream) == _capi.CLBM_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(out0[0].item(), lat.reduce_pair(a)[0].item(), rtol=1e-12)
    lat.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _capi.lib()
    dev = torch.device("cuda", 0)
    a = torch.zeros(4, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    rc = lib.clbm_reduce_pair_noalloc(_p(a), None, MAX_N + 1, _p(out), None)
    assert rc == _capi.CLBM_ERR_ARG
    assert b"134217728" in lib.clbm_last_error()
    assert lib.clbm_reduce_pair_noalloc(_p(a), None, -1, _p(out), None) == _capi.CLBM_ERR_ARG
