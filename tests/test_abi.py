"""CPU checks of the C-ABI boundary: the built library exports every entry
point that include/clbm.h declares, the binding declares them all, and host
argument validation rejects bad input before any CUDA call."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "clbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(clbm_[a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build libclbm.so")
    from paper_1801_04586_gb300 import _capi
    from paper_1801_04586_gb300.builder import build
    build()
    return _capi.lib()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for must in ("clbm_create", "clbm_destroy", "clbm_step", "clbm_init_equilibrium", "clbm_get_macros",
                 "clbm_set_force_field", "clbm_set_force_uniform", "clbm_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1801_04586_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == declared_functions()


def _params(**kw):
    from paper_1801_04586_gb300 import _capi
    base = dict(nx=8, ny=8, nz=8, walls=0, nu=0.1, s2b=1.0, s3=1.0, s4=1.0, storage=0, block_x=0, block_y=0,
                variant=0, lattice=0, pattern=0, s3b=0.0, s4b=0.0, s5=0.0, s6=0.0, model=0,
                slab=0, z0=0, reserved=0, wait_cycles=0, inject=0, reserved2=0)
    base.update(kw)
    return _capi.Params(**base)


@pytest.mark.parametrize("kw", [dict(nx=0), dict(ny=-3), dict(nz=70000), dict(walls=8), dict(nu=0.0),
                                dict(nu=-1.0), dict(s2b=2.0), dict(s3=0.0), dict(s4=float("nan")),
                                dict(storage=5), dict(block_x=48), dict(block_x=1024, block_y=1),
                                dict(nx=2048, ny=2048, nz=1024), dict(variant=3),
                                dict(lattice=21), dict(lattice=27, s5=2.5), dict(lattice=27, variant=2),
                                dict(lattice=27, block_x=512, block_y=1), dict(pattern=2),
                                dict(pattern=-1), dict(pattern=1, variant=2), dict(model=3), dict(model=-1),
                                dict(reserved=1), dict(model=2, variant=2), dict(slab=4), dict(slab=1, lattice=27),
                                dict(slab=2, model=1), dict(slab=3, pattern=1), dict(slab=1, variant=2),
                                dict(z0=5), dict(slab=1, z0=-1),
                                dict(slab=3, nx=1024, ny=1024, nz=8, z0=2100), dict(wait_cycles=-1),
                                dict(inject=2), dict(reserved2=1)])
def test_create_rejects_bad_parameters(lib, kw):
    from paper_1801_04586_gb300 import _capi
    h = ctypes.c_void_p()
    p = _params(**kw)
    assert lib.clbm_create(ctypes.byref(p), None, ctypes.byref(h)) == _capi.CLBM_ERR_ARG
    assert not h.value
    assert lib.clbm_last_error().decode().startswith("clbm_create")


def test_null_pointers_rejected(lib):
    from paper_1801_04586_gb300 import _capi
    h = ctypes.c_void_p()
    assert lib.clbm_create(None, None, ctypes.byref(h)) == _capi.CLBM_ERR_ARG
    assert lib.clbm_step(None, 1) == _capi.CLBM_ERR_ARG
    assert lib.clbm_get_macros(None, None, None) == _capi.CLBM_ERR_ARG
    assert lib.clbm_destroy(None) == _capi.CLBM_OK
    assert lib.clbm_slab_step(None, 0) == _capi.CLBM_ERR_ARG
    assert lib.clbm_slab_faces(None, None, None, None) == _capi.CLBM_ERR_ARG
    assert lib.clbm_status_string(_capi.CLBM_ERR_UNSTABLE).decode().startswith("unstable")
    assert lib.clbm_status_string(_capi.CLBM_ERR_TIMEOUT).decode().startswith("timeout")
