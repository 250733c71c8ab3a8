"""ctypes declarations of the C ABI in include/clbm.h (argument marshalling only).

Loading fails loudly when libclbm.so has not been built: there is no CPU or
PyTorch fallback for any step of the method.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libclbm.so")
# The bounds-checked debug build of the same library (builder.build(bounds_check=True)).
LIB_BC_PATH = os.path.join(PKG, "libclbm_bc.so")

CLBM_OK = 0
CLBM_ERR_ARG = -1
CLBM_ERR_OOM = -2
CLBM_ERR_CUDA = -3
CLBM_ERR_UNSTABLE = -4
CLBM_ERR_STATE = -5
CLBM_ERR_TIMEOUT = -6
CLBM_ERR_BOUNDS = -7

STORAGE = {"f32": 0, "f16": 1, "bf16": 2, "f16sr": 3, "bf16sr": 4}
PATTERN = {"ab": 0, "aa": 1}
MODEL = {"cascaded": 0, "srt": 1, "mrt": 2}
WALL_X, WALL_Y, WALL_Z = 1, 2, 4
SLAB_LO, SLAB_HI = 1, 2
SLAB_ALL, SLAB_FACES, SLAB_INTERIOR = 0, 1, 2
INJECT_DROP_COPY = 1


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("walls", ctypes.c_uint32), ("nu", ctypes.c_double), ("s2b", ctypes.c_double),
                ("s3", ctypes.c_double), ("s4", ctypes.c_double), ("storage", ctypes.c_int32),
                ("block_x", ctypes.c_int32), ("block_y", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("lattice", ctypes.c_int32), ("pattern", ctypes.c_int32), ("s3b", ctypes.c_double),
                ("s4b", ctypes.c_double), ("s5", ctypes.c_double), ("s6", ctypes.c_double),
                ("model", ctypes.c_int32), ("slab", ctypes.c_int32), ("z0", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("wait_cycles", ctypes.c_int64), ("inject", ctypes.c_int32),
                ("reserved2", ctypes.c_int32)]


class Domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("walls", ctypes.c_uint32), ("nu", ctypes.c_double), ("s2b", ctypes.c_double),
                ("s3", ctypes.c_double), ("s4", ctypes.c_double), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("fz", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("ndomains", ctypes.c_int32), ("ntiles", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("total_nodes", ctypes.c_int64), ("state_bytes", ctypes.c_int64), ("steps_done", ctypes.c_int64),
                ("pattern", ctypes.c_int32), ("buffers", ctypes.c_int32)]


BATCH_GRAPH, BATCH_DIRECT, BATCH_PER_DOMAIN = 0, 1, 2


class Info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("pop_stride", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("storage", ctypes.c_int32), ("block_x", ctypes.c_int32),
                ("block_y", ctypes.c_int32), ("s2", ctypes.c_double), ("nodes_per_thread", ctypes.c_int32),
                ("q", ctypes.c_int32), ("pattern", ctypes.c_int32), ("buffers", ctypes.c_int32),
                ("model", ctypes.c_int32), ("staged", ctypes.c_int32), ("slab", ctypes.c_int32),
                ("face_bytes", ctypes.c_int64)]


P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double

# name -> argument types; every function returns int unless listed in _STR
SIGNATURES = {
    "clbm_create": [ctypes.POINTER(Params), P, ctypes.POINTER(P)],
    "clbm_destroy": [P],
    "clbm_get_info": [P, ctypes.POINTER(Info)],
    "clbm_set_force_uniform": [P, D, D, D],
    "clbm_set_force_profile_z": [P, P],
    "clbm_set_force_field": [P, P],
    "clbm_set_force_decay": [P, D],
    "clbm_init_equilibrium": [P, P, P],
    "clbm_step": [P, I64],
    "clbm_get_macros": [P, P, P],
    "clbm_get_populations": [P, P, I32],
    "clbm_set_populations": [P, P, I32],
    "clbm_reduce_moments": [P, P],
    "clbm_reduce_pair": [P, P, P, I64, P],
    "clbm_check": [P, I32],
    "clbm_export_state": [P, P],
    "clbm_import_state": [P, P, I64],
    "clbm_save_state": [P, P, ctypes.POINTER(ctypes.c_size_t)],
    "clbm_load_state": [P, P, ctypes.c_size_t],
    "clbm_run_host": [P, P, P, I64, P, P, P],
    "clbm_step_raw": [P, P, P],
    "clbm_adjoint_seed": [P, P, P, P, P],
    "clbm_adjoint_step": [P, P, P, P, P],
    "clbm_adjoint_segment": [P, P, P, I64, P, P, P],
    "clbm_reduce_pair_noalloc": [P, P, I64, P, P],
    "clbm_slab_step": [P, I32],
    "clbm_slab_faces": [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64)],
    "clbm_batch_create": [P, I32, I32, P, ctypes.POINTER(P)],
    "clbm_batch_create_pattern": [P, I32, I32, I32, P, ctypes.POINTER(P)],
    "clbm_batch_destroy": [P],
    "clbm_batch_get_info": [P, P],
    "clbm_batch_set_tile": [P, I32],
    "clbm_batch_autotune": [P, I32, ctypes.POINTER(ctypes.c_int32)],
    "clbm_batch_init_equilibrium": [P],
    "clbm_batch_step": [P, I64, I32],
    "clbm_batch_get_macros": [P, I32, P, P],
    "clbm_batch_get_populations": [P, I32, P, I32],
    "clbm_batch_set_populations": [P, I32, P, I32],
    "clbm_batch_check": [P, I32],
    "clbm_status_string": [I32],
    "clbm_last_error": [],
}
_STR = {"clbm_status_string", "clbm_last_error"}

_lib = None


def lib():
    """Load libclbm.so (built by __graft_entry__.build() or builder.build()),
    or, when the environment variable CLBM_LIBRARY=bounds_check is set, its
    bounds-checked debug build libclbm_bc.so."""
    global _lib
    if _lib is None:
        path = LIB_BC_PATH if os.environ.get("CLBM_LIBRARY") == "bounds_check" else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1801_04586_gb300.builder.build() "
                               "(nvcc, sm_103a); there is no fallback implementation")
        L = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name in _STR else ctypes.c_int
        _lib = L
    return _lib


class CLBMError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        msg = L.clbm_last_error().decode() or L.clbm_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


class UnstableError(CLBMError):
    pass


def check(code: int, where: str) -> None:
    if code != CLBM_OK:
        if code == CLBM_ERR_UNSTABLE:
            raise UnstableError(code, where)
        raise CLBMError(code, where)
