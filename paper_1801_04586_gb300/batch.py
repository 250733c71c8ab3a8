"""Python front end of the batched C ABI: many independent D3Q19 lattices of
uneven sizes and parameters stepped with one launch per time step."""
from __future__ import annotations

import ctypes
from typing import List, Optional

import torch

from . import _capi
from ._capi import check


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Batch:
    """domains: list of dicts with nx, ny, nz, walls, nu and optional s2b, s3,
    s4 (default 1) and fx, fy, fz (default 0)."""

    GRAPH, DIRECT, PER_DOMAIN = _capi.BATCH_GRAPH, _capi.BATCH_DIRECT, _capi.BATCH_PER_DOMAIN

    def __init__(self, domains: List[dict], storage: str = "f32", device=None, pattern: str = "ab"):
        """pattern "ab": two population buffers; "aa": one, updated in place by
        alternating even and odd steps (half the memory, the same bits)."""
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the batch runs only in libclbm.so's kernels")
        self.lib = _capi.lib()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = torch.device("cuda", dev.index if dev.index is not None else torch.cuda.current_device())
        arr = (_capi.Domain * len(domains))()
        for k, d in enumerate(domains):
            arr[k] = _capi.Domain(int(d["nx"]), int(d["ny"]), int(d["nz"]), int(d.get("walls", 0)), float(d["nu"]),
                                  float(d.get("s2b", 1.0)), float(d.get("s3", 1.0)), float(d.get("s4", 1.0)),
                                  float(d.get("fx", 0.0)), float(d.get("fy", 0.0)), float(d.get("fz", 0.0)))
        self.domains = [dict(d) for d in domains]
        self.storage = storage
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            check(self.lib.clbm_batch_create_pattern(arr, len(domains), _capi.STORAGE[storage],
                                                     _capi.PATTERN[pattern],
                                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                  "clbm_batch_create_pattern")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.clbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = _capi.BatchInfo()
        check(self.lib.clbm_batch_get_info(self.h, ctypes.byref(i)), "clbm_batch_get_info")
        return {k: getattr(i, k) for k, _ in _capi.BatchInfo._fields_}

    def set_tile(self, threads: int):
        check(self.lib.clbm_batch_set_tile(self.h, int(threads)), "clbm_batch_set_tile")

    def autotune(self, trial_steps: int = 10) -> int:
        """Pick the fastest block size; returns threads per block."""
        t = ctypes.c_int32()
        check(self.lib.clbm_batch_autotune(self.h, int(trial_steps), ctypes.byref(t)), "clbm_batch_autotune")
        return t.value

    def init_equilibrium(self):
        check(self.lib.clbm_batch_init_equilibrium(self.h), "clbm_batch_init_equilibrium")

    def step(self, nsteps: int, mode: int = _capi.BATCH_GRAPH):
        check(self.lib.clbm_batch_step(self.h, int(nsteps), int(mode)), "clbm_batch_step")

    def _shape(self, d):
        dd = self.domains[d]
        return (int(dd["nz"]), int(dd["ny"]), int(dd["nx"]))

    def macros(self, d: int):
        shape = self._shape(d)
        rho = torch.empty(shape, device=self.device)
        u = torch.empty((3,) + shape, device=self.device)
        check(self.lib.clbm_batch_get_macros(self.h, int(d), _ptr(rho), _ptr(u)), "clbm_batch_get_macros")
        return rho, u

    def populations(self, d: int, deviation: bool = False):
        out = torch.empty((19,) + self._shape(d), device=self.device)
        check(self.lib.clbm_batch_get_populations(self.h, int(d), _ptr(out), int(deviation)),
              "clbm_batch_get_populations")
        return out

    def set_populations(self, d: int, f: torch.Tensor, deviation: bool = False):
        if f.dtype != torch.float32 or not f.is_contiguous() or f.numel() != 19 * torch.Size(self._shape(d)).numel():
            raise ValueError("f: expected a contiguous float32 (19, nz, ny, nx) tensor")
        check(self.lib.clbm_batch_set_populations(self.h, int(d), _ptr(f), int(deviation)),
              "clbm_batch_set_populations")

    def check(self, clear: bool = False):
        check(self.lib.clbm_batch_check(self.h, int(clear)), "clbm_batch_check")

    @property
    def total_nodes(self) -> int:
        return int(self.info()["total_nodes"])
