"""Python front end of the C ABI: a D3Q19 cascaded-LBM lattice on one GPU.

PyTorch supplies device memory for inputs/outputs and the CUDA stream; every
step of the method runs in libclbm.so's kernels. Shapes: scalar fields
(nz, ny, nx), vector fields (3, nz, ny, nx), populations (19, nz, ny, nx),
all float32 on the lattice's CUDA device.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Tuple

import torch

from . import _capi
from ._capi import check


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class _DeviceSpan:
    """A span of device memory owned by the library, exposed to PyTorch through
    the CUDA array interface (no copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def _device_bytes(ptr: int, nbytes: int, device) -> torch.Tensor:
    with torch.cuda.device(device):
        return torch.as_tensor(_DeviceSpan(ptr, nbytes), device=device)


class Lattice:
    """CLBM lattice (Fei, Luo & Li, arXiv:1801.04586): D3Q19 of Appendix A
    (lattice=19) or D3Q27 of Sec. II (lattice=27).

    nu sets s2 = 1/(3 nu + 1/2); s2b, s3, s4 are the bulk, third- and
    fourth-order rates (Eq. A3 / Eq. 13), s3b, s4b, s5, s6 the further D3Q27
    rates; walls is a CLBM_WALL_* bit mask (x=1, y=2, z=4; other axes
    periodic); storage is 'f32', 'f16', 'bf16', 'f16sr' or 'bf16sr'
    (populations stored as deviations f - w_i); pattern is 'ab' (two
    buffers, pull) or 'aa' (one buffer updated in place); model is
    'cascaded' (the paper's collision), or one of the comparison models
    'srt' (SRT-LBM at s2) and 'mrt' (non-orthogonal MRT of Appendix B).
    slab (SLAB_LO | SLAB_HI bits) and z0 make the lattice the z-slab
    z0 .. z0 + nz - 1 of a larger one whose z faces take their crossing
    populations from halo planes (see slab_step, faces and slabs.py).
    wait_cycles bounds the staged step's waits for its copies (0: about 2 s);
    inject = INJECT_DROP_COPY withholds the first tile's copies (failure-
    detection tests: the step then ends with CLBM_ERR_TIMEOUT).
    """

    def __init__(self, nx: int, ny: int, nz: int, nu: float, walls: int = 0, s2b: float = 1.0,
                 s3: float = 1.0, s4: float = 1.0, storage: str = "f32", block: Tuple[int, int] = (0, 0),
                 device=None, stream: Optional[torch.cuda.Stream] = None, variant: int = 0, lattice: int = 19,
                 s3b: float = 1.0, s4b: float = 1.0, s5: float = 1.0, s6: float = 1.0, pattern: str = "ab",
                 model: str = "cascaded", slab: int = 0, z0: int = 0, wait_cycles: int = 0, inject: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the lattice runs only in libclbm.so's kernels")
        self.lib = _capi.lib()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = torch.device("cuda", dev.index if dev.index is not None else torch.cuda.current_device())
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.shape = (self.nz, self.ny, self.nx)
        self.n = self.nx * self.ny * self.nz
        self.walls = int(walls)
        self.storage = storage
        self.pattern = pattern
        self.model = model
        self.q = 27 if int(lattice) == 27 else 19
        self.slab = int(slab)
        self.z0 = int(z0)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            p = _capi.Params(self.nx, self.ny, self.nz, self.walls, float(nu), float(s2b), float(s3), float(s4),
                             _capi.STORAGE[storage], int(block[0]), int(block[1]), int(variant), int(lattice),
                             _capi.PATTERN[pattern],
                             float(s3b), float(s4b), float(s5), float(s6), _capi.MODEL[model], self.slab,
                             self.z0, 0, int(wait_cycles), int(inject), 0)
            h = ctypes.c_void_p()
            check(self.lib.clbm_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                  "clbm_create")
        self.h = h
        self._force_ref = None  # keeps borrowed force tensors alive

    # ---- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.clbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = _capi.Info()
        check(self.lib.clbm_get_info(self.h, ctypes.byref(i)), "clbm_get_info")
        return {k: getattr(i, k) for k, _ in _capi.Info._fields_}

    # ---- helpers
    def _dev(self, t: torch.Tensor, shape, name):
        if t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous float32 tensor on {self.device}")
        if tuple(t.shape) != tuple(shape) and t.numel() != math.prod(shape):
            raise ValueError(f"{name}: expected shape {shape}, got {tuple(t.shape)}")
        return t

    def empty(self, *shape, dtype=torch.float32):
        return torch.empty(shape, dtype=dtype, device=self.device)

    # ---- force
    def set_force_uniform(self, fx: float, fy: float = 0.0, fz: float = 0.0):
        check(self.lib.clbm_set_force_uniform(self.h, fx, fy, fz), "clbm_set_force_uniform")
        self._force_ref = None

    def set_force_profile_z(self, F: torch.Tensor):
        self._dev(F, (3, self.nz), "F")
        check(self.lib.clbm_set_force_profile_z(self.h, _ptr(F)), "clbm_set_force_profile_z")
        self._force_ref = F

    def set_force_field(self, F: torch.Tensor):
        self._dev(F, (3,) + self.shape, "F")
        check(self.lib.clbm_set_force_field(self.h, _ptr(F)), "clbm_set_force_field")
        self._force_ref = F

    def set_force_decay(self, gamma: float):
        """Force in use at step t becomes F exp(-gamma t) (gamma = 0: static)."""
        check(self.lib.clbm_set_force_decay(self.h, float(gamma)), "clbm_set_force_decay")

    # ---- state
    def init_equilibrium(self, rho: Optional[torch.Tensor] = None, u: Optional[torch.Tensor] = None):
        if rho is not None:
            self._dev(rho, self.shape, "rho")
        if u is not None:
            self._dev(u, (3,) + self.shape, "u")
        check(self.lib.clbm_init_equilibrium(self.h, _ptr(rho), _ptr(u)), "clbm_init_equilibrium")

    def step(self, nsteps: int = 1):
        check(self.lib.clbm_step(self.h, int(nsteps)), "clbm_step")

    def macros(self, rho: Optional[torch.Tensor] = None, u: Optional[torch.Tensor] = None):
        rho = self.empty(*self.shape) if rho is None else self._dev(rho, self.shape, "rho")
        u = self.empty(3, *self.shape) if u is None else self._dev(u, (3,) + self.shape, "u")
        check(self.lib.clbm_get_macros(self.h, _ptr(rho), _ptr(u)), "clbm_get_macros")
        return rho, u

    def populations(self, deviation: bool = False, out: Optional[torch.Tensor] = None):
        out = self.empty(self.q, *self.shape) if out is None else self._dev(out, (self.q,) + self.shape, "out")
        check(self.lib.clbm_get_populations(self.h, _ptr(out), int(deviation)), "clbm_get_populations")
        return out

    def set_populations(self, f: torch.Tensor, deviation: bool = False):
        self._dev(f, (self.q,) + self.shape, "f")
        check(self.lib.clbm_set_populations(self.h, _ptr(f), int(deviation)), "clbm_set_populations")

    def reduce_moments(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """FP64 [sum rho, sum rho u_x, sum rho u_y, sum rho u_z] (Eq. 9), on the device."""
        out = torch.empty(4, dtype=torch.float64, device=self.device) if out is None else out
        check(self.lib.clbm_reduce_moments(self.h, _ptr(out)), "clbm_reduce_moments")
        return out

    def reduce_pair(self, a: torch.Tensor, b: Optional[torch.Tensor] = None,
                    out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """FP64 [sum (a-b)^2, sum b^2, sum a b] over all elements, on the device."""
        if a.dtype != torch.float32 or not a.is_contiguous() or a.device != self.device:
            raise ValueError("a: expected a contiguous float32 tensor on the lattice device")
        if b is not None and (b.dtype != torch.float32 or not b.is_contiguous() or b.numel() != a.numel()):
            raise ValueError("b: expected a contiguous float32 tensor like a")
        out = torch.empty(3, dtype=torch.float64, device=self.device) if out is None else out
        check(self.lib.clbm_reduce_pair(self.h, _ptr(a), _ptr(b), a.numel(), _ptr(out)), "clbm_reduce_pair")
        return out

    def check(self, clear: bool = False):
        check(self.lib.clbm_check(self.h, int(clear)), "clbm_check")

    def state_bytes(self) -> int:
        return int(self.info()["state_bytes"])

    def export_state(self, dst: Optional[torch.Tensor] = None) -> torch.Tensor:
        nb = self.state_bytes()
        dst = torch.empty(nb, dtype=torch.uint8, device=self.device) if dst is None else dst
        if dst.numel() * dst.element_size() < nb:
            raise ValueError("dst too small")
        check(self.lib.clbm_export_state(self.h, _ptr(dst)), "clbm_export_state")
        return dst

    def import_state(self, src: torch.Tensor, set_steps: int = -1):
        if src.numel() * src.element_size() < self.state_bytes():
            raise ValueError("src too small")
        check(self.lib.clbm_import_state(self.h, _ptr(src), int(set_steps)), "clbm_import_state")

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        check(self.lib.clbm_save_state(self.h, None, ctypes.byref(n)), "clbm_save_state")
        buf = ctypes.create_string_buffer(n.value)
        check(self.lib.clbm_save_state(self.h, buf, ctypes.byref(n)), "clbm_save_state")
        return buf.raw[: n.value]

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        check(self.lib.clbm_load_state(self.h, buf, len(data)), "clbm_load_state")

    def run_host(self, rho: Optional[torch.Tensor], u: Optional[torch.Tensor], nsteps: int,
                 rho_out: Optional[torch.Tensor] = None, u_out: Optional[torch.Tensor] = None,
                 moments: Optional[torch.Tensor] = None):
        """One job through host buffers (ideally pinned CPU tensors): upload rho/u,
        initialise, step, read per-step FP64 moments and the final rho/u back."""
        for name, t in (("rho", rho), ("u", u), ("rho_out", rho_out), ("u_out", u_out), ("moments", moments)):
            if t is not None and (t.device.type != "cpu" or not t.is_contiguous()):
                raise ValueError(f"{name}: expected a contiguous host tensor")
        check(self.lib.clbm_run_host(self.h, _ptr(rho), _ptr(u), int(nsteps), _ptr(rho_out), _ptr(u_out),
                                     _ptr(moments)), "clbm_run_host")

    @property
    def steps_done(self) -> int:
        return int(self.info()["steps_done"])

    # ---- z-slab decomposition
    def slab_step(self, part: int = _capi.SLAB_ALL):
        """One step of a z-slab (or its faces / interior part, SLAB_FACES then
        SLAB_INTERIOR); exchange faces (slabs.exchange_faces) before the next."""
        check(self.lib.clbm_slab_step(self.h, int(part)), "clbm_slab_step")

    def faces(self) -> Tuple[torch.Tensor, torch.Tensor]:
        """(send, recv): byte views of the newest state's send and receive
        planes, each 2 x face_bytes (first half: the lower neighbour's share,
        second half: the upper's). They alias library memory and are valid
        until the next step."""
        send, recv, nb = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        check(self.lib.clbm_slab_faces(self.h, ctypes.byref(send), ctypes.byref(recv), ctypes.byref(nb)),
              "clbm_slab_faces")
        return (_device_bytes(send.value, 2 * nb.value, self.device),
                _device_bytes(recv.value, 2 * nb.value, self.device))

    # ---- recomputation and adjoint (FP32 storage)
    def step_raw(self, src: torch.Tensor, dst: torch.Tensor):
        """One step from raw state buffer src into dst (context state untouched)."""
        nb = self.state_bytes()
        for name, b in (("src", src), ("dst", dst)):
            if b.device != self.device or b.numel() * b.element_size() < nb or not b.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous device buffer of >= {nb} bytes")
        check(self.lib.clbm_step_raw(self.h, _ptr(src), _ptr(dst)), "clbm_step_raw")

    def lam_numel(self) -> int:
        """Floats of an adjoint array: 19 x N in the post-streaming layout; a
        z-slab appends 20 planes (10 receive, 10 send; slabs.lam_faces)."""
        return 19 * self.nz * self.ny * self.nx + (20 * self.ny * self.nx if self.slab else 0)

    def empty_lam(self) -> torch.Tensor:
        return torch.zeros(self.lam_numel(), dtype=torch.float32, device=self.device)

    def _lam(self, t: torch.Tensor, name: str):
        if not self.slab:
            return self._dev(t, (19,) + self.shape, name)
        if t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous() or \
                t.numel() < self.lam_numel():
            raise ValueError(f"{name}: expected a contiguous float32 tensor of >= {self.lam_numel()} elements "
                             f"on {self.device} (a z-slab's adjoint array with its halo planes)")
        return t

    def adjoint_seed(self, gu: torch.Tensor, lam: torch.Tensor, gF: torch.Tensor,
                     state: Optional[torch.Tensor] = None):
        self._dev(gu, (3,) + self.shape, "gu")
        self._lam(lam, "lam")
        self._dev(gF, (3,) + self.shape, "gF")
        check(self.lib.clbm_adjoint_seed(self.h, _ptr(state), _ptr(gu), _ptr(lam), _ptr(gF)), "clbm_adjoint_seed")

    def adjoint_step(self, state: torch.Tensor, lam_next: torch.Tensor, lam: torch.Tensor, gF: torch.Tensor):
        self._lam(lam_next, "lam_next")
        self._lam(lam, "lam")
        self._dev(gF, (3,) + self.shape, "gF")
        if state.numel() * state.element_size() < self.state_bytes():
            raise ValueError("state: buffer too small")
        check(self.lib.clbm_adjoint_step(self.h, _ptr(state), _ptr(lam_next), _ptr(lam), _ptr(gF)),
              "clbm_adjoint_step")

    def adjoint_segment(self, ckpt: torch.Tensor, tape: Optional[torch.Tensor], k: int, lam: torch.Tensor,
                        lam_tmp: torch.Tensor, gF: torch.Tensor):
        """Backward over one checkpointed segment of k steps (recompute into tape,
        then k adjoint steps); lam holds the adjoint at the segment end on entry
        and at its start on return."""
        nb = self.state_bytes()
        if k > 1 and (tape is None or tape.numel() * tape.element_size() < (k - 1) * nb):
            raise ValueError("tape too small")
        for name, a in (("lam", lam), ("lam_tmp", lam_tmp)):
            self._dev(a, (19,) + self.shape, name)
        self._dev(gF, (3,) + self.shape, "gF")
        check(self.lib.clbm_adjoint_segment(self.h, _ptr(ckpt), _ptr(tape), int(k), _ptr(lam), _ptr(lam_tmp),
                                            _ptr(gF)), "clbm_adjoint_segment")
