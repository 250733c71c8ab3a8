"""ctypes binding of the FP64 C oracle (test infrastructure only).

The C source, ``clbm_oracle.c``, states what it computes and which passage of
the paper (Fei, Luo & Li, arXiv:1801.04586) each function follows. This module
only builds it with gcc and marshals numpy float64 arrays.

Array conventions: populations are ``(19, nz, ny, nx)`` float64 arrays
(structure of arrays, x fastest); vector fields are ``(3, nz, ny, nx)``;
scalar fields ``(nz, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "clbm_oracle.c"), os.path.join(_HERE, "oracle_node.inc")]
_LIBS = {19: os.path.join(_HERE, "libclbm_oracle.so"), 27: os.path.join(_HERE, "libclbm_oracle27.so")}
_PREFIX = {19: "ora_", 27: "ora27_"}

Q = 19


def lib_path(q: int = 19) -> str:
    return _LIBS[q]


def build(force: bool = False) -> str:
    """Compile the oracle (D3Q19 and D3Q27 builds of the same source) with gcc
    (OpenMP) if a shared object is stale."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    for q, lib in _LIBS.items():
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
            tmp = lib + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", f"-DORACLE_Q={q}",
                   "-o", tmp, _SRC[0], "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, lib)
    return _LIBS[19]


_libs = {}


class _Lib:
    """Exported functions of one build, by their unprefixed names."""

    def __init__(self, lib, prefix):
        self._lib, self._prefix = lib, prefix

    def __getattr__(self, name):
        return getattr(self._lib, self._prefix + name[len("ora_"):])


def _get(q: int = 19):
    if q not in _libs:
        build()
        lib = ctypes.CDLL(_LIBS[q])
        pre = _PREFIX[q]
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        sig = {
            "ora_velocities": [P], "ora_moment_exponents": [P], "ora_matrix_M": [P],
            "ora_matrix_Minv": [P], "ora_matrix_N": [P, P], "ora_matrix_S": [P, P],
            "ora_teq": [D, P], "ora_cforce": [P, P], "ora_central_moments": [P, P, P],
            "ora_macros_node": [P, P, P, P], "ora_collide": [P, P, P, P],
            "ora_equilibrium": [D, P, P], "ora_init": [P, P, P, P, P],
            "ora_step": [P, P, P, I, I], "ora_macros": [P, P, P, P, P],
            "ora_step_decay": [P, P, P, I, I, D, D],
            "ora_first_step_nodes": [P, P, P, P, I, P, P, I],
            "ora_adjoint_step": [P, P, P, P, P, P, I],
            "ora_adjoint_seed": [P, P, P, P, P, P],
            "ora_num_threads": [],
            "ora_feq_discrete": [D, P, P], "ora_guo_force": [P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, pre + name[len("ora_"):])
            fn.argtypes = args
            fn.restype = ctypes.c_int if name in (
                "ora_init", "ora_step", "ora_step_decay", "ora_macros", "ora_first_step_nodes",
                "ora_adjoint_step", "ora_adjoint_seed", "ora_num_threads") else None
        _libs[q] = _Lib(lib, pre)
    return _libs[q]


class _CLattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("walls", ctypes.c_int), ("s0", ctypes.c_double), ("s1", ctypes.c_double),
                ("s2", ctypes.c_double), ("s2b", ctypes.c_double), ("s3", ctypes.c_double),
                ("s4", ctypes.c_double), ("s3b", ctypes.c_double), ("s4b", ctypes.c_double),
                ("s5", ctypes.c_double), ("s6", ctypes.c_double), ("model", ctypes.c_int),
                ("pad", ctypes.c_int)]


@dataclass
class Lattice:
    """Lattice and relaxation rates. ``walls`` bit 0/1/2: x/y/z faces are
    halfway bounce-back walls (else periodic). ``s2`` follows from the
    kinematic viscosity, nu = (1/s2 - 1/2)/3 (Sec. II.B). ``q`` selects D3Q19
    (Appendix A) or D3Q27 (Sec. II); s3b, s4b, s5, s6 are the extra D3Q27
    rates of Eq. 13. ``model`` selects the collision: 0 the cascaded one
    (Sec. II), 1 the SRT-LBM at rate s2 with the discrete equilibrium of
    Sec. II.B and Guo's forcing, 2 the non-orthogonal raw-moment MRT of
    Appendix B (same M and S)."""
    nx: int
    ny: int
    nz: int
    walls: int = 0
    s2: float = 1.0
    s2b: float = 1.0
    s3: float = 1.0
    s4: float = 1.0
    s0: float = 1.0
    s1: float = 1.0
    q: int = 19
    s3b: float = 1.0
    s4b: float = 1.0
    s5: float = 1.0
    s6: float = 1.0
    model: int = 0

    @staticmethod
    def from_nu(nx, ny, nz, nu, walls=0, **kw):
        return Lattice(nx, ny, nz, walls, s2=1.0 / (3.0 * nu + 0.5), **kw)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def c(self) -> _CLattice:
        return _CLattice(self.nx, self.ny, self.nz, self.walls, self.s0, self.s1,
                         self.s2, self.s2b, self.s3, self.s4, self.s3b, self.s4b, self.s5, self.s6,
                         int(self.model), 0)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return _get().ora_num_threads()


def velocities(q: int = 19) -> np.ndarray:
    out = np.zeros((q, 3), dtype=np.int32)
    _get(q).ora_velocities(_ptr(out))
    return out


def moment_exponents(q: int = 19) -> np.ndarray:
    out = np.zeros((q, 3), dtype=np.int32)
    _get(q).ora_moment_exponents(_ptr(out))
    return out


def matrix_M(q: int = 19) -> np.ndarray:
    out = np.zeros((q, q))
    _get(q).ora_matrix_M(_ptr(out))
    return out


def matrix_Minv(q: int = 19) -> np.ndarray:
    out = np.zeros((q, q))
    _get(q).ora_matrix_Minv(_ptr(out))
    return out


def matrix_N(u, q: int = 19) -> np.ndarray:
    out = np.zeros((q, q))
    _get(q).ora_matrix_N(_ptr(_f64(u, (3,))), _ptr(out))
    return out


def matrix_S(lat: Lattice) -> np.ndarray:
    out = np.zeros((lat.q, lat.q))
    c = lat.c()
    _get(lat.q).ora_matrix_S(ctypes.byref(c), _ptr(out))
    return out


def teq(rho: float, q: int = 19) -> np.ndarray:
    out = np.zeros(q)
    _get(q).ora_teq(float(rho), _ptr(out))
    return out


def cforce(F, q: int = 19) -> np.ndarray:
    out = np.zeros(q)
    _get(q).ora_cforce(_ptr(_f64(F, (3,))), _ptr(out))
    return out


def central_moments(f, u, q: int = 19) -> np.ndarray:
    out = np.zeros(q)
    _get(q).ora_central_moments(_ptr(_f64(f, (q,))), _ptr(_f64(u, (3,))), _ptr(out))
    return out


def macros_node(f, F=(0.0, 0.0, 0.0), q: int = 19):
    rho = np.zeros(1)
    u = np.zeros(3)
    _get(q).ora_macros_node(_ptr(_f64(f, (q,))), _ptr(_f64(F, (3,))), _ptr(rho), _ptr(u))
    return float(rho[0]), u


def collide(lat: Lattice, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    out = np.zeros(lat.q)
    c = lat.c()
    _get(lat.q).ora_collide(ctypes.byref(c), _ptr(_f64(f, (lat.q,))), _ptr(_f64(F, (3,))), _ptr(out))
    return out


def equilibrium(rho: float, u, q: int = 19) -> np.ndarray:
    out = np.zeros(q)
    _get(q).ora_equilibrium(float(rho), _ptr(_f64(u, (3,))), _ptr(out))
    return out


def feq_discrete(rho: float, u, q: int = 19) -> np.ndarray:
    """The second-order discrete equilibrium of Sec. II.B at (rho, u)."""
    out = np.zeros(q)
    _get(q).ora_feq_discrete(float(rho), _ptr(_f64(u, (3,))), _ptr(out))
    return out


def guo_force(u, F, q: int = 19) -> np.ndarray:
    """Guo's forcing term as Appendix B quotes it, at (u, F)."""
    out = np.zeros(q)
    _get(q).ora_guo_force(_ptr(_f64(u, (3,))), _ptr(_f64(F, (3,))), _ptr(out))
    return out


def init(lat: Lattice, rho=None, u=None, F=None) -> np.ndarray:
    """Generalized equilibrium at (rho, u - F/(2 rho)); returns (19, nz, ny, nx)."""
    f = np.zeros((lat.q,) + lat.shape)
    c = lat.c()
    _get(lat.q).ora_init(ctypes.byref(c), _ptr(_f64(rho, lat.shape)), _ptr(_f64(u, (3,) + lat.shape)),
                    _ptr(_f64(F, (3,) + lat.shape)), _ptr(f))
    return f


def step(lat: Lattice, f, F=None, nsteps: int = 1, nthreads: int = 0) -> np.ndarray:
    """Advance the post-streaming state f by nsteps; returns a new array."""
    f = _f64(f, (lat.q,) + lat.shape).copy()
    c = lat.c()
    rc = _get(lat.q).ora_step(ctypes.byref(c), _ptr(_f64(F, (3,) + lat.shape)), _ptr(f), int(nsteps),
                         int(nthreads))
    if rc != 0:
        raise MemoryError("oracle step failed")
    return f


def step_decay(lat: Lattice, f, F, nsteps: int, t0: float, gamma: float, nthreads: int = 0) -> np.ndarray:
    """As step, with the force F(x) exp(-gamma t) at each collision time
    t = t0, t0 + 1, ..."""
    f = _f64(f, (lat.q,) + lat.shape).copy()
    c = lat.c()
    rc = _get(lat.q).ora_step_decay(ctypes.byref(c), _ptr(_f64(F, (3,) + lat.shape)), _ptr(f), int(nsteps), int(nthreads),
                               float(t0), float(gamma))
    if rc != 0:
        raise MemoryError("oracle step failed")
    return f


def macros(lat: Lattice, f, F=None):
    rho = np.zeros(lat.shape)
    u = np.zeros((3,) + lat.shape)
    c = lat.c()
    _get(lat.q).ora_macros(ctypes.byref(c), _ptr(_f64(f, (lat.q,) + lat.shape)),
                      _ptr(_f64(F, (3,) + lat.shape)), _ptr(rho), _ptr(u))
    return rho, u


def first_step_nodes(lat: Lattice, nodes, rho=None, u=None, F=None, nthreads: int = 0):
    """f(node, t=1) for the listed linear node indices, from the initial state
    that ``init`` builds; returns (len(nodes), 19)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((len(nodes), lat.q))
    c = lat.c()
    _get(lat.q).ora_first_step_nodes(ctypes.byref(c), _ptr(_f64(rho, lat.shape)),
                                _ptr(_f64(u, (3,) + lat.shape)), _ptr(_f64(F, (3,) + lat.shape)),
                                len(nodes), _ptr(nodes), _ptr(out), int(nthreads))
    return out


def adjoint_step(lat: Lattice, f_t, lam_next, F=None, gF=None, nthreads: int = 0):
    """Adjoint of one step. Returns lam_t; accumulates into gF (3, nz, ny, nx) if given."""
    lam_t = np.zeros((lat.q,) + lat.shape)
    c = lat.c()
    if gF is not None:
        assert gF.dtype == np.float64 and gF.flags.c_contiguous
    _get(lat.q).ora_adjoint_step(ctypes.byref(c), _ptr(_f64(f_t, (lat.q,) + lat.shape)),
                            _ptr(_f64(F, (3,) + lat.shape)), _ptr(_f64(lam_next, (lat.q,) + lat.shape)),
                            _ptr(lam_t), _ptr(gF), int(nthreads))
    return lam_t


def adjoint_seed(lat: Lattice, f_T, g, F=None, gF=None):
    """Seed lam^T from a cotangent g (3, nz, ny, nx) on the final velocity."""
    lam = np.zeros((lat.q,) + lat.shape)
    c = lat.c()
    if gF is not None:
        assert gF.dtype == np.float64 and gF.flags.c_contiguous
    _get(lat.q).ora_adjoint_seed(ctypes.byref(c), _ptr(_f64(f_T, (lat.q,) + lat.shape)),
                            _ptr(_f64(F, (3,) + lat.shape)), _ptr(_f64(g, (3,) + lat.shape)),
                            _ptr(lam), _ptr(gF))
    return lam
