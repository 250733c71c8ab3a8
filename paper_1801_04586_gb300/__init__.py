"""GB300 (sm_103a) D3Q19 cascaded lattice Boltzmann method with consistent
forcing (Fei, Luo & Li, arXiv:1801.04586): a C-ABI CUDA library (libclbm.so,
declared in include/clbm.h) and a thin PyTorch-facing binding.
"""
from .builder import build  # noqa: F401
from .lattice import Lattice  # noqa: F401
from .batch import Batch  # noqa: F401
from ._capi import CLBMError, UnstableError, WALL_X, WALL_Y, WALL_Z  # noqa: F401
