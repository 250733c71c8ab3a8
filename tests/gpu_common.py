"""Helpers for the GPU-vs-oracle parity tests.

Inputs come from paper_1801_04586_gb300.synthetic as float32; the oracle gets
the same values widened to float64. Nothing the GPU computes is fed to the
oracle.
"""
import json
import os

import numpy as np
import torch

import oracle
from paper_1801_04586_gb300 import Lattice

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).reshape(19, 1, 1, 1)

# Tolerance on FP32 populations after 100 steps: max_{x,i} |f_gpu - f_ora| / f_ora.
F32_REL_TOL = 1e-5


def dev():
    return torch.device("cuda", 0)


def t(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def s2_of(nu):
    return 1.0 / (3.0 * nu + 0.5)


def make_pair(nx, ny, nz, nu, walls=0, s2b=1.0, s3=1.0, s4=1.0, storage="f32", block=(0, 0), variant=0):
    g = Lattice(nx, ny, nz, nu, walls=walls, s2b=s2b, s3=s3, s4=s4, storage=storage, block=block, device=dev(),
                variant=variant)
    o = oracle.Lattice(nx, ny, nz, walls=walls, s2=s2_of(nu), s2b=s2b, s3=s3, s4=s4)
    return g, o


def gpu_f(g):
    """GPU state as float64 populations f = w + h (h read as deviations, exact)."""
    return g.populations(deviation=True).double().cpu().numpy() + W


def rel_err(f_gpu, f_ora):
    return float(np.max(np.abs(f_gpu - f_ora) / np.abs(f_ora)))


def dev_err(f_gpu, f_ora):
    """Error relative to the size of the deviations from the rest weights."""
    return float(np.max(np.abs(f_gpu - f_ora)) / max(np.max(np.abs(f_ora - W)), 1e-300))


def report(name, **values):
    """Append measured figures to the file named by CLBM_REPORT (if set)."""
    path = os.environ.get("CLBM_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"test": name, **values}) + "\n")
