"""Seeded synthetic inputs (numpy PCG64) shared by the tests, the benchmark
and the oracle comparisons. Workload definitions only: nothing here computes
any part of the lattice Boltzmann method.

All arrays are float32 (the precision the GPU library consumes); a caller that
feeds the same values to the FP64 oracle widens them exactly.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def kolmogorov_profile(nz: int, F0: float) -> np.ndarray:
    """Kolmogorov body force along x varying with z: F_x = F0 sin(2 pi z / nz),
    as a (3, nz) profile."""
    F = np.zeros((3, nz), dtype=np.float64)
    F[0] = F0 * np.sin(2.0 * np.pi * np.arange(nz) / nz)
    return F.astype(np.float32)


def profile_to_field(profile: np.ndarray, shape) -> np.ndarray:
    """Expand a (3, nz) profile to a (3, nz, ny, nx) field."""
    nz, ny, nx = shape
    return np.ascontiguousarray(np.broadcast_to(profile[:, :, None, None], (3, nz, ny, nx))).astype(np.float32)


def uniform_field(shape, F) -> np.ndarray:
    out = np.zeros((3,) + tuple(shape), dtype=np.float32)
    for a in range(3):
        out[a] = F[a]
    return out


def divfree_velocity(shape, seed: int, umax: float, kmin: float = 1.0, kmax: float = 4.0) -> np.ndarray:
    """Random periodic divergence-free field (3, nz, ny, nx): Gaussian Fourier
    amplitudes on wavenumbers kmin <= |k| <= kmax, projected onto the plane
    normal to k, real through Hermitian symmetry (irfftn), scaled so that
    max |u| = umax."""
    nz, ny, nx = shape
    g = rng(seed)
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    mask = (kk >= kmin) & (kk <= kmax)
    spec = (g.standard_normal((3,) + kk.shape) + 1j * g.standard_normal((3,) + kk.shape)) * mask
    k = np.stack(np.broadcast_arrays(kx, ky, kz)).astype(np.float64)  # components x, y, z
    kdot = (k * spec).sum(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        spec = spec - np.where(kk > 0, k * kdot / np.where(kk > 0, kk * kk, 1.0), 0.0)
    u = np.fft.irfftn(spec, s=(nz, ny, nx), axes=(1, 2, 3))
    speed = np.sqrt((u * u).sum(axis=0)).max()
    return (u * (umax / speed)).astype(np.float32)


def gaussian_force(shape, sigma: float, seed: int) -> np.ndarray:
    return (rng(seed).standard_normal((3,) + tuple(shape)) * sigma).astype(np.float32)


def uniform_perturbation(shape, amp: float, seed: int, components: int = 3) -> np.ndarray:
    return rng(seed).uniform(-amp, amp, (components,) + tuple(shape)).astype(np.float32)


def random_deviations(shape, amp: float, seed: int) -> np.ndarray:
    """Arbitrary (non-equilibrium) population deviations (19, nz, ny, nx),
    uniform in (-amp, amp): a random lattice state for parity checks."""
    return rng(seed).uniform(-amp, amp, (19,) + tuple(shape)).astype(np.float32)


def density_perturbation(shape, amp: float, seed: int) -> np.ndarray:
    return (1.0 + rng(seed).uniform(-amp, amp, tuple(shape))).astype(np.float32)


def batch_domains(count: int, seed: int, side_lo: int = 32, side_hi: int = 128,
                  nu_lo: float = 0.005, nu_hi: float = 0.1, f_lo: float = 1e-7, f_hi: float = 1e-5):
    """Independent channels/ducts: sides uniform in [side_lo, side_hi] per axis,
    walls on z (channel) or on y and z (duct) by a fair coin, nu and F_x
    uniform in the given ranges."""
    g = rng(seed)
    out = []
    for _ in range(count):
        nx, ny, nz = (int(v) for v in g.integers(side_lo, side_hi + 1, 3))
        duct = bool(g.integers(0, 2))
        out.append({"nx": nx, "ny": ny, "nz": nz, "walls": 6 if duct else 4,
                    "nu": float(g.uniform(nu_lo, nu_hi)), "fx": float(g.uniform(f_lo, f_hi))})
    return out
