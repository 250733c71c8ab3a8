"""Closed-form flow solutions used to pin the oracle and the GPU path.

Coordinates follow the halfway bounce-back placement of Sec. III.C: with n
nodes across a channel, the walls sit half a spacing outside the first and
last nodes, so node k is at k - (n - 1)/2 from the centre and the half-width
is n/2.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def nu_from_s2(s2: float) -> float:
    """Kinematic viscosity of Sec. II.B: nu = (1/s2 - 1/2) cs^2 (dt = 1)."""
    return (1.0 / s2 - 0.5) * CS2


def s2_from_nu(nu: float) -> float:
    return 1.0 / (3.0 * nu + 0.5)


def noslip_s3(s2: float) -> float:
    """No-slip rule of Sec. III.B: s3 = (16 - 8 s2)/(8 - s2)."""
    return (16.0 - 8.0 * s2) / (8.0 - s2)


def centred(n: int) -> np.ndarray:
    """Node positions relative to the channel centre for n nodes between walls."""
    return np.arange(n) - (n - 1) / 2.0


def poiseuille_steady(n: int, F: float, nu: float, rho: float = 1.0) -> np.ndarray:
    """Sec. III.B: u(z) = u0 (1 - z^2/L^2), u0 = F L^2 / (2 rho nu), L = n/2."""
    L = n / 2.0
    z = centred(n)
    return F * L * L / (2.0 * rho * nu) * (1.0 - z * z / (L * L))


def poiseuille_startup(n: int, F: float, nu: float, t: float, rho: float = 1.0,
                       terms: int = 400) -> np.ndarray:
    """Start-up from rest of the Sec. III.B channel: the steady parabola minus its
    cosine eigen-expansion decaying as exp(-n^2 pi^2 nu t / (4 L^2))."""
    L = n / 2.0
    z = centred(n)
    u0 = F * L * L / (2.0 * rho * nu)
    u = 1.0 - z * z / (L * L)
    for k in range(terms):
        m = 2 * k + 1
        coef = 32.0 * (-1.0) ** k / (m * np.pi) ** 3
        u = u - coef * np.cos(m * np.pi * z / (2 * L)) * np.exp(-m * m * np.pi ** 2 * nu * t / (4 * L * L))
    return u0 * u


def duct_steady(n: int, F: float, nu: float, rho: float = 1.0, terms: int = 200) -> np.ndarray:
    """Sec. III.C series for the developed square-duct flow, on an n x n node
    cross-section (half-width a = n/2). Returns u_x[z, y]."""
    a = n / 2.0
    y = centred(n)[None, :]
    z = centred(n)[:, None]
    u = np.zeros((n, n))
    for k in range(terms):
        m = 2 * k + 1
        # cosh ratio written with exponentials to stay finite for large m
        ratio = (np.exp(m * np.pi * (z / (2 * a) - 0.5)) + np.exp(-m * np.pi * (z / (2 * a) + 0.5))) / (
            1.0 + np.exp(-m * np.pi))
        u = u + (-1.0) ** k * (1.0 - ratio) * np.cos(m * np.pi * y / (2 * a)) / m ** 3
    return 16.0 * a * a * F / (rho * nu * np.pi ** 3) * u


def duct_transient(n: int, F: float, nu: float, t: float, rho: float = 1.0, terms: int = 120) -> np.ndarray:
    """Start-up from rest of the square duct: the double cosine series
    sum_{m,n odd} F_mn/(nu lam_mn) (1 - exp(-nu lam_mn t)) cos(m pi y/2a) cos(n pi z/2a),
    F_mn = 16 F (-1)^((m+n-2)/2) / (m n pi^2), lam_mn = (pi/2a)^2 (m^2 + n^2).
    Returns u_x[z, y]."""
    a = n / 2.0
    y = centred(n)
    z = centred(n)
    ms = 2 * np.arange(terms) + 1
    sgn = (-1.0) ** np.arange(terms)
    cy = np.cos(np.outer(ms, y) * np.pi / (2 * a))  # (terms, n)
    cz = np.cos(np.outer(ms, z) * np.pi / (2 * a))
    lam = (np.pi / (2 * a)) ** 2 * (ms[:, None] ** 2 + ms[None, :] ** 2)
    Fmn = 16.0 * F / rho * np.outer(sgn, sgn) / (np.outer(ms, ms) * np.pi ** 2)
    amp = Fmn / (nu * lam) * (1.0 - np.exp(-nu * lam * t))  # (m over y, n over z)
    return np.einsum("mn,my,nz->zy", amp, cy, cz)


def shear_wave_amplitude(ux_y: np.ndarray) -> float:
    """Amplitude of the sin(2 pi y / L) component of a periodic profile u_x(y)."""
    L = ux_y.shape[-1]
    y = np.arange(L)
    return 2.0 / L * float(np.sum(ux_y * np.sin(2 * np.pi * y / L)))


def taylor_green(L: int, u0: float, nu: float, t: float):
    """Sec. III.D: decaying Taylor-Green vortex on an L x L periodic box with
    k1 = k2 = 2 pi / L, node positions x = 0..L-1. Returns (u_x, u_y) as [y, x]
    arrays at time t."""
    k = 2.0 * np.pi / L
    x = np.arange(L)[None, :]
    y = np.arange(L)[:, None]
    d = np.exp(-2.0 * nu * k * k * t)
    return -u0 * np.cos(k * x) * np.sin(k * y) * d, u0 * np.sin(k * x) * np.cos(k * y) * d


def taylor_green_force(L: int, u0: float, rho: float = 1.0):
    """The body force of Sec. III.D at t = 0, (F_x, F_y) as [y, x] arrays; it
    decays as exp(-gamma t) with gamma = taylor_green_decay(L, nu)."""
    k = 2.0 * np.pi / L
    x = np.arange(L)[None, :] * np.ones((L, 1))
    y = np.arange(L)[:, None] * np.ones((1, L))
    return -(rho * k * u0 * u0 / 2.0) * np.sin(2.0 * k * x), -(rho * k * u0 * u0 / 2.0) * np.sin(2.0 * k * y)


def taylor_green_decay(L: int, nu: float) -> float:
    """Decay rate of the Taylor-Green force: 2 nu (k1^2 + k2^2)."""
    k = 2.0 * np.pi / L
    return 4.0 * nu * k * k


def taylor_green_time(L: int, nu: float, tstar: float) -> int:
    """Steps to reach T* = nu (k1^2 + k2^2) t / ln 2 (Sec. III.D)."""
    k = 2.0 * np.pi / L
    return int(round(tstar * np.log(2.0) / (2.0 * nu * k * k)))
