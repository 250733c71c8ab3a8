"""Bulk viscosity and sound speed of the oracle, from a standing sound wave.

Sec. II.B relates the rate s2b of the trace k200 + k020 + k002 to the bulk
viscosity, xi = (2/3)(1/s2b - 1/2) c_s^2, beside nu = (1/s2 - 1/2) c_s^2.
The linearised isothermal Navier-Stokes equations turn a density
perturbation A cos(kx) at rest into a damped oscillation
A e^{-gamma t} cos(omega t + phi) with gamma = ((4/3) nu + xi) k^2 / 2 and
omega^2 = c_s^2 k^2 - gamma^2 (c_s^2 = 1/3). Fitting gamma and omega to the
oracle's density mode on a periodic line of 64 nodes measures xi and the
sound speed. Relaxing the trace at s2 instead of s2b, or a wrong factor in
the trace block of S (Eq. A3), moves xi by tens of percent.
"""
import numpy as np
import pytest

import oracle as o

optimize = pytest.importorskip("scipy.optimize")

CS2 = 1.0 / 3.0
NU = 0.05
L = 64


def fit_mode(q, s2b, steps=1200, amplitude=1e-4):
    lat = o.Lattice.from_nu(L, 1, 1, NU, q=q, s2b=s2b)
    x = np.arange(L)
    k = 2.0 * np.pi / L
    rho = np.broadcast_to(1.0 + amplitude * np.cos(k * x), lat.shape).copy()
    f = o.init(lat, rho, np.zeros((3,) + lat.shape))
    a = np.empty(steps)
    for t in range(steps):
        r, _ = o.macros(lat, f)
        a[t] = (2.0 / L) * np.sum((r[0, 0] - 1.0) * np.cos(k * x))
        f = o.step(lat, f, nsteps=1)
    t = np.arange(steps)
    skip = 20  # the start-up layer of the equilibrium initial state

    def wave(t, a0, gamma, omega, phi):
        return a0 * np.exp(-gamma * t) * np.cos(omega * t + phi)

    p, _ = optimize.curve_fit(wave, t[skip:], a[skip:], p0=[amplitude, 1e-3, np.sqrt(CS2) * k, 0.0])
    return k, p[1], p[2]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("s2b", [0.8, 1.4, 1.7])
def test_bulk_viscosity_and_sound_speed(q, s2b):
    k, gamma, omega = fit_mode(q, s2b)
    xi = 2.0 * gamma / k**2 - 4.0 / 3.0 * NU
    xi_paper = 2.0 / 3.0 * (1.0 / s2b - 0.5) * CS2
    assert abs(xi / xi_paper - 1.0) < 5e-3, (xi, xi_paper)
    omega_th = np.sqrt(CS2 * k**2 - gamma**2)
    assert abs(omega / omega_th - 1.0) < 1e-3, (omega, omega_th)
