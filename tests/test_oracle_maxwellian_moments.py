"""The central-moment equilibria and forcing terms derived from the Maxwellian.

Sec. II.B sets the central-moment equilibria to the central moments of the
continuous Maxwell-Boltzmann distribution (Eq. 15; Eq. A5 for D3Q19):
  int f^M (xi - u)^(a, b, c) = rho c_s^(a+b+c) (a-1)!! (b-1)!! (c-1)!!
(zero unless a, b and c are all even). It obtains the forcing terms by
applying Eq. 6 to the generalized local equilibrium (Eq. 16; Eq. A6). They
coincide with the central moments of the force term acting on the Maxwellian,
which integration by parts of -F . grad_xi f^M / rho against (xi - u)^(a, b, c)
gives as
  C_abc = F_x a M_(a-1)bc + F_y b M_a(b-1)c + F_z c M_ab(c-1)
with M the moments above at rho = 1. The test derives every entry this way for
the moment sets of both lattices and compares with the oracle's T~eq and C. It
shares nothing with the values typed from the paper (pinned elsewhere) or with
the matrix route of Eq. 6.
"""
import numpy as np
import pytest

import oracle as o

CS2 = 1.0 / 3.0


def double_factorial_before(n):
    """(n - 1)!! for even n >= 0."""
    r = 1
    for k in range(n - 1, 0, -2):
        r *= k
    return r


def gaussian_central_moment(a, b, c):
    if a % 2 or b % 2 or c % 2:
        return 0.0
    return CS2 ** ((a + b + c) // 2) * double_factorial_before(a) * double_factorial_before(b) * \
        double_factorial_before(c)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("rho", [1.0, 0.83, 1.37])
def test_equilibrium_central_moments_are_the_maxwellians(q, rho):
    derived = np.array([rho * gaussian_central_moment(*map(int, e)) for e in o.moment_exponents(q)])
    np.testing.assert_allclose(o.teq(rho, q), derived, rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", [19, 27])
def test_forcing_central_moments_are_the_force_on_the_maxwellian(q):
    rng = np.random.default_rng(16)
    for F in [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]), rng.uniform(-1.0, 1.0, 3)]:
        derived = []
        for a, b, c in (tuple(map(int, e)) for e in o.moment_exponents(q)):
            v = 0.0
            if a:
                v += F[0] * a * gaussian_central_moment(a - 1, b, c)
            if b:
                v += F[1] * b * gaussian_central_moment(a, b - 1, c)
            if c:
                v += F[2] * c * gaussian_central_moment(a, b, c - 1)
            derived.append(v)
        np.testing.assert_allclose(o.cforce(F, q), np.array(derived), rtol=0, atol=1e-15)
