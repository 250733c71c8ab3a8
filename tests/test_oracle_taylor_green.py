"""Pin of the oracle under a space- and time-dependent force: the decaying
Taylor-Green vortex of Sec. III.D (Re = 50, u0 = 0.005, T* = 4), whose error
against the analytic solution must fall at second order with the grid."""
import numpy as np

import analytic as an
import oracle


def _tg_error(L, u0=0.005, Re=50.0, tstar=4.0):
    nu = u0 * L / Re
    lat = oracle.Lattice.from_nu(L, L, 1, nu)  # the flow is z-invariant: one plane
    ux, uy = an.taylor_green(L, u0, nu, 0.0)
    u = np.zeros((3, 1, L, L))
    u[0, 0], u[1, 0] = ux, uy
    fx, fy = an.taylor_green_force(L, u0)
    F = np.zeros((3, 1, L, L))
    F[0, 0], F[1, 0] = fx, fy
    gamma = an.taylor_green_decay(L, nu)
    T = an.taylor_green_time(L, nu, tstar)
    f = oracle.step_decay(lat, oracle.init(lat, None, u, F), F, T, 0.0, gamma)
    _, uu = oracle.macros(lat, f, F * np.exp(-gamma * T))
    ax, ay = an.taylor_green(L, u0, nu, T)
    return float(np.sqrt(((uu[0, 0] - ax) ** 2 + (uu[1, 0] - ay) ** 2).sum() / (ax ** 2 + ay ** 2).sum()))


def test_taylor_green_second_order():
    e16, e32 = _tg_error(16), _tg_error(32)
    order = np.log2(e16 / e32)
    assert 1.8 < order < 2.2
    assert e32 < 1e-2


def test_step_decay_matches_stepwise_force():
    """The decaying force equals stepping one step at a time with F e^{-gamma t}."""
    lat = oracle.Lattice(4, 3, 5, walls=4, s2=1.3)
    rng = np.random.default_rng(7)
    F = rng.normal(scale=1e-3, size=(3,) + lat.shape)
    f0 = oracle.init(lat, None, None, F)
    gamma = 0.05
    a = oracle.step_decay(lat, f0, F, 6, 0.0, gamma)
    b = f0
    for t in range(6):
        b = oracle.step(lat, b, F * np.exp(-gamma * t), 1)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
