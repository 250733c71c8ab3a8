"""Pins of the oracle's collision (Eq. 5), streaming (Eq. 8) and macroscopic
update (Eq. 9) against invariants, special cases and textbook reductions.

Paper: Fei, Luo & Li, arXiv:1801.04586.
"""
import numpy as np
import pytest

import oracle as o
from golden_io import load_matrix

CS2 = 1.0 / 3.0
M = load_matrix("d3q19_M.txt")
E = load_matrix("d3q19_velocities.txt").T.astype(int)  # (19, 3)
OPP = np.array([int(np.where((E == -E[i]).all(axis=1))[0][0]) for i in range(19)])
RNG = np.random.default_rng(1801)


def _rand_state(rng, amp=0.02):
    w = o.equilibrium(1.0, np.zeros(3))
    return w * (1.0 + rng.uniform(-amp, amp, 19))


def _rand_lat(rng, **kw):
    return o.Lattice(2, 2, 2, s2=rng.uniform(0.3, 1.9), s2b=rng.uniform(0.3, 1.9),
                     s3=rng.uniform(0.3, 1.9), s4=rng.uniform(0.3, 1.9), **kw)


def test_collision_conserves_mass_and_adds_F():
    """Eqs. 5, 7, 9: mass is conserved and the momentum sum_i f_i e_i grows by
    exactly F per collision, for any rates."""
    for _ in range(20):
        lat = _rand_lat(RNG, s0=RNG.uniform(0.1, 1.9), s1=RNG.uniform(0.1, 1.9))
        f = _rand_state(RNG, 0.2)
        F = RNG.normal(scale=1e-3, size=3)
        fs = o.collide(lat, f, F)
        assert fs.sum() == pytest.approx(f.sum(), abs=2e-15)
        np.testing.assert_allclose(E.T @ fs, E.T @ f + F, rtol=0, atol=2e-15)


def test_equilibrium_is_fixed_point_without_force():
    for _ in range(10):
        lat = _rand_lat(RNG)
        rho = RNG.uniform(0.9, 1.1)
        u = RNG.uniform(-0.15, 0.15, 3)
        feq = o.equilibrium(rho, u)
        np.testing.assert_allclose(o.collide(lat, feq), feq, rtol=0, atol=1e-15)


def test_result_independent_of_conserved_rates():
    """s0, s1 act on conserved central moments; the result does not depend on them."""
    f = _rand_state(RNG, 0.1)
    F = RNG.normal(scale=1e-3, size=3)
    a = o.collide(o.Lattice(2, 2, 2, s2=1.2, s2b=0.8, s3=1.1, s4=0.7, s0=1.0, s1=1.0), f, F)
    b = o.collide(o.Lattice(2, 2, 2, s2=1.2, s2b=0.8, s3=1.1, s4=0.7, s0=0.3, s1=1.7), f, F)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def _maxwell_raw(rho, u):
    g = lambda m, v: (1.0, v, v * v + CS2)[m]  # noqa: E731
    return np.array([rho * g(a, u[0]) * g(b, u[1]) * g(c, u[2]) for a, b, c in o.moment_exponents()])


def test_uniform_rates_reduce_to_srt_with_guo_forcing():
    """Sec. II.A: with all rates equal the scheme is SRT; its forcing term then
    carries Guo's moments up to second order: 0, F, u F + F u."""
    for _ in range(10):
        s = RNG.uniform(0.2, 1.9)
        lat = o.Lattice(2, 2, 2, s2=s, s2b=s, s3=s, s4=s, s0=s, s1=s)
        f = _rand_state(RNG, 0.1)
        F = RNG.normal(scale=1e-3, size=3)
        rho, u = o.macros_node(f, F)
        fs = o.collide(lat, f, F)
        guo = np.zeros(10)
        guo[1:4] = F
        guo[4] = u[0] * F[1] + u[1] * F[0]
        guo[5] = u[0] * F[2] + u[2] * F[0]
        guo[6] = u[1] * F[2] + u[2] * F[1]
        guo[7:10] = 2 * u * F
        expect = (1 - s) * (M @ f)[:10] + s * _maxwell_raw(rho, u)[:10] + (1 - s / 2) * guo
        np.testing.assert_allclose((M @ fs)[:10], expect, rtol=0, atol=2e-15)


def test_srt_without_force_relaxes_raw_moments_to_maxwellian():
    """With F = 0 and uniform rates every raw moment relaxes at rate s toward
    the Maxwellian raw moments (the generalized equilibrium)."""
    s = 1.37
    lat = o.Lattice(2, 2, 2, s2=s, s2b=s, s3=s, s4=s, s0=s, s1=s)
    f = _rand_state(RNG, 0.1)
    rho, u = o.macros_node(f)
    np.testing.assert_allclose(M @ o.collide(lat, f), (1 - s) * (M @ f) + s * _maxwell_raw(rho, u),
                               rtol=0, atol=2e-15)


def test_relaxation_groups_without_force():
    """Central moments about u relax group by group: k~110.. at s2, the trace of
    the second-order non-equilibrium part at s2b and its deviator at s2, the
    third order at s3 and the fourth order toward rho cs^4 at s4."""
    s2, s2b, s3, s4 = 1.3, 0.6, 1.1, 0.8
    lat = o.Lattice(2, 2, 2, s2=s2, s2b=s2b, s3=s3, s4=s4)
    f = _rand_state(RNG, 0.2)
    rho, u = o.macros_node(f)
    kt = o.central_moments(f, u)
    ks = o.central_moments(o.collide(lat, f), u)
    np.testing.assert_allclose(ks[4:7], (1 - s2) * kt[4:7], atol=1e-15)
    d, ds = kt[7:10] - rho * CS2, ks[7:10] - rho * CS2
    assert ds.sum() == pytest.approx((1 - s2b) * d.sum(), abs=1e-15)
    np.testing.assert_allclose(ds - ds.mean(), (1 - s2) * (d - d.mean()), atol=1e-15)
    np.testing.assert_allclose(ks[10:16], (1 - s3) * kt[10:16], atol=1e-15)
    np.testing.assert_allclose(ks[16:] - rho * CS2 ** 2, (1 - s4) * (kt[16:] - rho * CS2 ** 2), atol=1e-15)


def _pull_stream(f, walls):
    """Streaming of Eq. 8 written in pull form with numpy rolls: f_i(x) takes
    f_i(x - e_i), or f_ibar(x) when x - e_i lies beyond a wall face."""
    nz, ny, nx = f.shape[1:]
    out = np.empty_like(f)
    idx = np.indices((nz, ny, nx))  # z, y, x
    for i in range(19):
        ex, ey, ez = E[i]
        rolled = np.roll(f[i], shift=(ez, ey, ex), axis=(0, 1, 2))
        beyond = np.zeros((nz, ny, nx), bool)
        for axis, (c, n, e) in enumerate(((idx[2], nx, ex), (idx[1], ny, ey), (idx[0], nz, ez))):
            if walls & (1 << axis):
                src = c - e
                beyond |= (src < 0) | (src >= n)
        out[i] = np.where(beyond, f[OPP[i]], rolled)
    return out


@pytest.mark.parametrize("walls", [0, 1, 2, 4, 6, 7])
def test_pure_streaming_matches_roll(walls):
    """With every rate zero and F = 0 the collision is the identity, so a step is
    pure streaming; compare with the pull-form roll, including bounce-back."""
    lat = o.Lattice(5, 4, 3, walls=walls, s0=0, s1=0, s2=0, s2b=0, s3=0, s4=0)
    f = RNG.uniform(0.0, 1.0, (19,) + lat.shape)
    np.testing.assert_allclose(o.step(lat, f), _pull_stream(f, walls), rtol=0, atol=1e-14)


def test_lattice_conservation_periodic():
    lat = o.Lattice(4, 3, 5, walls=0, s2=1.4, s2b=0.9, s3=1.2, s4=1.0)
    f = np.stack([o.equilibrium(1.0, np.zeros(3))[i] * (1 + RNG.uniform(-0.05, 0.05, lat.shape))
                  for i in range(19)])
    F = RNG.normal(scale=1e-4, size=(3,) + lat.shape)
    m0 = f.sum()
    p0 = np.einsum("ia,izyx->a", E, f)
    g = o.step(lat, f, F, nsteps=7)
    assert g.sum() == pytest.approx(m0, rel=1e-14)
    np.testing.assert_allclose(np.einsum("ia,izyx->a", E, g), p0 + 7 * F.sum(axis=(1, 2, 3)),
                               rtol=0, atol=1e-13)


def test_lattice_mass_conservation_walls():
    lat = o.Lattice(3, 5, 4, walls=7, s2=1.1, s2b=1.0, s3=0.9, s4=1.0)
    f = np.stack([o.equilibrium(1.0, np.zeros(3))[i] * (1 + RNG.uniform(-0.05, 0.05, lat.shape))
                  for i in range(19)])
    F = RNG.normal(scale=1e-4, size=(3,) + lat.shape)
    assert o.step(lat, f, F, nsteps=9).sum() == pytest.approx(f.sum(), rel=1e-14)


def test_init_returns_prescribed_macros():
    """The initial state (generalized equilibrium at u - F/2rho) gives back the
    prescribed rho and u through Eq. 9."""
    lat = o.Lattice(3, 4, 2)
    rho = 1.0 + RNG.uniform(-0.01, 0.01, lat.shape)
    u = RNG.uniform(-0.05, 0.05, (3,) + lat.shape)
    F = RNG.normal(scale=1e-3, size=(3,) + lat.shape)
    f = o.init(lat, rho, u, F)
    r2, u2 = o.macros(lat, f, F)
    np.testing.assert_allclose(r2, rho, atol=1e-15)
    np.testing.assert_allclose(u2, u, atol=1e-15)


@pytest.mark.parametrize("walls", [0, 6, 7])
def test_first_step_nodes_matches_full_step(walls):
    lat = o.Lattice(5, 4, 6, walls=walls, s2=1.5, s2b=1.0, s3=1.0, s4=1.0)
    rho = 1.0 + RNG.uniform(-0.01, 0.01, lat.shape)
    u = RNG.uniform(-0.05, 0.05, (3,) + lat.shape)
    F = RNG.normal(scale=1e-3, size=(3,) + lat.shape)
    full = o.step(lat, o.init(lat, rho, u, F), F, 1).reshape(19, -1)
    nodes = RNG.choice(lat.n, 25, replace=False)
    np.testing.assert_allclose(o.first_step_nodes(lat, nodes, rho, u, F), full[:, nodes].T,
                               rtol=0, atol=1e-15)


def _rest_jacobian(lat):
    """Jacobian of the oracle collision at the rest state (central differences)."""
    q = lat.q
    w = o.equilibrium(1.0, np.zeros(3), q)
    J = np.zeros((q, q))
    h = 1e-7
    for k in range(q):
        d = np.zeros(q)
        d[k] = h
        J[:, k] = (o.collide(lat, w + d) - o.collide(lat, w - d)) / (2 * h)
    return J


def _spectral_radius(lat, nk=9):
    """Largest |eigenvalue| of one linearised step (streaming in Fourier space
    times the rest-state collision Jacobian) over a grid of wavevectors."""
    E = o.velocities(lat.q).astype(float)
    J = _rest_jacobian(lat)
    ks = np.linspace(0.0, np.pi, nk)
    r = 0.0
    for kx in ks:
        for ky in ks:
            for kz in ks:
                P = np.diag(np.exp(-1j * (E @ np.array([kx, ky, kz]))))
                r = max(r, float(np.abs(np.linalg.eigvals(P @ J)).max()))
    return r


def test_linear_stability_at_rest():
    """Von Neumann analysis of the oracle's step at the rest state: at k = 0
    the 4 conserved modes have eigenvalue 1 and the others 1 - s; at every
    wavevector the step does not amplify for the rates the tests use, and it
    does amplify when the bulk rate nears 2 (s2b = 1.9 at nu = 0.1), which is
    why no configuration here goes there."""
    s2 = 1.0 / (3 * 0.1 + 0.5)
    lat = o.Lattice(1, 1, 1, s2=s2, s2b=1.2, s3=1.1, s4=0.9)
    ev = np.sort(np.abs(np.linalg.eigvals(_rest_jacobian(lat))))[::-1]
    np.testing.assert_allclose(ev[:4], 1.0, atol=1e-7)
    expected = sorted([1.0] * 4 + [abs(1 - s2)] * 5 + [abs(1 - 1.2)] + [abs(1 - 1.1)] * 6 + [abs(1 - 0.9)] * 3,
                      reverse=True)
    np.testing.assert_allclose(ev, expected, atol=1e-7)
    for kw in (dict(s2b=1.2, s3=1.1, s4=0.9), dict(s2b=s2, s3=(16 - 8 * s2) / (8 - s2), s4=1.0)):
        assert _spectral_radius(o.Lattice(1, 1, 1, s2=s2, **kw)) < 1 + 1e-7
    assert _spectral_radius(o.Lattice(1, 1, 1, s2=s2, s2b=1.9, s3=(16 - 8 * s2) / (8 - s2), s4=1.0)) > 1.05
