"""Pins of the oracle's D3Q27 build (Sec. II, the paper's main development)
against the printed Eqs. 1, 14, 15 and 16, the non-zero counts the paper
states for M and M^-1, textbook D3Q27 weights, invariants and closed-form
flows.

Paper: Fei, Luo & Li, arXiv:1801.04586.
"""
import numpy as np
import pytest

import analytic as an
import oracle as o
from golden_io import load_matrix, load_symbolic

Q = 27
CS2 = 1.0 / 3.0
M27 = load_matrix("d3q27_M.txt")
E27 = load_matrix("d3q27_velocities.txt").T.astype(int)
RNG = np.random.default_rng(27)


def lat27(nx=2, ny=2, nz=2, **kw):
    return o.Lattice(nx, ny, nz, q=Q, **kw)


def test_velocities_and_M_match_eqs_1_and_14():
    np.testing.assert_array_equal(o.velocities(Q), E27)
    np.testing.assert_array_equal(o.matrix_M(Q), M27)


def test_nonzero_counts_stated_in_sec_II():
    """Sec. II.B: M and M^-1 have 343 and 216 non-zero elements."""
    assert (M27 != 0).sum() == 343
    Minv = o.matrix_Minv(Q)
    assert (np.abs(Minv) > 1e-12).sum() == 216
    np.testing.assert_allclose(Minv @ M27, np.eye(Q), atol=1e-14)


def test_moment_set_is_tensor_product():
    """Eq. 12 (with k~002 for the repeated k~020) holds every exponent triple in
    {0,1,2}^3 once."""
    exps = {tuple(r) for r in o.moment_exponents(Q)}
    assert exps == {(a, b, c) for a in range(3) for b in range(3) for c in range(3)}


def test_teq_and_C_match_printed_15_16():
    rho = 1.02
    np.testing.assert_allclose(o.teq(rho, Q), load_symbolic("Teq27", rho=rho, cs2=CS2), atol=1e-16)
    F = RNG.normal(size=3)
    np.testing.assert_allclose(o.cforce(F, Q), load_symbolic("C27", Fx=F[0], Fy=F[1], Fz=F[2], cs2=CS2),
                               atol=1e-16)


def test_rest_weights():
    w = o.equilibrium(1.0, np.zeros(3), Q)
    expect = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)
    np.testing.assert_allclose(w, expect, atol=1e-16)


def test_central_moments_two_routes_and_N_inverse():
    for _ in range(5):
        f = RNG.uniform(0.001, 0.3, Q)
        u = RNG.uniform(-0.3, 0.3, 3)
        N = o.matrix_N(u, Q)
        np.testing.assert_allclose(o.central_moments(f, u, Q), N @ M27 @ f, atol=1e-14)
        np.testing.assert_allclose(N @ o.matrix_N(-u, Q), np.eye(Q), atol=1e-15)
        assert np.all(np.triu(N, 1) == 0)


def test_generalized_equilibrium_is_maxwellian_on_all_moments():
    g = lambda m, v: (1.0, v, v * v + CS2)[m]  # noqa: E731
    for _ in range(5):
        rho, u = RNG.uniform(0.9, 1.1), RNG.uniform(-0.2, 0.2, 3)
        feq = o.equilibrium(rho, u, Q)
        expect = [rho * g(a, u[0]) * g(b, u[1]) * g(c, u[2]) for a, b, c in o.moment_exponents(Q)]
        np.testing.assert_allclose(M27 @ feq, expect, atol=1e-15)


def test_collision_invariants():
    w = o.equilibrium(1.0, np.zeros(3), Q)
    for _ in range(10):
        r = RNG.uniform(0.3, 1.9, 8)
        lat = lat27(s2=r[0], s2b=r[1], s3=r[2], s4=r[3], s3b=r[4], s4b=r[5], s5=r[6], s6=r[7],
                    s0=RNG.uniform(0.1, 1.9), s1=RNG.uniform(0.1, 1.9))
        f = w * (1 + RNG.uniform(-0.2, 0.2, Q))
        F = RNG.normal(scale=1e-3, size=3)
        fs = o.collide(lat, f, F)
        assert fs.sum() == pytest.approx(f.sum(), abs=2e-15)
        np.testing.assert_allclose(E27.T @ fs, E27.T @ f + F, rtol=0, atol=2e-15)
        rho, u = RNG.uniform(0.9, 1.1), RNG.uniform(-0.1, 0.1, 3)
        feq = o.equilibrium(rho, u, Q)
        np.testing.assert_allclose(o.collide(lat, feq), feq, atol=1e-15)


def test_uniform_rates_give_srt_with_guo_moments():
    g = lambda m, v: (1.0, v, v * v + CS2)[m]  # noqa: E731
    w = o.equilibrium(1.0, np.zeros(3), Q)
    s = 1.3
    lat = lat27(s2=s, s2b=s, s3=s, s4=s, s3b=s, s4b=s, s5=s, s6=s, s0=s, s1=s)
    f = w * (1 + RNG.uniform(-0.1, 0.1, Q))
    F = RNG.normal(scale=1e-3, size=3)
    rho, u = o.macros_node(f, F, Q)
    exps = o.moment_exponents(Q)
    maxw = np.array([rho * g(a, u[0]) * g(b, u[1]) * g(c, u[2]) for a, b, c in exps])
    guo = np.zeros(10)
    guo[1:4] = F
    guo[4] = u[0] * F[1] + u[1] * F[0]
    guo[5] = u[0] * F[2] + u[2] * F[0]
    guo[6] = u[1] * F[2] + u[2] * F[1]
    guo[7:10] = 2 * u * F
    expect = (1 - s) * (M27 @ f)[:10] + s * maxw[:10] + (1 - s / 2) * guo
    np.testing.assert_allclose((M27 @ o.collide(lat, f, F))[:10], expect, atol=2e-15)


def test_relaxation_groups_d3q27():
    r = dict(s2=1.3, s2b=0.6, s3=1.1, s3b=0.7, s4=0.8, s4b=1.5, s5=0.9, s6=1.2)
    lat = lat27(**r)
    w = o.equilibrium(1.0, np.zeros(3), Q)
    f = w * (1 + RNG.uniform(-0.2, 0.2, Q))
    rho, u = o.macros_node(f, np.zeros(3), Q)
    kt, ks = o.central_moments(f, u, Q), o.central_moments(o.collide(lat, f), u, Q)
    teq = o.teq(rho, Q)
    d, ds = kt - teq, ks - teq
    np.testing.assert_allclose(ds[4:7], (1 - r["s2"]) * d[4:7], atol=1e-15)
    assert ds[7:10].sum() == pytest.approx((1 - r["s2b"]) * d[7:10].sum(), abs=1e-15)
    np.testing.assert_allclose(ds[10:16], (1 - r["s3"]) * d[10:16], atol=1e-15)
    assert ds[16] == pytest.approx((1 - r["s3b"]) * d[16], abs=1e-15)
    np.testing.assert_allclose(ds[17:20], (1 - r["s4"]) * d[17:20], atol=1e-15)
    np.testing.assert_allclose(ds[20:23], (1 - r["s4b"]) * d[20:23], atol=1e-15)
    np.testing.assert_allclose(ds[23:26], (1 - r["s5"]) * d[23:26], atol=1e-15)
    assert ds[26] == pytest.approx((1 - r["s6"]) * d[26], abs=1e-15)


@pytest.mark.parametrize("walls", [0, 5, 7])
def test_pure_streaming_d3q27(walls):
    opp = np.array([int(np.where((E27 == -E27[i]).all(axis=1))[0][0]) for i in range(Q)])
    lat = lat27(4, 5, 3, walls=walls, s0=0, s1=0, s2=0, s2b=0, s3=0, s4=0, s3b=0, s4b=0, s5=0, s6=0)
    f = RNG.uniform(0, 1, (Q,) + lat.shape)
    nz, ny, nx = lat.shape
    idx = np.indices(lat.shape)
    expect = np.empty_like(f)
    for i in range(Q):
        ex, ey, ez = E27[i]
        rolled = np.roll(f[i], shift=(ez, ey, ex), axis=(0, 1, 2))
        beyond = np.zeros(lat.shape, bool)
        for axis, (c, n, e) in enumerate(((idx[2], nx, ex), (idx[1], ny, ey), (idx[0], nz, ez))):
            if walls & (1 << axis):
                beyond |= (c - e < 0) | (c - e >= n)
        expect[i] = np.where(beyond, f[opp[i]], rolled)
    np.testing.assert_allclose(o.step(lat, f), expect, atol=1e-14)


def test_shear_wave_viscosity_d3q27():
    L, nu = 101, 0.05
    lat = o.Lattice(1, L, 1, q=Q, s2=an.s2_from_nu(nu))
    y = np.arange(L)
    u = np.zeros((3, 1, L, 1))
    u[0, 0, :, 0] = 1e-4 * np.sin(2 * np.pi * y / L)
    f = o.step(lat, o.init(lat, None, u), None, 200)
    a1 = an.shear_wave_amplitude(o.macros(lat, f)[1][0, 0, :, 0])
    f = o.step(lat, f, None, 2000)
    a2 = an.shear_wave_amplitude(o.macros(lat, f)[1][0, 0, :, 0])
    assert np.log(a1 / a2) / ((2 * np.pi / L) ** 2 * 2000) == pytest.approx(nu, rel=1e-3)


def test_poiseuille_noslip_rule_d3q27():
    n, nu, F = 20, 0.1, 1e-6
    s2 = an.s2_from_nu(nu)
    Ff = np.zeros((3, n, 1, 1))
    Ff[0] = F
    steps = int(30 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu))
    lat = o.Lattice(1, 1, n, walls=4, q=Q, s2=s2, s2b=s2, s3=an.noslip_s3(s2))
    f = o.step(lat, o.init(lat, None, None, Ff), Ff, steps)
    ux = o.macros(lat, f, Ff)[1][0, :, 0, 0]
    ua = an.poiseuille_steady(n, F, nu)
    assert np.sqrt(((ux - ua) ** 2).sum() / (ua ** 2).sum()) < 1e-8


def test_adjoint_dot_product_d3q27():
    lat = o.Lattice(3, 2, 4, walls=4, q=Q, s2=1.5, s2b=1.1, s3=0.9, s4=1.2, s3b=1.3, s4b=0.8, s5=1.1, s6=0.7)
    w = o.equilibrium(1.0, np.zeros(3), Q).reshape(Q, 1, 1, 1)
    f = w * (1 + RNG.uniform(-0.05, 0.05, (Q,) + lat.shape))
    F = RNG.normal(scale=1e-3, size=(3,) + lat.shape)
    v, vF, wv = RNG.normal(size=f.shape), RNG.normal(size=F.shape), RNG.normal(size=f.shape)
    h = 1e-6
    jv = (o.step(lat, f + h * v, F + h * vF) - o.step(lat, f - h * v, F - h * vF)) / (2 * h)
    gF = np.zeros_like(F)
    lam = o.adjoint_step(lat, f, wv, F, gF)
    lhs, rhs = float((wv * jv).sum()), float((lam * v).sum() + (gF * vF).sum())
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)
