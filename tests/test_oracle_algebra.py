"""Pins of the oracle's transforms, equilibria and forcing vectors against what
the paper prints (Eqs. A1, A4, A5, A6, row N_4) and against closed forms.

Paper: Fei, Luo & Li, arXiv:1801.04586.
"""
import numpy as np
import pytest

import oracle as o
from golden_io import load_matrix, load_symbolic

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(20180114)


def test_velocities_match_eq_A1():
    e = o.velocities()
    golden = load_matrix("d3q19_velocities.txt").astype(int)  # rows ex, ey, ez
    np.testing.assert_array_equal(e.T, golden)


def test_M_matches_printed_eq_A4():
    """M built from its definition (Eq. 4 on the moment set of Eq. A2) equals the
    printed matrix, which also pins the exponent reading k~002 for the tenth moment."""
    np.testing.assert_array_equal(o.matrix_M(), load_matrix("d3q19_M.txt"))


def test_nonzero_counts():
    M = load_matrix("d3q19_M.txt")
    assert (M != 0).sum() == 127
    Minv = o.matrix_Minv()
    assert (np.abs(Minv) > 1e-12).sum() == 91
    # entries of M^-1 are in {0, +-1, +-1/2, +-1/4}
    vals = set(np.round(np.abs(Minv[np.abs(Minv) > 1e-12]), 12))
    assert vals <= {1.0, 0.5, 0.25}


def test_Minv_inverts_printed_M():
    M = load_matrix("d3q19_M.txt")
    np.testing.assert_allclose(o.matrix_Minv() @ M, np.eye(19), atol=1e-14)
    np.testing.assert_allclose(M @ o.matrix_Minv(), np.eye(19), atol=1e-14)


def test_N4_row_matches_printed_example():
    for _ in range(5):
        u = RNG.uniform(-0.3, 0.3, 3)
        golden = load_symbolic("N4", ux=u[0], uy=u[1], uz=u[2])
        np.testing.assert_allclose(o.matrix_N(u)[4], golden, rtol=0, atol=1e-15)


def test_N_structure_and_inverse():
    """Lower triangular in the degree ordering with unit diagonal (Sec. II.B:
    binomial expansion from the lowest order up), N(u)^-1 = N(-u)."""
    u = RNG.uniform(-0.2, 0.2, 3)
    N = o.matrix_N(u)
    np.testing.assert_array_equal(np.diag(N), np.ones(19))
    assert np.all(np.triu(N, 1) == 0)
    np.testing.assert_allclose(N @ o.matrix_N(-u), np.eye(19), atol=1e-15)
    assert (np.abs(N) > 0).sum() == 91


def test_central_moments_two_routes():
    """Step 1 by the direct definition (Eq. 2) equals the two-stage route
    T~ = N M f of Eq. 4 with the printed M."""
    M = load_matrix("d3q19_M.txt")
    for _ in range(10):
        f = RNG.uniform(0.01, 0.4, 19)
        u = RNG.uniform(-0.3, 0.3, 3)
        np.testing.assert_allclose(o.central_moments(f, u), o.matrix_N(u) @ M @ f, rtol=0, atol=1e-14)
    # at u = 0 central moments are the raw moments
    f = RNG.uniform(0.01, 0.4, 19)
    np.testing.assert_allclose(o.central_moments(f, np.zeros(3)), M @ f, atol=1e-15)


def test_teq_and_C_match_printed_A5_A6():
    rho = 1.0 + RNG.uniform(-0.1, 0.1)
    np.testing.assert_allclose(o.teq(rho), load_symbolic("Teq", rho=rho, cs2=CS2), atol=1e-16)
    F = RNG.normal(size=3)
    np.testing.assert_allclose(o.cforce(F), load_symbolic("C", Fx=F[0], Fy=F[1], Fz=F[2], cs2=CS2),
                               atol=1e-16)


def test_rest_equilibrium_is_standard_weights():
    """At u = 0 the generalized equilibrium reduces to the textbook D3Q19 weights."""
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    np.testing.assert_allclose(o.equilibrium(1.0, np.zeros(3)), w, atol=1e-16)
    np.testing.assert_allclose(o.equilibrium(1.3, np.zeros(3)), 1.3 * w, atol=1e-15)


def _maxwell_raw(rho, u, exps):
    """Raw moments of a continuous Maxwellian with density rho, velocity u and
    temperature cs^2, for exponents <= 2 per axis: products of the 1D moments
    1, u, u^2 + cs^2."""
    g = lambda m, v: (1.0, v, v * v + CS2)[m]  # noqa: E731
    return np.array([rho * g(a, u[0]) * g(b, u[1]) * g(c, u[2]) for a, b, c in exps])


def test_generalized_equilibrium_raw_moments_are_maxwellian():
    """Its raw moments over the moment set equal those of the continuous
    Maxwellian (Eq. 15: T~eq are continuous central moments)."""
    M = load_matrix("d3q19_M.txt")
    exps = o.moment_exponents()
    for _ in range(10):
        rho = RNG.uniform(0.8, 1.2)
        u = RNG.uniform(-0.2, 0.2, 3)
        feq = o.equilibrium(rho, u)
        np.testing.assert_allclose(M @ feq, _maxwell_raw(rho, u, exps), atol=1e-15)
        np.testing.assert_allclose(o.central_moments(feq, u), o.teq(rho), atol=1e-15)


def test_macros_node_eq9():
    e = load_matrix("d3q19_velocities.txt").T
    f = RNG.uniform(0.01, 0.4, 19)
    F = RNG.normal(scale=1e-3, size=3)
    rho, u = o.macros_node(f, F)
    assert rho == pytest.approx(f.sum(), abs=1e-15)
    np.testing.assert_allclose(u, (e.T @ f + F / 2) / f.sum(), atol=1e-16)


def test_S_block_eigenvalues():
    """The 3x3 block of Eq. A3 relaxes the trace at s2b and the two normal-stress
    differences at s2 (Sec. II.B); s_nu = s2 on the off-diagonal moments."""
    lat = o.Lattice(4, 4, 4, s2=1.3, s2b=0.7, s3=1.1, s4=0.9, s0=0.5, s1=0.6)
    S = o.matrix_S(lat)
    B = S[7:10, 7:10]
    np.testing.assert_allclose(B @ np.ones(3), 0.7 * np.ones(3), atol=1e-15)
    for d in (np.array([1.0, -1.0, 0.0]), np.array([1.0, 0.0, -1.0])):
        np.testing.assert_allclose(B @ d, 1.3 * d, atol=1e-15)
    np.testing.assert_allclose(np.diag(S)[[0, 1, 2, 3, 4, 5, 6]], [0.5, 0.6, 0.6, 0.6, 1.3, 1.3, 1.3])
    np.testing.assert_allclose(np.diag(S)[10:16], 1.1)
    np.testing.assert_allclose(np.diag(S)[16:], 0.9)
