"""Symbolic derivation of the shift matrix N(u) (Eq. 4) from the definition
of a central moment, against the oracle's N(u), for the moment sets of
Eq. A2 (D3Q19) and Eq. 12 (D3Q27).

Row (m, n, p) of N(u) holds the coefficients that express the central moment
sum_i f_i (e_ix - u_x)^m (e_iy - u_y)^n (e_iz - u_z)^p (Eq. 2) through the
raw moments. Expanding the product with sympy and reducing it on the velocity
set (components in {-1, 0, 1}, so e^3 = e and e^4 = e^2; on D3Q19 no velocity
has three non-zero components, so monomials in all three vanish) leaves a
combination of the raw-moment monomials; its coefficients are the row.
Nothing of the oracle's construction is used on this side.
"""
import numpy as np
import pytest

import oracle as o

sympy = pytest.importorskip("sympy")


def symbolic_N(q=19):
    ex, ey, ez, ux, uy, uz = sympy.symbols("ex ey ez ux uy uz")
    exps = [tuple(int(v) for v in row) for row in o.moment_exponents(q)]
    index = {e: k for k, e in enumerate(exps)}
    N = sympy.zeros(q, q)
    for r, (m, n, p) in enumerate(exps):
        poly = sympy.Poly(sympy.expand((ex - ux) ** m * (ey - uy) ** n * (ez - uz) ** p), ex, ey, ez)
        for (a, b, c), coeff in poly.terms():
            # reduce on {-1, 0, 1}: e^3 = e, e^4 = e^2
            a, b, c = [k if k <= 2 else 2 - (k % 2) for k in (a, b, c)]
            if q == 19 and a and b and c:
                continue  # no D3Q19 velocity has three non-zero components
            N[r, index[(a, b, c)]] += coeff
    return N, (ux, uy, uz)


@pytest.mark.parametrize("q", [19, 27])
def test_shift_matrix_rows_follow_from_the_definition(q):
    N, (ux, uy, uz) = symbolic_N(q)
    f = sympy.lambdify((ux, uy, uz), N, "numpy")
    rng = np.random.default_rng(1801)
    for u in [(0.0, 0.0, 0.0), (1 / 7, -2 / 9, 3 / 11)] + [tuple(rng.uniform(-0.3, 0.3, 3)) for _ in range(4)]:
        np.testing.assert_allclose(o.matrix_N(np.array(u), q), np.array(f(*u), dtype=float), rtol=0, atol=1e-14)


@pytest.mark.parametrize("q,degree", [(19, 4), (27, 6)])
def test_shift_matrix_is_a_polynomial_with_unit_diagonal(q, degree):
    """Entries are polynomials in u of degree at most four (D3Q19, whose
    highest moments are k_220-type) or six (D3Q27, k_222), and the diagonal
    is 1."""
    N, us = symbolic_N(q)
    for i in range(q):
        assert N[i, i] == 1
        for j in range(q):
            if N[i, j] != 0:
                assert sympy.Poly(N[i, j], *us).total_degree() <= degree
