"""The cascaded collision relaxes in the frame that moves with the fluid.

Its central-moment equilibria depend on the density alone (Eq. A5 for D3Q19,
Eq. 15 for D3Q27) and its forcing terms on the force alone (Eqs. A6, 16), so
the post-collision central moments about u (Eq. 2) are a function of the
pre-collision central moments, rho and F only (Eqs. 5 and 7), whatever u is.
The test builds, from the definition of a central moment, two node states that
have the same central moments about two different velocities, collides both
with the oracle and compares the post-collision central moments, each about
its own velocity. The raw-moment MRT and the SRT collision (Appendix B and
Sec. III.A), whose relaxation mixes the frame velocity in, must fail the same
comparison: the check can tell the collisions apart.
"""
import numpy as np
import pytest

import oracle as o


def frame_matrix(u, q):
    """A[r, i] = prod_a (e_ia - u_a)^k_ra: central moment r of population i
    about u, by the definition (Eq. 2)."""
    e = o.velocities(q).astype(float)
    k = o.moment_exponents(q)
    return np.prod((e[None, :, :] - np.asarray(u)[None, None, :]) ** k[:, None, :], axis=2)


def velocity(f, F, q):
    """Eq. 9 with the half-force term."""
    e = o.velocities(q).astype(float)
    return (f @ e + 0.5 * np.asarray(F)) / f.sum()


def lattice(q, model):
    kw = dict(s2=1.3, s2b=1.1, s3=1.6, s4=0.9, q=q, model=model)
    if q == 27:
        kw.update(s3b=1.45, s4b=0.8, s5=1.2, s6=1.7)
    return o.Lattice(1, 1, 1, **kw)


def post_collision_pair(q, model, seed):
    rng = np.random.default_rng(seed)
    F = np.array([1e-3, -2e-3, 5e-4])
    w = o.equilibrium(1.0, (0.0, 0.0, 0.0), q)
    fA = w * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, q))
    uA = velocity(fA, F, q)
    K = frame_matrix(uA, q) @ fA  # central moments of fA about its own velocity
    uB = uA + np.array([0.11, -0.07, 0.05])
    fB = np.linalg.solve(frame_matrix(uB, q), K)  # the same central moments about uB
    np.testing.assert_allclose(velocity(fB, F, q), uB, rtol=0, atol=1e-13)
    lat = lattice(q, model)
    KA = frame_matrix(uA, q) @ o.collide(lat, fA, F)
    KB = frame_matrix(uB, q) @ o.collide(lat, fB, F)
    return K, KA, KB


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cascaded_post_collision_central_moments_do_not_depend_on_u(q, seed):
    K, KA, KB = post_collision_pair(q, 0, seed)
    assert np.abs(KA - K).max() > 1e-4  # the collision did change the state
    np.testing.assert_allclose(KA, KB, rtol=0, atol=1e-13)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("model", [1, 2])
def test_raw_moment_collisions_depend_on_u(q, model):
    _, KA, KB = post_collision_pair(q, model, 0)
    assert np.abs(KA - KB).max() > 1e-4
