"""Pins of the oracle adjoint (complex-step Jacobians, transposed streaming)
against central finite differences of the oracle's own forward step, which the
other oracle tests pin to the paper.
"""
import numpy as np

import oracle as o

RNG = np.random.default_rng(4586)


def _state(lat, rng):
    w = o.equilibrium(1.0, np.zeros(3))
    return np.stack([w[i] * (1 + rng.uniform(-0.05, 0.05, lat.shape)) for i in range(19)])


def test_adjoint_step_dot_product_against_fd():
    for walls in (0, 4, 7):
        lat = o.Lattice(3, 4, 5, walls=walls, s2=1.6, s2b=1.1, s3=0.9, s4=1.2)
        f = _state(lat, RNG)
        F = RNG.normal(scale=1e-3, size=(3,) + lat.shape)
        v = RNG.normal(size=f.shape)
        vF = RNG.normal(size=F.shape)
        w = RNG.normal(size=f.shape)
        h = 1e-6
        jv = (o.step(lat, f + h * v, F + h * vF) - o.step(lat, f - h * v, F - h * vF)) / (2 * h)
        gF = np.zeros_like(F)
        lam = o.adjoint_step(lat, f, w, F, gF)
        lhs = float((w * jv).sum())
        rhs = float((lam * v).sum() + (gF * vF).sum())
        assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


def test_adjoint_seed_against_fd():
    lat = o.Lattice(2, 3, 2)
    f = _state(lat, RNG)
    F = RNG.normal(scale=1e-3, size=(3,) + lat.shape)
    g = RNG.normal(size=(3,) + lat.shape)
    v = RNG.normal(size=f.shape)
    vF = RNG.normal(size=F.shape)
    h = 1e-7
    du = (o.macros(lat, f + h * v, F + h * vF)[1] - o.macros(lat, f - h * v, F - h * vF)[1]) / (2 * h)
    gF = np.zeros_like(F)
    lam = o.adjoint_seed(lat, f, g, F, gF)
    lhs = float((g * du).sum())
    rhs = float((lam * v).sum() + (gF * vF).sum())
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


def test_unrolled_gradient_against_fd():
    """dL/dF for L = 1/2 sum |u(T) - u*|^2 after T steps from a fixed state,
    by the chained oracle adjoint versus central differences at a few entries."""
    lat = o.Lattice(4, 3, 4, walls=4, s2=1.3, s2b=1.0, s3=1.0, s4=1.0)
    T = 6
    f0 = _state(lat, RNG)
    F = RNG.normal(scale=1e-4, size=(3,) + lat.shape)
    ut = RNG.normal(scale=1e-3, size=(3,) + lat.shape)

    def loss(Fv):
        f = o.step(lat, f0, Fv, T)
        u = o.macros(lat, f, Fv)[1]
        return 0.5 * float(((u - ut) ** 2).sum())

    states = [f0]
    for _ in range(T):
        states.append(o.step(lat, states[-1], F, 1))
    u = o.macros(lat, states[-1], F)[1]
    gF = np.zeros_like(F)
    lam = o.adjoint_seed(lat, states[-1], u - ut, F, gF)
    for t in range(T - 1, -1, -1):
        lam = o.adjoint_step(lat, states[t], lam, F, gF)
    h = 1e-7
    for _ in range(6):
        idx = tuple(RNG.integers(0, s) for s in F.shape)
        Fp, Fm = F.copy(), F.copy()
        Fp[idx] += h
        Fm[idx] -= h
        fd = (loss(Fp) - loss(Fm)) / (2 * h)
        assert abs(fd - gF[idx]) <= 1e-5 * abs(fd) + 1e-12
