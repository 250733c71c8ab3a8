"""The hand-written adjoint kernel against the FP64 oracle adjoint
(complex-step Jacobians) and against central finite differences of the FP32
forward, for L = 1/2 sum |u(T) - u*|^2 as a function of a body-force field."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import W, dev, make_pair, report, t
from paper_1801_04586_gb300 import synthetic
from paper_1801_04586_gb300.autograd import final_velocity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("walls", [0, 4, 7])
def test_single_adjoint_step_matches_oracle(walls):
    nx, ny, nz = 13, 9, 7
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.03, walls=walls, s2b=1.2, s3=0.9, s4=1.3)
    h0 = synthetic.random_deviations(shape, 5e-3, seed=71)
    F = synthetic.gaussian_force(shape, 1e-3, seed=72)
    lam_next = synthetic.rng(73).normal(size=(19,) + shape).astype(np.float32)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    state = g.export_state()
    lam = g.empty(19, *shape)
    gF = torch.zeros(3, *shape, device=dev())
    g.adjoint_step(state, t(lam_next), lam, gF)
    gFo = np.zeros((3,) + shape)
    lam_o = oracle.adjoint_step(o, h0.astype(np.float64) + W, lam_next, F, gFo)
    lam_g = lam.double().cpu().numpy()
    err_l = np.max(np.abs(lam_g - lam_o)) / np.max(np.abs(lam_o))
    err_f = np.max(np.abs(gF.double().cpu().numpy() - gFo)) / np.max(np.abs(gFo))
    report("adjoint_step_vs_oracle", walls=walls, lam=float(err_l), gF=float(err_f))
    assert err_l < 1e-5
    assert err_f < 1e-5


def test_adjoint_seed_matches_oracle():
    nx, ny, nz = 11, 8, 6
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.03, walls=2)
    h0 = synthetic.random_deviations(shape, 5e-3, seed=74)
    F = synthetic.gaussian_force(shape, 1e-3, seed=75)
    gu = synthetic.rng(76).normal(size=(3,) + shape).astype(np.float32)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    lam = g.empty(19, *shape)
    gF = g.empty(3, *shape)
    g.adjoint_seed(t(gu), lam, gF)
    gFo = np.zeros((3,) + shape)
    lam_o = oracle.adjoint_seed(o, h0.astype(np.float64) + W, gu, F, gFo)
    np.testing.assert_allclose(lam.double().cpu().numpy(), lam_o, rtol=0, atol=1e-6 * np.abs(lam_o).max())
    np.testing.assert_allclose(gF.double().cpu().numpy(), gFo, rtol=0, atol=1e-6 * np.abs(gFo).max())


def _oracle_gradient(o, F, u_target, T):
    shape = o.shape
    states = [oracle.equilibrium(1.0, np.zeros(3)).reshape(19, 1, 1, 1) * np.ones((19,) + shape)]
    for _ in range(T):
        states.append(oracle.step(o, states[-1], F, 1))
    u = oracle.macros(o, states[-1], F)[1]
    gF = np.zeros((3,) + shape)
    lam = oracle.adjoint_seed(o, states[-1], u - u_target, F, gF)
    for k in range(T - 1, -1, -1):
        lam = oracle.adjoint_step(o, states[k], lam, F, gF)
    return gF, u


@pytest.mark.parametrize("walls,every", [(0, 4), (4, 5), (6, 7)])
def test_unrolled_gradient_matches_oracle(walls, every):
    """The autograd Function (forward with checkpoints, backward recomputation
    plus adjoint kernel) against the chained FP64 oracle adjoint."""
    nx, ny, nz, T = 10, 8, 6, 20
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.02, walls=walls, s2b=1.1, s3=1.2)
    F = synthetic.gaussian_force(shape, 1e-4, seed=81)
    ut = synthetic.gaussian_force(shape, 1e-3, seed=82)
    g.init_equilibrium()  # rest state, independent of F
    init = g.export_state().clone()
    Ft = t(F).requires_grad_(True)
    u = final_velocity(Ft, g, init, T, every)
    loss = 0.5 * ((u.double() - t(ut).double()) ** 2).sum()
    loss.backward()
    gFo, uo = _oracle_gradient(o, F, ut, T)
    np.testing.assert_allclose(u.detach().double().cpu().numpy(), uo, rtol=0, atol=1e-8)
    err = np.max(np.abs(Ft.grad.double().cpu().numpy() - gFo)) / np.max(np.abs(gFo))
    report("unrolled_gradient_vs_oracle", walls=walls, every=every, rel=float(err))
    assert err < 1e-4


def test_gradient_against_fp64_finite_differences_per_sample():
    """The gradient the library returns (FP32 forward with checkpoints every
    10 steps, recomputation and the adjoint kernel behind the autograd
    Function) against central differences of the FP64 oracle forward, sample
    by sample. A 12^3 periodic copy of the differentiable box: F ~ N(0,
    (1e-5)^2) per component (seed 3), nu = 0.02, 40 steps from rest, target a
    divergence-free field with max |u*| = 1e-3 (seed 4), L = 1/2 sum |u(T) -
    u*|^2 with u from Eq. 9. At 32 seeded nodes (seed 5), all three
    components: every one of the 96 samples within 1e-3 relative. The FP64
    differences carry no rounding noise at this step (L is quadratic in F up
    to O(|u|^2) relative terms, so h = 1e-7 has no visible truncation error
    either)."""
    n, nu, T, every = 12, 0.02, 40, 10
    shape = (n, n, n)
    g, o = make_pair(n, n, n, nu)
    F = synthetic.gaussian_force(shape, 1e-5, seed=3)
    ut = synthetic.divfree_velocity(shape, seed=4, umax=1e-3)
    g.init_equilibrium()
    init = g.export_state().clone()
    Ft = t(F).requires_grad_(True)
    u = final_velocity(Ft, g, init, T, every)
    (0.5 * ((u.double() - t(ut).double()) ** 2).sum()).backward()
    grad = Ft.grad.double().cpu().numpy().reshape(3, -1)
    g.close()
    f0 = np.broadcast_to(W, (19,) + shape).copy()
    F64 = F.astype(np.float64)
    ut64 = ut.astype(np.float64)

    def loss(Fv):
        f = oracle.step(o, f0, Fv, T)
        uu = oracle.macros(o, f, Fv)[1]
        return 0.5 * float(((uu - ut64) ** 2).sum())

    nodes = synthetic.rng(5).choice(n ** 3, 32, replace=False)
    h = 1e-7
    fds, ads = [], []
    for s in nodes:
        for a in range(3):
            Fp, Fm = F64.copy(), F64.copy()
            Fp.reshape(3, -1)[a, s] += h
            Fm.reshape(3, -1)[a, s] -= h
            fds.append((loss(Fp) - loss(Fm)) / (2 * h))
            ads.append(grad[a, s])
    fds, ads = np.array(fds), np.array(ads)
    rel = np.abs(ads - fds) / np.abs(fds)
    report("adjoint_vs_fp64_fd_12cube", max_rel=float(rel.max()), median_rel=float(np.median(rel)),
           min_abs_grad=float(np.abs(fds).min()), max_abs_grad=float(np.abs(fds).max()))
    assert rel.max() < 1e-3


def test_gradient_against_finite_differences_64cube():
    """The full differentiable box: 64^3 periodic, F ~ N(0, (1e-5)^2) per
    component (seed 3), nu = 0.02, 200 steps with checkpoints every 20, target
    a divergence-free field with max |u*| = 1e-3 (seed 4): dL/dF against
    central differences of the FP32 forward (FP64 loss by the library's
    reduction) at 32 seeded nodes, all three components, plus one
    random-direction derivative. The FP32 forward's rounding noise in a
    difference quotient is about 1e-3 of the smallest sampled gradients here,
    so this full-size check holds the 1e-3 tolerance in the L2 norm over the
    96 samples and pointwise relative to the largest sampled gradient; the
    per-sample 1e-3 check is the FP64 one above."""
    n, nu, T, every = 64, 0.02, 200, 20
    shape = (n, n, n)
    g, _ = make_pair(n, n, n, nu)
    F = t(synthetic.gaussian_force(shape, 1e-5, seed=3))
    ut = t(synthetic.divfree_velocity(shape, seed=4, umax=1e-3))
    g.init_equilibrium()
    init = g.export_state().clone()
    Ft = F.clone().requires_grad_(True)
    u = final_velocity(Ft, g, init, T, every)
    (0.5 * ((u.double() - ut.double()) ** 2).sum()).backward()
    grad = Ft.grad.detach()

    def loss(Fv):
        g.set_force_field(Fv)
        g.import_state(init, set_steps=0)
        g.step(T)
        _, uu = g.macros()
        return 0.5 * float(g.reduce_pair(uu, ut)[0].item())

    rng = np.random.default_rng(5)
    nodes = rng.choice(n ** 3, 32, replace=False)
    # L is quadratic in F up to O(|u|^2) ~ 1e-6 relative, so the central
    # difference has no visible truncation error even at h = 1e-5; a larger h
    # keeps the FP32 rounding noise of the forward below the signal.
    h = 1e-5
    fds, ads = [], []
    for s in nodes:
        for a in range(3):
            Fp = F.clone()
            Fm = F.clone()
            Fp.view(3, -1)[a, s] += h
            Fm.view(3, -1)[a, s] -= h
            step = float((Fp.view(3, -1)[a, s] - Fm.view(3, -1)[a, s]).item())  # exact FP32 step
            fds.append((loss(Fp) - loss(Fm)) / step)
            ads.append(float(grad.view(3, -1)[a, s].item()))
    fds, ads = np.array(fds), np.array(ads)
    l2 = float(np.linalg.norm(fds - ads) / np.linalg.norm(fds))
    # a random direction: dot product form
    v = torch.from_numpy(rng.normal(size=(3,) + shape).astype(np.float32)).to(dev())
    hv = 1e-7
    fd = (loss(F + hv * v) - loss(F - hv * v)) / (2 * hv)
    ad = float((grad.double() * v.double()).sum().item())
    rel = np.abs(fds - ads) / np.abs(fds)
    report("adjoint_vs_fd_64cube", h=h, l2_rel=l2, max_rel=float(rel.max()), median_rel=float(np.median(rel)),
           max_abs_err=float(np.abs(fds - ads).max()), max_abs_grad=float(np.abs(fds).max()),
           dir_rel=abs(fd - ad) / abs(fd))
    assert l2 < 1e-3
    assert np.abs(fds - ads).max() < 1e-3 * np.abs(fds).max()
    assert abs(fd - ad) < 1e-3 * abs(fd)
