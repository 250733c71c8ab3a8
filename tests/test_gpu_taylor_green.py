"""Space- and time-dependent forcing on the GPU: the decaying Taylor-Green
vortex of Sec. III.D (Re = 50, u0 = 0.005, 5 nodes along z, T* = 4), against
the FP64 oracle and as a grid-convergence study (the paper fits a slope of
2.0345 for L = 16..128)."""
import numpy as np
import pytest
import torch

import analytic as an
import oracle
from gpu_common import dev, make_pair, report, t

pytestmark = pytest.mark.gpu

U0, RE = 0.005, 50.0


def _setup(L, nz=5):
    nu = U0 * L / RE
    ux, uy = an.taylor_green(L, U0, nu, 0.0)
    fx, fy = an.taylor_green_force(L, U0)
    u = np.zeros((3, nz, L, L), np.float32)
    F = np.zeros((3, nz, L, L), np.float32)
    u[0], u[1] = ux, uy
    F[0], F[1] = fx, fy
    return nu, u, F


def _run_gpu(L, steps, nz=5):
    nu, u, F = _setup(L, nz)
    g, _ = make_pair(L, L, nz, nu)
    Ft = t(F)
    g.set_force_field(Ft)
    g.set_force_decay(an.taylor_green_decay(L, nu))
    g.init_equilibrium(None, t(u))
    g.step(steps)
    g.check()
    uu = g.macros()[1].double().cpu().numpy()
    g.close()
    return nu, uu


def test_taylor_green_matches_oracle():
    L = 16
    nu, u, F = _setup(L, 1)
    T = an.taylor_green_time(L, nu, 4.0)
    _, ug = _run_gpu(L, T)
    lat = oracle.Lattice.from_nu(L, L, 1, nu)
    gamma = an.taylor_green_decay(L, nu)
    f = oracle.step_decay(lat, oracle.init(lat, None, u, F), F, T, 0.0, gamma)
    _, uo = oracle.macros(lat, f, F.astype(np.float64) * np.exp(-gamma * T))
    err = np.max(np.abs(ug[:2] - uo[:2, 0][:, None])) / U0
    report("taylor_green_vs_oracle", L=L, steps=T, max_err_over_u0=float(err))
    assert err < 1e-5


def test_taylor_green_convergence():
    errs = {}
    for L in (16, 32, 64, 128):
        nu = U0 * L / RE
        T = an.taylor_green_time(L, nu, 4.0)
        _, ug = _run_gpu(L, T)
        ax, ay = an.taylor_green(L, U0, nu, T)
        num = ((ug[0] - ax[None]) ** 2 + (ug[1] - ay[None]) ** 2).sum()
        den = 5 * (ax ** 2 + ay ** 2).sum()
        errs[L] = float(np.sqrt(num / den))
    Ls = np.array(sorted(errs))
    slope = -np.polyfit(np.log(Ls), np.log([errs[L] for L in Ls]), 1)[0]
    report("taylor_green_convergence", slope=float(slope), **{f"E2_L{L}": errs[L] for L in Ls})
    assert 1.8 < slope < 2.2
