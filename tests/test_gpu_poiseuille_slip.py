"""The CUDA step between halfway bounce-back walls against the closed-form
Poiseuille slip, a property that holds at any size and needs no oracle run.

Sec. III.B's no-slip rule s3 = (16 - 8 s2)/(8 - s2) is the case
Lambda = (1/s2 - 1/2)(1/s3 - 1/2) = 3/16 of the bounce-back analysis it cites
(Ginzburg & d'Humieres, Phys. Rev. E 68, 066614, 2003). For any s3 the steady
force-driven profile is the exact parabola u0 (1 - z^2/L^2) plus a uniform
slip F (16 Lambda - 3) / (24 nu); with s2b = s2 this holds at Re = 10 too
(the FP64 oracle meets it to 1e-11). The FP32 step must meet it within its
rounding: at the fixed point one half-unit rounding per step, amplified by the
slowest mode's 1 / (1 - lambda) of about 400, bounds the error by about 0.7 %
of the smallest slip here, so the bound is 2 %.
"""
import numpy as np
import pytest

import analytic as an
from gpu_common import dev, report
from paper_1801_04586_gb300 import Lattice

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice,pattern", [(19, "ab"), (19, "aa"), (27, "ab")])
def test_gpu_poiseuille_slip_closed_form(lattice, pattern):
    n, nu, F = 20, 0.1, 1e-4  # 2L = 20, u0 = F L^2 / (2 nu) = 0.05, Re = 10
    s2 = an.s2_from_nu(nu)
    ua = an.poiseuille_steady(n, F, nu)
    steps = int(40 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu))
    for s3 in (0.6, 1.2, 1.5):
        g = Lattice(32, 2, n, nu, walls=4, s2b=s2, s3=s3, lattice=lattice, pattern=pattern, device=dev())
        g.set_force_uniform(F)
        g.init_equilibrium()
        g.step(steps)
        g.check()
        ux = g.macros()[1][0].double().cpu().numpy()  # (nz, ny, nx)
        g.close()
        assert np.ptp(ux, axis=(1, 2)).max() < 1e-9  # every column is the same profile
        d = ux[:, 0, 0] - ua
        lam = (1.0 / s2 - 0.5) * (1.0 / s3 - 0.5)
        slip = F * (16.0 * lam - 3.0) / (24.0 * nu)
        report("gpu_poiseuille_slip", lattice=lattice, pattern=pattern, s3=s3, slip=slip,
               rel_err=float(d.mean() / slip - 1.0), spread=float(np.ptp(d)))
        assert abs(d.mean() / slip - 1.0) < 2e-2
        assert np.ptp(d) < 2e-2 * abs(slip)
