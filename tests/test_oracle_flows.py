"""Pins of the oracle against closed-form flows: shear-wave viscosity
(Sec. III.A), Poiseuille flow with the no-slip rule (Sec. III.B) and the
square duct (Sec. III.C).

Paper: Fei, Luo & Li, arXiv:1801.04586.
"""
import numpy as np
import pytest

import analytic as an
import oracle as o


def _shear_wave_nu(L, nu, s2b=None, t1=200, t2=2200):
    s2 = an.s2_from_nu(nu)
    lat = o.Lattice(1, L, 1, s2=s2, s2b=s2b if s2b is not None else 1.0)
    y = np.arange(L)
    u = np.zeros((3, 1, L, 1))
    u[0, 0, :, 0] = 1e-4 * np.sin(2 * np.pi * y / L)
    f = o.step(lat, o.init(lat, None, u), None, t1)
    a1 = an.shear_wave_amplitude(o.macros(lat, f)[1][0, 0, :, 0])
    f = o.step(lat, f, None, t2 - t1)
    a2 = an.shear_wave_amplitude(o.macros(lat, f)[1][0, 0, :, 0])
    return np.log(a1 / a2) / ((2 * np.pi / L) ** 2 * (t2 - t1))


@pytest.mark.parametrize("nu,s2b", [(0.05, None), (0.1, 0.5)])
def test_shear_wave_viscosity(nu, s2b):
    """Decay of a shear wave measures nu = (1/s2 - 1/2) cs^2 (Sec. II.B) within
    0.1% on L = 101 (the paper reports 0.08% on 5 x 101 x 5); the bulk rate s2b
    does not enter a shear wave."""
    assert _shear_wave_nu(101, nu, s2b) == pytest.approx(nu, rel=1e-3)


def _poiseuille(n, nu, steps, s3=None, s2b=None, F=1e-6):
    s2 = an.s2_from_nu(nu)
    lat = o.Lattice(1, 1, n, walls=4, s2=s2, s2b=s2b if s2b is not None else 1.0,
                    s3=s3 if s3 is not None else 1.0)
    Ff = np.zeros((3, n, 1, 1))
    Ff[0] = F
    f = o.step(lat, o.init(lat, None, None, Ff), Ff, steps)
    return o.macros(lat, f, Ff)[1][0, :, 0, 0]


def _e2(u, ua):
    """Global relative error of Sec. III.B."""
    return float(np.sqrt(((u - ua) ** 2).sum() / (ua ** 2).sum()))


@pytest.mark.parametrize("nu", [0.1, 0.2])
def test_poiseuille_noslip_rule_is_exact(nu):
    """Sec. III.B: with s3 = (16 - 8 s2)/(8 - s2) and s2b = s2 the steady
    Poiseuille profile of the consistent forcing scheme carries no numerical slip
    (E2 'negligible'); with s3 = 1 it does."""
    n, F = 20, 1e-6
    s2 = an.s2_from_nu(nu)
    ua = an.poiseuille_steady(n, F, nu)
    steps = int(30 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu))
    exact = _poiseuille(n, nu, steps, s3=an.noslip_s3(s2), s2b=s2, F=F)
    assert _e2(exact, ua) < 1e-8
    slip = _poiseuille(n, nu, steps, s3=1.0, s2b=s2, F=F)
    assert _e2(slip, ua) > 1e-5


def test_poiseuille_startup_series():
    """Force-driven start-up from rest in a 32-node channel at nu = 0.1,
    F = 1e-6 (the shape of the 16 x 32 x 32 channel along z), 2000 steps,
    against the eigen-expansion of the Sec. III.B parabola."""
    n, nu, F, t = 32, 0.1, 1e-6, 2000
    ua = an.poiseuille_startup(n, F, nu, t)
    assert _e2(_poiseuille(n, nu, t, F=F), ua) < 5e-4
    s2 = an.s2_from_nu(nu)
    assert _e2(_poiseuille(n, nu, t, s3=an.noslip_s3(s2), s2b=s2, F=F), ua) < 1e-4


@pytest.mark.parametrize("q,nu", [(19, 0.05), (19, 0.1), (19, 0.2), (27, 0.1)])
def test_poiseuille_slip_closed_form(q, nu):
    """Sec. III.B's no-slip rule s3 = (16 - 8 s2)/(8 - s2) is the case
    Lambda = (1/s2 - 1/2)(1/s3 - 1/2) = 3/16 of the bounce-back analysis it
    cites (Ginzburg & d'Humieres, Phys. Rev. E 68, 066614, 2003): for any
    s3, the steady profile between halfway bounce-back walls is the exact
    parabola plus a uniform slip F (16 Lambda - 3) / (24 nu). On D3Q27 the
    rate s3b of the k111 group (Eq. 13) does not enter."""
    n, F = 20, 1e-6
    s2 = an.s2_from_nu(nu)
    ua = an.poiseuille_steady(n, F, nu)
    steps = int(40 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu))
    Ff = np.zeros((3, n, 1, 1))
    Ff[0] = F
    for s3 in (0.6, 0.9, 1.2, 1.5):
        lam = (1.0 / s2 - 0.5) * (1.0 / s3 - 0.5)
        lat = o.Lattice(1, 1, n, walls=4, s2=s2, s2b=s2, s3=s3, q=q, s3b=1.7 if q == 27 else 1.0)
        f = o.step(lat, o.init(lat, None, None, Ff), Ff, steps)
        d = o.macros(lat, f, Ff)[1][0, :, 0, 0] - ua
        assert d.max() - d.min() < 1e-13
        assert d.mean() == pytest.approx(F * (16.0 * lam - 3.0) / (24.0 * nu), rel=1e-6, abs=1e-14)


def test_poiseuille_error_linear_in_bulk_viscosity_offset():
    """Sec. III.B, on the separate trace rate of Eq. 13: at nu = 0.1 with the
    no-slip s3, the steady Poiseuille error E2 vanishes at xi = 2 nu / 3
    (s2b = s2) and grows in proportion to |xi - 2 nu / 3| on both sides.
    Re = 2 u0 L / nu = 10 (F = 1e-4, 2L = 20); xi = (2/3)(1/s2b - 1/2) c_s^2."""
    n, nu, F = 20, 0.1, 1e-4
    s2 = an.s2_from_nu(nu)
    ua = an.poiseuille_steady(n, F, nu)
    steps = int(30 * 4 * (n / 2) ** 2 / (np.pi ** 2 * nu))
    xi0 = 2.0 * nu / 3.0
    ratios = np.array([0.5, 0.75, 1.0, 1.5, 2.0, 3.0])  # xi / xi0
    e2 = []
    for r in ratios:
        s2b = 1.0 / (r * xi0 / (2.0 / 9.0) + 0.5)
        e2.append(_e2(_poiseuille(n, nu, steps, s3=an.noslip_s3(s2), s2b=s2b, F=F), ua))
    e2 = np.array(e2)
    at = ratios == 1.0
    assert e2[at][0] < 1e-11
    slope = e2[~at] / np.abs(ratios[~at] - 1.0)
    assert slope.min() > 1e-7
    np.testing.assert_allclose(slope, slope.mean(), rtol=1e-2)


def test_square_duct_series():
    """Sec. III.C duct at nu = 0.2, Fx = 2e-4 on a 16 x 16 cross-section: the
    steady series is met within 0.15% with the no-slip s3 (16/13 at nu = 0.2),
    and less well with s3 = 1 (the rule is only approximate in 2D)."""
    n, nu, F = 16, 0.2, 2e-4
    s2 = an.s2_from_nu(nu)
    ua = an.duct_steady(n, F, nu)
    errs = []
    for s3 in (an.noslip_s3(s2), 1.0):
        lat = o.Lattice(1, n, n, walls=6, s2=s2, s2b=s2, s3=s3)
        Ff = np.zeros((3, n, n, 1))
        Ff[0] = F
        f = o.step(lat, o.init(lat, None, None, Ff), Ff, 5500)
        errs.append(_e2(o.macros(lat, f, Ff)[1][0, :, :, 0], ua))
    assert errs[0] < 1.5e-3
    assert errs[1] > 2 * errs[0]


def test_noslip_rule_constants():
    """The two cases of Sec. III.B: nu = 0.1 gives s2 = 5/4 and s3 = 8/9;
    nu = 0.2 gives s2 = 10/11 (printed as 20/11) and s3 = 16/13 = 1.23077
    (printed as 1.33077 in Sec. III.C)."""
    assert an.s2_from_nu(0.1) == pytest.approx(5 / 4)
    assert an.noslip_s3(5 / 4) == pytest.approx(8 / 9)
    assert an.s2_from_nu(0.2) == pytest.approx(10 / 11)
    assert an.noslip_s3(10 / 11) == pytest.approx(16 / 13)


def test_duct_cross_section_error_minimal_near_the_noslip_rate():
    """Sec. III.C: the local error E(z) over a duct cross-section is smallest
    near the no-slip s3 for the central and intermediate sections (the rule
    is exact only for unidirectional flow, so near, not at: the scan's
    minimum sits at 1.18-1.23). At nu = 0.2 that rate is 16/13 = 1.23077;
    the paper prints 1.33077, whose error is at least 1.3 times larger
    (reading of the printed value)."""
    n, nu, F = 16, 0.2, 2e-4
    s2 = an.s2_from_nu(nu)
    target = an.noslip_s3(s2)
    assert target == pytest.approx(16 / 13, rel=1e-12)
    ua = an.duct_steady(n, F, nu)
    Ff = np.zeros((3, n, n, 1))
    Ff[0] = F
    steps = int(24 * n * n / (np.pi ** 2 * nu))
    sections = (n // 2, n // 2 + 3)  # z = 0.5 and 3.5 spacings from the centre
    E = {}
    for s3 in (1.10, 1.18, target, 1.28, 1.33077, 1.40):
        lat = o.Lattice(1, n, n, walls=6, s2=s2, s2b=s2, s3=s3)
        ux = o.macros(lat, o.step(lat, o.init(lat, None, None, Ff), Ff, steps), Ff)[1][0, :, :, 0]
        E[s3] = [np.sqrt(((ux[z] - ua[z]) ** 2).sum() / (ua[z] ** 2).sum()) for z in sections]
    for k in range(len(sections)):
        best = min(e[k] for e in E.values())
        assert E[target][k] < 1.25 * best
        assert E[1.33077][k] > 1.3 * E[target][k]
