"""Pins of the oracle's Peng-Robinson EOS (Eq. 14) and chemical potential
(Eq. 15) with the paper's constants a = 2/49, b = 2/21, R = 1 and the water
acentric factor 0.344: Gibbs-Duhem between the two printed formulas, Eq. 15
against the Eq. 13 route by quadrature, the textbook PR critical constants,
alpha(T), equal areas of the Maxwell construction, and a short stable run."""
import math

import numpy as np
import pytest

import oracle as O

integrate = pytest.importorskip("scipy.integrate")

A, B, RR, W = 2.0 / 49.0, 2.0 / 21.0, 1.0, 0.344


def pr(Tr):
    return O.eos_make(O.EOS_PR, A, B, RR, Tr, W)


@pytest.mark.parametrize("Tr", [0.5, 0.7, 0.95])
def test_gibbs_duhem(Tr):
    # rho dmu/drho = dp/drho for the printed pair (a typo in either breaks it)
    e = pr(Tr)
    for rho in (0.05, 0.8, 3.0, 7.5):
        h = 1e-5 * rho
        dmu = (O.eos_mu(e, rho + h) - O.eos_mu(e, rho - h)) / (2 * h)
        dp = (O.eos_pressure(e, rho + h) - O.eos_pressure(e, rho - h)) / (2 * h)
        assert rho * dmu == pytest.approx(dp, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("Tr", [0.6, 0.9])
def test_eq15_follows_the_eq13_route(Tr):
    # psi = rho (int p0 / rho^2 drho + C) (Eq. 13) gives psi' = int p0/rho^2 drho + p0/rho:
    # differences of Eq. 15 between two densities equal that expression's
    e = pr(Tr)
    p = lambda r: O.eos_pressure(e, r)
    for r0, r1 in ((0.02, 0.5), (0.5, 6.0), (1.0, 9.0)):
        integral, _ = integrate.quad(lambda r: p(r) / (r * r), r0, r1, epsabs=0, epsrel=1e-13, limit=200)
        want = integral + p(r1) / r1 - p(r0) / r0
        assert O.eos_mu(e, r1) - O.eos_mu(e, r0) == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_critical_constants_are_the_textbook_ones():
    rc, Tc = O.pr_critical(A, B, RR)
    # Peng-Robinson: R T_c b / a = 0.17014, b rho_c = 0.25307, Z_c = 0.30740
    assert RR * Tc * B / A == pytest.approx(0.170144, abs=2e-6)
    assert B * rc == pytest.approx(0.253077, abs=2e-6)
    e = O.eos_make(O.EOS_PR, A, B, RR, 1.0, W)
    pc = O.eos_pressure(e, rc)
    assert pc / (rc * RR * Tc) == pytest.approx(0.307401, abs=2e-6)
    # p' = p'' = 0 there
    h = 1e-4 * rc
    p = lambda r: O.eos_pressure(e, r)
    assert abs(p(rc + h) - p(rc - h)) / (2 * h) < 1e-8
    assert abs(p(rc + h) - 2 * p(rc) + p(rc - h)) / (h * h) < 1e-5


def test_alpha_of_temperature():
    Tc = O.pr_critical(A, B, RR)[1]
    assert O.pr_alpha(Tc, Tc, W) == 1.0
    kap = 0.37464 + 1.54226 * W - 0.26992 * W * W
    for Tr in (0.3, 0.7, 0.9):
        assert O.pr_alpha(Tr * Tc, Tc, W) == pytest.approx((1 + kap * (1 - math.sqrt(Tr))) ** 2, rel=1e-15)
    assert pr(0.7).alpha == pytest.approx((1 + kap * (1 - math.sqrt(0.7))) ** 2, rel=1e-15)


@pytest.mark.parametrize("Tr", [0.5, 0.7, 0.9])
def test_maxwell_equal_area(Tr):
    e = pr(Tr)
    g, l = O.eos_maxwell(e)
    p = lambda r: O.eos_pressure(e, r)
    ps = p(g)
    assert abs(p(l) - ps) < 1e-11 * A * e.alpha * l * l
    integrand = lambda s_: p(math.exp(s_)) * math.exp(-s_)
    lo, hi = math.log(g), math.log(l)
    area, _ = integrate.quad(integrand, lo, hi, limit=500, epsabs=0, epsrel=1e-13)
    size, _ = integrate.quad(lambda s_: abs(integrand(s_)), lo, hi, limit=500, epsabs=0, epsrel=1e-10)
    assert abs(area - ps * (1 / g - 1 / l)) < 1e-9 * size
    assert 0 < g < e.rho_c < l < 1 / B


def test_pr_droplet_runs_and_conserves_mass():
    # PR liquid densities are ~25 times the CS ones at these constants, so
    # kappa-hat is scaled down by as much (kappa-hat >= 0.05 is unstable here)
    s = O.Sim(nx=48, ny=48, Tr=0.8, k=0.2, kappa=0.01, scheme="EFDS4", eos="PR", a=A, b=B, R=RR, acentric=W)
    s.init_droplet(12.0)
    m0 = s.density().sum()
    assert s.step(200) == 0
    rho = s.density()
    assert rho.sum() == pytest.approx(m0, rel=1e-12)
    g, l = O.eos_maxwell(pr(0.8))
    assert rho[24, 24] > 0.5 * (g + l) > rho[0, 0]
