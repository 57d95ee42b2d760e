"""Pins of the oracle's van der Waals and Redlich-Kwong-Soave EOS, whose
chemical potentials follow from Eq. 13 (the paper prints only PR, Eq. 14-15):
Gibbs-Duhem, the Eq. 13 quadrature route, the closed-form critical constants
(VDW: b rho_c = 1/3, R T_c b / a = 8/27, Z_c = 3/8; RKS: b rho_c = 2^(1/3) - 1,
Z_c = 1/3), alpha(T_c) = 1, and equal areas of the Maxwell construction."""
import math

import pytest

import oracle as O

integrate = pytest.importorskip("scipy.integrate")

CASES = {O.EOS_VDW: (9.0 / 49.0, 2.0 / 21.0), O.EOS_RKS: (2.0 / 49.0, 2.0 / 21.0)}


def eos(kind, Tr):
    a, b = CASES[kind]
    return O.eos_make(kind, a, b, 1.0, Tr, 0.344)


@pytest.mark.parametrize("kind", [O.EOS_VDW, O.EOS_RKS])
@pytest.mark.parametrize("Tr", [0.5, 0.8, 0.95])
def test_gibbs_duhem(kind, Tr):
    e = eos(kind, Tr)
    for x in (0.01, 0.1, 0.3, 0.6):
        rho = x / CASES[kind][1]
        h = 1e-5 * rho
        dmu = (O.eos_mu(e, rho + h) - O.eos_mu(e, rho - h)) / (2 * h)
        dp = (O.eos_pressure(e, rho + h) - O.eos_pressure(e, rho - h)) / (2 * h)
        assert rho * dmu == pytest.approx(dp, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("kind", [O.EOS_VDW, O.EOS_RKS])
def test_mu_follows_the_eq13_route(kind):
    e = eos(kind, 0.7)
    p = lambda r: O.eos_pressure(e, r)
    b = CASES[kind][1]
    for x0, x1 in ((0.01, 0.2), (0.2, 0.7)):
        r0, r1 = x0 / b, x1 / b
        integral, _ = integrate.quad(lambda r: p(r) / (r * r), r0, r1, epsabs=0, epsrel=1e-13, limit=200)
        want = integral + p(r1) / r1 - p(r0) / r0
        assert O.eos_mu(e, r1) - O.eos_mu(e, r0) == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_critical_constants():
    a, b = CASES[O.EOS_VDW]
    rc, Tc = O.cubic_critical(O.EOS_VDW, a, b, 1.0)
    assert b * rc == pytest.approx(1.0 / 3.0, abs=1e-12)
    assert Tc * b / a == pytest.approx(8.0 / 27.0, abs=1e-12)
    e = eos(O.EOS_VDW, 1.0)
    assert O.eos_pressure(e, rc) / (rc * Tc) == pytest.approx(3.0 / 8.0, abs=1e-12)
    a, b = CASES[O.EOS_RKS]
    rc, Tc = O.cubic_critical(O.EOS_RKS, a, b, 1.0)
    x = 2 ** (1.0 / 3.0) - 1
    assert b * rc == pytest.approx(x, abs=1e-12)
    e = eos(O.EOS_RKS, 1.0)
    assert e.alpha == 1.0
    assert O.eos_pressure(e, rc) / (rc * Tc) == pytest.approx(1.0 / 3.0, abs=1e-12)


@pytest.mark.parametrize("kind", [O.EOS_VDW, O.EOS_RKS])
@pytest.mark.parametrize("Tr", [0.6, 0.9])
def test_maxwell_equal_area(kind, Tr):
    e = eos(kind, Tr)
    g, l = O.eos_maxwell(e)
    p = lambda r: O.eos_pressure(e, r)
    ps = p(g)
    integrand = lambda s_: p(math.exp(s_)) * math.exp(-s_)
    lo, hi = math.log(g), math.log(l)
    area, _ = integrate.quad(integrand, lo, hi, limit=500, epsabs=0, epsrel=1e-13)
    size, _ = integrate.quad(lambda s_: abs(integrand(s_)), lo, hi, limit=500, epsabs=0, epsrel=1e-10)
    assert abs(area - ps * (1 / g - 1 / l)) < 1e-9 * size
    assert 0 < g < e.rho_c < l < 1 / CASES[kind][1]
