"""Pins for the oracle's Carnahan-Starling EOS, chemical potential (Eq. 10-13)
and Maxwell construction.  Checked against numerical derivatives, the
textbook critical constants of the CS fluid, the ideal-gas limit and an
independent equal-area quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle as O

A, B, RR = 1.0, 4.0, 1.0


def test_gibbs_duhem():
    # Eq. 10 and Eq. 13 imply rho * dmu/drho = dp0/drho; central differences
    T = 0.07
    for rho in np.linspace(0.01, 0.7, 25):
        h = 1e-6 * rho
        dmu = (O.cs_mu(rho + h, A, B, RR, T) - O.cs_mu(rho - h, A, B, RR, T)) / (2 * h)
        dp = (O.cs_pressure(rho + h, A, B, RR, T) - O.cs_pressure(rho - h, A, B, RR, T)) / (2 * h)
        assert rho * dmu == pytest.approx(dp, rel=1e-7, abs=1e-10)


def test_ideal_gas_limit():
    # a = 0 and vanishing co-volume: p0 -> rho R T and mu -> R T ln rho (up to a constant)
    T = 0.3
    for rho in (1e-3, 0.1, 2.0):
        assert O.cs_pressure(rho, 0.0, 1e-12, RR, T) == pytest.approx(rho * RR * T, rel=1e-10)
        assert O.cs_mu(rho, 0.0, 1e-12, RR, T) == pytest.approx(RR * T * math.log(rho), abs=1e-10)


def test_critical_point():
    rc, Tc = O.cs_critical(A, B, RR)
    # textbook CS critical constants: eta_c = b rho_c / 4 = 0.1304, R T_c b / a = 0.3773
    assert B * rc / 4 == pytest.approx(0.13044, abs=2e-5)
    assert RR * Tc * B / A == pytest.approx(0.37731, abs=2e-5)
    # and independently: dp/drho and d2p/drho2 vanish there (numerical derivatives)
    h = 1e-4
    p = lambda r: O.cs_pressure(r, A, B, RR, Tc)
    d1 = (p(rc + h / 10) - p(rc - h / 10)) / (2 * h / 10)
    d2 = (p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2
    assert abs(d1) < 1e-9 and abs(d2) < 1e-5
    # scaling: Tc proportional to a/b, rho_c to 1/b
    rc2, Tc2 = O.cs_critical(2.0, 2.0, 1.0)
    assert rc2 == pytest.approx(rc * 2, rel=1e-12) and Tc2 == pytest.approx(Tc * 4, rel=1e-12)


@pytest.mark.parametrize("Tr", [0.95, 0.9, 0.8, 0.7, 0.5, 0.3, 0.2])
def test_maxwell_equal_area(Tr):
    Tc = O.cs_critical(A, B, RR)[1]
    T = Tr * Tc
    g, l = O.maxwell(T, A, B, RR)
    p = lambda r: O.cs_pressure(r, A, B, RR, T)
    ps = p(g)  # the gas pressure has no cancellation; p(l) is a difference of O(a l^2) terms
    # compare the two phase pressures on the scale of those terms
    scale = A * l * l
    assert abs(p(l) - ps) < 1e-13 * scale
    # equal areas in the p-v plane: int_{v_l}^{v_g} p dv = p_sat (v_g - v_l).  With
    # v = 1/rho and rho = e^s: int p(e^s) e^-s ds over [ln g, ln l].
    integrand = lambda s_: p(math.exp(s_)) * math.exp(-s_)
    mag = lambda s_: abs(integrand(s_))
    lo, hi = math.log(g), math.log(l)
    area, _ = integrate.quad(integrand, lo, hi, limit=500, epsabs=0, epsrel=1e-13)
    size, _ = integrate.quad(mag, lo, hi, limit=500, epsabs=0, epsrel=1e-10)
    assert abs(area - ps * (1 / g - 1 / l)) < 1e-9 * size
    # ordering: gas below the spinodal, liquid above
    assert 0 < g < O.cs_critical(A, B, RR)[0] < l < 4 / B


def test_maxwell_approaches_critical():
    rc, Tc = O.cs_critical(A, B, RR)
    g, l = O.maxwell(0.9999 * Tc, A, B, RR)
    assert abs(g - rc) < 0.03 * rc and abs(l - rc) < 0.03 * rc
    with pytest.raises(ValueError):
        O.maxwell(1.01 * Tc, A, B, RR)
