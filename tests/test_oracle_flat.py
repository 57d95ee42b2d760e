"""Pins of the oracle's equilibrium flat interface (Eq. 29) and the
derivative-error study built on it (Sec. 3.1, Fig. 3(a)).

The profile is checked against the equilibrium equation itself (uniform
chemical potential, Eq. 16, by sixth-order differences on a 16x finer
sampling), the bulk Maxwell densities at its ends, its midpoint, the
derivative it reports, and the 1/k scaling of the interface width (Fig. 4
inset).  The study reproduces the paper's statements: every scheme's error
falls as k falls; at the largest k the optimal compact scheme is the most
accurate; at small k the highest-order schemes are; the second-order scheme
deviates most."""
import numpy as np
import pytest

import oracle as O

Tr, KAP = 0.6, 0.1


def fine(k, n=64, y0=31.5, m=16):
    # rho(y) at y = j / m: the profile depends on k y / sqrt(kappa) only
    return O.flat_profile(n * m, y0 * m, Tr, k / m, KAP)


@pytest.mark.parametrize("k", [0.4, 0.2])
def test_profile_satisfies_uniform_chemical_potential(k):
    m = 16
    rho, _ = fine(k, m=m)
    h = 1.0 / m
    c = np.array([2, -27, 270, -490, 270, -27, 2]) / 180.0
    d2 = sum(c[i] * rho[i:len(rho) - 6 + i] for i in range(7)) / (h * h)
    r = rho[3:-3]
    mu = np.array([O.cs_mu(x, 1.0, 4.0, 1.0, Tr * O.cs_critical()[1]) for x in r])
    g = O.maxwell_tr(Tr)[0]
    mug = O.cs_mu(g, 1.0, 4.0, 1.0, Tr * O.cs_critical()[1])
    resid = k * k * (mu - mug) - KAP * d2
    scale = np.max(np.abs(k * k * (mu - mug)))
    assert np.max(np.abs(resid)) < 2e-6 * scale


def test_ends_midpoint_and_reported_derivative():
    g, l = O.maxwell_tr(Tr)
    rho, d = O.flat_profile(96, 48.0, Tr, 0.3, KAP)
    assert rho[0] == pytest.approx(g, rel=1e-9) and rho[-1] == pytest.approx(l, rel=1e-9)
    assert rho[48] == pytest.approx(0.5 * (g + l), rel=1e-12)
    m = 16
    rf, df = fine(0.3, n=96, y0=48.0, m=m)
    c = np.array([-1, 9, -45, 0, 45, -9, 1]) / 60.0
    d1 = sum(c[i] * rf[i:len(rf) - 6 + i] for i in range(7)) * m
    # df is per fine node (the fine profile is the same curve at k / m)
    assert np.max(np.abs(d1 - m * df[3:-3])) < 1e-7 * np.max(m * df)


def test_interface_width_scales_as_one_over_k():
    # rho(y; k) = rho(2 y; k / 2): node j at k = 0.2 is node 2 j at k = 0.1
    r1, _ = O.flat_profile(64, 31.5, Tr, 0.2, KAP)
    r2, _ = O.flat_profile(128, 63.0, Tr, 0.1, KAP)
    assert np.allclose(r1, r2[::2], rtol=1e-9, atol=0)


def periodic(n, k):
    half = n // 2
    r, d = O.flat_profile(half, half / 2 - 0.5, Tr, k, KAP)
    return np.concatenate([r, r[::-1]]), np.concatenate([d, -d[::-1]])


def errors(k):
    rho, dr = periodic(256, k)
    return {s: np.max(np.abs(O.deriv_line(s, rho) - dr)) / np.max(np.abs(dr))
            for s in ("EFDS2", "EFDS4", "EFDS6", "CFDS4", "CFDS6", "CFDS8", "OCFDS4")}


def test_derivative_errors_reproduce_fig3a():
    e = {k: errors(k) for k in (0.4, 0.3, 0.2, 0.1)}
    for s in e[0.4]:
        assert e[0.4][s] > e[0.3][s] > e[0.2][s] > e[0.1][s], s  # error falls with k
    assert min(e[0.4], key=e[0.4].get) == "OCFDS4"              # resolution wins at large k
    assert min(e[0.1], key=e[0.1].get) == "CFDS8"               # order wins at small k
    for k in e:
        assert max(e[k], key=e[k].get) == "EFDS2"               # the second-order scheme deviates most
