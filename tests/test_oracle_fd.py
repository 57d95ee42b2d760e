"""Pins for the oracle's difference operators (Sec. 2.3, Eq. 17-28, Table 1).

Each test checks the oracle against something the paper or mathematics fixes
independently of the oracle's code: the exact single-mode response of Eq. 28,
the truncation constants of Table 1, a dense linear solve of the periodic
compact system, and the order of isotropy of Eq. 25.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _frac(p):
    return Fraction(p[0], p[1])


def printed_coeffs(s):
    """(alpha, a, b, c) as printed in the paper, not taken from the oracle."""
    if s in GOLD["compact_coefficients"]:
        d = GOLD["compact_coefficients"][s]
        return tuple(float(_frac(d[k])) for k in ("alpha", "a", "b", "c"))
    if s in GOLD["explicit_coefficients"]:
        d = GOLD["explicit_coefficients"][s]
        return (0.0,) + tuple(float(_frac(d[k])) for k in ("a", "b", "c"))
    d = GOLD["ocfds4"]
    return (d["alpha"], d["a"], d["b"], d["c"])


LINE_SCHEMES = ["EFDS2", "EFDS4", "EFDS6", "CFDS4", "CFDS6", "CFDS8", "OCFDS4"]


def taylor_ocfds4():
    """OCFDS4 with the printed alpha and c, and a, b from the two fourth-order
    Taylor conditions of Eq. 21 (a + b + c = 1 + 2 alpha, a + 4b + 9c = 6 alpha)."""
    d = GOLD["ocfds4"]
    al, c = d["alpha"], d["c"]
    A = np.array([[1.0, 1.0], [1.0, 4.0]])
    a, b = np.linalg.solve(A, [1 + 2 * al - c, 6 * al - 9 * c])
    return al, a, b, c


def modified_wavenumber(s, w):
    """Eq. 28 (beta = 0): w' = (a sin w + b/2 sin 2w + c/3 sin 3w) / (1 + 2 alpha cos w)."""
    al, a, b, c = taylor_ocfds4() if s == "OCFDS4" else printed_coeffs(s)
    return (a * np.sin(w) + b / 2 * np.sin(2 * w) + c / 3 * np.sin(3 * w)) / (1 + 2 * al * np.cos(w))


@pytest.mark.parametrize("s", LINE_SCHEMES)
@pytest.mark.parametrize("n", [16, 37, 64])
def test_single_mode_response_eq28(s, n):
    # On a periodic grid a single Fourier mode is an eigenvector of every
    # scheme: D sin(w j) = w'(w) cos(w j) exactly (Eq. 27-28).
    j = np.arange(n)
    for m in range(1, n // 2):
        w = 2 * np.pi * m / n
        d = O.deriv_line(s, np.sin(w * j))
        expect = modified_wavenumber(s, w) * np.cos(w * j)
        assert np.max(np.abs(d - expect)) < 1e-13, (s, n, m)


def test_coefficients_match_paper():
    for s in LINE_SCHEMES:
        al, a, b, c = O.scheme_coeffs(s)
        pal, pa, pb, pc = printed_coeffs(s)
        if s == "OCFDS4":
            # printed a = 1.541, b = 0.40667: the oracle's values round to them
            assert round(a, 3) == pa and round(b, 5) == pb and al == pal and c == pc
            # and satisfy the fourth-order conditions of Eq. 21 exactly
            assert abs(a + b + c - (1 + 2 * al)) < 1e-15
            assert abs(a + 4 * b + 9 * c - 6 * al) < 1e-14
        else:
            assert (al, a, b, c) == pytest.approx((pal, pa, pb, pc), abs=1e-16)


def test_alpha_family_formulas():
    # Sec. 2.3.2: the 4th-order family a = 2(alpha+2)/3, b = (4alpha-1)/3 gives Eq. 22 at
    # alpha = 1/4 and Eq. 23 at alpha = 1/3; the 6th-order family gives Eq. 24 at 3/8.
    for s, al in (("CFDS4", Fraction(1, 4)), ("CFDS6", Fraction(1, 3))):
        d = GOLD["compact_coefficients"][s]
        assert _frac(d["a"]) == 2 * (al + 2) / 3 and _frac(d["b"]) == (4 * al - 1) / 3
    al = Fraction(3, 8)
    d = GOLD["compact_coefficients"]["CFDS8"]
    assert _frac(d["a"]) == (al + 9) / 6 and _frac(d["b"]) == (32 * al - 9) / 15 and _frac(d["c"]) == (1 - 3 * al) / 10


def derivative_constant(s):
    """Leading derivative error constant C in D f - f' = C h^p f^(p+1).

    Table 1 lists the truncation error of the relation Eq. 21; for a compact
    scheme the derivative error is that divided by the left operator's symbol
    at zero wavenumber, 1 + 2 alpha.  For OCFDS4 the paper prints the formula
    (12 b + 72 c - 4 alpha)/5!."""
    al = printed_coeffs(s)[0]
    if s == "OCFDS4":
        _, a, b, c = printed_coeffs(s)
        return 4, (12 * b + 72 * c - 4 * al) / 120 / (1 + 2 * al)
    t = GOLD["table1_truncation"][s]
    return t["order"], float(_frac(t["coef"])) / (1 + 2 * al)


@pytest.mark.parametrize("s", LINE_SCHEMES)
def test_convergence_order_and_table1_constant(s):
    p, C = derivative_constant(s)
    n0 = {2: 256, 4: 128, 6: 64, 8: 32}[p]
    errs = []
    for n in (n0, 2 * n0):
        h = 2 * np.pi / n
        x = h * np.arange(n)
        d = O.deriv_line(s, np.sin(x)) / h
        # f = sin: f^(p+1) = (-1)^(p/2) cos for even p
        fp1 = (-1) ** (p // 2) * np.cos(x)
        ratio = (d - np.cos(x))[0] / (h ** p * fp1[0])
        errs.append((h, np.max(np.abs(d - np.cos(x))), ratio))
    order = math.log(errs[0][1] / errs[1][1]) / math.log(2)
    assert abs(order - p) < 0.15, (s, order)
    assert errs[1][2] == pytest.approx(C, rel=0.03), (s, errs[1][2], C)


@pytest.mark.parametrize("s", ["CFDS4", "CFDS6", "CFDS8", "OCFDS4"])
@pytest.mark.parametrize("n", [7, 8, 11, 16])
def test_compact_dense_solve(s, n):
    # Brute force: assemble the periodic system of Eq. 21 (beta = 0) as dense
    # circulant matrices and solve it with LAPACK.
    al, a, b, c = O.scheme_coeffs(s)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for i in range(n):
        A[i, i] += 1
        A[i, (i + 1) % n] += al
        A[i, (i - 1) % n] += al
        for m, coef in ((1, a / 2), (2, b / 4), (3, c / 6)):
            B[i, (i + m) % n] += coef
            B[i, (i - m) % n] -= coef
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n)
    expect = np.linalg.solve(A, B @ f)
    assert np.max(np.abs(O.deriv_line(s, f) - expect)) < 1e-13


def _plane_wave_angle(scheme, j, n=512, mx=2, my=1):
    x = np.arange(n)
    kx, ky = 2 * np.pi * mx * j / n, 2 * np.pi * my * j / n
    phi = np.sin(kx * x[None, :] + ky * x[:, None])
    g = O.gradient(scheme, phi)
    gx, gy = g[0][0, 0], g[1][0, 0]  # phase 0: gradient along k
    return abs(math.atan2(gy, gx) - math.atan2(ky, kx)), math.hypot(kx, ky)


@pytest.mark.parametrize("scheme,order", [("EFDS2", 2), ("EFDS4", 4), ("E4", 4), ("E8", 8)])
def test_isotropy_order_of_gradient(scheme, order):
    # Eq. 25 with isotropic weights: the direction of the discrete gradient of a
    # plane wave deviates from the wave vector at O(k^order) (E4: the rank-4
    # moment is isotropic; E8: moments to rank 8; explicit line schemes: only
    # rank 2).  Measured slope of the angle deviation must match.
    a1, k1 = _plane_wave_angle(scheme, 8)
    a2, k2 = _plane_wave_angle(scheme, 16)
    slope = math.log(a2 / a1) / math.log(k2 / k1)
    assert abs(slope - order) < 0.3, (scheme, slope)


def test_e4_weights_printed():
    # Gradient of a unit spike at the origin: node e receives -w(|e|^2) e (Eq. 25a)
    n = 9
    phi = np.zeros((n, n))
    phi[0, 0] = 1.0
    g = O.gradient("E4", phi)
    w1 = float(_frac(GOLD["e4_weights"]["w1"]))
    w2 = float(_frac(GOLD["e4_weights"]["w2"]))
    # node (x=-1, y=0) sees the spike at offset e = (+1, 0): g_x = w(1) * 1
    assert g[0][0, n - 1] == pytest.approx(w1, abs=1e-16)
    assert g[0][n - 1, n - 1] == pytest.approx(w2, abs=1e-16)
    assert g[1][n - 1, n - 1] == pytest.approx(w2, abs=1e-16)


def test_e8_first_moment_and_3d_e4():
    # consistency: the isotropic gradient of a long-wave plane wave approaches k
    for scheme, shape in (("E8", (256, 256)), ("E4", (64, 64, 64))):
        n = shape[0]
        x = np.arange(n)
        k = 2 * np.pi / n
        if len(shape) == 2:
            phi = np.sin(k * x)[None, :] * np.ones(shape)
        else:
            phi = np.sin(k * x)[None, None, :] * np.ones(shape)
        g = O.gradient(scheme, phi)
        assert abs(g[0].flat[0] - k) < 2e-3 * k


@pytest.mark.parametrize("s,order", [("EFDS2", 2), ("EFDS4", 4), ("EFDS6", 6), ("CFDS8", 8), ("E4", 2), ("E8", 2)])
def test_laplacian_order(s, order):
    # Laplacian paired with each scheme: convergence to -k^2 sin for a
    # single mode; EFDS2's 3-point stencil equals -4 sin^2(w/2) exactly.
    errs = []
    n0 = {2: 128, 4: 64, 6: 32, 8: 16}[order]
    for n in (n0, 2 * n0):
        h = 2 * np.pi / n
        x = h * np.arange(n)
        phi = np.sin(x)[None, :] * np.ones((n, n))
        lap = O.laplacian(s, phi) / h ** 2
        errs.append(np.max(np.abs(lap[0] + np.sin(x))))
        if s == "EFDS2":
            w = h
            assert np.max(np.abs(O.laplacian(s, phi)[0] + 4 * np.sin(w / 2) ** 2 * np.sin(x))) < 1e-14
    p = math.log(errs[0] / errs[1]) / math.log(2)
    assert abs(p - order) < 0.2, (s, p)


def test_laplacian_isotropic_e4_plane_wave():
    # Eq. 25b: the E4 Laplacian of a plane wave is isotropic to O(k^4): two
    # directions with equal |k| give responses that agree to O(k^6).
    n = 400
    x = np.arange(n)
    res = []
    for (mx, my) in ((5, 0), (3, 4)):  # |m| = 5 in both
        kx, ky = 2 * np.pi * mx / n, 2 * np.pi * my / n
        phi = np.cos(kx * x[None, :] + ky * x[:, None])
        res.append(O.laplacian("E4", phi)[0, 0])
    k2 = (2 * np.pi * 5 / n) ** 2
    assert abs(res[0] - res[1]) < 0.05 * k2 ** 3
    assert res[0] == pytest.approx(-k2, rel=0.01)
