"""Pins for the oracle's LBM step: lattices (Eq. 2), equilibrium (Eq. 6),
exact-difference forcing (Eq. 8), collision and streaming, and whole-run
invariants (mass, symmetry, fixed points, shear-wave decay, coexistence)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_d2q9_matches_eq2():
    e, w = O.lattice(O.D2Q9)
    assert tuple(e[0]) == (0, 0, 0)
    for i in range(1, 5):
        ang = (i - 1) * math.pi / 2
        assert (e[i][0], e[i][1]) == (round(math.cos(ang)), round(math.sin(ang)))
    for i in range(5, 9):
        ang = (2 * i - 9) * math.pi / 4
        assert (e[i][0], e[i][1]) == (round(math.sqrt(2) * math.cos(ang)), round(math.sqrt(2) * math.sin(ang)))
    g = GOLD["d2q9_weights"]
    assert w[0] == pytest.approx(g["w0"][0] / g["w0"][1], abs=1e-16)
    assert np.allclose(w[1:5], g["w1_4"][0] / g["w1_4"][1], atol=1e-16)
    assert np.allclose(w[5:9], g["w5_8"][0] / g["w5_8"][1], atol=1e-16)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_lattice_isotropy(lat):
    e, w = O.lattice(lat)
    d = 2 if lat == O.D2Q9 else 3
    e = e[:, :d].astype(float)
    assert w.sum() == pytest.approx(1, abs=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), np.eye(d) / 3, atol=1e-16)
    I = np.eye(d)
    iso4 = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), iso4, atol=1e-16)
    # opposite directions exist for every velocity
    for v in e:
        assert any(np.array_equal(-v, u) for u in e)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_equilibrium_moments(lat):
    e, w = O.lattice(lat)
    d = 2 if lat == O.D2Q9 else 3
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = rng.uniform(0.01, 1)
        u = np.zeros(3)
        u[:d] = rng.uniform(-0.1, 0.1, d)
        f = O.feq(lat, rho, u)
        E = e.astype(float)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(E.T @ f, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, E, E)[:d, :d]
        assert np.allclose(P, rho / 3 * np.eye(d) + rho * np.outer(u[:d], u[:d]), atol=1e-15)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19])
def test_edm_moments(lat):
    # Eq. 8: sum F_i = 0 and sum e_i F_i = F (the force adds exactly F to the momentum)
    e, _ = O.lattice(lat)
    d = 2 if lat == O.D2Q9 else 3
    rng = np.random.default_rng(2)
    for _ in range(5):
        rho = rng.uniform(0.01, 1)
        u = np.zeros(3)
        F = np.zeros(3)
        u[:d] = rng.uniform(-0.1, 0.1, d)
        F[:d] = rng.uniform(-0.01, 0.01, d)
        Fi = O.edm(lat, rho, u, F)
        assert abs(Fi.sum()) < 1e-16
        assert np.allclose(e.astype(float).T @ Fi, F, atol=1e-16)


def test_uniform_state_is_fixed_point():
    for lat, shape in ((O.D2Q9, (12, 10, 1)), (O.D3Q19, (6, 7, 5))):
        s = O.Sim(lattice=lat, nx=shape[0], ny=shape[1], nz=shape[2], Tr=0.7, k=0.3, kappa=0.1, scheme="EFDS2")
        s.init_droplet(0.0, rho_l=0.2, rho_g=0.2)
        f0 = s.get_f()
        assert s.step(7) == 0
        assert np.max(np.abs(s.get_f() - f0)) < 1e-16


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_shear_wave_decay(tau):
    # uniform density, sinusoidal shear u_x(y): no nonideal force, and the LBM
    # reproduces the Navier-Stokes decay rate with nu = c_s^2 (tau - 1/2).
    # The rate is measured between two times, after the start-up transient.
    n = 64
    s = O.Sim(nx=4, ny=n, Tr=0.7, k=0.3, kappa=0.1, tau=tau, scheme="EFDS4")
    rho0, U = 0.3, 1e-4
    f = np.zeros((9, n, 4))
    for y in range(n):
        f[:, y, :] = O.feq(O.D2Q9, rho0, [U * math.sin(2 * math.pi * y / n), 0, 0])[:, None]
    s.set_f(f)
    kk = 2 * math.pi / n

    def amp():
        ux = s.fields()["u"][0][:, 0]
        return np.sum(ux * np.sin(kk * np.arange(n))) * 2 / n

    assert s.step(100) == 0
    a1 = amp()
    assert s.step(800) == 0
    a2 = amp()
    nu = (tau - 0.5) / 3
    assert math.log(a1 / a2) / 800 == pytest.approx(nu * kk * kk, rel=2e-3)


def test_streaming_direction_and_relaxation():
    # A non-equilibrium perturbation that leaves rho and j unchanged (+d on
    # f_1 and f_3, -2d on f_0) relaxes by (1 - 1/tau) and is pushed along each
    # velocity: f_1 moves to x + 1, f_3 to x - 1 (Eq. 1, left side; Eq. 2).
    tau = 2.0
    s = O.Sim(nx=8, ny=8, Tr=0.7, k=0.3, kappa=0.1, tau=tau, scheme="EFDS2")
    s.init_droplet(0.0, rho_l=0.25, rho_g=0.25)
    f = s.get_f()
    base = f.copy()
    d = 1e-6
    f[1, 3, 2] += d
    f[3, 3, 2] += d
    f[0, 3, 2] -= 2 * d
    s.set_f(f)
    m0 = f.sum()
    s.step(1)
    f1 = s.get_f()
    assert f1[1, 3, 3] - base[1, 3, 3] == pytest.approx(d * (1 - 1 / tau), rel=1e-9)
    assert f1[3, 3, 1] - base[3, 3, 1] == pytest.approx(d * (1 - 1 / tau), rel=1e-9)
    assert f1[0, 3, 2] - base[0, 3, 2] == pytest.approx(-2 * d * (1 - 1 / tau), rel=1e-9)
    assert f1.sum() == pytest.approx(m0, rel=1e-15)


def test_droplet_mass_and_symmetry():
    s = O.Sim(nx=48, ny=48, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS4")
    s.init_droplet(12)
    m0 = s.observables()["mass"]
    assert s.step(300) == 0
    rho = s.density()
    o = s.observables()
    assert o["mass"] == pytest.approx(m0, rel=1e-13)
    c = 24
    r = rho[c - 20:c + 21, c - 20:c + 21]
    assert np.max(np.abs(r - r.T)) < 1e-12          # reflection about the diagonal
    assert np.max(np.abs(r - r[::-1, :])) < 1e-12   # reflection about y = c
    assert np.max(np.abs(r - r[:, ::-1])) < 1e-12


def test_flat_slab_has_no_tangential_flow_and_matches_maxwell():
    # Flat interface (Sec. 3.4): v_x is zero by symmetry, and with a
    # high-order scheme the bulk densities approach the Maxwell values.
    Tr = 0.8
    g, l = O.maxwell_tr(Tr)
    s = O.Sim(nx=4, ny=400, Tr=Tr, k=0.2, kappa=0.1, scheme="EFDS6")
    s.init_slab(1, 200, width=20)
    assert s.step(20000) == 0
    fl = s.fields()
    assert np.max(np.abs(fl["u"][0])) < 1e-15
    o = s.observables()
    assert o["max_v"] < 1e-3
    assert o["rho_center"] == pytest.approx(l, rel=2e-3)
    assert o["rho_corner"] == pytest.approx(g, rel=3e-2)


def test_initial_observables():
    # at t = 0 u = 0, so v = F / (2 rho) and max|u| = 0
    s = O.Sim(nx=32, ny=32, Tr=0.7, k=0.25, kappa=0.1, scheme="EFDS4")
    s.init_droplet(8)
    fl = s.fields()
    o = s.observables()
    vmax = np.max(np.sqrt((fl["F"] ** 2).sum(0)) / (2 * fl["rho"]))
    assert o["max_u"] == 0 and o["max_v"] == pytest.approx(vmax, rel=1e-14)
    g, l = O.maxwell_tr(0.7)
    # Eq. 26 at the centre node (r = 0), r0 = 8, W = 10
    assert o["rho_center"] == pytest.approx((l + g) / 2 - (l - g) / 2 * math.tanh(2 * (0 - 8) / 10), rel=1e-14)
    assert o["rho_corner"] == fl["rho"][0, 0]


def test_instability_is_reported():
    # second-order gradients at T_r = 0.7 with tau = 1 do not settle; the oracle
    # stops at the first non-positive density and reports the step
    s = O.Sim(nx=64, ny=64, Tr=0.7, k=0.25, kappa=0.1, scheme="EFDS2")
    s.init_droplet(16)
    rc = s.step(2000)
    o = s.observables()
    assert rc == O.EUNSTABLE and o["status"] == O.EUNSTABLE and 0 < o["step"] < 2000
