"""Pins of the oracle's chemical-potential wall boundary (Appendix A): wall
layers, the Eq. A.1 densities on them, the wall chemical potential, halfway
bounce-back (mass conservation, a resting uniform fluid stays at rest),
mirror symmetry of a droplet on a flat wall, and wettability that follows the
wall chemical potential."""
import numpy as np
import pytest

import oracle as O

Tr, K, KAP = 0.8, 0.25, 0.1


def wall_sim(nx=40, ny=32, rows=4, scheme="EFDS4", mu_w=None, **kw):
    s = O.Sim(nx=nx, ny=ny, Tr=Tr, k=K, kappa=KAP, scheme=scheme, **kw)
    mask = np.zeros((ny, nx), np.uint8)
    mask[:rows, :] = 1
    return s, mask


def mu_sat():
    g = O.maxwell_tr(Tr)[0]
    return K * K * O.cs_mu(g, 1.0, 4.0, 1.0, Tr * O.cs_critical()[1])


def test_wall_layers():
    s, mask = wall_sim(rows=10, ny=40)
    s.set_solid(mask, 0.0)
    # a periodic 10-row wall: layers from both faces, deeper rows beyond the third
    assert list(s.solid_layers()[:10, 7]) == [1, 2, 3, 4, 4, 4, 4, 3, 2, 1]
    assert np.all(s.solid_layers()[10:] == 0)


def test_eq_a1_densities():
    s, mask = wall_sim(rows=6, nx=24, ny=24)
    rng = np.random.default_rng(3)
    rho = 0.1 + 0.02 * rng.random((24, 24))
    s.set_f(np.stack([w * rho for w in O.lattice(O.D2Q9)[1]]))
    s.set_solid(mask, -0.02)
    fr = s.fields()["rho"]
    # layer 1 below the fluid (row 5): weights 1/9 straight up, 1/36 on the diagonals
    for x in (0, 7, 23):
        up = rho[6]
        want = (up[x] / 9 + (up[(x - 1) % 24] + up[(x + 1) % 24]) / 36) / (1 / 9 + 2 / 36)
        assert fr[5, x] == pytest.approx(want, rel=1e-14)
    # layer 2 (row 4) from layer 1 (row 5)
    for x in (3, 11):
        l1 = fr[5]
        want = (l1[x] / 9 + (l1[x - 1] + l1[x + 1]) / 36) / (1 / 9 + 2 / 36)
        assert fr[4, x] == pytest.approx(want, rel=1e-14)
    # the wall carries mu_w
    assert np.all(s.fields()["mu"][:6] == -0.02)


def test_resting_uniform_fluid_stays_at_rest():
    s, mask = wall_sim()
    rho0 = 0.2
    s.init_droplet(0.0, rho_l=rho0, rho_g=rho0)
    s.set_solid(mask, K * K * O.cs_mu(rho0, 1.0, 4.0, 1.0, Tr * O.cs_critical()[1]))
    f0 = s.get_f()
    assert s.step(20) == 0
    fluid = mask == 0
    assert np.max(np.abs((s.get_f() - f0)[:, fluid])) < 1e-15


def test_bounce_back_conserves_mass_and_a_centred_droplet_stays_symmetric():
    s, mask = wall_sim(nx=48, ny=40)
    s.init_droplet(10.0, center=[24.0, 4 + 7.0, 0.0])
    s.set_solid(mask, mu_sat())
    m0 = s.observables()["mass"]
    assert s.step(400) == 0
    o = s.observables()
    assert o["mass"] == pytest.approx(m0, rel=1e-12)
    rho = s.density()[4:]
    # mirror about x = 24 (the droplet centre node)
    assert np.max(np.abs(rho[:, 1:24] - rho[:, 47:24:-1])) < 1e-12


def test_wettability_follows_the_wall_chemical_potential():
    g, l = O.maxwell_tr(Tr)
    wetted = []
    for dmu in (-0.02, 0.0, 0.02):
        s, mask = wall_sim(nx=96, ny=64)
        s.init_droplet(14.0, center=[48.0, 14.0, 0.0])
        s.set_solid(mask, mu_sat() + dmu)
        assert s.step(2000) == 0
        wetted.append(int(np.sum(s.density()[4] > 0.5 * (g + l))))
    # a lower wall chemical potential pulls the liquid along the wall
    assert wetted[0] > wetted[1] > wetted[2]


def test_walls_need_an_explicit_scheme():
    s, mask = wall_sim(scheme="CFDS4")
    with pytest.raises(ValueError):
        s.set_solid(mask, 0.0)
