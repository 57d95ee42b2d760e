"""Pins of the oracle's MRT collision (Eq. 1, 3-5; D2Q9): the printed matrix,
the moment polynomials it encodes, its inverse, the reduction to single
relaxation when every rate is 1/tau (stated after Eq. 5), conservation, the
shear viscosity nu = c_s^2 (tau - 1/2) set by s_8 = s_9 = 1/tau, and the
relaxation of each non-conserved moment by its own rate."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))["mrt_d2q9"]


def velocities():
    return np.array(O.lattice(O.D2Q9)[0], dtype=float)[:, :2]


def test_matrix_is_the_printed_one():
    assert np.array_equal(O.mrt_matrix(), np.array(GOLD["M"], dtype=float))


def test_rows_are_the_moment_polynomials():
    # density, energy, energy squared, momentum, energy flux, stress: the
    # polynomials in e_i that define the rows (checks every printed entry)
    e = velocities()
    ex, ey = e[:, 0], e[:, 1]
    e2 = ex * ex + ey * ey
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 * e2, ex, (-5 + 3 * e2) * ex, ey,
            (-5 + 3 * e2) * ey, ex * ex - ey * ey, ex * ey]
    assert np.array_equal(O.mrt_matrix(), np.array(rows))


def test_orthogonal_rows_and_inverse():
    M = O.mrt_matrix()
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))  # "orthogonal transformation matrix"
    assert np.allclose(O.mrt_inverse(), np.linalg.inv(M), rtol=0, atol=1e-15)


def test_equal_rates_reduce_to_single_relaxation():
    for tau in (0.7, 1.0, 1.6):
        kw = dict(nx=24, ny=20, Tr=0.8, k=0.25, kappa=0.1, tau=tau, scheme="EFDS4")
        a = O.Sim(collision="BGK", **kw)
        b = O.Sim(collision="MRT", mrt_s=[1.0 / tau] * 9, **kw)
        for s in (a, b):
            s.init_droplet(6.0)
            assert s.step(15) == 0
        assert np.max(np.abs(a.get_f() - b.get_f())) < 1e-14


def test_collision_conserves_mass_and_adds_the_force_momentum():
    rng = np.random.default_rng(5)
    e = velocities()
    for _ in range(5):
        f = O.feq(O.D2Q9, 0.3, [0.02, -0.01, 0]) + 1e-3 * rng.standard_normal(9)
        rho = f.sum()
        u = [(e[:, 0] @ f) / rho, (e[:, 1] @ f) / rho, 0.0]
        F = [1e-4, -2e-4, 0.0]
        post = O.mrt_collide(f, O.feq(O.D2Q9, rho, u), O.edm(O.D2Q9, rho, u, F), O.mrt_rates(0.9))
        assert post.sum() == pytest.approx(rho, rel=1e-15)
        assert e[:, 0] @ post == pytest.approx(e[:, 0] @ f + F[0], abs=1e-15)
        assert e[:, 1] @ post == pytest.approx(e[:, 1] @ f + F[1], abs=1e-15)


@pytest.mark.parametrize("row,rate", [(1, 1.64), (2, 1.54), (4, 1.7), (6, 1.7), (7, 1.0 / 0.9), (8, 1.0 / 0.9)])
def test_each_moment_relaxes_at_its_own_rate(row, rate):
    # a non-equilibrium part along one moment direction relaxes by (1 - s_k)
    # in that moment and leaves every other moment at equilibrium
    M = O.mrt_matrix()
    rho, u = 0.25, [0.01, 0.02, 0.0]
    feq = O.feq(O.D2Q9, rho, u)
    dm = np.zeros(9)
    dm[row] = 1e-4
    f = feq + np.linalg.solve(M, dm)
    post = O.mrt_collide(f, feq, np.zeros(9), O.mrt_rates(0.9))
    got = M @ (post - feq)
    want = np.zeros(9)
    want[row] = (1 - rate) * 1e-4
    assert np.allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_mrt_shear_wave_decays_with_the_shear_rate(tau):
    # a long wave (128 nodes) keeps the O(k^2) correction, which depends on the
    # other rates, below the tolerance
    n = 128
    s = O.Sim(nx=4, ny=n, Tr=0.7, k=0.3, kappa=0.1, tau=tau, scheme="EFDS4", collision="MRT")
    rho0, U = 0.3, 1e-4
    f = np.zeros((9, n, 4))
    for y in range(n):
        f[:, y, :] = O.feq(O.D2Q9, rho0, [U * math.sin(2 * math.pi * y / n), 0, 0])[:, None]
    s.set_f(f)
    kk = 2 * math.pi / n

    def amp():
        ux = s.fields()["u"][0][:, 0]
        return np.sum(ux * np.sin(kk * np.arange(n))) * 2 / n

    assert s.step(200) == 0
    a1 = amp()
    assert s.step(3200) == 0
    a2 = amp()
    nu = (tau - 0.5) / 3
    assert math.log(a1 / a2) / 3200 == pytest.approx(nu * kk * kk, rel=2e-3)


def test_mrt_is_d2q9_only():
    with pytest.raises(ValueError):
        O.Sim(lattice=O.D3Q19, nx=8, ny=8, nz=8, collision="MRT")
