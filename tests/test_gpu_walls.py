"""GPU parity of the chemical-potential wall boundary (Appendix A) with the
oracle: Eq. A.1 wall densities, mu_w on wall nodes, halfway bounce-back and
fluid-only observables, for EFDS2/4/6 on D2Q9 (BGK and MRT) and D3Q19, FP64
to 1e-12 and FP32 deviation storage to 1e-5 of rho_l, on a flat wall and on a
round post; refusals."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

Tr, K, KAP = 0.8, 0.25, 0.1


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


def mu_sat():
    g = O.maxwell_tr(Tr)[0]
    return K * K * O.cs_mu(g, 1.0, 4.0, 1.0, Tr * O.cs_critical()[1])


def flat_wall(shape, rows):
    # the first `rows` lines of the slowest axis (y in 2D, z in 3D)
    m = np.zeros(shape, np.uint8)
    m[:rows] = 1
    return m


def post(shape, cx, cy, r):
    y, x = np.mgrid[0:shape[0], 0:shape[1]]
    return ((x - cx) ** 2 + (y - cy) ** 2 <= r * r).astype(np.uint8)


def pair(L, lattice, shape, scheme, precision=0, collision="BGK", tau=1.0):
    dims = dict(nx=shape[-1], ny=shape[-2], nz=shape[0] if len(shape) == 3 else 1)
    kw = dict(Tr=Tr, k=K, kappa=KAP, tau=tau, scheme=scheme, collision=collision, **dims)
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9 if lattice == 2 else L.LBM_D3Q19, precision=precision, **kw))
    o = O.Sim(lattice=O.D2Q9 if lattice == 2 else O.D3Q19, **kw)
    return g, o


def compare(g, o, mask, tol_rel, steps):
    g.lbm_step(steps)
    assert o.step(steps) == 0
    fluid = mask == 0
    rl = O.maxwell_tr(Tr)[1]
    f_g, f_o = g.lbm_get_f(), o.get_f()
    assert np.max(np.abs(f_g[:, fluid] - f_o[:, fluid])) / rl < tol_rel
    fo = o.fields()
    layers = o.solid_layers()
    near = layers <= 3  # fluid and the wall layers a stencil reaches
    rho_g = g.lbm_get_density()
    assert np.max(np.abs(rho_g[near] - fo["rho"][near])) / rl < tol_rel
    F, mu = g.lbm_get_force()
    D = F.shape[0]
    Fo = fo["F"][:D]
    scale = np.max(np.abs(Fo))
    assert np.max(np.abs(F - Fo)) / scale < 100 * tol_rel
    assert np.max(np.abs(mu[near] - fo["mu"][near])) / np.max(np.abs(fo["mu"])) < 100 * tol_rel
    walls = mask != 0
    assert np.all(F[:, walls] == 0.0)
    og, oo = g.lbm_observables(), o.observables()
    assert og["mass"] == pytest.approx(oo["mass"], rel=tol_rel)
    assert og["max_u"] == pytest.approx(oo["max_u"], rel=100 * tol_rel, abs=1e-12)
    assert og["max_v"] == pytest.approx(oo["max_v"], rel=100 * tol_rel, abs=1e-12)


@pytest.mark.parametrize("scheme", ["EFDS2", "EFDS4", "EFDS6"])
def test_fp64_flat_wall_d2q9(L, scheme):
    shape = (40, 48)
    g, o = pair(L, 2, shape, scheme)
    g.lbm_init_droplet(9.0, center=[24.0, 4 + 6.0, 0.0])
    o.init_droplet(9.0, center=[24.0, 4 + 6.0, 0.0])
    mask = flat_wall(shape, 4)
    g.lbm_set_solid(mask, mu_sat() - 0.01)
    o.set_solid(mask, mu_sat() - 0.01)
    compare(g, o, mask, 1e-12, 60)


def test_fp64_mrt_flat_wall_d2q9(L):
    shape = (36, 40)
    g, o = pair(L, 2, shape, "EFDS4", collision="MRT", tau=0.8)
    g.lbm_init_droplet(8.0, center=[20.0, 4 + 5.0, 0.0])
    o.init_droplet(8.0, center=[20.0, 4 + 5.0, 0.0])
    mask = flat_wall(shape, 4)
    g.lbm_set_solid(mask, mu_sat() + 0.01)
    o.set_solid(mask, mu_sat() + 0.01)
    compare(g, o, mask, 1e-12, 60)


def test_fp64_round_post_d2q9(L):
    # convex wall of every orientation; droplet touching it
    shape = (48, 56)
    mask = post(shape, 20, 24, 7.5)
    g, o = pair(L, 2, shape, "EFDS6")
    g.lbm_init_droplet(8.0, center=[34.0, 24.0, 0.0])
    o.init_droplet(8.0, center=[34.0, 24.0, 0.0])
    g.lbm_set_solid(mask, mu_sat() - 0.005)
    o.set_solid(mask, mu_sat() - 0.005)
    compare(g, o, mask, 1e-12, 80)


@pytest.mark.parametrize("scheme", ["EFDS4", "EFDS6"])
def test_fp32dev_flat_wall_d2q9(L, scheme):
    shape = (48, 64)
    g, o = pair(L, 2, shape, scheme, precision=1)
    g.lbm_init_droplet(11.0, center=[32.0, 4 + 8.0, 0.0])
    o.init_droplet(11.0, center=[32.0, 4 + 8.0, 0.0])
    mask = flat_wall(shape, 4)
    g.lbm_set_solid(mask, mu_sat() - 0.01)
    o.set_solid(mask, mu_sat() - 0.01)
    compare(g, o, mask, 1e-5, 100)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_flat_wall_d3q19(L, precision, tol):
    shape = (18, 20, 24)  # z, y, x
    g, o = pair(L, 3, shape, "EFDS4", precision=precision)
    c = [12.0, 10.0, 3 + 5.0]
    g.lbm_init_droplet(6.0, center=c)
    o.init_droplet(6.0, center=c)
    mask = flat_wall(shape, 3)
    g.lbm_set_solid(mask, mu_sat() - 0.01)
    o.set_solid(mask, mu_sat() - 0.01)
    compare(g, o, mask, tol, 30)


def test_walls_are_refused_where_they_do_not_apply(L):
    shape = (32, 32)
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=32, ny=32, Tr=Tr, k=K, kappa=KAP, scheme="CFDS4"))
    with pytest.raises(L.LBMError) as e:
        g.lbm_set_solid(flat_wall(shape, 4), 0.0)
    assert e.value.code == L.LBM_ENOTSUP
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=32, ny=32, Tr=Tr, k=K, kappa=KAP, scheme="EFDS4"))
    with pytest.raises(L.LBMError) as e:
        g.lbm_set_solid(np.ones(shape, np.uint8), 0.0)
    assert e.value.code == L.LBM_EINVAL


def test_removing_the_walls_restores_the_periodic_step(L):
    shape = (32, 40)
    kw = dict(lattice=L.LBM_D2Q9, nx=40, ny=32, Tr=Tr, k=K, kappa=KAP, scheme="EFDS4")
    a, b = L.Sim(L.make_params(**kw)), L.Sim(L.make_params(**kw))
    for s in (a, b):
        s.lbm_init_droplet(8.0)
    b.lbm_set_solid(flat_wall(shape, 4), 0.0)
    b.lbm_set_solid(None)
    a.lbm_step(20)
    b.lbm_step(20)
    assert np.array_equal(a.lbm_get_density(), b.lbm_get_density())


@pytest.mark.parametrize("eos,a,b,kap,rho", [("CS", 1.0, 4.0, 0.1, 0.2), ("PR", 2 / 49, 2 / 21, 0.01, 3.0),
                                             ("VDW", 9 / 49, 2 / 21, 0.01, 3.0), ("RKS", 2 / 49, 2 / 21, 0.01, 3.0)])
def test_bulk_mu_is_the_mu_of_a_uniform_fluid(L, eos, a, b, kap, rho):
    # the host value callers pick mu_w against carries the kernels' additive constant
    p = L.make_params(lattice=L.LBM_D2Q9, nx=32, ny=32, eos=eos, a=a, b=b, Tr=0.8, k=0.3, kappa=kap, scheme="EFDS4")
    s = L.Sim(p)
    s.lbm_init_density(np.full((32, 32), rho))
    _, mu = s.lbm_get_force()
    want = L.lbm_bulk_mu(p, rho)
    assert np.max(np.abs(mu - want)) <= 1e-13 * abs(want) + 1e-15


@pytest.mark.parametrize("lattice,shape,scheme,precision,tol,steps",
                         [(2, (29, 37), "EFDS4", 0, 1e-12, 60), (3, (11, 13, 17), "EFDS6", 0, 1e-12, 30),
                          (3, (11, 13, 17), "EFDS6", 1, 1e-5, 30)])
def test_scattered_obstacles_on_ragged_lattices(L, lattice, shape, scheme, precision, tol, steps):
    # isolated wall nodes and small clusters (seed 7, ~6-8% of the nodes),
    # lattice sizes that fill no tile or warp evenly
    rng = np.random.default_rng(7)
    mask = (rng.random(shape) < (0.08 if lattice == 2 else 0.06)).astype(np.uint8)
    g, o = pair(L, lattice, shape, scheme, precision=precision)
    c = [shape[-1] // 2, shape[-2] // 2, shape[0] // 2 if lattice == 3 else 0]
    r = 7.0 if lattice == 2 else 4.0
    g.lbm_init_droplet(r, center=[float(v) for v in c])
    o.init_droplet(r, center=[float(v) for v in c])
    g.lbm_set_solid(mask, mu_sat())
    o.set_solid(mask, mu_sat())
    compare(g, o, mask, tol, steps)
