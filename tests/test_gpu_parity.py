"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs.  FP64 mode: 1e-12 relative; FP32 deviation storage:
1e-5 on densities relative to the liquid density."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


def pair(L, lattice, precision=0, mu_fp64=0, **kw):
    lat_g = L.LBM_D2Q9 if lattice == 2 else L.LBM_D3Q19
    lat_o = O.D2Q9 if lattice == 2 else O.D3Q19
    g = L.Sim(L.make_params(lattice=lat_g, precision=precision, mu_fp64=mu_fp64, **kw))
    o = O.Sim(lattice=lat_o, **kw)
    return g, o


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


SCHEMES_2D = ["EFDS2", "EFDS4", "EFDS6", "E4", "E8", "CFDS4", "CFDS6", "CFDS8", "OCFDS4"]
SCHEMES_3D = ["EFDS2", "EFDS4", "EFDS6", "E4", "CFDS4", "CFDS6", "CFDS8", "OCFDS4"]


@pytest.mark.parametrize("scheme", SCHEMES_2D)
def test_d2q9_fp64_fields_and_steps(L, scheme):
    # 40 x 24: one full and one ragged tile in x (32 + 8), three tiles in y
    kw = dict(nx=40, ny=24, Tr=0.8, k=0.25, kappa=0.1, scheme=scheme)
    g, o = pair(L, 2, **kw)
    g.lbm_init_droplet(7.0, center=[19.0, 11.5, 0.0])
    o.init_droplet(7.0, center=[19.0, 11.5, 0.0])
    F, mu = g.lbm_get_force()
    fo = o.fields()
    assert relerr(mu, fo["mu"]) < TOL64
    assert relerr(F, fo["F"]) < 1e-11
    for n in (1, 9, 40):
        g.lbm_step(n)
        assert o.step(n) == 0
        assert relerr(g.lbm_get_density(), o.density()) < TOL64, (scheme, n)
    assert relerr(g.lbm_get_f(), o.get_f()) < TOL64


@pytest.mark.parametrize("scheme", SCHEMES_3D)
def test_d3q19_fp64_steps(L, scheme):
    # 36 x 20 x 40: ragged tiles in x and y, two z chunks (32 + 8)
    kw = dict(nx=36, ny=20, nz=40, Tr=0.8, k=0.25, kappa=0.1, scheme=scheme)
    g, o = pair(L, 3, **kw)
    g.lbm_init_droplet(6.0, center=[17.0, 9.0, 21.0])
    o.init_droplet(6.0, center=[17.0, 9.0, 21.0])
    F, mu = g.lbm_get_force()
    fo = o.fields()
    assert relerr(mu, fo["mu"]) < TOL64
    assert relerr(F, fo["F"]) < 1e-11
    g.lbm_step(6)
    assert o.step(6) == 0
    assert relerr(g.lbm_get_density(), o.density()) < TOL64
    assert relerr(g.lbm_get_f(), o.get_f()) < TOL64


@pytest.mark.parametrize("lattice,shape,scheme", [(2, (64, 48, 1), "EFDS6"), (2, (64, 48, 1), "OCFDS4"),
                                                  (3, (32, 24, 40), "EFDS6"), (3, (32, 24, 40), "E4")])
@pytest.mark.parametrize("mu_fp64", [0, 1])
def test_fp32dev_against_oracle(L, lattice, shape, scheme, mu_fp64):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, Tr=0.8, k=0.25, kappa=0.1, scheme=scheme)
    g, o = pair(L, lattice, precision=L.LBM_FP32DEV, mu_fp64=mu_fp64, **kw)
    g.lbm_init_droplet(10.0)
    o.init_droplet(10.0)
    rl = O.maxwell_tr(0.8)[1]
    g.lbm_step(100)
    assert o.step(100) == 0
    err = np.max(np.abs(g.lbm_get_density() - o.density())) / rl
    assert err < TOL32, err


# nx % 4 == 0 takes the 16-byte (vector) mu and collision kernels, other nx the
# 4-byte ones; 68 = 64 + 4 leaves a 4-wide vector block, 8^3 wraps every halo
# several times around the lattice.  The collision pass cuts the lattice into
# tiles of 32 columns and bands of 11 rows whose edge columns and rows are
# completed by atomic additions and whose corners by fixed-point ones: ny = 45
# and 12 leave a last band of one row, which takes a row from the band before
# it; ny = 11 is one band whose two edge rows feed each other across the seam;
# nx = 33 and 65 leave a last tile of one column, which takes a column from
# the tile before it; nx < 32 is one tile whose edge columns feed each other
@pytest.mark.parametrize("shape", [(68, 40, 36), (42, 26, 20), (8, 8, 8), (12, 9, 10), (64, 45, 20), (36, 12, 10),
                                   (40, 11, 12), (33, 20, 12), (65, 23, 10)])
@pytest.mark.parametrize("scheme", ["EFDS2", "EFDS6"])
def test_fp32dev_kernel_variants_against_oracle(L, shape, scheme):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, Tr=0.9, k=0.3, kappa=0.1, scheme=scheme)
    g, o = pair(L, 3, precision=L.LBM_FP32DEV, **kw)
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    rho = 0.15 + 0.01 * rng.standard_normal((nz, ny, nx))
    g.lbm_init_density(rho)
    o.set_f(np.stack([w * rho for w in O.lattice(O.D3Q19)[1]]))
    g.lbm_step(30)
    assert o.step(30) == 0
    err = np.max(np.abs(g.lbm_get_density() - o.density())) / 0.15
    assert err < TOL32, err


def test_fp32dev_split_step_is_bitwise_reproducible(L):
    # the band edge rows and tile edge columns receive exactly two atomic
    # additions onto zero, whose result does not depend on their order, and the
    # tile corners exact integer additions: repeated runs agree bit for bit
    kw = dict(lattice=L.LBM_D3Q19, nx=64, ny=45, nz=24, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
              precision=L.LBM_FP32DEV)
    outs = []
    for _ in range(3):
        g = L.Sim(L.make_params(**kw))
        g.lbm_init_droplet(10.0)
        g.lbm_step(25)
        outs.append((g.lbm_get_f(), g.lbm_get_density()))
    for f, r in outs[1:]:
        assert np.array_equal(f, outs[0][0]) and np.array_equal(r, outs[0][1])


def test_observables_parity(L):
    kw = dict(nx=48, ny=40, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS4")
    g, o = pair(L, 2, **kw)
    g.lbm_init_droplet(10.0)
    o.init_droplet(10.0)
    for n in (0, 30, 200):
        g.lbm_step(n)
        o.step(n)
        og, oo = g.lbm_observables(), o.observables()
        assert og["status"] == 0 and og["step"] == oo["step"]
        for key in ("max_v", "max_u", "rho_center", "rho_corner", "mass", "max_drho"):
            assert og[key] == pytest.approx(oo[key], rel=1e-11, abs=1e-300), key


def test_first_config_instability_agrees(L):
    # 64 x 64, r0 = 16, T_r = 0.7, second-order scheme, tau = 1: the oracle
    # reports a non-positive density; the GPU must report it at the same step
    kw = dict(nx=64, ny=64, Tr=0.7, k=0.25, kappa=0.1, scheme="EFDS2")
    g, o = pair(L, 2, **kw)
    g.lbm_init_droplet(16.0)
    o.init_droplet(16.0)
    g.lbm_step(40)
    o.step(40)
    assert relerr(g.lbm_get_density(), o.density()) < 1e-11
    assert o.step(3000) == O.EUNSTABLE
    oo = o.observables()
    g.lbm_step(3000 - 40)
    og = g.lbm_observables()
    assert og["status"] == L.LBM_EUNSTABLE
    assert abs(og["step"] - oo["step"]) <= 2, (og["step"], oo["step"])


def test_deterministic_fp64(L):
    kw = dict(nx=40, ny=40, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6")
    outs = []
    for _ in range(2):
        g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, **kw))
        g.lbm_init_droplet(9.0)
        g.lbm_step(25)
        outs.append((g.lbm_get_f(), g.lbm_observables()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_init_variants_match_oracle(L):
    kw = dict(nx=33, ny=27, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS4")
    g, o = pair(L, 2, **kw)
    g.lbm_init_slab(1, 12.0, width=6.0)
    o.init_slab(1, 12.0, width=6.0)
    assert relerr(g.lbm_get_density(), o.density()) < 1e-14
    r = np.linspace(0.0, 20.0, 41)
    prof = 0.2 + 0.1 * np.tanh(8.0 - r)
    g.lbm_init_profile(r, prof)
    o.init_profile(r, prof)
    assert relerr(g.lbm_get_density(), o.density()) < 1e-14
    rng = np.random.default_rng(7)
    rho = 0.2 + 0.01 * rng.standard_normal((27, 33))
    g.lbm_init_density(rho)
    f = np.stack([w * rho for w in O.lattice(O.D2Q9)[1]])
    o.set_f(f)
    g.lbm_step(5)
    o.step(5)
    assert relerr(g.lbm_get_density(), o.density()) < TOL64


@pytest.mark.parametrize("shape", [(8, 8, 1), (65, 33, 1), (8, 8, 8), (9, 13, 11)])
def test_small_and_ragged_lattices(L, shape):
    nx, ny, nz = shape
    lat = 2 if nz == 1 else 3
    kw = dict(nx=nx, ny=ny, nz=nz, Tr=0.9, k=0.3, kappa=0.1, scheme="EFDS4")
    g, o = pair(L, lat, **kw)
    rng = np.random.default_rng(nx * 100 + ny)
    shp = (ny, nx) if lat == 2 else (nz, ny, nx)
    rho = 0.15 + 0.01 * rng.standard_normal(shp)
    g.lbm_init_density(rho)
    o.set_f(np.stack([w * rho for w in O.lattice(O.D2Q9 if lat == 2 else O.D3Q19)[1]]))
    g.lbm_step(7)
    o.step(7)
    assert relerr(g.lbm_get_density(), o.density()) < TOL64
    assert relerr(g.lbm_get_f(), o.get_f()) < TOL64


def test_zero_steps_and_invalid_arguments(L):
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=16, ny=16, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS4"))
    g.lbm_init_droplet(4.0)
    r0 = g.lbm_get_density()
    g.lbm_step(0)
    assert np.array_equal(r0, g.lbm_get_density())
    with pytest.raises(L.LBMError) as e:
        g.lbm_step(-1)
    assert e.value.code == L.LBM_EINVAL
    for bad in (dict(nx=4), dict(tau=0.5), dict(Tr=-1.0), dict(scheme=99), dict(nz=2)):
        kw = dict(lattice=L.LBM_D2Q9, nx=16, ny=16, Tr=0.8)
        kw.update(bad)
        with pytest.raises(L.LBMError) as e:
            L.Sim(L.make_params(**kw))
        assert e.value.code == L.LBM_EINVAL
    with pytest.raises(L.LBMError) as e:
        L.Sim(L.make_params(lattice=L.LBM_D3Q19, nx=16, ny=16, nz=16, scheme="E8"))
    assert e.value.code == L.LBM_ENOTSUP


def test_zchunk_and_autotune_do_not_change_results(L):
    kw = dict(lattice=L.LBM_D3Q19, nx=48, ny=40, nz=44, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
              precision=L.LBM_FP32DEV)
    outs = []
    for zc in (0, 5, 11, 44, -1):
        g = L.Sim(L.make_params(**kw))
        if zc < 0:
            assert g.lbm_autotune() > 0
        else:
            g.lbm_set_zchunk(zc)
        g.lbm_init_droplet(9.0)
        g.lbm_step(12)
        outs.append(g.lbm_get_f())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("ny", [40, 48])
def test_compact_zchunk_and_autotune_do_not_change_results(L, ny):
    # the compact schemes' tiled collision pass marches z-chunks too; the
    # tuner times them on the handle's lattice
    kw = dict(lattice=L.LBM_D3Q19, nx=64, ny=ny, nz=36, Tr=0.8, k=0.25, kappa=0.1, scheme="OCFDS4",
              precision=L.LBM_FP32DEV)
    outs = []
    for zc in (0, 5, 11, 36, -1):
        g = L.Sim(L.make_params(**kw))
        if zc < 0:
            assert g.lbm_autotune() > 0
        else:
            g.lbm_set_zchunk(zc)
        g.lbm_init_droplet(9.0)
        g.lbm_step(12)
        outs.append(g.lbm_get_f())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


# compact schemes in 3D with FP32 deviation storage: z-marching mu pass (orders
# 4 and 6; the node-parallel one for CFDS8), line solves, and the tiled
# collision pass reading the derivative fields (64: tensor-copy and 16-byte
# variants by tile; 42: the 4-byte variant everywhere).  Lines whose length is
# a multiple of 32 are solved in registers (64 x 96 x 64: every axis; 64 x 40
# x 36: x only), the others in shared memory; a cube of such lines (64^3) has
# all three axes solved in one launch.
@pytest.mark.parametrize("shape", [(64, 40, 36), (42, 26, 20), (64, 96, 64), (64, 64, 64)])
@pytest.mark.parametrize("scheme", ["OCFDS4", "CFDS6", "CFDS8"])
def test_fp32dev_compact_3d_against_oracle(L, shape, scheme):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, Tr=0.9, k=0.3, kappa=0.1, scheme=scheme)
    g, o = pair(L, 3, precision=L.LBM_FP32DEV, **kw)
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    rho = 0.15 + 0.01 * rng.standard_normal((nz, ny, nx))
    g.lbm_init_density(rho)
    o.set_f(np.stack([w * rho for w in O.lattice(O.D3Q19)[1]]))
    g.lbm_step(30)
    assert o.step(30) == 0
    err = np.max(np.abs(g.lbm_get_density() - o.density())) / 0.15
    assert err < TOL32, err


# D2Q9 FP32 deviation storage: nx % 4 == 0 takes the y-marching vector mu pass
# (68: a 4-node chunk past one 64-wide group; 40: a partial group; 8: every
# stencil wraps the lattice), 42 the tiled one
@pytest.mark.parametrize("shape", [(68, 37), (40, 24), (8, 8), (42, 26)])
@pytest.mark.parametrize("scheme", ["EFDS2", "EFDS4", "EFDS6"])
def test_fp32dev_2d_mu_variants_against_oracle(L, shape, scheme):
    nx, ny = shape
    kw = dict(nx=nx, ny=ny, Tr=0.9, k=0.3, kappa=0.1, scheme=scheme)
    g, o = pair(L, 2, precision=L.LBM_FP32DEV, **kw)
    rng = np.random.default_rng(nx * 100 + ny)
    rho = 0.15 + 0.01 * rng.standard_normal((ny, nx))
    g.lbm_init_density(rho)
    o.set_f(np.stack([w * rho for w in O.lattice(O.D2Q9)[1]]))
    g.lbm_step(40)
    assert o.step(40) == 0
    err = np.max(np.abs(g.lbm_get_density() - o.density())) / 0.15
    assert err < TOL32, err


@pytest.mark.parametrize("scheme", ["EFDS6", "E8"])
def test_d2q9_tile_rows_give_identical_results(L, scheme):
    # the split D2Q9 step on tiles of 16, 32 and 64 rows: the same arithmetic
    # per node, bitwise equal states; the tuner picks one of them
    kw = dict(lattice=L.LBM_D2Q9, nx=100, ny=90, Tr=0.8, k=0.25, kappa=0.1, scheme=scheme,
              precision=L.LBM_FP32DEV)
    out = {}
    for rows in (1, 2, 4):
        s = L.Sim(L.make_params(**kw))
        s.lbm_set_tile_rows(rows)
        s.lbm_init_droplet(20.0)
        s.lbm_step(30)
        out[rows] = s.lbm_get_density()
    assert np.array_equal(out[1], out[2]) and np.array_equal(out[4], out[2])
    s = L.Sim(L.make_params(**kw))
    assert s.lbm_autotune() in (1, 2, 4)
    with pytest.raises(L.LBMError):
        s.lbm_set_tile_rows(3)
