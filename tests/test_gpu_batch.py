"""Batched droplets in one persistent graph-captured launch: results equal
the single-case path, replays continue the run, per-case instability is
reported, and a stalled device barrier returns LBM_ETIMEOUT (no hang)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


CASES = [dict(nx=64, ny=48, Tr=0.8, k=0.25, scheme="EFDS4", r=12.0),
         dict(nx=40, ny=72, Tr=0.9, k=0.3, scheme="E4", r=10.0),
         dict(nx=96, ny=96, Tr=0.8, k=0.2, scheme="EFDS6", r=20.0),
         dict(nx=33, ny=35, Tr=0.85, k=0.25, scheme="E8", r=8.0),
         dict(nx=64, ny=64, Tr=0.7, k=0.25, scheme="EFDS2", r=16.0)]  # goes unstable


def params(L, c, precision):
    return L.make_params(lattice=L.LBM_D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1,
                         scheme=c["scheme"], precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_case_path(L, precision):
    b = L.Batch([params(L, c, precision) for c in CASES])
    b.lbm_batch_init_droplets([c["r"] for c in CASES])
    b.lbm_batch_step(30)
    b.lbm_batch_step(30)  # graph replay continues the run
    assert b.lbm_batch_get_step() == 60
    rc, obs = b.lbm_batch_observables(raise_errors=False)
    assert rc == 0
    for i, c in enumerate(CASES[:4]):
        s = L.Sim(params(L, c, precision))
        s.lbm_init_droplet(c["r"])
        s.lbm_step(60)
        # same tile code, compiled in another unit: equal up to rounding
        rb, rs = b.lbm_batch_get_density(i), s.lbm_get_density()
        assert np.max(np.abs(rb - rs)) / np.max(rs) < (1e-12 if precision == 0 else 1e-6), c
        o = s.lbm_observables()
        assert obs[i]["status"] == 0
        for key in ("max_v", "max_u", "mass", "rho_center", "rho_corner"):
            assert obs[i][key] == pytest.approx(o[key], rel=1e-10 if precision == 0 else 1e-3), (c, key)


def test_batch_fp64_matches_oracle(L):
    c = CASES[0]
    b = L.Batch([params(L, c, 0) for c in CASES[:2]])
    b.lbm_batch_init_droplets([c["r"] for c in CASES[:2]])
    b.lbm_batch_step(25)
    o = O.Sim(lattice=O.D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1, scheme=c["scheme"])
    o.init_droplet(c["r"])
    assert o.step(25) == 0
    ro = o.density()
    assert np.max(np.abs(b.lbm_batch_get_density(0) - ro)) / np.max(ro) < 1e-12


def test_batch_reports_unstable_case(L):
    b = L.Batch([params(L, c, 1) for c in CASES])
    b.lbm_batch_init_droplets([c["r"] for c in CASES])
    b.lbm_batch_step(1500)
    rc, obs = b.lbm_batch_observables(raise_errors=False)
    assert rc == 0
    assert obs[4]["status"] == L.LBM_EUNSTABLE and 0 < obs[4]["step"] < 1500
    assert all(obs[i]["status"] == 0 for i in range(4))


def test_stalled_barrier_times_out(L):
    import time
    b = L.Batch([params(L, c, 1) for c in CASES[:3]])
    b.lbm_batch_init_droplets([c["r"] for c in CASES[:3]])
    _, _, grid = b.lbm_batch_size()
    b.lbm_batch_inject_stall(grid - 1)
    t0 = time.time()
    b.lbm_batch_step(3)
    rc, _ = b.lbm_batch_observables(raise_errors=False)
    assert rc == L.LBM_ETIMEOUT
    assert time.time() - t0 < 30
    b.lbm_batch_inject_stall(-1)
    # the context stays usable
    s = L.Sim(params(L, CASES[0], 1))
    s.lbm_init_droplet(CASES[0]["r"])
    s.lbm_step(5)
    assert s.lbm_observables()["status"] == 0


def test_tile_shapes_give_identical_results(L):
    # the same arithmetic per node in every tile shape: bitwise equal states
    cases = CASES[:4]
    dens = {}
    for rows in (1, 2, 4):
        b = L.Batch([params(L, c, 1) for c in cases])
        b.lbm_batch_set_tiles(rows)
        b.lbm_batch_init_droplets([c["r"] for c in cases])
        b.lbm_batch_step(25)
        dens[rows] = [b.lbm_batch_get_density(i) for i in range(len(cases))]
        nc, nitems, grid = b.lbm_batch_size()
        assert nc == len(cases) and nitems > 0 and grid > 0
        b.close()
    for rows in (1, 4):
        for a, d in zip(dens[rows], dens[2]):
            assert np.array_equal(a, d), rows


def test_autotune_keeps_a_shape_and_caches_it(L, tmp_path):
    cases = CASES[:4]
    cache = str(tmp_path / "tiles.json")
    b = L.Batch([params(L, c, 1) for c in cases])
    b.lbm_batch_init_droplets([c["r"] for c in cases])
    rows = b.lbm_batch_autotune(steps=2, cache=cache)
    assert rows in (1, 2, 4)
    b.lbm_batch_init_droplets([c["r"] for c in cases])
    b.lbm_batch_step(10)
    ref = L.Batch([params(L, c, 1) for c in cases])
    ref.lbm_batch_init_droplets([c["r"] for c in cases])
    ref.lbm_batch_step(10)
    for i in range(len(cases)):
        assert np.array_equal(b.lbm_batch_get_density(i), ref.lbm_batch_get_density(i))
    # a second batch of the same shapes takes the cached choice
    c2 = L.Batch([params(L, c, 1) for c in cases])
    assert c2.lbm_batch_autotune(steps=2, cache=cache) == rows
    import json
    assert list(json.load(open(cache)).values()) == [rows]
    with pytest.raises(L.LBMError) as e:
        b.lbm_batch_set_tiles(3)
    assert e.value.code == L.LBM_EINVAL
    for x in (b, ref, c2):
        x.close()


def test_many_cases_dealt_dynamically_match_single_runs(L):
    # enough work that every CTA claims several guided runs of collision items
    # and every warp several mu units, across phases, steps and graph replays;
    # seed 11, 48 cases of 128..384 nodes a side, all five schemes, stable T_r
    rng = np.random.default_rng(11)
    schemes = ["EFDS2", "EFDS4", "EFDS6", "E4", "E8"]
    cases = []
    for i in range(48):
        nx, ny = int(rng.integers(128, 385)), int(rng.integers(128, 385))
        cases.append(dict(nx=nx, ny=ny, Tr=float(rng.uniform(0.8, 0.95)), k=float(rng.uniform(0.15, 0.35)),
                          scheme=schemes[i % 5], r=float(rng.uniform(8, min(nx, ny) / 4))))
    dens = {}
    for rows in (2, 1):
        b = L.Batch([params(L, c, 1) for c in cases])
        b.lbm_batch_set_tiles(rows)
        b.lbm_batch_init_droplets([c["r"] for c in cases])
        for _ in range(3):
            b.lbm_batch_step(8)
        assert b.lbm_batch_get_step() == 24
        _, nitems, grid = b.lbm_batch_size()
        assert nitems > 4 * grid
        rc, obs = b.lbm_batch_observables(raise_errors=False)
        assert rc == 0 and all(o["status"] == 0 for o in obs)
        dens[rows] = [b.lbm_batch_get_density(i) for i in range(len(cases))]
        b.close()
    for a, d in zip(dens[1], dens[2]):
        assert np.array_equal(a, d)
    for i, c in enumerate(cases):
        s = L.Sim(params(L, c, 1))
        s.lbm_init_droplet(c["r"])
        s.lbm_step(24)
        rs = s.lbm_get_density()
        assert np.max(np.abs(dens[2][i] - rs)) / np.max(rs) < 1e-6, c
        s.close()


# compact schemes (Eq. 21-24; OCFDS4 of Sec. 3.1) inside the persistent launch:
# mu field, line solves for grad mu and grad rho along x and y as work items,
# then the collision reading the derivative fields, each phase behind the
# bounded barrier; mixed with an explicit case and uneven, ragged sizes
COMPACT = [dict(nx=64, ny=48, Tr=0.8, k=0.25, scheme="OCFDS4", r=12.0),
           dict(nx=40, ny=72, Tr=0.85, k=0.3, scheme="CFDS4", r=10.0),
           dict(nx=96, ny=80, Tr=0.8, k=0.2, scheme="CFDS6", r=18.0),
           dict(nx=36, ny=44, Tr=0.9, k=0.25, scheme="CFDS8", r=8.0),
           dict(nx=48, ny=48, Tr=0.8, k=0.25, scheme="EFDS6", r=10.0)]


def oracle_density(c, steps):
    o = O.Sim(lattice=O.D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1, scheme=c["scheme"])
    o.init_droplet(c["r"])
    assert o.step(steps) == 0
    return o.density(), o


def test_batch_compact_fp64_matches_oracle(L):
    b = L.Batch([params(L, c, 0) for c in COMPACT])
    b.lbm_batch_init_droplets([c["r"] for c in COMPACT])
    b.lbm_batch_step(15)
    b.lbm_batch_step(10)  # a replay continues the run
    rc, obs = b.lbm_batch_observables(raise_errors=False)
    assert rc == 0
    for i, c in enumerate(COMPACT):
        ro, o = oracle_density(c, 25)
        assert np.max(np.abs(b.lbm_batch_get_density(i) - ro)) / np.max(ro) < 1e-12, c
        oo = o.observables()
        assert obs[i]["status"] == 0
        for key in ("max_v", "max_u", "mass", "rho_center", "rho_corner"):
            assert obs[i][key] == pytest.approx(oo[key], rel=1e-10, abs=1e-300), (c, key)


@pytest.mark.parametrize("mu_fp64", [0, 1])
def test_batch_compact_fp32_matches_oracle_and_single_case(L, mu_fp64):
    ps = [L.make_params(lattice=L.LBM_D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1,
                        scheme=c["scheme"], precision=L.LBM_FP32DEV, mu_fp64=mu_fp64) for c in COMPACT]
    b = L.Batch(ps)
    b.lbm_batch_init_droplets([c["r"] for c in COMPACT])
    b.lbm_batch_step(25)
    rc, obs = b.lbm_batch_observables(raise_errors=False)
    assert rc == 0
    for i, c in enumerate(COMPACT):
        ro, o = oracle_density(c, 25)
        rl = O.maxwell_tr(c["Tr"])[1]
        rb = b.lbm_batch_get_density(i)
        assert np.max(np.abs(rb - ro)) / rl < 1e-5, c
        s = L.Sim(ps[i])
        s.lbm_init_droplet(c["r"])
        s.lbm_step(25)
        rs = s.lbm_get_density()
        assert np.max(np.abs(rb - rs)) / np.max(rs) < 1e-6, c
        so = s.lbm_observables()
        for key in ("max_v", "max_u", "mass", "rho_center", "rho_corner"):
            assert obs[i][key] == pytest.approx(so[key], rel=1e-3), (c, key)
        s.close()


def test_batch_compact_tile_shapes_identical(L):
    dens = {}
    ps = [params(L, c, 1) for c in COMPACT]
    for rows in (1, 2, 4):
        b = L.Batch(ps)
        b.lbm_batch_set_tiles(rows)
        b.lbm_batch_init_droplets([c["r"] for c in COMPACT])
        b.lbm_batch_step(20)
        dens[rows] = [b.lbm_batch_get_density(i) for i in range(len(COMPACT))]
        b.close()
    for rows in (1, 4):
        for a, d in zip(dens[rows], dens[2]):
            assert np.array_equal(a, d), rows
