"""lbm_step_observe: n steps whose last one also reports the observables of the
state it started from.  On the split D3Q19 FP32-deviation path the collision
pass computes them in passing; the result must match lbm_observables taken
before that step (FP32 rounding apart) and the oracle's observables of the
same state, and the stepped state must match plain stepping.  Elsewhere the
call observes, then steps, and must equal doing exactly that."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

KEYS = ("max_v", "max_u", "mass", "rho_center", "rho_corner", "max_drho")


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


def make(L, shape, **kw):
    nx, ny, nz = shape
    lat = L.LBM_D2Q9 if nz == 1 else L.LBM_D3Q19
    args = dict(lattice=lat, nx=nx, ny=ny, nz=nz, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
                precision=L.LBM_FP32DEV)
    args.update(kw)
    s = L.Sim(L.make_params(**args))
    s.lbm_init_droplet(min(nx, ny) / 4.0)
    s.lbm_observables()  # snapshot at t = 0 for max |d rho / dt|
    return s


def close(a, b, rel, keys=KEYS):
    for k in keys:
        assert a[k] == pytest.approx(b[k], rel=rel, abs=1e-12 * max(1.0, abs(b[k]))), k


# nx % 4 == 0 takes the 16-byte copy variant of the collision pass, 42 the 4-byte one;
# mu_fp64 = 1: the same passes with the EOS chemical potential evaluated in FP64;
# 65 and 33 leave a last tile of one column, which joins the tile before it
@pytest.mark.parametrize("shape,scheme,mu_fp64", [((48, 40, 44), "EFDS6", 0), ((42, 36, 40), "EFDS4", 0),
                                                  ((40, 40, 40), "EFDS2", 0), ((48, 40, 44), "EFDS6", 1),
                                                  ((65, 23, 20), "EFDS6", 0), ((33, 24, 22), "EFDS4", 0)])
def test_fused_observation_matches_observe_then_step(L, shape, scheme, mu_fp64):
    a, b = make(L, shape, scheme=scheme, mu_fp64=mu_fp64), make(L, shape, scheme=scheme, mu_fp64=mu_fp64)
    t_prev = 0
    for n in (12, 5):  # two cycles: the second max |d rho / dt| uses the fused kernel's snapshot
        a.lbm_step(n - 1)
        oa = a.lbm_observables()
        a.lbm_step(1)
        ob = b.lbm_step_observe(n)
        assert ob["status"] == 0 and ob["step"] == oa["step"] == b.lbm_get_step() - 1
        close(ob, oa, 2e-6, keys=[k for k in KEYS if k != "max_drho"])
        # after the first cycle the two states differ by the FP32 rounding of the
        # observing step (bounded below by 1e-6 of max rho): max |d rho / dt|, a
        # difference of two such states, agrees to that bound over dt, not to a
        # relative tolerance of its own small value
        dt = ob["step"] - t_prev
        assert abs(ob["max_drho"] - oa["max_drho"]) <= 1e-6 * oa["rho_center"] / dt
        t_prev = ob["step"]
    ra, rb = a.lbm_get_density(), b.lbm_get_density()
    assert np.max(np.abs(ra - rb)) < 1e-6 * np.max(ra)
    assert np.max(np.abs(a.lbm_get_f() - b.lbm_get_f())) < 1e-6 * np.max(np.abs(a.lbm_get_f()))


def test_fused_observation_matches_oracle(L):
    shape = (40, 36, 44)
    b = make(L, shape)
    o = O.Sim(lattice=O.D3Q19, nx=40, ny=36, nz=44, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6")
    o.init_droplet(9.0)
    o.observables()
    ob = b.lbm_step_observe(16)
    o.step(15)
    oo = o.observables()
    assert ob["step"] == oo["step"] == 15
    # FP32 deviation storage against the FP64 oracle (the parity tolerance of the
    # densities; velocities to 1e-3 of their own scale: max |v| here is ~1e-2,
    # above 1e3 times the FP32 noise floor measured on flat slabs, ~5e-7)
    rl = O.maxwell_tr(0.8)[1]
    for k in ("rho_center", "rho_corner"):
        assert abs(ob[k] - oo[k]) < 1e-5 * rl, k
    assert ob["mass"] == pytest.approx(oo["mass"], rel=1e-6)
    for k in ("max_v", "max_u"):
        assert ob[k] == pytest.approx(oo[k], rel=1e-3, abs=1e-7), k


@pytest.mark.parametrize("shape,kw", [((48, 40, 1), dict(precision=0)), ((48, 40, 1), dict()),
                                      ((24, 24, 24), dict(scheme="OCFDS4")), ((24, 24, 24), dict(scheme="E4")),
                                      ((24, 24, 24), dict(precision=0, scheme="EFDS4"))])
def test_other_paths_observe_then_step(L, shape, kw):
    a, b = make(L, shape, **kw), make(L, shape, **kw)
    a.lbm_step(6)
    oa = a.lbm_observables()
    a.lbm_step(1)
    ob = b.lbm_step_observe(7)
    assert ob == oa
    assert np.array_equal(a.lbm_get_density(), b.lbm_get_density())


def test_step_observe_rejects_zero_steps(L):
    s = make(L, (16, 16, 1))
    with pytest.raises(L.LBMError) as e:
        s.lbm_step_observe(0)
    assert e.value.code == L.LBM_EINVAL


@pytest.mark.parametrize("shape,kw", [((48, 40, 44), dict()), ((48, 40, 1), dict()), ((24, 24, 24), dict(scheme="E4")),
                                      ((48, 40, 1), dict(precision=0)), ((32, 24, 28), dict(scheme="OCFDS4")),
                                      ((48, 40, 1), dict(scheme="EFDS4", walls=True))])
def test_async_observation_equals_the_synchronous_one(L, shape, kw):
    # the same kernels in the same order: bit-identical records, written by the
    # stream into page-locked host memory and into device memory
    import ctypes
    import torch
    kw = dict(kw)
    walls = kw.pop("walls", False)
    a, b = make(L, shape, **kw), make(L, shape, **kw)
    if walls:  # a flat wall of 4 rows (Appendix A) on both handles
        mask = np.zeros((shape[1], shape[0]), np.uint8)
        mask[:4] = 1
        mu_w = L.lbm_bulk_mu(a.params, L.lbm_maxwell(a.params)[0])  # saturation
        for s in (a, b):
            s.lbm_set_solid(mask, mu_w)
    size = ctypes.sizeof(L.lbm_obs)
    host = torch.empty(3 * size, dtype=torch.uint8).pin_memory()
    dev = torch.empty(size, dtype=torch.uint8, device="cuda")
    sync = [a.lbm_step_observe(n) for n in (9, 1, 4)]
    for k, n in enumerate((9, 1)):
        b.lbm_step_observe_async(n, host.data_ptr() + k * size)
    b.lbm_step_observe_async(4, dev.data_ptr())
    torch.cuda.synchronize()
    host[2 * size:] = dev.cpu()
    recs = [L.lbm_obs.from_address(host.data_ptr() + k * size).as_dict() for k in range(3)]
    assert recs == sync
    assert np.array_equal(a.lbm_get_density(), b.lbm_get_density())
