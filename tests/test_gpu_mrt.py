"""GPU parity of the D2Q9 MRT collision (Eq. 1, 3-5, the paper's rates) with
the oracle: FP64 to 1e-12 for every D2Q9 scheme at tau = 1 and tau = 0.8,
FP32 deviation storage to 1e-5 of rho_l; the single-relaxation reduction
inside the library; the batch against single cases; D3Q19 refused."""
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


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("scheme", ["EFDS2", "EFDS4", "EFDS6", "E4", "E8", "CFDS4", "OCFDS4"])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_fp64_mrt_matches_oracle(L, scheme, tau):
    # 40 x 24: one full and one ragged tile in x, several in y
    kw = dict(nx=40, ny=24, Tr=0.85, k=0.3, kappa=0.1, tau=tau, scheme=scheme)
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, collision="MRT", **kw))
    o = O.Sim(lattice=O.D2Q9, collision="MRT", **kw)
    g.lbm_init_droplet(7.0)
    o.init_droplet(7.0)
    g.lbm_step(25)
    assert o.step(25) == 0
    assert relerr(g.lbm_get_density(), o.density()) < 1e-12
    assert relerr(g.lbm_get_f(), o.get_f()) < 1e-12


@pytest.mark.parametrize("scheme", ["EFDS6", "E4"])
def test_fp32dev_mrt_matches_oracle(L, scheme):
    kw = dict(nx=64, ny=48, Tr=0.8, k=0.25, kappa=0.1, tau=0.9, scheme=scheme)
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, collision="MRT", precision=L.LBM_FP32DEV, **kw))
    o = O.Sim(lattice=O.D2Q9, collision="MRT", **kw)
    g.lbm_init_droplet(12.0)
    o.init_droplet(12.0)
    g.lbm_step(100)
    assert o.step(100) == 0
    rl = O.maxwell_tr(0.8)[1]
    assert np.max(np.abs(g.lbm_get_density() - o.density())) / rl < 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_equal_rates_reproduce_single_relaxation(L, precision):
    tau = 0.75
    kw = dict(lattice=L.LBM_D2Q9, nx=48, ny=40, Tr=0.8, k=0.25, kappa=0.1, tau=tau, scheme="EFDS4",
              precision=precision)
    a = L.Sim(L.make_params(**kw))
    b = L.Sim(L.make_params(collision="MRT", mrt_s=[1.0 / tau] * 9, **kw))
    for s in (a, b):
        s.lbm_init_droplet(9.0)
        s.lbm_step(40)
    tol = 1e-13 if precision == 0 else 2e-6
    assert relerr(a.lbm_get_density(), b.lbm_get_density()) < tol


def test_batch_mrt_matches_single_cases(L):
    cases = [dict(nx=72, ny=64, Tr=0.8, k=0.25, scheme="EFDS6", r=12.0),
             dict(nx=96, ny=80, Tr=0.75, k=0.3, scheme="E8", r=15.0),
             dict(nx=64, ny=100, Tr=0.85, k=0.2, scheme="EFDS4", r=10.0)]
    params = [L.make_params(lattice=L.LBM_D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1, tau=0.9,
                            scheme=c["scheme"], precision=L.LBM_FP32DEV, collision="MRT") for c in cases]
    b = L.Batch(params)
    b.lbm_batch_init_droplets([c["r"] for c in cases])
    b.lbm_batch_step(30)
    for i, (c, p) in enumerate(zip(cases, params)):
        s = L.Sim(p)
        s.lbm_init_droplet(c["r"])
        s.lbm_step(30)
        assert relerr(b.lbm_batch_get_density(i), s.lbm_get_density()) < 1e-6
    b.close()


def test_mrt_on_d3q19_is_refused(L):
    with pytest.raises(L.LBMError) as e:
        L.Sim(L.make_params(lattice=L.LBM_D3Q19, nx=16, ny=16, nz=16, collision="MRT"))
    assert e.value.code == L.LBM_ENOTSUP
