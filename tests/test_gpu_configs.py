"""Parity on the shapes of the paper-derived workloads: the 512^2 D2Q9 scheme
sweep (schemes x reduced temperature x proportional coefficient, FP64 and FP32
deviation storage) for a few steps from the tanh start, against the oracle."""
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


@pytest.mark.parametrize("scheme", ["EFDS2", "EFDS4", "EFDS6", "E4", "E8", "OCFDS4"])
@pytest.mark.parametrize("Tr,k", [(0.9, 0.1), (0.5, 0.4)])
def test_sweep_512_fp64_and_fp32(L, scheme, Tr, k):
    kw = dict(nx=512, ny=512, Tr=Tr, k=k, kappa=0.1, scheme=scheme)
    o = O.Sim(lattice=O.D2Q9, **kw)
    o.init_droplet(100.0)
    assert o.step(8) == 0
    ro = o.density()
    rl = O.maxwell_tr(Tr)[1]
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, precision=prec, **kw))
        g.lbm_init_droplet(100.0)
        g.lbm_step(8)
        err = np.max(np.abs(g.lbm_get_density() - ro)) / (np.max(ro) if prec == 0 else rl)
        assert err < tol, (prec, err)
