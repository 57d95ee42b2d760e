"""Full-size parity on the benchmark workload (D3Q19 256^3 droplet, EFDS6,
FP32 deviation storage, the launch configuration bench.py times): one GPU step
is checked on sampled sub-boxes, each advanced by the FP64 oracle from the
GPU's own input populations.  The oracle's sub-box is periodic, so only its
core (at least 2R + 2 = 8 nodes from the sub-box faces, beyond the reach of
one step's stencils) is compared."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

N = 256
MARGIN = 8
CORE = 8


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


def take_box(a, z0, y0, x0, n):
    """a[..., z, y, x] periodic sub-box of edge n starting at (z0, y0, x0)."""
    iz = np.arange(z0, z0 + n) % a.shape[-3]
    iy = np.arange(y0, y0 + n) % a.shape[-2]
    ix = np.arange(x0, x0 + n) % a.shape[-1]
    return a[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def test_bench_workload_one_step_sampled(L):
    kw = dict(Tr=0.8, k=0.25, kappa=0.1, tau=1.0, scheme="EFDS6")
    sim = L.Sim(L.make_params(lattice=L.LBM_D3Q19, nx=N, ny=N, nz=N, precision=L.LBM_FP32DEV, **kw))
    sim.lbm_autotune()
    sim.lbm_init_droplet(60.0)
    sim.lbm_step(3)  # leave the exact initial state: inputs with nonzero velocity
    f0 = sim.lbm_get_f()
    sim.lbm_step(1)
    r1 = sim.lbm_get_density()
    rl = O.maxwell_tr(0.8)[1]
    n = CORE + 2 * MARGIN
    c = N // 2
    # interface (x = c + 60), bulk liquid (centre), bulk gas across the periodic corner
    for (z0, y0, x0) in ((c - n // 2, c - n // 2, c + 60 - n // 2), (c - n // 2, c - n // 2, c - n // 2),
                         (N - n // 2, N - n // 2, N - n // 2)):
        fb = take_box(f0, z0, y0, x0, n)
        o = O.Sim(lattice=O.D3Q19, nx=n, ny=n, nz=n, **kw)
        o.set_f(fb)
        assert o.step(1) == 0
        ro = o.density()[MARGIN:MARGIN + CORE, MARGIN:MARGIN + CORE, MARGIN:MARGIN + CORE]
        rg = take_box(r1, z0 + MARGIN, y0 + MARGIN, x0 + MARGIN, CORE)
        err = np.max(np.abs(rg - ro)) / rl
        assert err < 1e-5, ((z0, y0, x0), err)
