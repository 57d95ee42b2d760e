"""Learned warm start: the solver generates converged profiles, the library's
MLP kernels fit them, and a predicted profile starts a held-out droplet closer
to its converged state than the tanh profile of Eq. 26; the warm-started run
relaxes to the same densities as the cold-started one (both relaxed until
max |d rho / dt| stagnates at the FP32 rounding floor), to 1e-5 of the liquid
density."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import warmstart
    return warmstart


def test_warm_start_gain_and_agreement(W):
    L = W.L
    n = 48
    train = [dict(Tr=tr, k=k, R=R, scheme="EFDS6") for tr in (0.65, 0.75) for k in (0.25, 0.35) for R in (11.0, 14.0)]
    X, Y, info = W.generate(train, n=n, tol=1e-6, max_steps=6000, check_every=200)
    assert len(X) >= 6
    net, loss, _ = W.train(X, Y, iters=1500, lr=2e-3)
    assert loss < 0.02
    case = dict(Tr=0.7, k=0.3, R=12.5, scheme="EFDS6")
    # cold start: tanh profile; relax and take the converged profile
    sim, p = W.make_sim(n, case["Tr"], case["k"])
    sim.lbm_init_droplet(case["R"])
    c = (n // 2, n // 2, n // 2)
    r = W.window(case["R"])
    cold0 = W.radial_profile(sim.lbm_get_density(), c, r)
    steps_c, _, ok_c, obs_c, _ = W.relax(sim, 1e-10, 40000, 200, fp32_floor=True)
    conv = W.radial_profile(sim.lbm_get_density(), c, r)
    assert ok_c
    # warm start from the network
    sim2, p2 = W.make_sim(n, case["Tr"], case["k"])
    rr, rho = W.predict(net, case["Tr"], case["k"], case["R"], case["scheme"], p2, n=n)
    sim2.lbm_init_profile(rr, rho)
    warm0 = W.radial_profile(sim2.lbm_get_density(), c, r)
    assert np.linalg.norm(warm0 - conv) < np.linalg.norm(cold0 - conv)
    steps_w, _, ok_w, obs_w, _ = W.relax(sim2, 1e-10, 40000, 200, fp32_floor=True)
    assert ok_w
    # the droplet survives (centre is liquid) and both starts reach the same state
    rl = L.lbm_maxwell(p)[1]
    assert obs_c["rho_center"] > 0.5 * rl
    assert abs(obs_w["rho_center"] - obs_c["rho_center"]) / rl < 1e-5
    assert abs(obs_w["rho_corner"] - obs_c["rho_corner"]) / rl < 1e-5
