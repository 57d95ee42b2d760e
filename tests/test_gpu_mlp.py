"""Warm-start network kernels against the FP64 oracle: forward values,
loss and gradients (FP32 kernels, relative tolerance 1e-4), and an Adam
training run that follows the oracle's own Adam on the same data."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SIZES = [4, 128, 128, 128, 64]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


def init_params(sizes, seed):
    rng = np.random.default_rng(seed)
    p = []
    for l in range(len(sizes) - 1):
        p.append(rng.standard_normal(sizes[l + 1] * sizes[l]) / np.sqrt(sizes[l]))
        p.append(0.1 * rng.standard_normal(sizes[l + 1]))
    return np.concatenate(p)


@pytest.mark.parametrize("batch", [1, 31, 100, 257])
def test_forward_and_gradient_match_oracle(L, batch):
    p = init_params(SIZES, 1).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(batch)
    x = rng.uniform(-1, 1, (batch, 4)).astype(np.float32).astype(np.float64)
    t = rng.uniform(0, 1, (batch, 64)).astype(np.float32).astype(np.float64)
    m = L.MLP(SIZES, 512)
    m.lbm_mlp_set_params(p)
    y = m.lbm_mlp_forward(x)
    yo = O.mlp_forward(SIZES, p, x)
    assert np.max(np.abs(y - yo)) < 1e-4 * max(1.0, np.max(np.abs(yo)))
    loss, g = m.lbm_mlp_loss_grad(x, t)
    lo, go = O.mlp_loss_grad(SIZES, p, x, t)
    assert loss == pytest.approx(lo, rel=1e-4)
    assert np.max(np.abs(g - go)) < 1e-4 * np.max(np.abs(go))


def test_adam_training_follows_oracle(L):
    sizes = [4, 32, 32, 16]
    p0 = init_params(sizes, 2).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (64, 4)).astype(np.float32).astype(np.float64)
    t = np.tanh(x @ rng.standard_normal((4, 16))).astype(np.float32).astype(np.float64)
    m = L.MLP(sizes, 64)
    m.lbm_mlp_set_params(p0)
    m.lbm_mlp_set_data(x, t)
    m.lbm_mlp_train(20, lr=1e-2)
    pg = m.lbm_mlp_get_params()
    po, mo, vo = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for it in range(1, 21):
        _, g = O.mlp_loss_grad(sizes, po, x, t)
        O.adam_step(po, mo, vo, g, 1e-2, it)
    # Adam normalises each step, so parameters whose gradient is at the FP32
    # noise level may take differently signed steps: compare the bulk and the loss
    d = np.abs(pg - po)
    assert np.quantile(d, 0.99) < 1e-3 and np.median(d) < 1e-4
    l0 = O.mlp_loss_grad(sizes, p0, x, t)[0]
    lg, lo = O.mlp_loss_grad(sizes, pg.astype(np.float64), x, t)[0], O.mlp_loss_grad(sizes, po, x, t)[0]
    assert lo < 0.7 * l0 and lg == pytest.approx(lo, rel=2e-2)
