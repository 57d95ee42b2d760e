"""Host-side logic of the learned warm start (no GPU): the predicted profile is
placed so that its lattice mass equals that of the tanh start it replaces, for
a realistic profile (matched by the radial shift) and for a flat one that no
shift can match (matched by the uniform remainder)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def W():
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import warmstart
    return warmstart


class FakeNet:
    """Stands in for the MLP: returns a fixed normalised profile."""

    def __init__(self, y):
        self.y = np.asarray(y, dtype=np.float32)

    def lbm_mlp_forward(self, x):
        return np.repeat(self.y[None, :], len(x), axis=0)


def lattice_mass(W, n, r, rho):
    return float(np.sum(np.interp(W.lattice_radii(n), r, rho)))


@pytest.mark.parametrize("shape", ["tanh", "flat"])
def test_predicted_profile_holds_the_tanh_mass(W, shape):
    L = W.L
    n, R = 32, 9.0
    p = L.make_params(lattice=L.LBM_D3Q19, nx=n, ny=n, nz=n, Tr=0.75, k=0.3, kappa=0.1, scheme="EFDS6")
    g, l = L.lbm_maxwell(p)
    r = W.window(R)
    target = W.tanh_mass(n, R, p)
    if shape == "tanh":  # a profile one node wider than the tanh start
        y = 0.5 - 0.5 * np.tanh(2.0 * (r - R - 1.0) / 8.0)
    else:  # uniform, 1% above the mean density of the tanh start: no shift can help
        y = np.full(W.NPROF, (1.01 * target / n ** 3 - g) / (l - g))
    rr, rho = W.predict(FakeNet(y), 0.75, 0.3, R, "EFDS6", p, n=n)
    assert lattice_mass(W, n, rr, rho) == pytest.approx(target, rel=1e-6)
    if shape == "tanh":  # matched by moving the interface inwards, far field untouched
        assert abs(rho[-1] - (g + (l - g) * y[-1])) < 1e-4 * l


def test_unplaceable_profile_gives_no_warm_start(W):
    L = W.L
    n, R = 32, 9.0
    p = L.make_params(lattice=L.LBM_D3Q19, nx=n, ny=n, nz=n, Tr=0.75, k=0.3, kappa=0.1, scheme="EFDS6")
    assert W.predict(FakeNet(np.full(W.NPROF, 0.5)), 0.75, 0.3, R, "EFDS6", p, n=n) is None
