"""How much float storage alone can move the FP64 oracle (CPU, oracle only).

FP32 deviation storage keeps f_i - w_i rho_g in float.  Rounding only the
stored populations of an FP64 run to float after every step, and comparing with
the unrounded run, measures the floor that the problem itself puts under any
float-storage result.  On the 128^2 droplet of the low-temperature parity tests
that floor is ~1e-7 of rho_l after 100 steps, except for the optimised compact
scheme (OCFDS4, Sec. 3.1) at T_r 0.2 with k = 0.25, where the start transient
of the tanh profile (Eq. 26) amplifies the rounding to ~4e-5 of rho_l; with a
wider interface (k = 0.15, inside the paper's 0.1-0.4 range) the amplification
is gone.  The GPU parity tests run that case at k = 0.15 for this reason.
"""
import numpy as np
import pytest

import oracle as O


def storage_floor(scheme, Tr, k, steps=100):
    kw = dict(lattice=O.D2Q9, nx=128, ny=128, Tr=Tr, k=k, kappa=0.1, scheme=scheme)
    a, b = O.Sim(**kw), O.Sim(**kw)
    a.init_droplet(32.0)
    b.init_droplet(32.0)
    rg, rl = O.maxwell_tr(Tr)
    w = O.lattice(O.D2Q9)[1].reshape(9, 1, 1)
    for _ in range(steps):
        f = b.get_f()
        b.set_f(w * rg + (f - w * rg).astype(np.float32).astype(np.float64))
        assert a.step(1) == 0 and b.step(1) == 0
    return float(np.max(np.abs(a.density() - b.density()))) / rl


@pytest.mark.parametrize("scheme,Tr,k", [("EFDS6", 0.2, 0.25), ("OCFDS4", 0.2, 0.15), ("OCFDS4", 0.3, 0.25)])
def test_float_storage_floor_is_small(scheme, Tr, k):
    assert storage_floor(scheme, Tr, k) < 1e-6


def test_ocfds4_low_temperature_narrow_interface_is_ill_conditioned():
    assert storage_floor("OCFDS4", 0.2, 0.25) > 1e-5
