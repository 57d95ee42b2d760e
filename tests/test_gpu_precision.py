"""Reduced-precision contract of FP32 deviation storage against the FP64 oracle,
down to the low reduced temperatures of the paper's coexistence study (Sec. 3.4,
Fig. 13: T_r to 0.2), with the EOS chemical potential in FP32 (mu_fp64 = 0) and
in FP64 (mu_fp64 = 1).

* Densities: |rho_gpu - rho_oracle| / rho_l <= 1e-5 node-wise after 100 steps
  from the tanh start (Eq. 26), on D2Q9 128^2 and D3Q19 48^3, sixth-order
  central (EFDS6) and optimised compact (OCFDS4, Sec. 3.1) differences, at
  T_r 0.5, 0.3 and 0.2.  The gas density's relative error is reported apart
  (it is 1e-11 of rho_l at T_r 0.2 and carries no weight in the node-wise bar).
  OCFDS4 at T_r 0.2 runs at k = 0.15: with k = 0.25 the start transient
  amplifies float rounding by two orders of magnitude (see
  tests/test_oracle_conditioning.py: the oracle itself moves by 4e-5 of rho_l
  when only its stored populations are rounded to float each step), so no
  float storage can meet 1e-5 there; both sides must still agree that it goes
  unstable.
* Spurious currents at equilibrium (the ~1e-5 magnitudes of the paper's
  conclusion): a relaxed droplet's max |v| and max |u| agree to 1e-3 relative
  where the oracle's value exceeds 1e3 times the FP32 noise floor, else to the
  floor.  The floor is measured, not assumed: max |v| of the same FP32 path on a
  flat slab whose exact velocity (the oracle's) has decayed to nothing.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL_RHO = 1e-5      # node-wise density bar, relative to the liquid density
TOL_V = 1e-3        # spurious-current bar, relative, above 1e3 x the noise floor


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm
    return lbm


_ORACLE = {}


def oracle_run(lat, shape, Tr, scheme, k, init, steps):
    """FP64 oracle state after `steps` (cached: the two mu variants share it)."""
    key = (lat, shape, Tr, scheme, k, init, steps)
    if key not in _ORACLE:
        nx, ny, nz = shape
        o = O.Sim(lattice=O.D2Q9 if lat == 2 else O.D3Q19, nx=nx, ny=ny, nz=nz, Tr=Tr, k=k, kappa=0.1,
                  scheme=scheme)
        kind, size = init
        if kind == "droplet":
            o.init_droplet(size)
        else:
            o.init_slab(1, size)
        o.observables()
        rc = o.step(steps)
        _ORACLE[key] = (rc, o.density(), o.observables())
    return _ORACLE[key]


def gpu_run(L, lat, shape, Tr, scheme, k, init, steps, mu_fp64):
    nx, ny, nz = shape
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9 if lat == 2 else L.LBM_D3Q19, nx=nx, ny=ny, nz=nz, Tr=Tr, k=k,
                            kappa=0.1, scheme=scheme, precision=L.LBM_FP32DEV, mu_fp64=mu_fp64))
    kind, size = init
    if kind == "droplet":
        g.lbm_init_droplet(size)
    else:
        g.lbm_init_slab(1, size)
    g.lbm_observables()
    g.lbm_step(steps)
    return g.lbm_get_density(), g.lbm_observables()


LOW_T = [(0.5, "EFDS6", 0.25), (0.3, "EFDS6", 0.25), (0.2, "EFDS6", 0.25),
         (0.5, "OCFDS4", 0.25), (0.3, "OCFDS4", 0.25), (0.2, "OCFDS4", 0.15)]
LATTICES = [(2, (128, 128, 1), 32.0), (3, (48, 48, 48), 12.0)]


@pytest.mark.parametrize("mu_fp64", [0, 1])
@pytest.mark.parametrize("Tr,scheme,k", LOW_T)
@pytest.mark.parametrize("lat,shape,radius", LATTICES)
def test_low_temperature_densities(L, lat, shape, radius, Tr, scheme, k, mu_fp64):
    rg, rl = O.maxwell_tr(Tr)
    rc, ro, oo = oracle_run(lat, shape, Tr, scheme, k, ("droplet", radius), 100)
    assert rc == 0
    rho, og = gpu_run(L, lat, shape, Tr, scheme, k, ("droplet", radius), 100, mu_fp64)
    assert og["status"] == 0 and og["step"] == oo["step"] == 100
    err = float(np.max(np.abs(rho - ro))) / rl
    assert err < TOL_RHO, err
    # the gas phase, relative to its own density (reported; at T_r 0.2 the
    # Maxwell gas density is 1.2e-11 and the lattice's gas has not reached it)
    gas = ro < 2.0 * rg + 1e-3 * rl
    gas_rel = float(np.max(np.abs(rho[gas] - ro[gas]) / ro[gas])) if gas.any() else 0.0
    print("T_r %g %s k %g mu_fp64 %d: max |drho| / rho_l %.2e, gas relative %.2e, rho_corner relative %.2e"
          % (Tr, scheme, k, mu_fp64, err, gas_rel, abs(og["rho_corner"] / oo["rho_corner"] - 1)))
    # FP32 collision conserves mass only to its rounding: ~1.5e-6 after 100 steps
    assert abs(og["mass"] / oo["mass"] - 1) < TOL_RHO


def test_ill_conditioned_case_agrees_on_instability(L):
    # OCFDS4, T_r 0.2, k 0.25 on the 128^2 droplet: the oracle reports a
    # non-positive density within the first 1500 steps (at step s, to 50
    # steps); FP32 storage must be stable 200 steps before s and unstable 200
    # steps after it
    o = O.Sim(lattice=O.D2Q9, nx=128, ny=128, Tr=0.2, k=0.25, kappa=0.1, scheme="OCFDS4")
    o.init_droplet(32.0)
    step_o = None
    for n in range(0, 1500, 50):
        if o.step(50) != 0:
            step_o = n + 50
            break
    assert step_o is not None and step_o > 200
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=128, ny=128, Tr=0.2, k=0.25, kappa=0.1, scheme="OCFDS4",
                            precision=L.LBM_FP32DEV))
    g.lbm_init_droplet(32.0)
    g.lbm_step(step_o - 200)
    assert g.lbm_observables()["status"] == 0
    g.lbm_step(400)
    assert g.lbm_observables()["status"] == L.LBM_EUNSTABLE


EQ = [("EFDS6", 0.8), ("OCFDS4", 0.8), ("EFDS6", 0.5)]


@pytest.mark.parametrize("mu_fp64", [0, 1])
@pytest.mark.parametrize("scheme,Tr", EQ)
def test_equilibrium_spurious_currents(L, scheme, Tr, mu_fp64):
    # the FP32 noise floor: a flat slab (same parameters) whose exact velocity
    # has decayed; what the FP32 path still shows there is its rounding noise
    slab = (16, 64, 1)
    rc, _, os_ = oracle_run(2, slab, Tr, scheme, 0.25, ("slab", 32.0), 15000)
    assert rc == 0
    _, gs = gpu_run(L, 2, slab, Tr, scheme, 0.25, ("slab", 32.0), 15000, mu_fp64)
    floor = gs["max_v"]
    assert os_["max_v"] < 1e-2 * floor  # the slab's exact velocity is below the floor
    # a droplet relaxed for 5000 steps (equilibrium spurious currents)
    drop = (64, 64, 1)
    rc, _, od = oracle_run(2, drop, Tr, scheme, 0.25, ("droplet", 16.0), 5000)
    assert rc == 0
    _, gd = gpu_run(L, 2, drop, Tr, scheme, 0.25, ("droplet", 16.0), 5000, mu_fp64)
    assert gd["status"] == 0
    # max |u| = max |v - F / (2 rho)| stays at the interface force's scale
    # (~4e-2): far above the floor, it takes the relative bar
    for key in ("max_v", "max_u"):
        diff = abs(gd[key] - od[key])
        if od[key] > 1e3 * floor:
            assert diff <= TOL_V * od[key], (key, diff / od[key])
        else:
            assert diff <= floor, (key, diff, floor)
        print("%s T_r %g mu_fp64 %d %s: oracle %.4e, FP32 %.4e, |diff| %.2e, floor %.2e"
              % (scheme, Tr, mu_fp64, key, od[key], gd[key], diff, floor))
