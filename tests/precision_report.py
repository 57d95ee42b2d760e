"""Error of every observable of the FP32-deviation path against the FP64 oracle.

Run on a machine with the GPU (python tests/precision_report.py [out.md]); it
calls only the oracle and the library through its C ABI, and prints one
markdown table:

* transient rows: droplets (Eq. 26 start) after 100 steps, D2Q9 128^2 (r0 = 32)
  and D3Q19 48^3 (r0 = 12), EFDS6 and OCFDS4, T_r 0.8 / 0.5 / 0.3 / 0.2, k = 0.25
  (OCFDS4 at T_r 0.2: k = 0.15, the k = 0.25 case being ill-conditioned),
  FP32 chemical potential (mu32) and FP64 chemical potential (mu64), plus the
  FP64 storage mode for reference;
* equilibrium rows: D2Q9 64^2 droplet (r0 = 16) relaxed for 5000 steps, with
  the FP32 noise floor of max |v| measured on a 16 x 64 flat slab after 15000
  steps (the oracle's slab velocity having decayed below it), and one droplet
  run for 40000 steps.

Columns: relative errors of max |v|, max |u|, rho at the centre node, rho at the
corner node (the gas), total mass and max |d rho / dt| (over the last 100 steps
for transients, 1000 for equilibrium; where the oracle's has converged below
1e-9 per step both absolute values are shown), and the node-wise
max |drho| / rho_l.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

KEYS = ("max_v", "max_u", "rho_center", "rho_corner", "mass", "max_drho")


def pair(L, lat, shape, Tr, scheme, k, prec, mu64):
    nx, ny, nz = shape
    g = L.Sim(L.make_params(lattice=L.LBM_D2Q9 if lat == 2 else L.LBM_D3Q19, nx=nx, ny=ny, nz=nz, Tr=Tr, k=k,
                            kappa=0.1, scheme=scheme, precision=prec, mu_fp64=mu64))
    return g


def run_gpu(L, lat, shape, Tr, scheme, k, prec, mu64, init, steps, last):
    g = pair(L, lat, shape, Tr, scheme, k, prec, mu64)
    (g.lbm_init_droplet if init[0] == "droplet" else (lambda s: g.lbm_init_slab(1, s)))(init[1])
    g.lbm_step(steps - last)
    g.lbm_observables()
    g.lbm_step(last)
    return g.lbm_get_density(), g.lbm_observables()


_OR = {}


def run_oracle(lat, shape, Tr, scheme, k, init, steps, last):
    key = (lat, shape, Tr, scheme, k, init, steps, last)
    if key not in _OR:
        nx, ny, nz = shape
        o = O.Sim(lattice=O.D2Q9 if lat == 2 else O.D3Q19, nx=nx, ny=ny, nz=nz, Tr=Tr, k=k, kappa=0.1, scheme=scheme)
        if init[0] == "droplet":
            o.init_droplet(init[1])
        else:
            o.init_slab(1, init[1])
        rc = o.step(steps - last)
        o.observables()
        rc |= o.step(last)
        _OR[key] = (rc, o.density(), o.observables())
    return _OR[key]


def rel(a, b):
    return abs(a - b) / abs(b) if b else abs(a)


def main(out=None):
    import torch
    assert torch.cuda.is_available(), "the report needs the GPU"
    import paper_2205_09186_gb300 as pkg
    pkg.build()
    from paper_2205_09186_gb300 import lbm as L
    modes = [("FP64", L.LBM_FP64, 0), ("FP32DEV mu32", L.LBM_FP32DEV, 0), ("FP32DEV mu64", L.LBM_FP32DEV, 1)]
    lines = ["| case | mode | max_v | max_u | rho_center | rho_corner | mass | max_drho | max drho / rho_l |",
             "|---|---|---|---|---|---|---|---|---|"]
    cases = []
    for lat, shape, r in ((2, (128, 128, 1), 32.0), (3, (48, 48, 48), 12.0)):
        for Tr in (0.8, 0.5, 0.3, 0.2):
            for scheme in ("EFDS6", "OCFDS4"):
                k = 0.15 if (scheme == "OCFDS4" and Tr == 0.2) else 0.25
                cases.append((lat, shape, Tr, scheme, k, ("droplet", r), 100, 100,
                              "%s %s T_r %g k %g, 100 steps" % ("D2Q9 128^2" if lat == 2 else "D3Q19 48^3", scheme,
                                                                Tr, k)))
    for scheme, Tr in (("EFDS6", 0.8), ("OCFDS4", 0.8), ("EFDS6", 0.5)):
        cases.append((2, (64, 64, 1), Tr, scheme, 0.25, ("droplet", 16.0), 5000, 1000,
                      "D2Q9 64^2 %s T_r %g k 0.25, equilibrium (5000 steps)" % (scheme, Tr)))
    # a long run: the slow drift that FP32 rounding of the chemical potential
    # leaves in the equilibrium, and that the FP64 chemical potential removes
    cases.append((2, (64, 64, 1), 0.8, "EFDS6", 0.25, ("droplet", 16.0), 40000, 1000,
                  "D2Q9 64^2 EFDS6 T_r 0.8 k 0.25, 40000 steps"))
    for lat, shape, Tr, scheme, k, init, steps, last, name in cases:
        rg, rl = O.maxwell_tr(Tr)
        rc, ro, oo = run_oracle(lat, shape, Tr, scheme, k, init, steps, last)
        if rc != 0:
            lines.append("| %s | oracle unstable | | | | | | | |" % name)
            continue
        for mname, prec, mu64 in modes:
            rho, og = run_gpu(L, lat, shape, Tr, scheme, k, prec, mu64, init, steps, last)
            if og["status"] != 0:
                lines.append("| %s | %s | unstable | | | | | | |" % (name, mname))
                continue
            # a converged max |d rho / dt| (the oracle's ~1e-13 per step) has
            # no meaningful relative error: both absolute values are shown
            errs = [("%.1e" % rel(og[k_], oo[k_])) if not (k_ == "max_drho" and abs(oo[k_]) < 1e-9)
                    else "abs %.0e vs %.0e" % (og[k_], oo[k_]) for k_ in KEYS]
            lines.append("| %s | %s | %s | %.1e |" % (name, mname, " | ".join(errs),
                                                      float(np.max(np.abs(rho - ro))) / rl))
        if steps == 5000:
            _, _, os_ = run_oracle(2, (16, 64, 1), Tr, scheme, 0.25, ("slab", 32.0), 15000, 100)
            for mname, prec, mu64 in modes[1:]:
                _, gs = run_gpu(L, 2, (16, 64, 1), Tr, scheme, 0.25, prec, mu64, ("slab", 32.0), 15000, 100)
                lines.append("| %s: flat-slab noise floor of max_v | %s | %.1e (oracle %.1e; droplet oracle max_v %.3e) "
                             "| | | | | | |" % (name.split(",")[0], mname, gs["max_v"], os_["max_v"], oo["max_v"]))
    text = "\n".join(lines) + "\n"
    print(text)
    if out:
        with open(out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
