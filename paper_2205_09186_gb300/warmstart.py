"""Learned warm start for droplet runs (no counterpart in the paper).

The solver itself produces training data: D3Q19 droplets relaxed from the
tanh profile of Eq. 26 until the density stops changing; the converged radial
density profile of each run is the target.  A small GELU network (4 inputs ->
3 x 128 -> 64 outputs) is trained on the GPU by the library's own kernels
(lbm_mlp_*), then predicts the initial profile of new droplets.  Warm and
cold (tanh) starts are relaxed by the same solver to the same criterion; the
cold-start result judges the warm start's final densities.

Network input: (T_r, ln k, R / 64, scheme id / 8).  Output: 64 samples of
(rho - rho_g) / (rho_l - rho_g) (Maxwell densities) at r_j = max(0, R - 16) +
j / 2, j = 0..63; the profile is held at its end values outside the window.
"""
import math
import time

import numpy as np

from . import lbm as L

SIZES = [4, 128, 128, 128, 64]
NPROF = 64


def window(R):
    r0 = max(0.0, R - 16.0)
    return r0 + 0.5 * np.arange(NPROF)


def features(Tr, k, R, scheme):
    s = L.SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    return np.array([Tr, math.log(k), R / 64.0, s / 8.0], dtype=np.float64)


def radial_profile(rho, center, r):
    """Average of the six axis rays through `center` (3D field rho[z, y, x]),
    linearly interpolated at radii r."""
    nz, ny, nx = rho.shape
    cz, cy, cx = int(center[2]), int(center[1]), int(center[0])
    rays = [rho[cz, cy, cx:], rho[cz, cy, cx::-1], rho[cz, cy:, cx], rho[cz, cy::-1, cx], rho[cz:, cy, cx],
            rho[cz::-1, cy, cx]]
    n = min(len(a) for a in rays)
    prof = np.mean([a[:n] for a in rays], axis=0)
    return np.interp(r, np.arange(n), prof)


def relax(sim, tol, max_steps, check_every=100):
    """Step until max |d rho / dt| over a check interval falls below tol.
    Returns (steps, device seconds of the stepping, converged, observables)."""
    import torch
    stream = torch.cuda.current_stream()
    steps, dev_ms = 0, 0.0
    sim.lbm_observables()
    obs = None
    while steps < max_steps:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.lbm_step(check_every)
        e1.record(stream)
        obs = sim.lbm_observables()
        dev_ms += e0.elapsed_time(e1)
        steps += check_every
        if obs["status"] != 0:
            return steps, dev_ms * 1e-3, False, obs
        if obs["max_drho"] < tol:
            return steps, dev_ms * 1e-3, True, obs
    return steps, dev_ms * 1e-3, False, obs


def make_sim(n, Tr, k, scheme="EFDS6", precision=L.LBM_FP32DEV):
    p = L.make_params(lattice=L.LBM_D3Q19, nx=n, ny=n, nz=n, Tr=Tr, k=k, kappa=0.1, scheme=scheme,
                      precision=precision)
    return L.Sim(p), p


def generate(cases, n=80, tol=1e-7, max_steps=20000, check_every=200):
    """Relax tanh-initialised droplets; return features X, normalised profiles Y, info."""
    X, Y, info = [], [], []
    for c in cases:
        sim, p = make_sim(n, c["Tr"], c["k"], c.get("scheme", "EFDS6"))
        sim.lbm_init_droplet(c["R"])
        steps, dev_s, ok, obs = relax(sim, tol, max_steps, check_every)
        if not ok:
            info.append(dict(c, steps=steps, converged=False))
            continue
        g, l = L.lbm_maxwell(p)
        rho = sim.lbm_get_density()
        prof = radial_profile(rho, (n // 2, n // 2, n // 2), window(c["R"]))
        X.append(features(c["Tr"], c["k"], c["R"], c.get("scheme", "EFDS6")))
        Y.append((prof - g) / (l - g))
        info.append(dict(c, steps=steps, converged=True, device_s=dev_s))
        sim.close()
    return np.array(X), np.array(Y), info


def train(X, Y, iters=3000, lr=1e-3, seed=0):
    rng = np.random.default_rng(seed)
    p = []
    for l in range(len(SIZES) - 1):
        p.append(rng.standard_normal(SIZES[l + 1] * SIZES[l]) * math.sqrt(2.0 / SIZES[l]))
        p.append(np.zeros(SIZES[l + 1]))
    net = L.MLP(SIZES, max(len(X), 32))
    net.lbm_mlp_set_params(np.concatenate(p))
    net.lbm_mlp_set_data(X, Y)
    loss = net.lbm_mlp_train(iters, lr)
    return net, loss


def predict(net, Tr, k, R, scheme, params):
    y = net.lbm_mlp_forward(features(Tr, k, R, scheme)[None, :])[0].astype(np.float64)
    g, l = L.lbm_maxwell(params)
    rho = g + (l - g) * y
    return window(R), np.maximum(rho, 0.5 * g)


def compare(net, cases, n=80, tol=1e-7, max_steps=20000, check_every=200):
    """Warm (network profile) vs cold (Eq. 26 tanh) start on each case."""
    rows = []
    for c in cases:
        out = {}
        for arm in ("cold", "warm"):
            sim, p = make_sim(n, c["Tr"], c["k"], c.get("scheme", "EFDS6"))
            if arm == "cold":
                sim.lbm_init_droplet(c["R"])
            else:
                r, rho = predict(net, c["Tr"], c["k"], c["R"], c.get("scheme", "EFDS6"), p)
                sim.lbm_init_profile(r, rho)
            steps, dev_s, ok, obs = relax(sim, tol, max_steps, check_every)
            out[arm] = dict(steps=steps, device_s=dev_s, converged=ok, rho_center=obs["rho_center"],
                            rho_corner=obs["rho_corner"], max_v=obs["max_v"])
            sim.close()
        out["case"] = c
        rl = max(abs(out["cold"]["rho_center"]), 1e-30)
        out["density_err"] = max(abs(out["warm"]["rho_center"] - out["cold"]["rho_center"]) / rl,
                                 abs(out["warm"]["rho_corner"] - out["cold"]["rho_corner"]) / rl)
        rows.append(out)
    return rows


def sample_cases(n, seed, Tr=(0.6, 0.9), k=(0.15, 0.3), R=(10.0, 20.0), scheme="EFDS6"):
    rng = np.random.default_rng(seed)
    return [dict(Tr=float(rng.uniform(*Tr)), k=float(math.exp(rng.uniform(math.log(k[0]), math.log(k[1])))),
                 R=float(rng.uniform(*R)), scheme=scheme) for _ in range(n)]


def experiment(n_train=48, n_test=16, n=80, tol=1e-7, iters=4000, seed=2205):
    t0 = time.time()
    train_cases = sample_cases(n_train, seed)
    test_cases = sample_cases(n_test, seed + 1)
    X, Y, info = generate(train_cases, n=n, tol=tol)
    net, loss = train(X, Y, iters=iters)
    rows = compare(net, test_cases, n=n, tol=tol)
    conv = [r for r in rows if r["warm"]["converged"] and r["cold"]["converged"]]
    res = {"lattice": "D3Q19 %d^3, EFDS6, FP32DEV" % n, "tol_max_drho": tol, "train_cases": len(X),
           "train_loss": loss, "test_cases": len(rows), "both_converged": len(conv),
           "cold_steps": sum(r["cold"]["steps"] for r in conv), "warm_steps": sum(r["warm"]["steps"] for r in conv),
           "cold_device_s": sum(r["cold"]["device_s"] for r in conv),
           "warm_device_s": sum(r["warm"]["device_s"] for r in conv),
           "max_density_err_vs_cold": max([r["density_err"] for r in conv], default=None),
           "train_generation_device_s": sum(i.get("device_s", 0.0) for i in info), "wall_s": time.time() - t0}
    return res, rows
