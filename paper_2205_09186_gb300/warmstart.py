"""Learned warm start for droplet runs (no counterpart in the paper).

The solver itself produces training data: D3Q19 droplets relaxed from the
tanh profile of Eq. 26 until the density stops changing; the converged radial
density profile of each run is the target.  A small GELU network (4 inputs ->
3 x 128 -> 64 outputs) is trained on the GPU by the library's own kernels
(lbm_mlp_*), then predicts the initial profile of new droplets.  Warm and
cold (tanh) starts are relaxed by the same solver to the same criterion; the
cold-start result judges the warm start's final densities.  Droplets that
evaporate (too small for their temperature) are left out of training and
counted apart in the comparison.

Network input: (T_r, ln k, R / 64, scheme id / 8).  Output: 64 samples of
(rho - rho_g) / (rho_l - rho_g) (Maxwell densities) at r_j = max(0, R - 16) +
j / 2, j = 0..63; the profile is held at its end values outside the window and
shifted radially (plus a uniform remainder) so that it holds the same mass as
the tanh start: both arms then relax towards the same equilibrium, which the
cold start defines.
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


STAG_CAP = 1e-8     # FP32 stagnation: max |d rho / dt| below this ...
STAG_CHECKS = 5     # ... and not 10% lower than the smallest of the previous checks


def relax(sim, tol, max_steps, check_every=100, fp32_floor=False):
    """Step until max |d rho / dt| over a check interval falls below tol, or,
    with fp32_floor (FP32 deviation storage), until it stagnates: below
    STAG_CAP and no longer falling (not 10% below the smallest of the previous
    STAG_CHECKS checks), the state moving only by the rounding drift of FP32
    storage, which stays above the FP64 criterion.  Returns (steps, device
    seconds of the stepping, converged, observables, how: "tol" or "stagnation")."""
    import torch
    stream = torch.cuda.current_stream()
    steps, dev_ms = 0, 0.0
    sim.lbm_observables()
    obs = None
    hist = []
    while steps < max_steps:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.lbm_step(check_every)
        e1.record(stream)
        obs = sim.lbm_observables()
        dev_ms += e0.elapsed_time(e1)
        steps += check_every
        if obs["status"] != 0:
            return steps, dev_ms * 1e-3, False, obs, None
        d = obs["max_drho"]
        if d < tol:
            return steps, dev_ms * 1e-3, True, obs, "tol"
        if fp32_floor and len(hist) >= STAG_CHECKS and d < STAG_CAP and d > 0.9 * min(hist[-STAG_CHECKS:]):
            return steps, dev_ms * 1e-3, True, obs, "stagnation"
        hist.append(d)
    return steps, dev_ms * 1e-3, False, obs, None


def survived(obs, g, l):
    """A droplet is left at the centre (centre density above the Maxwell midpoint)."""
    return obs["rho_center"] > 0.5 * (g + l)


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
        steps, dev_s, ok, obs, _ = relax(sim, tol, max_steps, check_every, fp32_floor=True)
        if not ok:
            info.append(dict(c, steps=steps, converged=False))
            continue
        g, l = L.lbm_maxwell(p)
        if not survived(obs, g, l):  # the droplet evaporated: no interface to learn
            info.append(dict(c, steps=steps, converged=True, survived=False, device_s=dev_s))
            sim.close()
            continue
        rho = sim.lbm_get_density()
        prof = radial_profile(rho, (n // 2, n // 2, n // 2), window(c["R"]))
        X.append(features(c["Tr"], c["k"], c["R"], c.get("scheme", "EFDS6")))
        Y.append((prof - g) / (l - g))
        info.append(dict(c, steps=steps, converged=True, survived=True, device_s=dev_s))
        sim.close()
    return np.array(X), np.array(Y), info


def train(X, Y, iters=3000, lr=1e-3, seed=0):
    """Adam on the MSE of the profiles, on the GPU; returns (net, final loss,
    device seconds of the training)."""
    import torch
    rng = np.random.default_rng(seed)
    p = []
    for l in range(len(SIZES) - 1):
        p.append(rng.standard_normal(SIZES[l + 1] * SIZES[l]) * math.sqrt(2.0 / SIZES[l]))
        p.append(np.zeros(SIZES[l + 1]))
    net = L.MLP(SIZES, max(len(X), 32))
    net.lbm_mlp_set_params(np.concatenate(p))
    net.lbm_mlp_set_data(X, Y)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    loss = net.lbm_mlp_train(iters, lr)
    e1.record(stream)
    e1.synchronize()
    return net, loss, e0.elapsed_time(e1) * 1e-3


def lattice_radii(n):
    """Distance of every node of an n^3 lattice to the centre node (n/2, n/2, n/2)."""
    c = n // 2
    x = np.arange(n) - c
    return np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)


def tanh_mass(n, R, params, width=10.0):
    """Mass of the Eq. 26 initial droplet on the n^3 lattice (Maxwell densities)."""
    g, l = L.lbm_maxwell(params)
    r = lattice_radii(n)
    return float(np.sum(0.5 * (l + g) - 0.5 * (l - g) * np.tanh(2.0 * (r - R) / width)))


MAX_REMAINDER = 0.05  # largest uniform mass remainder, as a fraction of the gas density


def predict(net, Tr, k, R, scheme, params, n=None):
    """Network profile (r, rho).  With n given, the profile is shifted radially so
    that its mass on the n^3 lattice equals that of the tanh start it replaces:
    the warm and cold starts then hold the same fluid and relax to the same state.
    Returns None when the shift leaves a remainder above MAX_REMAINDER x rho_g."""
    y = net.lbm_mlp_forward(features(Tr, k, R, scheme)[None, :])[0].astype(np.float64)
    g, l = L.lbm_maxwell(params)
    rho = np.maximum(g + (l - g) * y, 0.5 * g)
    r = window(R)
    if n is None:
        return r, rho
    rr = lattice_radii(n)
    target = tanh_mass(n, R, params)

    def placed(shift):
        rs = r + shift
        keep = rs >= 0
        return rs[keep], rho[keep]

    def mass(shift):
        return float(np.sum(np.interp(rr, *placed(shift))))

    lo, hi = -8.0, 8.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if mass(mid) < target:
            lo = mid
        else:
            hi = mid
    shift = 0.5 * (lo + hi)
    # what the shift cannot match (a profile that is nearly flat, or a shift
    # beyond the search range) is spread uniformly: every node takes its value
    # from the profile, so the masses are then equal
    rs, vs = placed(shift)
    rem = (target - mass(shift)) / rr.size
    if abs(rem) > MAX_REMAINDER * g:
        return None  # the network's profile cannot hold this mass: no warm start
    return rs, vs + rem


def compare(net, cases, n=80, tol=1e-10, max_steps=60000, check_every=200, plain=0):
    """Warm (network profile) vs cold (Eq. 26 tanh) start on each case, both
    with FP32 deviation storage; for the first `plain` cases also the plain
    run: FP64 storage from the tanh start."""
    rows = []
    for ic, c in enumerate(cases):
        out = {}
        for arm in ("cold", "warm", "plain") if ic < plain else ("cold", "warm"):
            prec = L.LBM_FP64 if arm == "plain" else L.LBM_FP32DEV
            sim, p = make_sim(n, c["Tr"], c["k"], c.get("scheme", "EFDS6"), precision=prec)
            if arm in ("cold", "plain"):
                sim.lbm_init_droplet(c["R"])
            else:
                prof = predict(net, c["Tr"], c["k"], c["R"], c.get("scheme", "EFDS6"), p, n=n)
                out["fallback"] = prof is None
                if prof is None:
                    sim.lbm_init_droplet(c["R"])
                else:
                    sim.lbm_init_profile(*prof)
            steps, dev_s, ok, obs, how = relax(sim, tol, max_steps, check_every, fp32_floor=(arm != "plain"))
            out[arm] = dict(steps=steps, device_s=dev_s, converged=ok, how=how, rho_center=obs["rho_center"],
                            rho_corner=obs["rho_corner"], max_v=obs["max_v"], max_drho=obs["max_drho"])
            sim.close()
        out["case"] = c
        g, rl = L.lbm_maxwell(L.make_params(Tr=c["Tr"]))
        out["survived"] = survived(out["cold"], g, rl)
        out["density_err"] = max(abs(out["warm"]["rho_center"] - out["cold"]["rho_center"]) / rl,
                                 abs(out["warm"]["rho_corner"] - out["cold"]["rho_corner"]) / rl)
        rows.append(out)
    return rows


def sample_cases(n, seed, Tr=(0.6, 0.85), k=(0.2, 0.35), R=(14.0, 22.0), scheme="EFDS6"):
    rng = np.random.default_rng(seed)
    return [dict(Tr=float(rng.uniform(*Tr)), k=float(math.exp(rng.uniform(math.log(k[0]), math.log(k[1])))),
                 R=float(rng.uniform(*R)), scheme=scheme) for _ in range(n)]


def experiment(n_train=48, n_test=16, n=80, tol=1e-10, iters=4000, seed=2205, plain=0, train_tol=1e-7,
               max_steps=60000, R=(14.0, 22.0)):
    """Generate, train, compare; the totals count the test cases where both arms
    converged and the cold-start droplet survived (an evaporating droplet has
    no profile to predict; those cases are counted separately).  Training
    profiles are relaxed to train_tol (a shape for the network to learn);
    the compared arms to tol (FP64: max |d rho / dt| < tol; FP32 storage: tol or
    stagnation at its rounding floor).  The warm arm is charged its training
    data and training as well as its own runs."""
    t0 = time.time()
    train_cases = sample_cases(n_train, seed, R=R)
    test_cases = sample_cases(n_test, seed + 1, R=R)
    X, Y, info = generate(train_cases, n=n, tol=train_tol, max_steps=max_steps)
    net, loss, train_s = train(X, Y, iters=iters)
    rows = compare(net, test_cases, n=n, tol=tol, plain=plain, max_steps=max_steps)
    both = [r for r in rows if r["warm"]["converged"] and r["cold"]["converged"]]
    conv = [r for r in both if r["survived"]]
    res = {"lattice": "D3Q19 %d^3, EFDS6, FP32DEV" % n, "tol_max_drho": tol, "train_cases": len(X),
           "train_evaporated": sum(1 for i in info if i.get("survived") is False),
           "train_loss": loss, "test_cases": len(rows), "both_converged": len(both),
           "test_evaporated": len(both) - len(conv), "counted": len(conv),
           "warm_fallbacks": sum(1 for r in rows if r["fallback"]),
           "max_density_err_evaporated": max([r["density_err"] for r in both if not r["survived"]], default=None),
           "cold_steps": sum(r["cold"]["steps"] for r in conv), "warm_steps": sum(r["warm"]["steps"] for r in conv),
           "cold_device_s": sum(r["cold"]["device_s"] for r in conv),
           "warm_device_s": sum(r["warm"]["device_s"] for r in conv),
           "max_density_err_vs_cold": max([r["density_err"] for r in conv], default=None),
           "warm_failed": sum(1 for r in rows if not r["warm"]["converged"]),
           "cold_failed": sum(1 for r in rows if not r["cold"]["converged"]),
           "train_generation_device_s": sum(i.get("device_s", 0.0) for i in info), "train_device_s": train_s,
           "fp32_arms_stopped_by": {h: sum(1 for r in conv for a in ("cold", "warm") if r[a]["how"] == h)
                                    for h in ("tol", "stagnation")},
           "wall_s": time.time() - t0}
    res["warm_total_device_s"] = res["warm_device_s"] + res["train_generation_device_s"] + train_s
    res["device_s_ratio_cold_over_warm"] = res["cold_device_s"] / res["warm_device_s"] if res["warm_device_s"] else None
    res["device_s_ratio_cold_over_warm_total"] = (res["cold_device_s"] / res["warm_total_device_s"]
                                                  if res["warm_total_device_s"] else None)
    if plain:
        # the plain arm: FP64 storage, tanh start, one case at a time
        both_p = [r for r in conv if "plain" in r and r["plain"]["converged"]]
        res.update(plain_counted=len(both_p),
                   plain_failed=sum(1 for r in rows if "plain" in r and not r["plain"]["converged"]),
                   plain_steps=sum(r["plain"]["steps"] for r in both_p),
                   plain_device_s=sum(r["plain"]["device_s"] for r in both_p),
                   warm_device_s_same_cases=sum(r["warm"]["device_s"] for r in both_p),
                   max_density_err_warm_vs_plain=max(
                       [max(abs(r["warm"]["rho_center"] - r["plain"]["rho_center"]),
                            abs(r["warm"]["rho_corner"] - r["plain"]["rho_corner"]))
                        / L.lbm_maxwell(L.make_params(Tr=r["case"]["Tr"]))[1] for r in both_p], default=None))
        res["device_s_ratio_plain_over_warm"] = (res["plain_device_s"] / res["warm_device_s_same_cases"]
                                                 if res["warm_device_s_same_cases"] else None)
        res["max_density_err_cold_vs_plain"] = max(
            [max(abs(r["cold"]["rho_center"] - r["plain"]["rho_center"]),
                 abs(r["cold"]["rho_corner"] - r["plain"]["rho_corner"]))
             / L.lbm_maxwell(L.make_params(Tr=r["case"]["Tr"]))[1] for r in both_p], default=None)
    res["wall_s"] = time.time() - t0
    return res, rows
