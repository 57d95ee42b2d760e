#!/usr/bin/env python
"""Benchmark: fused D3Q19 chemical-potential LBM step on one GB300.

Workload (one step = one full time step of the hot path over the lattice):
D3Q19, 256^3 periodic, droplet r0 = 60, Carnahan-Starling EOS (a=1, b=4,
R=1), T_r = 0.8, k = 0.25, kappa = 0.1, tau = 1, sixth-order central
differences (EFDS6), populations stored in FP32 as deviations from w_i rho_g,
the density field as an FP32 deviation from rho_g, the chemical potential in
FP32 (reductions in FP64).  The f arrays (1.27 GB) are far larger than L2, so
no flush is needed between steps.  Extra legs: the same droplet at T_r 0.5
and 0.2 and with the FP64 chemical potential, the 512-case D2Q9 batch, D2Q9
512^2 / 4096^2, the compact schemes, the warm start.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead,
on a bounded sample of the same workload.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM-peak fraction of fused step; device-s to converged sweep vs plain"
UNIT = "MLUPS"
WORKLOAD = dict(lattice="D3Q19", nx=256, ny=256, nz=256, radius=60.0, Tr=0.8, k=0.25, kappa=0.1, tau=1.0,
                scheme="EFDS6", precision="FP32DEV", mu="fp32")
# algorithmic bytes per lattice update of the step: read + write the 19 FP32
# populations (152), read + write the FP32 density deviation (8), write + read
# the FP32 chemical potential field of the mu pass (8)
B_ALG = 19 * 4 * 2 + 4 * 2 + 4 * 2
# of which the collision/streaming pass (the dominant kernel) moves: populations
# read + write, density read + write, mu read
B_COLL = 19 * 4 * 2 + 4 * 2 + 4
B_MU = 4 + 4
SAMPLE_N = 128  # oracle sample lattice (same parameters, radius scaled)


def reduce_max_ms(total_ms, dist=None, device="cpu"):
    """Max over ranks of a rank's timed-region milliseconds (all ranks get it)."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank, steps, world, total_ms):
    """Whole-job throughput: lattice updates of all ranks over the slowest rank's time."""
    return nodes_per_rank * steps * world / (total_ms * 1e-3) / 1e6


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[2:]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


KERNEL_SOURCES = ["paper_2205_09186_gb300/csrc/step3d_split.cuh", "paper_2205_09186_gb300/csrc/lbm_device.cuh",
                  "paper_2205_09186_gb300/csrc/step3d_fast.cuh", "paper_2205_09186_gb300/csrc/step3d.cuh",
                  "paper_2205_09186_gb300/csrc/step3d_mu.cuh", "paper_2205_09186_gb300/csrc/coll3d_launch.cuh"]
TRAFFIC_FILE = "profiles/k_coll3d_d3q19_fp32dev_traffic.txt"


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(n_nodes):
    """DRAM bytes per launch of the collision pass from the committed ncu
    capture, scaled to n_nodes by bytes per lattice update; None when the
    kernel sources changed since the capture."""
    try:
        kv = {}
        with open(os.path.join(ROOT, TRAFFIC_FILE)) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha256_16") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_lu"]) * n_nodes
    except Exception:
        return None


def oracle_sample(steps, n=SAMPLE_N):
    """Time the FP64 oracle on an n^3 sample with the workload's parameters."""
    import oracle as O
    w = WORKLOAD
    s = O.Sim(lattice=O.D3Q19, nx=n, ny=n, nz=n, Tr=w["Tr"], k=w["k"], kappa=w["kappa"], tau=w["tau"],
              scheme=w["scheme"])
    s.init_droplet(w["radius"] * n / w["nx"])
    t = time.perf_counter()
    rc = s.step(steps)
    dt = time.perf_counter() - t
    assert rc == 0
    return n ** 3 * steps / dt / 1e6, dt


SWEEP_SCHEMES = ["EFDS2", "EFDS4", "EFDS6", "E4", "E8", "OCFDS4"]


def batch_cases(n=512, seed=2205, schemes=None):
    """Seeded sweep of D2Q9 droplets: sizes uniform in {64..512}^2, radius uniform
    in [8, L/4], T_r uniform in [0.2, 0.95], k log-uniform in [0.1, 0.4], scheme
    uniform over the sweep set: second-, fourth- and sixth-order central,
    isotropic E4 and E8, and the optimised compact OCFDS4 (Sec. 3.1)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    schemes = schemes or SWEEP_SCHEMES
    out = []
    for _ in range(n):
        lx, ly = int(rng.integers(64, 513)), int(rng.integers(64, 513))
        r0 = float(rng.uniform(8, min(lx, ly) / 4))
        tr = float(rng.uniform(0.2, 0.95))
        k = float(np.exp(rng.uniform(np.log(0.1), np.log(0.4))))
        sch = schemes[int(rng.integers(0, len(schemes)))]
        out.append(dict(nx=lx, ny=ly, r=r0, Tr=tr, k=k, scheme=sch))
    return out


def run_batch(L, steps=50, warmup=10, ncases=512, schemes=None):
    """ncases (512) D2Q9 droplets of uneven sizes in one persistent graph-captured
    launch per lbm_batch_step (FP32 deviation storage); returns MLUPS and case
    counts."""
    import torch
    cases = batch_cases(ncases, schemes=schemes)
    params = [L.make_params(lattice=L.LBM_D2Q9, nx=c["nx"], ny=c["ny"], Tr=c["Tr"], k=c["k"], kappa=0.1,
                            scheme=c["scheme"], precision=L.LBM_FP32DEV) for c in cases]
    b = L.Batch(params)
    # tile shape by timing on the initial droplets (the tuning advances the
    # state: initialise again afterwards)
    b.lbm_batch_init_droplets([c["r"] for c in cases])
    rows = b.lbm_batch_autotune(steps=steps)  # launches as long as the timed one
    b.lbm_batch_init_droplets([c["r"] for c in cases])
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    b.lbm_batch_step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.lbm_batch_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rc, obs = b.lbm_batch_observables(raise_errors=False)
    stable = sum(1 for o in obs if o["status"] == 0)
    # the unstable cases (low T_r with second-order or isotropic gradients)
    # keep stepping on non-finite values inside the timed launches: also
    # count only the nodes of the cases still stable at the end (a lower bound
    # on useful work, since they were stepped for part of the run)
    stable_nodes = sum(c["nx"] * c["ny"] for c, o in zip(cases, obs) if o["status"] == 0)
    by_scheme = {}
    for c, o in zip(cases, obs):
        d = by_scheme.setdefault(c["scheme"], [0, 0])
        d[0] += 1
        d[1] += int(o["status"] == 0)
    ncases, nitems, grid = b.lbm_batch_size()
    b.close()
    return {"workload": "%d D2Q9 droplets, sizes U{64..512}^2 (seed 2205), FP32DEV, one persistent launch" % ncases,
            "schemes": sorted(by_scheme), "nodes": nodes, "steps": steps, "ms": ms,
            "mlups": nodes * steps / (ms * 1e-3) / 1e6,
            "mlups_stable_cases": stable_nodes * steps / (ms * 1e-3) / 1e6,
            "hbm_frac": nodes * steps * (9 * 4 * 2 + 4 * 2) / (ms * 1e-3) / 1e9 / measured_peak()[0],
            "stable_cases": stable, "cases_stable_by_scheme": by_scheme, "work_items": nitems,
            "resident_ctas": grid, "tile_rows_per_thread": rows, "status": rc}


def run_cfg2_sweep(L, steps=50, warmup=5):
    """The 512^2 droplet sweep (r0 = 100): schemes {EFDS2, EFDS4, EFDS6, E4, E8,
    OCFDS4} x T_r {0.9, 0.7, 0.5, 0.3, 0.2} x k {0.1, 0.4}, each half of the
    storage choice (FP32 deviations, FP64) as one persistent batch: MLUPS of
    each half and the cases still stable after warmup + steps."""
    import torch
    out = {"workload": "D2Q9 512^2 droplets r0=100, 6 schemes x 5 T_r x 2 k, per storage mode one batch"}
    for name, prec in (("fp32dev", L.LBM_FP32DEV), ("fp64", L.LBM_FP64)):
        params = [L.make_params(lattice=L.LBM_D2Q9, nx=512, ny=512, Tr=tr, k=k, kappa=0.1, scheme=sch, precision=prec)
                  for sch in SWEEP_SCHEMES for tr in (0.9, 0.7, 0.5, 0.3, 0.2) for k in (0.1, 0.4)]
        b = L.Batch(params)
        b.lbm_batch_init_droplets([100.0] * len(params))
        b.lbm_batch_step(warmup)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.lbm_batch_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rc, obs = b.lbm_batch_observables(raise_errors=False)
        nodes = 512 * 512 * len(params)
        out[name] = {"cases": len(params), "steps": steps, "ms": ms, "mlups": nodes * steps / (ms * 1e-3) / 1e6,
                     "stable_cases": sum(1 for o in obs if o["status"] == 0), "status": rc}
        b.close()
    return out


def run_2d(L, steps=200, warmup=20):
    """D2Q9 512^2 droplet (r0 = 100, T_r = 0.8, k = 0.25, EFDS6, FP32 deviation
    storage): BGK and the MRT operator of Eq. 1, 3-5; MLUPS and the roofline of
    the collision pass (84 B per lattice update); the same droplet on a wall."""
    import numpy as np
    import torch
    out = {"workload": "D2Q9 512^2 droplet r0=100, T_r 0.8, k 0.25, EFDS6, FP32DEV, tau 1"}
    for col in ("BGK", "MRT"):
        s = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=512, ny=512, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
                                precision=L.LBM_FP32DEV, collision=col))
        s.lbm_init_droplet(100.0)
        rows = s.lbm_autotune()  # tile rows by timing (leaves the state undefined)
        s.lbm_init_droplet(100.0)
        s.lbm_step(warmup)
        torch.cuda.synchronize()
        ms = s.lbm_step_timed(steps)
        n = 512 * 512
        coll_ms = ms[1] / steps
        out[col.lower()] = {"mlups": n * steps / (ms[2] * 1e-3) / 1e6, "ms_per_step": ms[2] / steps,
                            "coll_ms": coll_ms, "mu_ms": ms[0] / steps,
                            "coll_frac": 84 * n / (coll_ms * 1e-3) / 1e9 / measured_peak()[0],
                            "tile_rows_per_thread": rows, "status": s.lbm_observables()["status"]}
        s.close()
    # a lattice larger than L2: 4096^2 (1.2 GB of populations), r0 = 800
    s = L.Sim(L.make_params(lattice=L.LBM_D2Q9, nx=4096, ny=4096, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
                            precision=L.LBM_FP32DEV))
    s.lbm_init_droplet(800.0)
    rows = s.lbm_autotune()  # tile rows by timing (leaves the state undefined)
    s.lbm_init_droplet(800.0)
    s.lbm_step(5)
    torch.cuda.synchronize()
    ms = s.lbm_step_timed(20)
    n = 4096 * 4096
    out["bgk_4096"] = {"mlups": n * 20 / (ms[2] * 1e-3) / 1e6, "ms_per_step": ms[2] / 20, "coll_ms": ms[1] / 20,
                       "mu_ms": ms[0] / 20, "coll_frac": 84 * n / (ms[1] / 20 * 1e-3) / 1e9 / measured_peak()[0],
                       "tile_rows_per_thread": rows,
                       "status": s.lbm_observables()["status"]}
    s.close()
    # the same droplet sitting on a flat wall of 8 rows (Appendix A), wall
    # chemical potential 0.005 below saturation; node-parallel wall step
    p = L.make_params(lattice=L.LBM_D2Q9, nx=512, ny=512, Tr=0.8, k=0.25, kappa=0.1, scheme="EFDS6",
                      precision=L.LBM_FP32DEV)
    s = L.Sim(p)
    s.lbm_init_droplet(100.0, center=[256.0, 8.0 + 80.0, 0.0])
    mask = np.zeros((512, 512), np.uint8)
    mask[:8] = 1
    s.lbm_set_solid(mask, L.lbm_bulk_mu(p, L.lbm_maxwell(p)[0]) - 0.005)
    s.lbm_step(warmup)
    torch.cuda.synchronize()
    ms = s.lbm_step_timed(steps)
    n = 512 * 512
    out["walls"] = {"mlups": n * steps / (ms[2] * 1e-3) / 1e6, "ms_per_step": ms[2] / steps,
                    "status": s.lbm_observables()["status"]}
    s.close()
    return out


def run_compact(L, steps=20, warmup=5, n=192):
    """D3Q19 n^3 droplet (r0 = 45, T_r 0.8, k 0.25) with the compact schemes
    (Sec. 3.1: OCFDS4; Eq. 23: CFDS6), FP32 deviation storage: mu field, one
    periodic tridiagonal line solve per field and axis, then the collision pass
    reading the derivative fields."""
    import torch
    out = {"workload": "D3Q19 %d^3 droplet r0=45, T_r 0.8, k 0.25, FP32DEV, tau 1" % n}
    for sch in ("OCFDS4", "CFDS6"):
        s = L.Sim(L.make_params(lattice=L.LBM_D3Q19, nx=n, ny=n, nz=n, Tr=0.8, k=0.25, kappa=0.1, scheme=sch,
                                precision=L.LBM_FP32DEV))
        s.lbm_init_droplet(45.0)
        zc = s.lbm_autotune()  # the collision pass's z-chunk, timed (the state is then undefined)
        s.lbm_init_droplet(45.0)
        s.lbm_step(warmup)
        torch.cuda.synchronize()
        ms = s.lbm_step_timed(steps)
        out[sch.lower()] = {"mlups": n ** 3 * steps / (ms[2] * 1e-3) / 1e6, "ms_per_step": ms[2] / steps,
                            "zchunk": zc, "status": s.lbm_observables()["status"]}
        s.close()
    return out


def run_cfg3_legs(L, zc, steps=20, warmup=5, n=256, check_steps=300):
    """The 256^3 droplet (r0 = 60, EFDS6, FP32 deviation storage) at the other
    temperatures of the configuration and with the FP64 chemical potential:
    MLUPS, the step's HBM fraction at 168 B per lattice update, and the status
    after check_steps steps (first bad step if unstable).  At T_r 0.2 the
    k = 0.25 droplet goes unstable (the oracle on the same droplet scaled to
    96^3 fails at the same step as the GPU there); it is recorded, and the
    T_r 0.2 leg also runs at k = 0.15, inside the paper's 0.1-0.4 range."""
    import torch
    peak = measured_peak()[0]
    out = {"workload": "D3Q19 %d^3 droplet r0=60, EFDS6, kappa 0.1, FP32DEV, tau 1" % n}
    legs = [("Tr0.5", 0.5, 0.25, 0), ("Tr0.2_k0.25", 0.2, 0.25, 0), ("Tr0.2_k0.15", 0.2, 0.15, 0),
            ("Tr0.8_mu_fp64", 0.8, 0.25, 1), ("Tr0.2_k0.15_mu_fp64", 0.2, 0.15, 1)]
    for name, Tr, k, mu64 in legs:
        s = L.Sim(L.make_params(lattice=L.LBM_D3Q19, nx=n, ny=n, nz=n, Tr=Tr, k=k, kappa=0.1, scheme="EFDS6",
                                precision=L.LBM_FP32DEV, mu_fp64=mu64))
        if zc:
            s.lbm_set_zchunk(zc)
        s.lbm_init_droplet(60.0 * n / 256)
        s.lbm_step(warmup)
        torch.cuda.synchronize()
        ms = s.lbm_step_timed(steps)
        s.lbm_step(check_steps - warmup - steps)
        o = s.lbm_observables()
        out[name] = {"Tr": Tr, "k": k, "mu": "fp64" if mu64 else "fp32", "mlups": n ** 3 * steps / (ms[2] * 1e-3) / 1e6,
                     "ms_per_step": ms[2] / steps,
                     "step_frac": B_ALG * n ** 3 / (ms[2] / steps * 1e-3) / 1e9 / peak,
                     "status": o["status"], "steps_checked": check_steps,
                     "first_bad_step": o["step"] if o["status"] != 0 else None,
                     "rho_center": o["rho_center"], "rho_corner": o["rho_corner"], "max_v": o["max_v"]}
        s.close()
    return out


def _oracle_replica(args):
    """One oracle replica of the all-core CPU leg (a process of its own)."""
    steps, n, barrier, q = args
    import oracle as O
    w = WORKLOAD
    s = O.Sim(lattice=O.D3Q19, nx=n, ny=n, nz=n, Tr=w["Tr"], k=w["k"], kappa=w["kappa"], tau=w["tau"],
              scheme=w["scheme"])
    s.init_droplet(w["radius"] * n / w["nx"])
    barrier.wait()
    t0 = time.perf_counter()
    rc = s.step(steps)
    q.put((t0, time.perf_counter(), rc))


def oracle_sample_all_cores(steps, n=SAMPLE_N):
    """The oracle as it stands, one replica per host core (processes started
    with spawn), all stepping the same n^3 sample at once: aggregate MLUPS."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    barrier, q = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=((steps, n, barrier, q),)) for _ in range(cores)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join()
    assert all(r[2] == 0 for r in res)
    wall = max(r[1] for r in res) - min(r[0] for r in res)
    return cores * n ** 3 * steps / wall / 1e6, wall, cores


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(1)
    vals = []
    total = 0.0
    for _ in range(args.steps):
        v, dt = oracle_sample(1)
        vals.append(v)
        total += dt
    value = SAMPLE_N ** 3 * args.steps / total / 1e6
    sample = "%d^3 lattice, same parameters (r0 scaled), one oracle step per timed step" % SAMPLE_N
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(workload="D3Q19 droplet, FP64 CPU oracle sample", **WORKLOAD),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    if args.size != WORKLOAD["nx"]:
        WORKLOAD.update(nx=args.size, ny=args.size, nz=args.size, radius=60.0 * args.size / 256)
    import numpy as np
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_2205_09186_gb300 as pkg
    if rank == 0 or world == 1:
        pkg.build()
    if dist:
        dist.barrier()
    from paper_2205_09186_gb300 import lbm as L
    w = WORKLOAD
    params = L.make_params(lattice=L.LBM_D3Q19, nx=w["nx"], ny=w["ny"], nz=w["nz"], Tr=w["Tr"], k=w["k"],
                           kappa=w["kappa"], tau=w["tau"], scheme=w["scheme"], precision=L.LBM_FP32DEV, mu_fp64=0)
    stream = torch.cuda.current_stream()
    sim = L.Sim(params)
    if args.zchunk > 0:
        sim.lbm_set_zchunk(args.zchunk)
        zc = args.zchunk
    else:
        zc = sim.lbm_autotune()  # z-chunk of the D3Q19 kernel; leaves the state undefined
    sim.lbm_init_droplet(w["radius"])
    N = w["nx"] * w["ny"] * w["nz"]
    for _ in range(args.warmup):
        sim.lbm_step(1)
    torch.cuda.synchronize()
    obs0 = sim.lbm_observables()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        # one step per launch group; CUDA events between the mu pass and the
        # collision pass time the dominant kernel on the handle's own stream
        phase_ms = sim.lbm_step_timed(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    if dist:
        total_ms = reduce_max_ms(total_ms, dist, "cuda")
        dist.barrier()
    obs = sim.lbm_observables()
    ok = obs["status"] == 0 and abs(obs["mass"] / obs0["mass"] - 1) < 1e-6
    mlups = job_mlups(N, args.steps, world, total_ms)
    coll_ms = phase_ms[1] / args.steps   # collision/streaming pass (dominant kernel), per launch
    mu_ms = phase_ms[0] / args.steps     # mu pass, per launch
    achieved = B_COLL * N / (coll_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()

    # end to end through the public API with pinned host buffers: upload the
    # initial density (H2D), step with the observables of every step read back
    # (D2H; lbm_step_observe_async reports the state each step started from), read
    # back the final density (D2H)
    host_rho0 = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    host_rho0[:] = sim.lbm_get_density().reshape(-1)
    host_rho = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    # one page-locked lbm_obs record per step, filled by the stream
    rec_size = ctypes.sizeof(L.lbm_obs)
    host_obs = torch.empty(rec_size * args.steps, dtype=torch.uint8).pin_memory()
    # three complete runs (upload, K observed steps, read-back); the median
    # is reported, the host side of the box being shared
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.lbm_init_density(host_rho0)
        for k in range(args.steps):
            sim.lbm_step_observe_async(1, host_obs.data_ptr() + rec_size * k)
        sim.lbm_get_density(out=host_rho)  # synchronises the stream
        torch.cuda.synchronize()
        runs.append(time.perf_counter() - t0)
    e2e_s = statistics.median(runs)
    e2e_last = L.lbm_obs.from_address(host_obs.data_ptr() + rec_size * (args.steps - 1))
    e2e = {"value": N * args.steps * world / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": N * 8 / args.steps, "d2h_bytes_per_step": rec_size + N * 8 / args.steps,
           "runs": 3, "run_values": [N * args.steps * world / r / 1e6 for r in runs],
           "last_status": e2e_last.status}

    sim.close()
    extra = {}
    if not args.no_cfg3:
        extra["d3q19_256_legs"] = run_cfg3_legs(L, zc, n=w["nx"])
    if not args.no_batch:
        extra["batch2d"] = run_batch(L, steps=args.batch_steps, ncases=args.batch_cases)
        # the same seeded sweep over the explicit and isotropic schemes only
        extra["batch2d_explicit"] = run_batch(L, steps=args.batch_steps, ncases=args.batch_cases,
                                              schemes=SWEEP_SCHEMES[:5])
        extra["d2q9_512"] = run_2d(L)
        extra["d2q9_512_sweep_batched"] = run_cfg2_sweep(L)
        extra["d3q19_compact"] = run_compact(L)
    if not args.no_warmstart:
        from paper_2205_09186_gb300 import warmstart as W
        # the plain arm (FP64 storage, tanh start) on the first 4 test cases;
        # --warmstart-full: 64 held-out droplets on 192^3 lattices, warm against
        # cold FP32 only (FP64 storage at this size takes ~17 ms per step here)
        if args.warmstart_full:
            res, _ = W.experiment(n_train=32, n_test=64, n=192, tol=1e-10, iters=4000, plain=0, R=(30.0, 50.0),
                                  max_steps=100000)
        else:
            res, _ = W.experiment(n_train=32, n_test=12, n=80, tol=1e-10, iters=4000, plain=4)
        extra["warmstart"] = res
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # all host cores: one oracle replica per core on the same sample (the
        # oracle is single-threaded as written); the single-core figure beside it
        va, dta, cores = oracle_sample_all_cores(args.cpu_steps)
        v, dt = oracle_sample(args.cpu_steps)
        cpu = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d replicas (one per host core, processes) of a %d^3 lattice with the same parameters "
                         "(r0 scaled), %d FP64 oracle steps each, %.1f s" % (cores, SAMPLE_N, args.cpu_steps, dta),
               "single_core": {"value": v, "unit": UNIT, "cores": 1,
                               "sample": "one %d^3 replica, %d steps, %.1f s" % (SAMPLE_N, args.cpu_steps, dt)}}
    line = {"metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload="D3Q19 droplet %d^3 r0=%g, CS EOS, EFDS6, FP32-deviation populations, "
                                    "FP32 density deviation; inputs larger than L2 (no flush)" % (w["nx"], w["radius"]),
                           parallelism="replicas", zchunk=zc,
                           **WORKLOAD),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": captured_traffic(N), "peak_kind": peak_kind,
                         "bytes_per_lu": B_COLL,
                         "kernel": "k_coll3d (grad mu, grad rho, force, BGK+EDM, push, next density)"
                                   " + k_coll3d_corners (tile-corner densities), timed together",
                         "kernel_ms": coll_ms, "mu_pass": {"kernel": "k_mu3d_zm", "ms": mu_ms, "bytes_per_lu": B_MU,
                                                           "achieved": B_MU * N / (mu_ms * 1e-3) / 1e9 if mu_ms > 0 else None},
                         "step_bytes_per_lu": B_ALG, "step_frac": B_ALG * N / (total_ms / args.steps * 1e-3) / 1e9 / peak},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 3 * args.steps,
            "clocks": clk.summary(), "check": {"status": obs["status"], "mass_rel_change": obs["mass"] / obs0["mass"] - 1,
                                               "ok": ok},
            "extra": extra}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 2D sweep measurement")
    ap.add_argument("--batch-cases", type=int, default=512, help="cases of the batched 2D sweep (small: profiling)")
    ap.add_argument("--batch-steps", type=int, default=50, help="steps per timed launch of the batched 2D sweep")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the warm-start experiment")
    ap.add_argument("--no-cfg3", action="store_true", help="skip the other-temperature and FP64-mu 256^3 legs")
    ap.add_argument("--compact-only", action="store_true",
                    help="profiling: only the D3Q19 192^3 compact-scheme leg (one JSON line of its own)")
    ap.add_argument("--warmstart-full", action="store_true",
                    help="the warm-start experiment at full size (64 held-out 192^3 droplets; tens of minutes)")
    ap.add_argument("--zchunk", type=int, default=0, help="fix the z-chunk instead of autotuning (profiling runs)")
    ap.add_argument("--size", type=int, default=256,
                    help="lattice edge (profiling runs only; the benchmark workload is 256)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.compact_only:
        import paper_2205_09186_gb300 as pkg
        pkg.build()
        from paper_2205_09186_gb300 import lbm as L
        print(json.dumps({"d3q19_compact": run_compact(L, steps=args.steps, warmup=args.warmup)}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
