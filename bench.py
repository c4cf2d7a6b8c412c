#!/usr/bin/env python3
"""Throughput benchmark of the dsDNA engine (arXiv:1608.03722 model) on GB300.

Workload (default): 1 Mbp dsDNA, 2e6 nucleotides, confined self-avoiding helix
in a periodic cube at volume fraction 0.05, Langevin at kT = 1, FP32 forces
with FP64 accumulation.  One bench step = ``--md-steps`` (default 100)
Langevin timesteps of the whole system (forces of App. A, Langevin update,
neighbour-list rebuilds as needed), queued through the C ABI.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (one Langevin step of the same workload per bench step).
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nucleotide-timesteps/s at 1 Mbp (fraction of HBM roofline); batched/surrogate vs plain"
UNIT = "nucleotide-timesteps/s"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, x: float, device) -> float:
    """Largest x over all ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_workload(name: str, seed: int = 0, n_bp: int = 1_000_000):
    from paper_1608_03722_gb300 import inputs as I
    if name == "c3":
        cfg = I.c3_walk(n_bp=n_bp, seed=seed)
        desc = (f"confined self-avoiding dsDNA, {n_bp:,} bp = {2 * n_bp:,} nucleotides, self-avoiding walk of "
                f"30 bp helical segments (joints <= 30 deg) in a periodic cube L={cfg.box[0]:.2f} nm "
                f"(volume fraction 0.05), Langevin kT=1, dt=0.005")
    elif name == "c3rows":
        cfg = I.c3_confined(n_bp=n_bp, seed=seed)
        desc = (f"confined self-avoiding dsDNA, {n_bp:,} bp = {2 * n_bp:,} nucleotides, rows along x joined by "
                f"U-turns in a periodic cube L={cfg.box[0]:.2f} nm (volume fraction 0.05), Langevin kT=1, dt=0.005")
    elif name == "c2":
        cfg = I.c2_tethered(force=5.0, torque=2.0, seed=seed)
        desc = "tethered linear dsDNA, 10 kbp = 20,000 nucleotides, f=5 kT/nm, torque 2 kT"
    elif name == "c4":
        cfg = I.c4_batch(seed=seed)
        desc = f"256 independent molecules, lengths log-uniform 500-20000 bp ({cfg.n_nt} nucleotides)"
    elif name == "paper960":
        cfg = I.paper_array(40, 40, 600, seed=seed)
        desc = "paper benchmark geometry: 40x40 array of 600 bp strands (960 kbp, 1,920,000 nucleotides), periodic"
    elif name == "c1":
        cfg = I.c1_linear(200, seed=seed)
        desc = "linear dsDNA, 200 bp = 400 nucleotides, open boundaries"
    else:
        raise SystemExit(f"unknown workload {name}")
    return cfg, desc


# DRAM bytes (read + write) per nucleotide-step of the mixed-precision step
# kernel from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of
# the bench's multi-step launches on the 1 Mbp confined workload, pair halving),
# keyed by a hash of the kernel sources it was taken on and by the skin: a
# changed kernel, or a skin without a capture, reports no traffic.
ENGINE_TRAFFIC = {("2798d66a242bfac2", "c3", 0.3): 214.5,
                  ("2798d66a242bfac2", "c3", 0.35): 215.8,
                  ("2798d66a242bfac2", "c3", 0.4): 218.0}
ENGINE_SOURCES = ("engine.cuh", "engine_kernels.cuh", "kern_mixed.cu")   # the step kernel's code


def engine_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, "paper_1608_03722_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def engine_traffic_per_nt_step(prec, workload, skin):
    from paper_1608_03722_gb300 import dsdna as D
    if prec != D.PREC_MIXED:
        return None
    return ENGINE_TRAFFIC.get((engine_source_hash(), workload, round(float(skin), 2)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def wait_first(self, timeout: float = 10.0):
        """Block until nvidia-smi has written its first sample: its start-up
        holds the driver long enough to starve a short timed region."""
        t0 = time.time()
        while self.p is not None and time.time() - t0 < timeout:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.05)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def run_cpu_oracle(cfg, steps: int, seconds_cap: float = 25.0, chunk: int = 1, seed: int = 0):
    """Time the FP64 oracle (as it stands, cell-hash pair search) on whole
    Langevin steps of the workload, `chunk` steps per call, one thread."""
    import oracle as O
    p = O.params(box=cfg.box, seed=seed) if cfg.box[0] > 0 else O.params(seed=seed)
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    done = 0
    t0 = time.perf_counter()
    w0 = time.time()
    while done < steps:
        n = min(chunk, steps - done)
        O.run(p, cfg.n_bp, X, V, u, Om, n, step0=done, ext_f=cfg.ext_f, ext_t=cfg.ext_t, tether=cfg.tether,
              cells=True)
        done += n
        if time.perf_counter() - t0 > seconds_cap:
            break
    dt = time.perf_counter() - t0
    return cfg.n_nt * done / dt, done, dt, (w0, time.time())


def _oracle_worker(job):
    """One independent replica of the workload on one host core (spawned process)."""
    path, seed, steps, cap, chunk = job
    sys.path.insert(0, ROOT)
    from paper_1608_03722_gb300 import inputs as I
    d = np.load(path)
    opt = lambda k: d[k] if d[k].size else None
    cfg = I.Config("replica", d["n_bp"], d["X"], d["u"], d["V"], d["Om"], box=tuple(d["box"]), tether=opt("tether"),
                   ext_f=opt("ext_f"), ext_t=opt("ext_t"))
    _, done, _, (w0, w1) = run_cpu_oracle(cfg, steps, cap, chunk, seed)
    return cfg.n_nt * done, w0, w1


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_cpu_oracle_all_cores(cfg, steps: int, seconds_cap: float, chunk: int = 1, workers: int | None = None):
    """The oracle as it stands on every host core: one independent replica of
    the workload per core (its own noise seed), started together in spawned
    processes; nucleotide-steps of all replicas over the span from the first
    start to the last finish."""
    import multiprocessing as mp
    workers = workers or host_cores()
    none = np.zeros(0)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "cfg.npz")
        np.savez(path, n_bp=cfg.n_bp, X=cfg.X, u=cfg.u, V=cfg.V, Om=cfg.Om, box=np.asarray(cfg.box, float),
                 tether=none if cfg.tether is None else cfg.tether, ext_f=none if cfg.ext_f is None else cfg.ext_f,
                 ext_t=none if cfg.ext_t is None else cfg.ext_t)
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(path, 1000 + r, steps, seconds_cap, chunk) for r in range(workers)])
    total = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return total / span, total, span, workers


def cpu_baseline(cfg, c3_steps=2, c3_cap=20.0, c1_steps=10_000):
    """The oracle on the host: the bench's workload (whole steps, one thread and
    all cores) and the 200 bp molecule for its full 10^4 steps."""
    from paper_1608_03722_gb300 import inputs as I
    cores = host_cores()
    v1, done, dt, _ = run_cpu_oracle(cfg, c3_steps, c3_cap)
    va, tot, span, w = run_cpu_oracle_all_cores(cfg, c3_steps, c3_cap)
    c1 = I.c1_linear(200)
    u1, d1, t1, _ = run_cpu_oracle(c1, c1_steps, 120.0, chunk=500)
    ua, tot1, span1, _ = run_cpu_oracle_all_cores(c1, c1_steps, 120.0, chunk=500)
    return {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{c3_steps} whole Langevin steps of the full workload ({cfg.n_nt} nucleotides) on each of "
                      f"{w} cores, one independent replica per core ({span:.1f} s)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{done} whole Langevin steps of the full workload, {dt:.1f} s"},
            "c1_200bp_1e4_steps": {"single_thread": {"value": u1, "unit": UNIT, "steps": d1, "seconds": t1},
                                   "all_cores": {"value": ua, "unit": UNIT, "cores": w, "seconds": span1,
                                                 "sample": f"{c1_steps} steps of 200 bp on each core"}}}


def timed_steps(ctx, torch, steps, reps):
    """Device time of reps x ctx.step(steps) after a warm-up, CUDA events on the context's stream."""
    ctx.step(steps)
    ctx.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.step(steps)
    e1.record()
    ctx.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def _batch_rate(D, torch, cfg, p, steps, reps):
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether)
    for m in range(len(cfg.n_bp)):
        ctx.set_external_force_torque(m, cfg.ext_f[m], cfg.ext_t[m])
    t = timed_steps(ctx, torch, steps, reps)
    ctx.close()
    return cfg.n_nt * steps * reps / t


def _per_molecule_rate(D, torch, cfg, prec, steps):
    """Every molecule in a context of its own (default launch parameters),
    run one after the other: nucleotide-steps over the summed device time."""
    off = np.concatenate([[0], np.cumsum(cfg.n_bp)])
    nt_steps, secs = 0, 0.0
    for m in range(len(cfg.n_bp)):
        sl = slice(2 * off[m], 2 * off[m + 1])
        c1 = D.Context(D.dsdna_default_params(precision=prec), [int(cfg.n_bp[m])], X=cfg.X[sl], V=cfg.V[sl],
                       u=cfg.u[sl], Om=cfg.Om[sl], tether=[1])
        c1.set_external_force_torque(0, cfg.ext_f[m], cfg.ext_t[m])
        secs += timed_steps(c1, torch, steps, 1)
        nt_steps += 2 * int(cfg.n_bp[m]) * steps
        c1.close()
    return nt_steps / secs


def compare_batched(D, torch, n_mol=256, steps=100):
    """C4, 256 ragged tethered molecules with their own loads, four ways on
    the same molecules: batched (one context, one graph-driven persistent
    launch, autotuned) or one molecule per context, each in mixed precision
    and in FP64, so the gain splits into its batching and precision parts;
    and the batched mixed run with the molecules in random orientations and
    places."""
    from paper_1608_03722_gb300 import inputs as I
    cfg = I.c4_batch(n_mol=n_mol, seed=0)
    out = {"workload": f"{n_mol} tethered molecules log-uniform 500-20000 bp ({cfg.n_nt} nucleotides), own force "
                       f"and torque each, {steps}-step runs"}
    for name, prec in (("mixed", D.PREC_MIXED), ("fp64", D.PREC_FP64)):
        p, _ = D.dsdna_autotune(D.dsdna_default_params(precision=prec), cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om,
                                tether=cfg.tether, trial_steps=30)
        out["batched_" + name] = {"value": _batch_rate(D, torch, cfg, p, steps, 3), "unit": UNIT, "skin": p.skin,
                                  "block_threads": p.block_threads}
        out["per_molecule_" + name] = {"value": _per_molecule_rate(D, torch, cfg, prec, steps), "unit": UNIT,
                                       "molecules": n_mol}
    b = {k: out[k]["value"] for k in ("batched_mixed", "batched_fp64", "per_molecule_mixed", "per_molecule_fp64")}
    out["speedup"] = b["batched_mixed"] / b["per_molecule_fp64"]
    out["batching_gain_mixed"] = b["batched_mixed"] / b["per_molecule_mixed"]
    out["batching_gain_fp64"] = b["batched_fp64"] / b["per_molecule_fp64"]
    out["precision_gain_batched"] = b["batched_mixed"] / b["batched_fp64"]
    out["precision_gain_per_molecule"] = b["per_molecule_mixed"] / b["per_molecule_fp64"]
    rp = I.c4_batch(n_mol=n_mol, seed=0, random_pose=True)
    p, _ = D.dsdna_autotune(D.dsdna_default_params(), rp.n_bp, X=rp.X, V=rp.V, u=rp.u, Om=rp.Om, tether=rp.tether,
                            trial_steps=30)
    out["batched_mixed_random_pose"] = {"value": _batch_rate(D, torch, rp, p, steps, 3), "unit": UNIT,
                                        "skin": p.skin, "block_threads": p.block_threads,
                                        "pose": "uniformly random rotation about base pair 0, origin uniform in a "
                                                "200 nm cube, load along the molecule's own axis"}
    return out


# Paper's time unit: tau_Br = 2.28e-9 s and dt = 0.005 tau_Br (App. A), so
# simulated milliseconds per wall-clock day = steps/s * dt * 86400 s * 1e3.
MS_PER_DAY_PER_STEP_S = 0.005 * 2.28e-9 * 86400.0 * 1e3
# The paper's strong-scaling figures on ARCHER (Cray XC30, 24-core Ivy Bridge nodes), Sec. 6 / Fig. 11.
PAPER_FIG11 = {"10x10": "about 2 ms/day on 512 cores",
               "40x40": "about 0.4 ms/day on 2048 cores, up to 1 ms/day on 8192 cores"}


def compare_paper(D, torch, steps=100, reps=5):
    """The paper's benchmark geometry (regular arrays of 600 bp strands) run
    through the batched engine; simulated time per wall-clock day beside the
    paper's Fig. 11 figures."""
    from paper_1608_03722_gb300 import inputs as I
    out = {}
    for nx in (10, 40):
        cfg = I.paper_array(nx, nx, 600)
        p, _ = D.dsdna_autotune(D.dsdna_default_params(box=cfg.box), cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om,
                                trial_steps=50)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
        t = timed_steps(ctx, torch, steps, reps)
        ctx.close()
        steps_s = steps * reps / t
        key = f"{nx}x{nx}"
        out[key] = {"workload": f"{nx}x{nx} array of 600 bp strands ({cfg.n_nt} nucleotides), periodic box "
                                f"{cfg.box[0]:.0f}x{cfg.box[1]:.0f}x{cfg.box[2]:.0f} nm",
                    "value": cfg.n_nt * steps_s, "unit": UNIT, "steps_per_s": steps_s,
                    "autotuned": {"skin": p.skin, "block_threads": p.block_threads, "blocks_per_sm": p.blocks_per_sm},
                    "ms_per_day": steps_s * MS_PER_DAY_PER_STEP_S, "paper": PAPER_FIG11[key]}
    return out


def compare_ring(D, torch, n_bp=500, lk=47, samples=(0, 50_000, 100_000, 200_000, 400_000), n_batch=64,
                 steps=1000, reps=3):
    """Sec. 6 / Fig. 10: a 500 bp ring wound 47 turns instead of 50 (Delta Lk
    = -3, sigma = -0.06).  Twist, writhe and linking number along one
    trajectory (Lk must stay 47 while twist turns into writhe), and the step
    rate of one ring and of a batch of rings (the ring kernel instance with its
    junction pass)."""
    from paper_1608_03722_gb300 import inputs as I
    X, u = I.ring_helix(n_bp, lk)
    ctx = D.Context(D.dsdna_default_params(seed=1), [n_bp], X=X, u=u, circular=[1])
    traj, done = [], 0
    for s in samples:
        ctx.step(s - done)
        done = s
        o = ctx.observables(0, flags=D.OBS_TW | D.OBS_LK)
        traj.append({"step": s, "tw": o["tw"], "wr": o["wr"], "lk": o["lk"]})
    t1 = timed_steps(ctx, torch, steps, reps)
    ctx.close()
    Xs = np.concatenate([I.ring_helix(n_bp, lk, center=(40.0 * (m % 8), 40.0 * (m // 8), 0.0))[0] for m in range(n_batch)])
    us = np.concatenate([u] * n_batch)
    ctx = D.Context(D.dsdna_default_params(seed=2), [n_bp] * n_batch, X=Xs, u=us, circular=[1] * n_batch)
    tb = timed_steps(ctx, torch, steps, reps)
    ctx.close()
    return {"workload": f"{n_bp} bp ring, Lk {lk} (Delta Lk = {lk - n_bp // 10}), Langevin kT=1, dt=0.005",
            "trajectory": traj,
            "one_ring_steps_per_s": steps * reps / t1,
            "batch": {"rings": n_batch, "value": 2 * n_bp * n_batch * steps * reps / tb, "unit": UNIT,
                      "steps_per_s": steps * reps / tb}}


def reference_arm(args, ws, rank):
    if rank != 0:
        return 0
    cfg, desc = build_workload(args.workload, n_bp=args.n_bp)
    import oracle as O
    O.build()
    # every host core runs an independent replica of the workload; a bench step is
    # one whole Langevin step of every replica
    value, total, span, cores = run_cpu_oracle_all_cores(cfg, args.steps, seconds_cap=max(30.0, 20.0 * args.steps))
    done = int(round(total / cfg.n_nt / cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": done,
        "warmup": args.warmup, "ms_per_step": 1e3 * span / max(done, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "md_steps_per_step": 1, "l2": "state larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} whole Langevin steps of the full workload ({cfg.n_nt} nucleotides) on each "
                                   f"of {cores} cores, one independent replica per core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c3rows", "c4", "paper960"])
    ap.add_argument("--md-steps", type=int, default=100)
    ap.add_argument("--n-bp", type=int, default=1_000_000, help="base pairs of the confined workload")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--skin", type=float, default=None, help="fixed skin (skips the autotuner)")
    ap.add_argument("--block-threads", type=int, default=None, help="fixed CTA size (skips the autotuner)")
    ap.add_argument("--no-compare", action="store_true", help="skip the batched / FP64 per-molecule comparison")
    ap.add_argument("--list-build", type=int, default=0, choices=[0, 1],
                    help="periodic neighbour-list build: 0 chain window, 1 cell walk")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1608_03722_gb300 import dsdna as D

    cfg, desc = build_workload(args.workload, seed=rank, n_bp=args.n_bp)
    prec = D.PREC_MIXED if args.precision == "mixed" else D.PREC_FP64
    p = D.dsdna_default_params(precision=prec, box=cfg.box, seed=rank, list_build=args.list_build)
    tuned = None
    if args.skin is not None or args.block_threads is not None:
        args.no_autotune = True
        if args.skin is not None:
            p.skin = args.skin
        if args.block_threads is not None:
            p.block_threads = args.block_threads
    if not args.no_autotune:
        p, ns = D.dsdna_autotune(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether, trial_steps=30)
        tuned = {"skin": p.skin, "block_threads": p.block_threads, "blocks_per_sm": p.blocks_per_sm,
                 "list_build": p.list_build, "trial_ns_per_nt_step": ns}
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether)
    if cfg.ext_f is not None:
        for m in range(len(cfg.n_bp)):
            ctx.set_external_force_torque(m, cfg.ext_f[m], cfg.ext_t[m])
    K, W, S = args.steps, args.warmup, args.md_steps
    for _ in range(W):
        ctx.step(S)
    ctx.synchronize()
    info0 = ctx.info()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(gpu_uuid(torch, local)) if rank == 0 else None
    if sampler:
        sampler.wait_first()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        ctx.step(S)
    e1.record()
    barrier()
    clocks = sampler.stop() if sampler else None
    ctx.synchronize()
    ms = e0.elapsed_time(e1)
    info1 = ctx.info()
    ms_max = max_over_ranks(dist, ms, "cuda")
    nt_steps = cfg.n_nt * S * K * ws
    value = nt_steps / (ms_max * 1e-3)

    graph_chunk = ctx.params.steps_per_graph or 50
    graph_launches = K * ((S + graph_chunk - 1) // graph_chunk)
    rebuilds = info1["rebuilds"] - info0["rebuilds"]
    engine_launches = info1["engine_launches"] - info0["engine_launches"]
    # kernels of the timed region: per graph launch one loop-init kernel; per loop
    # iteration one loop-head kernel and one persistent step kernel; per rebuild five
    # (chain-window build, or a cell walk without pair halving) or six (a cell walk
    # and its pair-halving pack), none when the step kernel rebuilds the list itself
    per_rebuild = 5 if (info1["chain_list"] or info1["halved_tiles"] == 0) else 6
    gpu_launches = graph_launches + 2 * engine_launches + (0 if info1["rebuild_in_step"] else per_rebuild * rebuilds)

    # Roofline of the dominant kernel: K x S further steps queued launch by launch
    # (dsdna_step_profiled), each step-kernel launch bracketed by CUDA events on
    # the context stream.
    prof = {"steps": 0, "engine_launches": 0, "engine_ms": 0.0, "rebuild_launches": 0, "rebuild_ms": 0.0}
    for _ in range(K):
        pr = ctx.step_profiled(S)
        for k in prof:
            prof[k] += pr[k]
    # neighbours per bead (full list), for the algorithmic byte count; under pair
    # halving a pair within one 32-slot tile is evaluated once, one across tiles twice
    pairs = ctx.neighbor_pairs()
    nbar = 2.0 * len(pairs) / cfg.n_nt
    halved = ctx.info()["halved_tiles"] > 0
    same_tile = int(np.count_nonzero((pairs[:, 0] >> 5) == (pairs[:, 1] >> 5))) if len(pairs) else 0
    ebar = (2.0 * len(pairs) - same_tile) / cfg.n_nt

    # algorithmic bytes per nucleotide-step of the fused force + Langevin kernel:
    # mixed: read X, V (FP64 24 + 24), Omega (FP32 12), kref 12, mirror (its fourth word
    # is the image word) + orientation (16 + 16), topology 4, count 4, and the list: 4 n
    # entries, or under pair halving 8 bytes of entry codes, the tile's evaluated pairs
    # (4 e per nucleotide) and its pair count (4 per 32); write X, V, Omega, next mirror
    # + orientation (24 + 24 + 12 + 16 + 16).  FP64: X, u, V, Omega 24 each read and
    # written, kref 12, topology, count, image (periodic) 4 each.
    periodic = 1 if cfg.box[0] > 0 else 0
    if prec == D.PREC_MIXED:
        b_nt = 112 + 92 + (8 + 4 * ebar + 4.0 / 32 if halved else 4 * nbar)
    else:
        b_nt = (96 + 12 + 8 + 4 * periodic) + 96 + 4 * nbar
    steps_per_launch = prof["steps"] / max(prof["engine_launches"], 1)
    per_launch_bytes = b_nt * cfg.n_nt * steps_per_launch
    launch_s = prof["engine_ms"] * 1e-3 / max(prof["engine_launches"], 1)
    hbm, peak_kind = peaks()
    achieved = per_launch_bytes / launch_s / 1e9
    traffic = engine_traffic_per_nt_step(prec, args.workload, ctx.params.skin)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None if traffic is None else traffic * cfg.n_nt * steps_per_launch,
            "traffic_capture": None if traffic is None else
            f"{traffic} B per nucleotide-step from ncu at skin {round(float(ctx.params.skin), 2)}, scaled by "
            f"nucleotide-steps per launch",
            "peak_kind": peak_kind, "bytes_per_nt_step": b_nt, "neighbors_per_bead": nbar,
            "pair_halving": halved, "evaluated_pairs_per_nucleotide": ebar if halved else nbar,
            "algorithmic_bytes_per_launch": per_launch_bytes, "steps_per_launch": steps_per_launch,
            "launch_ms": launch_s * 1e3, "launches_timed": prof["engine_launches"],
            "rebuild_ms_per_rebuild": prof["rebuild_ms"] / max(prof["rebuild_launches"], 1),
            "share_of_step_time": prof["engine_ms"] / max(prof["engine_ms"] + prof["rebuild_ms"], 1e-30),
            "timing": "CUDA events around every step-kernel launch on the context stream, "
                      "K x md_steps steps run right after the timed region",
            "kernel": "engine_kernel<float,STEP> (fused forces + Langevin, persistent cooperative)"}

    # end to end through the C ABI with pinned host buffers: upload the state
    # (X, V, u, Omega), step, download the state, every bench step
    e2e = None
    if not args.no_e2e and rank == 0:
        host = tuple(torch.empty((cfg.n_nt, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(4))
        ctx.get_state(out=host)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, min(K, 3))
        for _ in range(n_e2e):
            ctx.set_state(-1, *host)
            ctx.step(S)
            ctx.get_state(out=host)
        dt_e2e = time.perf_counter() - t0
        e2e = {"value": cfg.n_nt * S * n_e2e / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * 3 * 8 * cfg.n_nt,
               "d2h_bytes_per_step": 4 * 3 * 8 * cfg.n_nt, "steps": n_e2e, "host_buffers": "pinned"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg)

    compare = None
    if rank == 0 and not args.no_compare:
        compare = compare_batched(D, torch)
        compare["paper_benchmark"] = compare_paper(D, torch)
        compare["supercoiled_ring"] = compare_ring(D, torch)
        from paper_1608_03722_gb300 import surrogate as SUR
        t_s = time.perf_counter()
        st = SUR.run_sweep_study(n_train=2000, n_test=200, n_query=100, length=(500, 20000), steps=8000,
                                 measure_from=2000, every=200, iters=3000, query_rounds=3)
        compare["surrogate"] = {
            "workload": "sweep of tethered molecules 500-20000 bp, force 0.1-10 kT/nm, torque -5..5 kT, kT 0.8-1.4 "
                        "(2000 training / 200 held-out points, 8000 steps each; 3 rounds of 100 committee-picked "
                        "against 100 random additions)",
            "held_out_r2": st["held_out"]["r2"], "held_out_rmse": st["held_out"]["rmse"],
            "replicate_noise": st["replicate_noise"],
            "rmse_over_replicate_noise": st["held_out"]["rmse_over_replicate_noise"],
            "dropped_points": st["dropped_points"],
            "simulation_s_per_point": st["simulation_s_per_point"],
            "surrogate_s_per_point": st["surrogate_s_per_point"], "speedup_per_point": st["speedup_per_point"],
            "r2_after_committee_queries": [r["committee"]["r2"] for r in st["query_rounds"]],
            "r2_after_random_queries": [r["random"]["r2"] for r in st["query_rounds"]],
            "committee_minus_random_r2": st["committee_minus_random_r2"],
            "seconds": time.perf_counter() - t_s}
        rows_cfg, rows_desc = build_workload("c3rows", n_bp=args.n_bp)
        pr_, _ = D.dsdna_autotune(D.dsdna_default_params(box=rows_cfg.box), rows_cfg.n_bp, X=rows_cfg.X, V=rows_cfg.V,
                                  u=rows_cfg.u, Om=rows_cfg.Om, trial_steps=30)
        rc_ = D.Context(pr_, rows_cfg.n_bp, X=rows_cfg.X, V=rows_cfg.V, u=rows_cfg.u, Om=rows_cfg.Om)
        t_r = timed_steps(rc_, torch, S, 3)
        rc_.close()
        compare["confined_rows"] = {"workload": rows_desc, "value": rows_cfg.n_nt * S * 3 / t_r, "unit": UNIT,
                                    "skin": pr_.skin, "block_threads": pr_.block_threads}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == D.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": desc, "md_steps_per_step": S, "n_nucleotides": cfg.n_nt,
                       "parallelism": f"replicas x{ws}", "l2": "inputs larger than L2 (state > 129 MB)",
                       "rebuilds_in_timed_region": rebuilds, "graph_steps_per_launch": graph_chunk,
                       "list_build": "chain window" if info1["chain_list"] else "cell walk",
                       "autotuned": tuned},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "compare": compare,
            "gpu_launches": gpu_launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
