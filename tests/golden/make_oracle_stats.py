"""Write tests/golden/oracle_tethered_stats.txt: ensemble statistics of the
FP64 oracle for the statistical-agreement test of the CUDA engine.

Calls only oracle/ (and the seeded configuration generator, which holds none
of the model's arithmetic).  Each replica is a tethered 300 bp molecule
(base pair 0 anchored, force f e_z and torque Gamma e_z on the last base
pair, Sec. 4.1-4.2), started as a relaxed straight helix with its own
Maxwell-Boltzmann velocities and Philox seed, and run with the oracle's
Langevin integrator; its labels are the averages over samples every EVERY
steps from FROM to STEPS of the extension R_z (Sec. 4.1), the excess twist
Tw - Tw_relaxed in turns (Sec. 3.2, App. B) and the denatured fraction
(Sec. 5).  The file holds the mean over replicas and its standard error.

    python tests/golden/make_oracle_stats.py [--replicas 24] [--workers 8]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(ROOT, "tests", "golden", "oracle_tethered_stats.txt")

N_BP = 300
FORCE = 5.0        # kT/nm along z on the last base pair
TORQUE = 2.0       # kT about z on the last base pair
STEPS = 60000
FROM = 10000
EVERY = 100
CONDITIONS = {"k2_6": 6.0, "k2_2": 2.0}   # hydrogen-bond stiffness K2 (Table 1: 6)


def replica(args):
    cond, k2, r = args
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1608_03722_gb300 import inputs as I
    cfg = I.c2_tethered(n_bp=N_BP, force=FORCE, torque=TORQUE, seed=100 + r)
    p = O.params(K2=k2, seed=5000 + r)
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    acc = np.zeros(3)
    ns = 0
    done = 0
    while done < STEPS:
        O.run(p, cfg.n_bp, X, V, u, Om, EVERY, step0=done, ext_f=cfg.ext_f, ext_t=cfg.ext_t, tether=cfg.tether,
              cells=True)
        done += EVERY
        if done >= FROM:
            o = O.observables(p, cfg.n_bp, X, u)
            acc += (o["rz"], o["tw"] - o["tw_ideal"], o["denat"])
            ns += 1
    return cond, acc / ns


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicas", type=int, default=24)
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    a = ap.parse_args()
    jobs = [(c, k2, r) for c, k2 in CONDITIONS.items() for r in range(a.replicas)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = pool.map(replica, jobs)
    lines = [
        "# Ensemble statistics of the FP64 oracle: tethered 300 bp dsDNA, force 5 kT/nm and torque 2 kT",
        "# about z on the last base pair, base pair 0 anchored (Sec. 4.1-4.2), relaxed straight start.",
        "# Written by tests/golden/make_oracle_stats.py (oracle only); per replica the average of samples",
        "# every `every` steps from `from` to `steps`; mean over replicas and its standard error.",
        f"n_bp = {N_BP}", f"force = {FORCE}", f"torque = {TORQUE}", f"steps = {STEPS}", f"from = {FROM}",
        f"every = {EVERY}", f"replicas = {a.replicas}",
    ]
    for c, k2 in CONDITIONS.items():
        v = np.array([m for cc, m in res if cc == c])
        lines.append(f"{c}.K2 = {k2}")
        for j, name in enumerate(("rz", "dtw", "denat")):
            lines.append(f"{c}.{name}_mean = {v[:, j].mean():.10g}")
            lines.append(f"{c}.{name}_se = {v[:, j].std(ddof=1) / np.sqrt(len(v)):.10g}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
