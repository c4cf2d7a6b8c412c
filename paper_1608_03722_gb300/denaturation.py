"""Denaturation time courses of Sec. 5 / Fig. 9 with the engine: the
fraction of open base pairs f(t) of linear molecules at several hydrogen-bond
stiffnesses K2, with the bubble rule on, and where along the chain the
pairs open (the paper sees melting nucleate at the ends).

A base pair is open when its patch distance exceeds rc (Sec. 2).  Each K2 is
one batched context of `copies` molecules starting as relaxed straight
helices; f comes from the engine's observable kernel, the profile along the
chain (end segments against the middle) from the state the engine holds.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def time_course(K2_values=(1.0, 1.2, 1.4, 2.0), n_bp=1000, copies=16, steps=1_000_000, samples=20,
                bubble_rule=2, end_bp=100, seed=0, dt=0.005, log=None):
    from . import dsdna as D
    out = []
    every = steps // samples
    for i, K2 in enumerate(K2_values):
        p = D.dsdna_default_params(K2=K2, bubble_rule=bubble_rule, seed=seed + i, dt=dt)
        ctx = D.Context(p, [n_bp] * copies)
        rows = []
        t0 = time.time()
        for s in range(samples):
            ctx.step(every)
            f = np.mean([ctx.observables(m, flags=D.OBS_DENAT)["denat"] for m in range(copies)])
            X, _, u, _ = ctx.get_state()
            pt = X + 0.5 * p.ell * u
            op = (np.linalg.norm(pt[1::2] - pt[0::2], axis=1) > p.rc_hb).reshape(copies, n_bp)
            ends = np.concatenate([op[:, :end_bp], op[:, -end_bp:]], axis=1).mean()
            mid = op[:, n_bp // 2 - end_bp: n_bp // 2 + end_bp].mean()
            rows.append({"step": (s + 1) * every, "time_tau": (s + 1) * every * dt, "f": float(f),
                         "f_ends": float(ends), "f_middle": float(mid)})
            if log:
                log(f"K2 {K2} sample {s + 1}/{samples}")
        ctx.close()
        out.append({"K2": K2, "rows": rows, "seconds": time.time() - t0})
    return {"n_bp": n_bp, "copies": copies, "bubble_rule": bubble_rule, "end_bp": end_bp, "dt": dt, "runs": out}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=1_000_000)
    ap.add_argument("--samples", type=int, default=20)
    ap.add_argument("--bubble-rule", type=int, default=2)
    ap.add_argument("--dt", type=float, default=0.005)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    import torch
    torch.cuda.init()
    r = time_course(steps=a.steps, samples=a.samples, bubble_rule=a.bubble_rule, dt=a.dt)
    for run in r["runs"]:
        print(f"K2 = {run['K2']}:")
        for row in run["rows"][:: max(1, len(run["rows"]) // 10)]:
            print(f"  t {row['time_tau']:8.1f} tau  f {row['f']:.3f}  ends {row['f_ends']:.3f}  middle {row['f_middle']:.3f}")
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)


if __name__ == "__main__":
    main()
