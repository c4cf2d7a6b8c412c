"""Bending and torsional persistence lengths of the model (Sec. 3.1, 3.2),
measured with the engine on many independent chains.

Sec. 3.1: the centreline runs through the base-pair centres (patch
midpoints); with unit tangents t(n) along it, <t(n) . t(n + s)> decays as
exp(-s / l_p) (the paper finds l_p = 143 +- 7 bp on a 300 bp chain, ends of
about 5 bp left out).  Sec. 3.2: with the twist increments between
consecutive base-pair frames (App. B), the residual total twist over m steps,
DeltaOmega(m) = Omega(m) - m theta0 with theta0 = 36 degrees, gives
<cos DeltaOmega(m)> = exp(-m / l_tau) (the paper: l_tau = 512 +- 18 bp).

The chains start as ideal helices and are equilibrated before sampling; the
profiles come from the engine's observable kernels (dsdna_profiles), the
correlators and the exponential fits are plain statistics on the host.  Error
bars: the spread of the fits over independent groups of molecules.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

THETA0 = 2.0 * math.pi / 10.0   # 36 degrees per base pair (Sec. 2)


def _fit_decay(c: np.ndarray, lo: int, hi: int) -> float:
    """Decay length of c[k] ~ exp(-k / l) by least squares of log c over k in [lo, hi]."""
    k = np.arange(lo, hi + 1)
    y = c[lo:hi + 1]
    ok = y > 0.05
    if ok.sum() < 3:
        return float("nan")
    slope = np.polyfit(k[ok], np.log(y[ok]), 1)[0]
    return -1.0 / slope if slope < 0 else float("inf")


class Correlators:
    """Running sums of <t(n).t(n+s)> and <cos DeltaOmega(m)> per molecule group."""

    def __init__(self, groups: int, s_max: int, m_max: int):
        self.ct = np.zeros((groups, s_max + 1)); self.nt = np.zeros((groups, s_max + 1))
        # cos and sin of DeltaOmega(m) (theta0 = 36 deg): any other reference
        # twist per bp follows from cos(x - m d) = cos x cos md + sin x sin md
        self.cw = np.zeros((groups, m_max + 1)); self.sw = np.zeros((groups, m_max + 1))
        self.nw = np.zeros((groups, m_max + 1))
        self.twist_sum = 0.0; self.twist_n = 0

    def add(self, group: int, centre: np.ndarray, twist_turns: np.ndarray, trim: int):
        t = np.diff(centre, axis=0)
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        t = t[trim:len(t) - trim]
        for s in range(min(self.ct.shape[1], len(t))):
            self.ct[group, s] += np.einsum("ij,ij->", t[:len(t) - s], t[s:])
            self.nt[group, s] += len(t) - s
        d = 2.0 * math.pi * twist_turns[trim:len(twist_turns) - trim]
        self.twist_sum += d.sum(); self.twist_n += len(d)
        cum = np.concatenate([[0.0], np.cumsum(d - THETA0)])
        for m in range(min(self.cw.shape[1], len(cum))):
            x = cum[m:] - cum[:len(cum) - m]
            self.cw[group, m] += np.cos(x).sum()
            self.sw[group, m] += np.sin(x).sum()
            self.nw[group, m] += len(cum) - m

    def twist_corr(self, g=None, d: float = 0.0) -> np.ndarray:
        """<cos(Omega(m) - m (theta0 + d))> of group g (None: all)."""
        sl = slice(None) if g is None else slice(g, g + 1)
        n = self.nw[sl].sum(0)
        m = np.arange(self.cw.shape[1])
        return (self.cw[sl].sum(0) * np.cos(m * d) + self.sw[sl].sum(0) * np.sin(m * d)) / n

    def result(self, s_fit: tuple, m_fit: tuple, s_short: int = 20) -> dict:
        ct = self.ct.sum(0) / self.nt.sum(0)
        G = len(self.ct)
        d = self.twist_sum / max(1, self.twist_n) - THETA0      # measured mean twist - 36 deg
        lp_g = [_fit_decay(self.ct[g] / self.nt[g], *s_fit) for g in range(G)]
        lps_g = [_fit_decay(self.ct[g] / self.nt[g], 1, s_short) for g in range(G)]
        lt_g = [_fit_decay(self.twist_corr(g), *m_fit) for g in range(G)]
        ltm_g = [_fit_decay(self.twist_corr(g, d), *m_fit) for g in range(G)]
        err = lambda v: float(np.std(v, ddof=1) / math.sqrt(G))
        return {"l_p_bp": _fit_decay(ct, *s_fit), "l_p_err_bp": err(lp_g),
                "l_p_short_bp": _fit_decay(ct, 1, s_short), "l_p_short_err_bp": err(lps_g),
                "l_tau_bp": _fit_decay(self.twist_corr(), *m_fit), "l_tau_err_bp": err(lt_g),
                "l_tau_mean_twist_bp": _fit_decay(self.twist_corr(None, d), *m_fit), "l_tau_mean_twist_err_bp": err(ltm_g),
                "twist_per_bp_deg": math.degrees(THETA0 + d),
                "tangent_correlator": ct.tolist(), "twist_correlator": self.twist_corr().tolist()}


def measure(n_mol=512, n_bp=300, equil=1_000_000, every=10_000, samples=100, seed=0, trim=5, groups=8,
            s_max=120, m_max=150, s_fit=(1, 100), m_fit=(1, 150), precision=None, init_lp=None, overrides=None,
            log=None):
    """Run n_mol independent n_bp chains (one context), equilibrate, then sample
    `samples` times every `every` steps; returns the fitted lengths in bp.
    The chains start straight, or (init_lp) along worm-like axes of that
    persistence length, so that equilibration can be checked from both sides."""
    from . import dsdna as D
    from . import inputs as I
    p = D.dsdna_default_params(seed=seed, **(overrides or {}))
    if precision is not None:
        p.precision = precision
    X = u = None
    if init_lp:
        rng = np.random.default_rng(seed)
        parts = [I.wlc_helix(n_bp, init_lp, rng) for _ in range(n_mol)]
        X = np.concatenate([q[0] for q in parts]); u = np.concatenate([q[1] for q in parts])
    ctx = D.Context(p, [n_bp] * n_mol, X=X, u=u)
    t0 = time.time()
    ctx.step(equil)
    ctx.synchronize()
    t_eq = time.time() - t0
    acc = Correlators(groups, s_max, m_max)
    for k in range(samples):
        ctx.step(every)
        for m in range(n_mol):
            cen, tw = ctx.profiles(m)
            acc.add(m * groups // n_mol, cen, tw, trim)
        if log:
            log(f"sample {k + 1}/{samples}")
    ctx.close()
    out = acc.result(s_fit, m_fit)
    out.update({"n_mol": n_mol, "n_bp": n_bp, "equilibration_steps": equil, "sample_every": every,
                "samples": samples, "trim_bp": trim, "init_lp_bp": init_lp, "overrides": overrides or {},
                "seconds": time.time() - t0,
                "seconds_equilibration": t_eq, "paper": {"l_p_bp": "143 +- 7", "l_tau_bp": "512 +- 18"}})
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n-mol", type=int, default=512)
    ap.add_argument("--n-bp", type=int, default=300)
    ap.add_argument("--equil", type=int, default=1_000_000)
    ap.add_argument("--every", type=int, default=10_000)
    ap.add_argument("--samples", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init-lp", type=float, default=None, help="start along worm-like axes of this l_p (bp)")
    ap.add_argument("--param", action="append", default=[], metavar="NAME=VALUE",
                    help="override a model parameter (e.g. K5=400), repeatable")
    ap.add_argument("--out", default=None, help="write the JSON result here")
    a = ap.parse_args()
    import torch
    torch.cuda.init()
    ov = {k: (int(v) if v.lstrip("-").isdigit() else float(v)) for k, v in (x.split("=", 1) for x in a.param)}
    r = measure(a.n_mol, a.n_bp, a.equil, a.every, a.samples, a.seed, init_lp=a.init_lp, overrides=ov)
    short = {k: v for k, v in r.items() if not k.endswith("correlator")}
    print(json.dumps(short))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)


if __name__ == "__main__":
    main()
