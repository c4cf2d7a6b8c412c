"""Single-molecule experiments of Sec. 4 with the engine: force-extension of
a 300 bp chain (Sec. 4.1, Eq. 5, Figs. 5-6) and the twist response of a
600 bp chain under 16 pN (Sec. 4.2, Eq. 7, Figs. 7-8).

Every (load, copy) pair is an independent molecule of one batched context:
base pair 0 anchored, a force F e_z (and a torque Gamma e_z) on the last base
pair.  Units: nm, kT = 1, so a force of 1 kT/nm is 4.11 pN at 298 K.

* Force-extension: <R_z>(F) is fitted with the worm-like-chain law of Eq. 5,
  F l_p / kT = x + 1/(4 (1 - x)^2) - 1/4 with x = R_z / L, for L and l_p
  (the paper: L = 100.3 +- 1.7 nm, l_p = 47 +- 2 nm).
* Twist response: sigma = (Tw - Tw0) / Tw0 with Tw0 = N / 10 turns, and
  C = (a0 / theta0) dGamma / dsigma / kT with a0 = 0.34 nm, theta0 = 2 pi / 10
  (Eq. 7; the paper: C = 88 nm).

The observables come from the engine's kernels (dsdna_observables); the fits
are plain least squares on the host.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

PN_PER_KT_NM = 4.114    # 1 kT/nm in pN at 298 K
A0 = 0.34               # nm per base pair (Sec. 4.2)
THETA0 = 2.0 * math.pi / 10.0


def wlc_force(x: np.ndarray, lp: float) -> np.ndarray:
    """Eq. 5: force (kT/nm) at relative extension x for persistence length lp (nm)."""
    return (x + 0.25 / (1.0 - x) ** 2 - 0.25) / lp


def fit_wlc(F: np.ndarray, Rz: np.ndarray, L0: float) -> tuple:
    """Least-squares fit of Eq. 5 to (F, <R_z>): returns (L, l_p, their errors)."""
    from scipy.optimize import curve_fit

    def model(rz, L, lp):
        return wlc_force(np.clip(rz / L, 0.0, 0.999), lp)
    p, cov = curve_fit(model, Rz, F, p0=(L0, 50.0), bounds=([0.5 * L0, 1.0], [2.0 * L0, 1000.0]))
    err = np.sqrt(np.diag(cov))
    return float(p[0]), float(p[1]), float(err[0]), float(err[1])


def fit_torsion(gamma: np.ndarray, sigma: np.ndarray) -> tuple:
    """Slope dGamma/dsigma by least squares and C of Eq. 7 (nm), with its error."""
    A = np.vstack([sigma, np.ones_like(sigma)]).T
    coef, res, _, _ = np.linalg.lstsq(A, gamma, rcond=None)
    slope = coef[0]
    n = len(sigma)
    s2 = float(res[0]) / max(1, n - 2) if len(res) else 0.0
    se = math.sqrt(s2 / max(1e-300, ((sigma - sigma.mean()) ** 2).sum()))
    k = A0 / THETA0
    return k * slope, k * se


def run_batch(n_bp: int, loads, copies: int, equil: int, every: int, samples: int, seed: int, flags, log=None,
              init_lp=None):
    """One context of len(loads) x copies anchored molecules; loads are
    (force, torque) pairs along e_z.  The molecules start straight along e_z,
    or (init_lp, bp) along smooth worm-like axes, so that slow relaxation can
    be bracketed from both sides.  Returns per-load mean observables."""
    from . import dsdna as D
    from . import inputs as I
    n_mol = len(loads) * copies
    if init_lp:
        rng = np.random.default_rng(seed)
        parts = [I.wlc_helix(n_bp, init_lp, rng) for _ in range(n_mol)]
        X = np.concatenate([q[0] for q in parts]); u = np.concatenate([q[1] for q in parts])
    else:
        X, u = I.straight_helix(n_bp)
        X = np.concatenate([X] * n_mol); u = np.concatenate([u] * n_mol)
    ctx = D.Context(D.dsdna_default_params(seed=seed), [n_bp] * n_mol, X=X, u=u, tether=[1] * n_mol)
    for m in range(n_mol):
        f, g = loads[m // copies]
        ctx.set_external_force_torque(m, [0.0, 0.0, f], [0.0, 0.0, g])
    ctx.step(equil)
    acc = {k: np.zeros(len(loads)) for k in ("rz", "tw", "wr", "lk")}
    for s in range(samples):
        ctx.step(every)
        for m in range(n_mol):
            o = ctx.observables(m, flags=flags)
            for k in acc:
                acc[k][m // copies] += o[k]
        if log:
            log(f"sample {s + 1}/{samples}")
    ctx.close()
    return {k: (v / (copies * samples)).tolist() for k, v in acc.items()}


def force_extension(n_bp=300, forces=(0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0), copies=24,
                    equil=500_000, every=5_000, samples=100, seed=0, init_lp=None, log=None):
    from . import dsdna as D
    t0 = time.time()
    r = run_batch(n_bp, [(f, 0.0) for f in forces], copies, equil, every, samples, seed, D.OBS_EXT, log, init_lp)
    F = np.array(forces); Rz = np.array(r["rz"])
    L, lp, eL, elp = fit_wlc(F, Rz, A0 * n_bp)
    return {"n_bp": n_bp, "forces_kT_per_nm": list(forces), "forces_pN": [f * PN_PER_KT_NM for f in forces],
            "Rz_nm": Rz.tolist(), "L_nm": L, "L_err_nm": eL, "l_p_nm": lp, "l_p_err_nm": elp,
            "l_p_bp": lp / A0, "copies": copies, "equilibration_steps": equil, "samples": samples, "init_lp_bp": init_lp,
            "sample_every": every, "seconds": time.time() - t0,
            "paper": {"L_nm": "100.3 +- 1.7", "l_p_nm": "47 +- 2"}}


def twist_response(n_bp=600, force_pN=16.0, torques=(-2.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0), copies=16,
                   equil=300_000, every=5_000, samples=60, seed=1, log=None):
    from . import dsdna as D
    t0 = time.time()
    f = force_pN / PN_PER_KT_NM
    r = run_batch(n_bp, [(f, g) for g in torques], copies, equil, every, samples, seed,
                  D.OBS_EXT | D.OBS_TW | D.OBS_LK, log)
    tw0 = n_bp / 10.0
    sigma_tw = (np.array(r["tw"]) - tw0) / tw0
    sigma_lk = (np.array(r["lk"]) - tw0) / tw0
    G = np.array(torques)
    C, eC = fit_torsion(G, sigma_tw)
    C_lk, eC_lk = fit_torsion(G, sigma_lk)
    return {"n_bp": n_bp, "force_pN": force_pN, "torques_kT": list(torques), "sigma_from_twist": sigma_tw.tolist(),
            "sigma_from_lk": sigma_lk.tolist(), "writhe": r["wr"], "C_nm": C, "C_err_nm": eC,
            "C_from_lk_nm": C_lk, "C_from_lk_err_nm": eC_lk, "copies": copies, "equilibration_steps": equil,
            "samples": samples, "sample_every": every, "seconds": time.time() - t0, "paper": {"C_nm": "88"}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--which", choices=("stretch", "twist", "both"), default="both")
    ap.add_argument("--equil", type=int, default=None)
    ap.add_argument("--samples", type=int, default=None)
    ap.add_argument("--every", type=int, default=None)
    ap.add_argument("--init-lp", type=float, default=None, help="stretch runs start along worm-like axes (bp)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    import torch
    torch.cuda.init()
    out = {}
    kw = {k: v for k, v in (("equil", a.equil), ("samples", a.samples), ("every", a.every)) if v is not None}
    if a.which in ("stretch", "both"):
        out["force_extension"] = force_extension(init_lp=a.init_lp, **kw)
        print(json.dumps({k: v for k, v in out["force_extension"].items() if k != "Rz_nm"}), flush=True)
    if a.which in ("twist", "both"):
        out["twist_response"] = twist_response(**kw)
        print(json.dumps(out["twist_response"]), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
