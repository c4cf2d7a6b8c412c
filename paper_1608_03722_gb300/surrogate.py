"""Sweep surrogate: an MLP that maps (force, torque, length, kT) to the mean
extension / contour length, the excess twist (Tw - Tw0)/Tw0 and the
denatured-bp fraction of a tethered molecule, trained on sweeps the engine
itself simulates.

The network runs in libdsdna.so (dsdna_mlp_*: BF16 tensor-core forward and
backward, FP32 accumulation, Adam); this module only marshals arguments,
holds an ensemble for query-by-committee selection, and drives the batched
engine to produce labels.  The full simulation stays the fallback and the
judge: ``Surrogate.predict`` returns the committee spread so that uncertain
points can be sent to ``simulate_sweep``.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import dsdna as D

NI, NO = 4, 3
KT_LEVELS = np.round(np.linspace(0.8, 1.4, 7), 3)   # kT is a per-context parameter: points are run at these levels


def _lib():
    L = D.load()
    if not getattr(L, "_mlp_ready", False):
        P = C.POINTER
        L.dsdna_mlp_create.argtypes = [C.c_int, P(D.dsdna_allocator), C.c_void_p, P(C.c_void_p)]
        L.dsdna_mlp_num_params.argtypes = []
        L.dsdna_mlp_set_params.argtypes = [C.c_void_p] + [P(C.c_float)] * 5
        L.dsdna_mlp_get_params.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float)]
        L.dsdna_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.dsdna_mlp_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, P(C.c_float)]
        L.dsdna_mlp_adam_step.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]
        L.dsdna_mlp_destroy.argtypes = [C.c_void_p]
        L.dsdna_mlp_destroy.restype = None
        L._mlp_ready = True
    return L


def _fp(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


class Mlp:
    """One network on the device (dsdna_mlp)."""

    def __init__(self, max_batch: int = 4096, stream=None):
        import torch
        self.torch = torch
        self.L = _lib()
        self.stream = torch.cuda.current_stream().cuda_stream if stream is None else stream
        self._alloc = D._TorchAllocator(self.stream)
        self.h = C.c_void_p()
        rc = self.L.dsdna_mlp_create(int(max_batch), C.byref(self._alloc.struct), C.c_void_p(self.stream), C.byref(self.h))
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_create failed")
        self.np = self.L.dsdna_mlp_num_params()
        self.max_batch = max_batch

    def set_params(self, params=None, in_mean=None, in_scale=None, out_mean=None, out_scale=None):
        keep = [_fp(x) for x in (params, in_mean, in_scale, out_mean, out_scale)]
        rc = self.L.dsdna_mlp_set_params(self.h, *[None if k is None else k[1] for k in keep])
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_set_params failed")

    def get_params(self):
        p = np.zeros(self.np, np.float32); g = np.zeros(self.np, np.float32)
        rc = self.L.dsdna_mlp_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                         g.ctypes.data_as(C.POINTER(C.c_float)))
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_get_params failed")
        return p, g

    def forward(self, X, Y):
        """X, Y: CUDA float32 tensors [B, 4], [B, 3]."""
        rc = self.L.dsdna_mlp_forward(self.h, C.c_void_p(X.data_ptr()), int(X.shape[0]), C.c_void_p(Y.data_ptr()))
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_forward failed")

    def backward(self, T, want_loss=True):
        loss = C.c_float()
        rc = self.L.dsdna_mlp_backward(self.h, C.c_void_p(T.data_ptr()), int(T.shape[0]),
                                       C.byref(loss) if want_loss else None)
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_backward failed")
        return loss.value

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        rc = self.L.dsdna_mlp_adam_step(self.h, float(lr), float(beta1), float(beta2), float(eps), float(weight_decay))
        if rc != 0:
            raise D.DsdnaError(rc, "dsdna_mlp_adam_step failed")

    def close(self):
        if self.h is not None and self.h.value:
            self.L.dsdna_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def input_norm(X):
    """Affine scaling of every input onto [-1, 1] over the training range."""
    lo, hi = np.asarray(X).min(0), np.asarray(X).max(0)
    return (lo + hi) / 2.0, np.maximum((hi - lo) / 2.0, 1e-6)


def _he_init(seed):
    """He-style initial parameters for W1[64][4] b1 W2[64][64] b2 W3[3][64] b3."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / NI), 64 * NI), np.zeros(64), rng.normal(0, math.sqrt(2.0 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, math.sqrt(1.0 / 64), NO * 64), np.zeros(NO)]
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    """Committee of networks (different initial weights and minibatch orders)."""

    def __init__(self, n_models: int = 4, max_batch: int = 4096, seed: int = 0):
        import torch
        self.torch = torch
        self.models = [Mlp(max_batch) for _ in range(n_models)]
        self.seed = seed
        self.norm = None

    def fit(self, X, T, iters: int = 3000, batch: int = 256, lr: float = 3e-3, weight_decay: float = 1e-2,
            val_frac: float = 0.2, check_every: int = 25, patience: int = 10):
        """Train every member with Adam (decoupled weight decay on the weights,
        learning rate decayed tenfold over `iters`) on random minibatches.

        Sweep labels are time averages of short simulations and carry sampling
        noise, so each member holds out its own random `val_frac` of the points,
        checks its loss on them every `check_every` iterations, and keeps the
        parameters of the lowest one, stopping after `patience` checks without
        improvement.  Points with non-finite labels are skipped.  Returns the
        members' best validation losses (training losses when nothing is held out)."""
        torch = self.torch
        X = np.asarray(X, np.float32); T = np.asarray(T, np.float32)
        ok = np.isfinite(T).all(1)          # points whose simulation broke carry NaN labels
        X, T = X[ok], T[ok]
        in_mean, in_scale = input_norm(X)
        out_mean, out_scale = T.mean(0), np.maximum(T.std(0), 1e-4)
        self.norm = (in_mean, in_scale, out_mean, out_scale)
        Xd = torch.tensor(X, device="cuda"); Td = torch.tensor(T, device="cuda")
        n = X.shape[0]
        Yd = torch.empty((max(batch, n), NO), device="cuda")
        losses = []
        for k, m in enumerate(self.models):
            m.set_params(_he_init(self.seed + k), in_mean, in_scale, out_mean, out_scale)
            rng = np.random.default_rng(self.seed + 100 + k)
            perm = rng.permutation(n)
            nv = int(round(val_frac * n)) if n >= 10 else 0
            vi, ti = perm[:nv], perm[nv:]
            Xt, Tt = Xd[torch.tensor(ti, device="cuda")].contiguous(), Td[torch.tensor(ti, device="cuda")].contiguous()
            if nv:
                Xv = Xd[torch.tensor(vi, device="cuda")].contiguous()
                Tv = Td[torch.tensor(vi, device="cuda")].contiguous()
            nt = len(ti)
            best_loss, best_p, bad = math.inf, None, 0
            for it in range(iters):
                idx = torch.tensor(rng.choice(nt, size=min(batch, nt), replace=False), device="cuda")
                xb = Xt[idx].contiguous(); tb = Tt[idx].contiguous()
                m.forward(xb, Yd[: xb.shape[0]])
                m.backward(tb, want_loss=False)
                m.adam(lr * (0.1 ** (it / iters)), weight_decay=weight_decay)
                if nv and (it + 1) % check_every == 0:
                    m.forward(Xv, Yd[:nv])
                    lv = m.backward(Tv)
                    if lv < best_loss:
                        best_loss, best_p, bad = lv, m.get_params()[0], 0
                    else:
                        bad += 1
                        if bad >= patience:
                            break
            if best_p is not None:
                m.set_params(best_p)
                losses.append(best_loss)
            else:
                m.forward(Xt, Yd[:nt])
                losses.append(m.backward(Tt))
        return losses

    def predict(self, X):
        """Committee mean and spread of the outputs, [B, 3] each."""
        torch = self.torch
        Xd = torch.tensor(np.ascontiguousarray(X, np.float32), device="cuda")
        outs = []
        for m in self.models:
            Yd = torch.empty((Xd.shape[0], NO), device="cuda")
            m.forward(Xd, Yd)
            outs.append(Yd)
        Y = torch.stack(outs).cpu().numpy()
        return Y.mean(0), Y.std(0)

    def select(self, candidates, k: int):
        """Query by committee: the k candidates on which the members disagree most
        (spread summed over outputs in units of each output's scale)."""
        _, sd = self.predict(candidates)
        score = (sd / self.norm[3]).sum(1)
        return np.argsort(-score)[:k]

    def close(self):
        for m in self.models:
            m.close()


def sample_points(n: int, seed: int = 0, length=(500, 20000), force=(0.1, 10.0), torque=(-5.0, 5.0)):
    """Sweep inputs: force and torque uniform, length log-uniform, kT on the run levels."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(*force, n)
    g = rng.uniform(*torque, n)
    L = np.exp(rng.uniform(math.log(length[0]), math.log(length[1]), n)).round()
    kT = rng.choice(KT_LEVELS, n)
    return np.stack([f, g, L, kT], 1)


def sweep_dt(kT: float) -> float:
    """Timestep of a sweep run at temperature kT: 0.005 tau_Br with the
    Brownian time tau_Br = gamma sigma^2 / kT of the run (App. A units), so
    the step is 0.005 at kT = 1 and shrinks as the noise grows."""
    return 0.005 / float(kT)


def _broken_molecules(ctx, lengths, R0):
    """Molecules to drop after a device error: those with a non-finite
    coordinate or a backbone bond beyond 0.9 R0 in the post-mortem state, else
    the one whose longest bond is closest to R0 (the state is the one after
    the update of the step whose forces saw the bond at R0)."""
    X, V, u, Om = ctx.get_state()
    off = np.concatenate([[0], np.cumsum(lengths)]) * 2
    bad, score = [], np.zeros(len(lengths))
    for m in range(len(lengths)):
        Xm, um = X[off[m]:off[m + 1]], u[off[m]:off[m + 1]]
        if not (np.isfinite(Xm).all() and np.isfinite(V[off[m]:off[m + 1]]).all() and np.isfinite(um).all()):
            bad.append(m)
            continue
        b = Xm - 0.25 * um
        score[m] = np.linalg.norm(b[2:] - b[:-2], axis=1).max() / R0 if len(b) > 2 else 0.0
        if score[m] >= 0.9:
            bad.append(m)
    if not bad:
        bad = [int(np.argmax(score))]
    return bad


def _run_group(lengths, loads, kT, seed, steps, measure_from, every, refine=1):
    """One context of tethered molecules at one kT; returns (labels, None) or
    (None, indices of the molecules that broke) after a device error.  With
    refine = r the timestep is sweep_dt(kT) / r and every step count is
    multiplied by r, so the samples fall at the same physical times."""
    from . import inputs as I
    cfg = I.ragged_batch(lengths, seed=seed)
    p = D.dsdna_default_params(kT=float(kT), dt=sweep_dt(kT) / refine, seed=seed + 1000)
    steps, measure_from, every = steps * refine, measure_from * refine, every * refine
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, u=cfg.u, tether=np.ones(len(lengths), np.int32))
    try:
        for m, (f, g) in enumerate(loads):
            ctx.set_external_force_torque(m, [0.0, 0.0, f], [0.0, 0.0, g])
        acc = np.zeros((len(lengths), NO)); ns = 0
        done = 0
        try:
            while done < steps:
                ctx.step(every)
                done += every
                if done >= measure_from:
                    for m in range(len(lengths)):
                        o = ctx.observables(m, D.OBS_EXT | D.OBS_DENAT | D.OBS_TW)
                        N = lengths[m]
                        acc[m, 0] += o["rz"] / (0.34 * max(N - 1, 1))
                        acc[m, 1] += (o["tw"] - o["tw_ideal"]) / o["tw_ideal"] if o["tw_ideal"] else 0.0
                        acc[m, 2] += o["denat"]
                    ns += 1
        except D.DsdnaError as e:
            if e.status not in ("EFENE", "ENAN"):
                raise
            return None, _broken_molecules(ctx, lengths, p.R0)
        return acc / max(ns, 1), None
    finally:
        ctx.close()


def simulate_sweep(points, steps: int = 4000, measure_from: int = 2000, every: int = 200, seed: int = 0,
                   max_nt_per_context: int = 3_000_000):
    """Full simulations of the sweep points with the batched engine.

    Every point is one tethered molecule of its length (relaxed helix along
    z, base pair 0 anchored) with force f e_z and torque Gamma e_z on its
    last base pair; points of one kT level run together in one context
    (chunked by size) at the timestep ``sweep_dt(kT)``.  The labels are the
    averages over the samples taken every ``every`` steps from
    ``measure_from`` on of: R_z / (0.34 (N-1)), (Tw - Tw0) / Tw0 and the
    denatured fraction.  A molecule whose backbone breaks (FENE reaches R0,
    an integration failure of the stiff bond under large loads) is taken out
    of its group, which is run again without it, and is then simulated once
    more at half the timestep; if it breaks again its labels are NaN.
    """
    pts = np.asarray(points, np.float64)
    out = np.zeros((len(pts), NO))
    order = np.argsort(pts[:, 3], kind="stable")
    groups = []
    for kT in np.unique(pts[:, 3]):
        idx = [i for i in order if pts[i, 3] == kT]
        cur, tot = [], 0
        for i in idx:
            nt = 2 * int(pts[i, 2])
            if cur and tot + nt > max_nt_per_context:
                groups.append((kT, cur)); cur, tot = [], 0
            cur.append(i); tot += nt
        if cur:
            groups.append((kT, cur))
    def run(groups, refine):
        broken = []
        for gi, (kT, idx) in enumerate(groups):
            idx = list(idx)
            for _attempt in range(8):
                if not idx:
                    break
                lengths = [int(pts[i, 2]) for i in idx]
                loads = [(pts[i, 0], pts[i, 1]) for i in idx]
                lab, bad = _run_group(lengths, loads, kT, seed + gi + 977 * (refine - 1), steps, measure_from, every,
                                      refine)
                if bad is None:
                    out[idx] = lab
                    break
                for m in bad:
                    out[idx[m]] = np.nan
                    broken.append(idx[m])
                idx = [i for m, i in enumerate(idx) if m not in set(bad)]
            else:
                out[idx] = np.nan
                broken += idx
        return broken

    broken = run(groups, 1)
    if broken:
        again = {}
        for i in broken:
            again.setdefault(pts[i, 3], []).append(i)
        run(sorted(again.items()), 2)
    return out


def _metrics(Y, T):
    ok = np.isfinite(T).all(1)
    Y, T = Y[ok], T[ok]
    err = Y - T
    rmse = np.sqrt((err ** 2).mean(0))
    var = ((T - T.mean(0)) ** 2).mean(0)
    r2 = 1.0 - (err ** 2).mean(0) / np.maximum(var, 1e-30)
    return {"rmse": rmse.tolist(), "r2": r2.tolist()}


def run_sweep_study(n_train: int = 2000, n_test: int = 200, n_query: int = 100, length=(500, 20000),
                    steps: int = 8000, measure_from: int = 2000, every: int = 200, models: int = 4,
                    iters: int = 3000, seed: int = 0, query_rounds: int = 1) -> dict:
    """Train on n_train simulated sweep points, evaluate on n_test held-out
    simulated points; then add n_query points chosen by the committee or at
    random and compare the held-out error of the two retrained surrogates
    (query_rounds times, each with its own candidate pool, random pick and
    initial weights, for the spread of the difference).  The held-out points
    are simulated a second time with another seed: the RMS difference /
    sqrt(2) is the sampling noise of one simulated label, the yardstick for
    the surrogate's error."""
    import time
    import torch

    def sim(pts, s):
        t = time.perf_counter()
        y = simulate_sweep(pts, steps=steps, measure_from=measure_from, every=every, seed=s)
        torch.cuda.synchronize()
        return y, time.perf_counter() - t

    train = sample_points(n_train, seed, length)
    test = sample_points(n_test, seed + 1, length)
    Ttrain, t_train = sim(train, seed)
    Ttest, t_test = sim(test, seed + 1)
    Trep, _ = sim(test, seed + 6)
    both = np.isfinite(Ttest).all(1) & np.isfinite(Trep).all(1)
    rep_noise = np.sqrt(((Ttest[both] - Trep[both]) ** 2).mean(0) / 2)
    sur = Surrogate(models, max_batch=max(4096, n_train + n_query), seed=seed)
    t = time.perf_counter()
    sur.fit(train, Ttrain, iters=iters)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t
    t = time.perf_counter()
    Y, sd = sur.predict(test)
    t_pred = time.perf_counter() - t
    base = _metrics(Y, Ttest)
    base["rmse_over_replicate_noise"] = (np.asarray(base["rmse"]) / np.maximum(rep_noise, 1e-30)).tolist()
    # query by committee vs random additions of the same size
    rounds = []
    for q in range(query_rounds):
        sq = seed + 100 * q
        if q:
            sur.close()
            sur = Surrogate(models, max_batch=max(4096, n_train + n_query), seed=sq)
            sur.fit(train, Ttrain, iters=iters)
        cand = sample_points(20 * n_query, sq + 2, length)
        pick = sur.select(cand, n_query)
        rnd = np.random.default_rng(sq + 3).choice(len(cand), n_query, replace=False)
        Tq, _ = sim(cand[pick], sq + 4)
        Tr, _ = sim(cand[rnd], sq + 5)
        sur.fit(np.concatenate([train, cand[pick]]), np.concatenate([Ttrain, Tq]), iters=iters)
        qbc = _metrics(sur.predict(test)[0], Ttest)
        sur.fit(np.concatenate([train, cand[rnd]]), np.concatenate([Ttrain, Tr]), iters=iters)
        random_add = _metrics(sur.predict(test)[0], Ttest)
        rounds.append({"committee": qbc, "random": random_add})
    sur.close()
    gain = np.array([np.asarray(r["committee"]["r2"]) - np.asarray(r["random"]["r2"]) for r in rounds])
    return {
        "train_points": n_train, "test_points": n_test, "lengths_bp": list(length), "steps": steps,
        "outputs": ["extension/contour", "excess twist (Tw-Tw0)/Tw0", "denatured fraction"],
        "label_spread": np.nanstd(Ttest, 0).tolist(), "replicate_noise": rep_noise.tolist(),
        "dropped_points": {"train": int((~np.isfinite(Ttrain).all(1)).sum()),
                           "test": int((~np.isfinite(Ttest).all(1)).sum())},
        "held_out": base, "after_committee_queries": rounds[0]["committee"],
        "after_random_queries": rounds[0]["random"], "query_rounds": rounds,
        "committee_minus_random_r2": {"mean": gain.mean(0).tolist(),
                                      "std": (gain.std(0, ddof=1) if len(gain) > 1 else np.zeros(NO)).tolist()},
        "seconds": {"simulate_train": t_train, "simulate_test": t_test, "fit": t_fit, "predict_test": t_pred},
        "simulation_s_per_point": t_test / n_test, "surrogate_s_per_point": t_pred / n_test,
        "speedup_per_point": (t_test / n_test) / max(t_pred / n_test, 1e-12),
    }


def kernel_passes(rows: int = 4096, passes: int = 3, seed: int = 0) -> float:
    """`passes` training iterations (forward, backward, Adam) of one network on
    `rows` random sweep points: a short run of the tensor-core kernels alone,
    e.g. for a profiler.  Returns the last loss."""
    import torch
    pts = sample_points(rows, seed)
    lab = np.stack([1.0 - 0.5 / np.sqrt(pts[:, 0] + 0.5), 0.01 * pts[:, 1], 0.05 * np.exp(-pts[:, 0] / 3)], 1)
    net = Mlp(max_batch=rows)
    m, sc = input_norm(pts)
    net.set_params(_he_init(seed), m, sc, lab.mean(0), lab.std(0) + 1e-6)
    X = torch.tensor(pts, dtype=torch.float32, device="cuda")
    T = torch.tensor(lab, dtype=torch.float32, device="cuda")
    Y = torch.empty((rows, NO), dtype=torch.float32, device="cuda")
    loss = float("nan")
    for _ in range(passes):
        net.forward(X, Y)
        loss = net.backward(T)
        net.adam(lr=1e-3)
    torch.cuda.synchronize()
    net.close()
    return loss


if __name__ == "__main__":
    import argparse
    import json
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "--kernels":    # --kernels [rows]: the kernels alone
        print(json.dumps({"loss": kernel_passes(int(sys.argv[2]) if len(sys.argv) > 2 else 4096)}))
        sys.exit(0)
    ap = argparse.ArgumentParser(description="sweep surrogate study (train / held-out / committee queries)")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--query", type=int, default=100)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--min-bp", type=int, default=500)
    ap.add_argument("--max-bp", type=int, default=20000)
    ap.add_argument("--iters", type=int, default=3000)
    a = ap.parse_args()
    print(json.dumps(run_sweep_study(a.train, a.test, a.query, (a.min_bp, a.max_bp), a.steps, iters=a.iters)))
