"""Trajectories of the step path against the FP64 oracle (same seed, same
Philox noise), in the periodic box of the throughput benchmark as well as in
an open box, and the error of the mixed-precision path stated per quantity.

Bounds: the FP64 engine differs from the oracle only by rounding order, so
its trajectory stays within 1e-9 nm of the oracle's for 200 steps.  The
mixed engine rounds every force to FP32 (relative 6e-8 of the per-site term
sum) and keeps X, V in FP64: it stays within 1e-4 nm for 100 steps, after
which the chaotic dynamics amplify the rounding differences.
"""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I
from tests.conftest import c3_walk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


def dense_walk(n_bp=3000, seed=1):
    """Random-walk helix packed into a small periodic box (L = 27.6 nm):
    contacts across periodic images and beads crossing the box faces."""
    cfg = I.random_walk_helix(n_bp=n_bp, phi=0.15, clearance=1.7, seed=seed)
    rng = np.random.default_rng(seed)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, rng, dx=0.01, dtheta=0.02)
    return cfg


def run_both(cfg, prec, seed, chunks, skin=None, tether=None):
    """Advance engine and oracle from the same state in chunks of steps; the
    largest |dX|, |dV|, |du|, |dOm| after each chunk."""
    kw = dict(precision=prec, box=cfg.box, seed=seed)
    if skin is not None:
        kw["skin"] = skin
    ctx = D.Context(D.dsdna_default_params(**kw), cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=tether)
    if cfg.ext_f is not None:
        for m in range(len(cfg.n_bp)):
            ctx.set_external_force_torque(m, cfg.ext_f[m], cfg.ext_t[m])
    po = O.params(box=cfg.box, seed=seed) if cfg.box[0] > 0 else O.params(seed=seed)
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    done, rows = 0, []
    for n in chunks:
        O.run(po, cfg.n_bp, X, V, u, Om, n, step0=done, ext_f=cfg.ext_f, ext_t=cfg.ext_t, tether=tether, cells=True)
        ctx.step(n)
        done += n
        Xg, Vg, ug, Og = ctx.get_state()
        rows.append((done, np.abs(Xg - X).max(), np.abs(Vg - V).max(), np.abs(ug - u).max(), np.abs(Og - Om).max()))
    info = ctx.info()
    ctx.close()
    return rows, info, (X, V, u, Om)


def _show(name, rows):
    for s, dx, dv, du, do in rows:
        print(f"{name} step {s:5d}: |dX| {dx:.2e}  |dV| {dv:.2e}  |du| {du:.2e}  |dOm| {do:.2e}")


def test_fp64_periodic_trajectory_matches_oracle():
    """Periodic box with pair contacts across images: skin 0.1 rebuilds the
    list every few steps, so the image words, the wrap of the build positions
    and the rebuilds across box faces all run; 200 steps to round-off."""
    cfg = dense_walk()
    rows, info, _ = run_both(cfg, D.PREC_FP64, 17, [50] * 4, skin=0.1)
    _show("fp64 periodic", rows)
    assert info["rebuilds"] > 10
    _, dx, dv, du, do = rows[-1]
    assert dx < 1e-9 and du < 1e-9 and dv < 1e-7 and do < 1e-7, rows[-1]


def test_mixed_periodic_trajectory_tracks_oracle():
    """The headline path (FP32 forces, FP64 X and V, periodic box, skin 0.1)
    stays on the oracle's trajectory for 100 steps."""
    cfg = dense_walk()
    rows, info, _ = run_both(cfg, D.PREC_MIXED, 18, [20] * 5, skin=0.1)
    _show("mixed periodic", rows)
    assert info["rebuilds"] > 5
    assert rows[-1][1] < 1e-4, rows


def test_c3_full_size_fp64_steps_match_oracle():
    """The 1 Mbp confined workload of the throughput benchmark (2e6
    nucleotides, periodic cube at volume fraction 0.05): 10 steps of the FP64
    engine against 10 oracle steps."""
    cfg = c3_walk()
    rows, info, _ = run_both(cfg, D.PREC_FP64, 3, [10])
    _show("fp64 1 Mbp", rows)
    assert rows[-1][1] < 1e-9 and rows[-1][3] < 1e-9, rows


def test_tethered_10kbp_first_thousand_steps():
    """Tethered 10 kbp molecule, f = 5 kT/nm, torque 2 kT: the mixed engine
    against the FP64 oracle on the first 10^3 steps (same noise).  The
    largest centre difference grows slowly (about 2e-5 nm at step 1000) and
    stays within 1e-4 nm over all 10^3 steps: no chaotic divergence yet."""
    cfg = I.c2_tethered(n_bp=10_000, force=5.0, torque=2.0, seed=0)
    rows, info, (X, _, _, _) = run_both(cfg, D.PREC_MIXED, 21, [100] * 10, tether=cfg.tether)
    _show("mixed tethered 10 kbp", rows)
    assert max(r[1] for r in rows) < 1e-4, rows
    assert max(r[3] for r in rows) < 1e-3, rows


def _quantities(cfg, prec, X, u):
    """Forces, energies, virial and observables of the engine on state (X, u)."""
    ctx = D.Context(D.dsdna_default_params(precision=prec, box=cfg.box), cfg.n_bp, X=X, V=np.zeros_like(X), u=u,
                    Om=np.zeros_like(X))
    Fb, Fp = ctx.compute_forces()
    E, W = ctx.energy_virial()
    obs = ctx.observables(0, D.OBS_EXT | D.OBS_DENAT | D.OBS_TW | D.OBS_LK)
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    return Fb, Fp, E, W, obs, Xs, us


@pytest.mark.parametrize("which", ["open_200bp", "periodic_dense"])
def test_mixed_precision_error_per_quantity(which):
    """The error of the mixed-precision engine against the FP64 oracle,
    quantity by quantity, printed as a table and bounded:

    * on one configuration (the one the engine holds): site forces relative
      to the larger of |F_i| and the RMS force, each energy term relative to
      the sum of |E_term|, the virial relative to its norm, R_z, twist,
      linking number and denatured fraction;
    * after 100 same-noise steps: X, V, u and Omega.
    """
    if which == "open_200bp":
        cfg = I.c1_linear(200)            # the trajectory starts from the relaxed helix
        rng = np.random.default_rng(31)
        Xp, up = I.perturb(cfg.X, cfg.u, rng, dx=0.03, dtheta=0.06)   # a thermal-like configuration
    else:
        cfg = dense_walk(1200, seed=33)
        Xp, up = cfg.X, cfg.u
    Fb, Fp, E, W, obs, Xs, us = _quantities(cfg, D.PREC_MIXED, Xp, up)
    po = O.params(box=cfg.box) if cfg.box[0] > 0 else O.params()
    r = O.forces(po, cfg.n_bp, Xs, us)
    F = np.concatenate([r["Fb"], r["Fp"]])
    Fg = np.concatenate([Fb, Fp])
    frms = np.sqrt((F * F).sum(1).mean())
    f_err = (np.linalg.norm(Fg - F, axis=1) / np.maximum(np.linalg.norm(F, axis=1), frms)).max()
    Eo, Wo = O.energy(po, cfg.n_bp, Xs, np.zeros_like(Xs), us, np.zeros_like(Xs), 0)
    e_scale = np.abs(Eo[0][:8]).sum()
    e_err = np.abs(E[:8] - Eo[0][:8]) / e_scale
    w_err = np.abs(W - Wo[0]).max() / np.abs(Wo[0]).max()
    oo = O.observables(po, cfg.n_bp, Xs, us, with_lk=True)
    o_err = {k: abs(obs[k] - oo[k]) for k in ("rz", "tw", "lk", "denat")}
    rows, _, _ = run_both(cfg, D.PREC_MIXED, 41, [100], skin=0.1)
    _, dx, dv, du, do = rows[-1]
    table = {"force (rel. max(|F|, F_rms))": f_err}
    table.update({f"energy {O.TERM_NAMES[k]} (rel. sum |E|)": e_err[k] for k in range(8)})
    table["virial (rel. max |W|)"] = w_err
    table.update({f"{k} (abs)": v for k, v in o_err.items()})
    table.update({"X after 100 steps (nm)": dx, "V after 100 steps": dv, "u after 100 steps": du,
                  "Omega after 100 steps": do})
    print(f"\n{which}:")
    for k, v in table.items():
        print(f"  {k:40s} {v:.2e}")
    assert f_err < 1e-5
    assert e_err.max() < 1e-6 and w_err < 1e-5
    assert o_err["rz"] < 1e-6 and o_err["tw"] < 1e-6 and o_err["lk"] < 1e-6 and o_err["denat"] == 0.0
    assert dx < 1e-4 and du < 1e-4 and dv < 1e-2 and do < 1e-1
