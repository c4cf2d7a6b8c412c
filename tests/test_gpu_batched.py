"""Batched engine, autotuner and the tethered single-molecule workload on the GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    yield


def _batch(seed=3):
    cfg = I.ragged_batch([130, 1, 64, 257, 2, 33, 500], seed=seed, spread=0.03)
    return cfg


@pytest.mark.parametrize("prec", [D.PREC_MIXED, D.PREC_FP64])
def test_batch_forces_equal_each_molecule_alone(prec):
    """Molecules never interact and every force sum runs in a fixed order, so a
    molecule's forces in a batch are bit for bit its forces alone."""
    cfg = _batch()
    p = D.dsdna_default_params(precision=prec)
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
    Fb, Fp = ctx.compute_forces()
    ctx.close()
    off = np.concatenate([[0], np.cumsum(cfg.n_bp)])
    for m, nb in enumerate(cfg.n_bp):
        sl = slice(2 * off[m], 2 * off[m + 1])
        c1 = D.Context(p, [int(nb)], X=cfg.X[sl], V=cfg.V[sl], u=cfg.u[sl], Om=cfg.Om[sl])
        fb, fp = c1.compute_forces()
        c1.close()
        assert np.array_equal(fb, Fb[sl]) and np.array_equal(fp, Fp[sl]), m


def test_periodic_array_molecules_equal_alone_and_oracle():
    """Paper's benchmark geometry in small (3 x 3 strands of 40 bp, periodic box,
    linear cell table with >= 3 cells per edge): each molecule's forces in the
    array equal its forces alone in the same box bit for bit, and the array's
    forces match the FP64 oracle."""
    cfg = I.paper_array(3, 3, 40, spacing=5.0, seed=2)
    X, u = I.perturb(cfg.X, cfg.u, np.random.default_rng(3), dx=0.02, dtheta=0.05)
    p = D.dsdna_default_params(box=cfg.box)
    ctx = D.Context(p, cfg.n_bp, X=X, V=cfg.V, u=u, Om=cfg.Om)
    Fb, Fp = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    off = np.concatenate([[0], np.cumsum(cfg.n_bp)])
    for m in range(len(cfg.n_bp)):
        sl = slice(2 * off[m], 2 * off[m + 1])
        c1 = D.Context(p, [int(cfg.n_bp[m])], X=X[sl], V=cfg.V[sl], u=u[sl], Om=cfg.Om[sl])
        fb, fp = c1.compute_forces()
        c1.close()
        assert np.array_equal(fb, Fb[sl]) and np.array_equal(fp, Fp[sl]), m
    po = O.params(box=cfg.box)
    r = O.forces(po, cfg.n_bp, Xs, us, cells=True)
    Sb, Sp = O.force_scale(po, cfg.n_bp, Xs, us)
    for Fg, Fo, Sc in ((Fb, r["Fb"], Sb), (Fp, r["Fp"], Sp)):
        assert (np.linalg.norm(Fg - Fo, axis=1) / (1e-5 * Sc + 5e-4)).max() < 1.0


def test_autotune_picks_a_candidate_and_keeps_the_forces():
    cfg = I.ragged_batch([130, 1, 64, 257, 2, 33, 500], seed=4)   # relaxed helices: the trials run dynamics
    p0 = D.dsdna_default_params()
    best, ns = D.dsdna_autotune(p0, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, trial_steps=20)
    assert round(best.skin, 3) in (0.2, 0.3, 0.4, 0.5, 0.6)
    assert best.block_threads in (128, 256) and best.blocks_per_sm in (0, 2)
    assert ns > 0.0
    a = D.Context(p0, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
    b = D.Context(best, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
    Fa = a.compute_forces()
    Fb_ = b.compute_forces()
    assert np.array_equal(Fa[0], Fb_[0]) and np.array_equal(Fa[1], Fb_[1])
    a.close(); b.close()


def test_batched_run_with_loads_stays_finite_and_stretches():
    """Each molecule carries its own load: after a short run the stretched
    molecules are longer than the unloaded one, and nothing diverges."""
    lengths = [60, 60, 60]
    cfg = I.ragged_batch(lengths, seed=5)
    p = D.dsdna_default_params(seed=9)
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=[1, 1, 1])
    for m, f in enumerate((0.0, 5.0, 20.0)):
        ctx.set_external_force_torque(m, [0.0, 0.0, f], [0.0, 0.0, 0.0])
    rz = np.zeros(3)
    for k in range(20):
        ctx.step(200)
        for m in range(3):
            rz[m] += ctx.observables(m, D.OBS_EXT)["rz"]
    X, V, u, Om = ctx.get_state()
    assert np.isfinite(X).all() and np.isfinite(V).all()
    assert rz[2] > rz[1] > rz[0]
    ctx.close()


def test_tethered_10kbp_tracks_the_oracle_first_steps():
    """Tethered 10 kbp molecule pulled with f = 5 kT/nm and twisted with 2 kT:
    mixed-precision engine against the FP64 oracle on the first 200 steps
    (same Philox noise)."""
    cfg = I.c2_tethered(n_bp=10_000, force=5.0, torque=2.0, seed=0)
    p = D.dsdna_default_params(seed=21)
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether)
    ctx.set_external_force_torque(0, cfg.ext_f[0], cfg.ext_t[0])
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    po = O.params(seed=21)
    errs = []
    for chunk in range(4):
        O.run(po, cfg.n_bp, X, V, u, Om, 50, step0=50 * chunk, ext_f=cfg.ext_f, ext_t=cfg.ext_t, tether=cfg.tether,
              cells=True)
        ctx.step(50)
        Xg = ctx.get_state()[0]
        errs.append(np.abs(Xg - X).max())
    assert errs[-1] < 1e-4, errs
    assert np.abs(Xg[:2] - cfg.X[:2]).max() == 0.0      # the anchored base pair never moves
    ctx.close()
