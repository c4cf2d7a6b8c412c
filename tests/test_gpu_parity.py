"""GPU parity: the CUDA engine (through the C ABI) against the FP64 oracle.

Forces are compared on identical configurations: the oracle evaluates the
state the engine holds (read back with get_state; in mixed precision the
orientation u is stored in FP32).  Per site i the bound is
    |F_gpu - F_oracle| <= rel * S_i + abs
with S_i the oracle's sum over all terms acting on the site of |term force|
(the condition scale of a floating-point force sum; FENE and its WCA counted
separately).  Mixed engine: rel = 1e-5, abs = 5e-4 kT/nm (twice the stiffest
term, 2 K4 lambda^2 = 3840 kT/nm^2, times the FP32 spacing of a 0.5 nm
displacement).  FP64 engine: rel = 1e-9, abs = 1e-10 kT/nm.
"""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I
from tests.conftest import c3_walk

pytestmark = pytest.mark.gpu

PRECS = [D.PREC_MIXED, D.PREC_FP64]
TOL = {D.PREC_MIXED: (1e-5, 5e-4), D.PREC_FP64: (1e-9, 1e-10)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


def oparams(cfg, **kw):
    return O.params(box=cfg.box, **kw) if cfg.box[0] > 0 else O.params(**kw)


def ctx_for(cfg, prec, X=None, u=None, **kw):
    p = D.dsdna_default_params(precision=prec, box=cfg.box, **kw)
    return D.Context(p, cfg.n_bp, X=cfg.X if X is None else X, V=cfg.V, u=cfg.u if u is None else u, Om=cfg.Om,
                     tether=cfg.tether)


def excess(Fg, Fo, S, prec):
    """Largest ratio of the force difference to its allowed bound (must stay < 1)."""
    rel, ab = TOL[prec]
    return (np.linalg.norm(Fg - Fo, axis=1) / (rel * S + ab)).max()


def check_forces(cfg, prec, X=None, u=None, ext=False):
    X = cfg.X if X is None else X
    u = cfg.u if u is None else u
    ctx = ctx_for(cfg, prec, X=X, u=u)
    if ext:
        for m in range(len(cfg.n_bp)):
            ctx.set_external_force_torque(m, cfg.ext_f[m], cfg.ext_t[m])
    Fb, Fp = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()          # the configuration the engine holds
    ef = cfg.ext_f if ext else None
    et = cfg.ext_t if ext else None
    r = O.forces(oparams(cfg), cfg.n_bp, Xs, us, ext_f=ef, ext_t=et)
    Sb, Sp = O.force_scale(oparams(cfg), cfg.n_bp, Xs, us, ext_f=ef, ext_t=et)
    eb, ep = excess(Fb, r["Fb"], Sb, prec), excess(Fp, r["Fp"], Sp, prec)
    ctx.close()
    assert eb < 1.0 and ep < 1.0, (eb, ep)
    return eb, ep


def dense_walk(n_bp=3000, seed=1):
    """Random-walk helix packed into a small periodic box: WCA contacts across images."""
    cfg = I.random_walk_helix(n_bp=n_bp, phi=0.15, clearance=1.7, seed=seed)
    rng = np.random.default_rng(seed)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, rng, dx=0.01, dtheta=0.02)
    return cfg


@pytest.mark.parametrize("prec", PRECS)
def test_forces_ideal_helix(prec):
    check_forces(I.c1_linear(200), prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_bp", [1, 2, 3, 127, 128, 129, 200, 515])
def test_forces_perturbed_lengths(prec, n_bp):
    """Lengths around the 128-bp segment of a 256-thread CTA, plus the degenerate 1-3 bp molecules."""
    cfg = I.c1_linear(n_bp)
    rng = np.random.default_rng(n_bp)
    X, u = I.perturb(cfg.X, cfg.u, rng, dx=0.03, dtheta=0.08)
    check_forces(cfg, prec, X, u)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_ragged_batch(prec):
    cfg = I.ragged_batch([1, 5, 130, 64, 257, 2, 33], seed=3, spread=0.03)
    check_forces(cfg, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_periodic_dense(prec):
    cfg = dense_walk()
    r = O.forces(oparams(cfg), cfg.n_bp, cfg.X, cfg.u)
    assert r["energy"][0, 3] > 1.0, "configuration must exercise the pair forces"
    check_forces(cfg, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_with_applied_load(prec):
    cfg = I.c4_batch(n_mol=5, lo=20, hi=300, seed=2)
    rng = np.random.default_rng(4)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, rng, dx=0.02, dtheta=0.05)
    check_forces(cfg, prec, ext=True)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_with_applied_load_random_poses(prec):
    """Molecules turned in random directions and placed anywhere in an open
    box (hashed cell table off its favourable axis), each loaded along its
    own axis."""
    cfg = I.c4_batch(n_mol=6, lo=20, hi=400, seed=5, random_pose=True, spread=30.0)
    rng = np.random.default_rng(6)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, rng, dx=0.02, dtheta=0.05)
    check_forces(cfg, prec, ext=True)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_with_the_ghost_size_for_steric_pairs_across_strands(prec):
    """The other reading of Sec. 2 (A1): steric beads of opposite strands at
    the ghost size sigma_cross = 0.5 (sigma_cross_steric <= 0), on the dense
    periodic walk; forces and the list against the oracle run with the same
    reading.  (The default, sigma = 1 for every steric pair, runs in every
    other parity test.)"""
    cfg = dense_walk(1500, seed=21)
    kw = dict(sigma_cross_steric=0.0)
    ctx = D.Context(D.dsdna_default_params(precision=prec, box=cfg.box, **kw), cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u,
                    Om=cfg.Om)
    Fb, Fp = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()
    got = {tuple(x) for x in ctx.neighbor_pairs()}
    skin = ctx.params.skin + 0.01
    ctx.close()
    po = O.params(box=cfg.box, **kw)
    r = O.forces(po, cfg.n_bp, Xs, us)
    Sb, Sp = O.force_scale(po, cfg.n_bp, Xs, us)
    eb, ep = excess(Fb, r["Fb"], Sb, prec), excess(Fp, r["Fp"], Sp, prec)
    assert eb < 1.0 and ep < 1.0, (eb, ep)
    lo = {tuple(x) for x in O.pairs(po, cfg.n_bp, Xs, us, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(po, cfg.n_bp, Xs, us, extra=skin + 1e-4)}
    assert lo <= got <= hi
    # the default reading lists more pairs (steric pairs across strands out to 1.43 nm)
    assert len(got) < len(O.pairs(O.params(box=cfg.box), cfg.n_bp, Xs, us, extra=skin))


@pytest.mark.parametrize("prec", PRECS)
def test_neighbor_pairs_equal_brute_force(prec):
    cfg = dense_walk(1500, seed=5)
    ctx = ctx_for(cfg, prec)
    got = {tuple(x) for x in ctx.neighbor_pairs()}
    skin = ctx.params.skin + 0.01   # the list radius carries a 0.01 margin over the skin
    want = {tuple(x) for x in O.pairs(oparams(cfg), cfg.n_bp, cfg.X, cfg.u, extra=skin)}
    # pairs within 1e-4 of the list radius may fall either way in FP32
    lo = {tuple(x) for x in O.pairs(oparams(cfg), cfg.n_bp, cfg.X, cfg.u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(oparams(cfg), cfg.n_bp, cfg.X, cfg.u, extra=skin + 1e-4)}
    assert lo <= got <= hi
    assert len(want) > 1000
    ctx.close()


def test_fp64_trajectory_matches_oracle():
    """Same seed, same uniform Philox noise: FP64 engine and oracle agree to round-off over 200 steps."""
    cfg = I.c1_linear(200)
    p = O.params(seed=11)
    ctx = ctx_for(cfg, D.PREC_FP64, seed=11)
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    O.run(p, cfg.n_bp, X, V, u, Om, 200)
    ctx.step(200)
    Xg, Vg, ug, Og = ctx.get_state()
    assert np.abs(Xg - X).max() < 1e-9
    assert np.abs(Vg - V).max() < 1e-7
    assert np.abs(ug - u).max() < 1e-9
    ctx.close()


def test_mixed_trajectory_tracks_oracle():
    """FP32 forces with FP64 accumulation stay on the oracle trajectory before chaotic divergence."""
    cfg = I.c1_linear(200)
    p = O.params(seed=12)
    ctx = ctx_for(cfg, D.PREC_MIXED, seed=12)
    X, V, u, Om = (a.copy() for a in (cfg.X, cfg.V, cfg.u, cfg.Om))
    errs = []
    for chunk in range(5):
        O.run(p, cfg.n_bp, X, V, u, Om, 20, step0=20 * chunk)
        ctx.step(20)
        Xg, Vg, ug, Og = ctx.get_state()
        errs.append(np.abs(Xg - X).max())
    assert errs[-1] < 1e-4, errs
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_energy_and_virial_match_oracle(prec):
    cfg = dense_walk(800, seed=7)
    ctx = ctx_for(cfg, prec)
    E, W = ctx.energy_virial()
    Eo, Wo = O.energy(oparams(cfg), cfg.n_bp, cfg.X, cfg.V, cfg.u, cfg.Om, 0)
    tol = 1e-9 if prec == D.PREC_FP64 else 2e-5
    scale = np.abs(Eo[0]).sum()
    assert np.abs(E - Eo[0]).max() < tol * scale, (E, Eo[0])
    assert np.abs(W - Wo[0]).max() < tol * np.abs(Wo[0]).sum() * 10
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_observables_match_oracle(prec):
    cfg = I.c1_linear(150)
    rng = np.random.default_rng(9)
    X, u = I.perturb(cfg.X, cfg.u, rng, dx=0.03, dtheta=0.05)
    X[1::2][:10, 0] += 0.5      # break ten hydrogen bonds
    ctx = ctx_for(cfg, prec, X=X, u=u)
    o = ctx.observables(0, D.OBS_EXT | D.OBS_DENAT | D.OBS_TW | D.OBS_LK)
    oo = O.observables(O.params(), cfg.n_bp, X, u, with_lk=True)
    un = u / np.linalg.norm(u, axis=1, keepdims=True)
    uf = np.ascontiguousarray(un.astype(np.float32).astype(np.float64))   # the engine keeps u in FP32
    oo2 = O.observables(O.params(), cfg.n_bp, X, uf, with_lk=True)
    for k in ("rz", "denat", "tw", "lk", "wr"):
        ref = oo if prec == D.PREC_FP64 else oo2
        assert abs(o[k] - ref[k]) < 1e-6 * max(1.0, abs(ref[k])), (k, o[k], ref[k])
    assert o["denat"] == 10 / 150
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_checkpoint_resume_is_bitwise(prec):
    """get_state at step 70 into a fresh context whose counter also stands at 70
    continues bit for bit like the uninterrupted run (counter-based noise)."""
    cfg = I.c1_linear(300)
    a = ctx_for(cfg, prec, seed=3)
    a.step(120)
    ref = a.get_state()
    b = ctx_for(cfg, prec, seed=3)
    b.step(70)
    s = b.get_state()
    c = ctx_for(cfg, prec, seed=3)
    c.step(70)
    c.set_state(-1, *s)
    c.step(50)
    got = c.get_state()
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    for h in (a, b, c):
        h.close()


@pytest.mark.parametrize("prec", PRECS)
def test_profiled_steps_follow_the_same_trajectory(prec):
    """dsdna_step_profiled queues the same kernels launch by launch: the
    state equals the graph-driven run bit for bit, and every launch is timed."""
    cfg = I.c1_linear(300)
    a = ctx_for(cfg, prec, seed=5)
    b = ctx_for(cfg, prec, seed=5)
    a.step(120)
    n0 = b.info()["engine_launches"]
    pr = b.step_profiled(120)
    assert pr["steps"] == 120 and b.step_counter == 120
    assert pr["engine_launches"] >= 1 and pr["engine_ms"] > 0.0
    assert pr["rebuild_launches"] >= 1 and pr["rebuild_ms"] > 0.0
    assert b.info()["engine_launches"] - n0 == pr["engine_launches"]
    assert a.info()["engine_launches"] >= pr["engine_launches"]
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    a.close(); b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_langevin_equipartition(prec):
    """App. A Eq. 8 thermostat: 3/2 kT translational and kT rotational (two axes
    normal to u) kinetic energy per nucleotide, averaged over a 200 bp run."""
    cfg = I.c1_linear(200)
    ctx = ctx_for(cfg, prec, seed=11)
    ctx.step(1000)
    kt, kr = [], []
    for _ in range(60):
        ctx.step(50)
        E, _ = ctx.energy_virial()
        kt.append(E[D.E_KIN_T] / cfg.n_nt)
        kr.append(E[D.E_KIN_R] / cfg.n_nt)
    ctx.close()
    assert abs(np.mean(kt) - 1.5) < 0.06, np.mean(kt)
    assert abs(np.mean(kr) - 1.0) < 0.05, np.mean(kr)


def test_broken_backbone_reports_efene_and_poisons():
    cfg = I.c1_linear(40)
    X = cfg.X.copy()
    X[2 * 20:, 2] += 0.5          # stretch one backbone bond past R0
    ctx = ctx_for(cfg, D.PREC_MIXED, X=X)
    with pytest.raises(D.DsdnaError) as e:
        ctx.compute_forces()
    assert e.value.status == "EFENE"
    with pytest.raises(D.DsdnaError) as e2:
        ctx.step(1)
    assert e2.value.status == "ESTATE"
    Xpm = ctx.get_state()[0]          # post-mortem read shows the broken bond
    assert np.abs(Xpm - X).max() < 1e-6
    ctx.set_state(-1, X=cfg.X, u=cfg.u)
    Fb, Fp = ctx.compute_forces()
    assert np.isfinite(Fb).all()
    ctx.close()


def test_neighbor_overflow_is_reported():
    cfg = dense_walk(600, seed=8)
    ctx = ctx_for(cfg, D.PREC_MIXED, max_neighbors=1)
    with pytest.raises(D.DsdnaError) as e:
        ctx.compute_forces()
    assert e.value.status == "EOVERFLOW"
    ctx.close()


def test_invalid_arguments_are_rejected():
    p = D.dsdna_default_params(block_threads=100)
    with pytest.raises(D.DsdnaError) as e:
        D.Context(p, [10])
    assert e.value.status == "EINVAL"
    p = D.dsdna_default_params(box=(10.0, 0.0, 10.0))
    with pytest.raises(D.DsdnaError):
        D.Context(p, [10])
    ctx = D.Context(D.dsdna_default_params(), [10])
    with pytest.raises(D.DsdnaError):
        ctx.set_external_force_torque(3, [0, 0, 1], [0, 0, 0])
    with pytest.raises(D.DsdnaError):
        ctx.step(-1)
    ctx.close()


def test_library_builds_default_helix_like_oracle():
    p = O.params(seed=21)
    ctx = D.Context(D.dsdna_default_params(seed=21, precision=D.PREC_FP64), [64, 9], tether=[1, 0])
    X, V, u, Om = ctx.get_state()
    Xo, uo = O.ideal_helix(p, 64)
    Vo, Omo = O.mb_velocities(p, 0, 64, uo, tether=1)
    assert np.allclose(X[:128], Xo, atol=1e-12) and np.allclose(u[:128], uo, atol=1e-12)
    assert np.allclose(V[:128], Vo, atol=1e-12) and np.allclose(Om[:128], Omo, atol=1e-12)
    Vo1, Omo1 = O.mb_velocities(p, 1, 9, O.ideal_helix(p, 9)[1])
    assert np.allclose(V[128:], Vo1, atol=1e-12)
    ctx.close()


@pytest.mark.parametrize("layout", ["walk", "rows"])
def test_c3_full_size_sampled_forces(layout):
    """The 1 Mbp confined helix (2e6 nucleotides) of the throughput benchmark
    (the self-avoiding walk; also the rows-and-U-turns layout), at its launch
    configuration, on a sample of nucleotides the oracle evaluates one by one."""
    cfg = c3_walk() if layout == "walk" else I.c3_confined()
    ctx = ctx_for(cfg, D.PREC_MIXED)
    Fb, Fp = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(cfg.n_nt, size=300, replace=False))
    ob, op, sb, sp = O.forces_sampled(oparams(cfg), cfg.n_bp, Xs, us, idx, with_scale=True)
    assert excess(Fb[idx], ob, sb, D.PREC_MIXED) < 1.0
    assert excess(Fp[idx], op, sp, D.PREC_MIXED) < 1.0
    ctx.step(20)
    ctx.synchronize()
    assert ctx.info()["rebuilds"] >= 1
    ctx.close()


def _open_pairs(X, bps, shift=0.5):
    """Move the strand-B nucleotide of each listed (global) base pair 0.5 nm
    radially off its partner: the pair's patches leave the 0.3 nm range."""
    X = X.copy()
    for k in bps:
        r = X[2 * k + 1, :2] - X[2 * k, :2]
        X[2 * k + 1, :2] += shift * r / np.linalg.norm(r)
    return X


@pytest.mark.parametrize("prec", PRECS)
def test_denaturation_rules_match_oracle(prec):
    """Sec. 5: bubble rule and A.T / G.C hydrogen-bond stiffness.  Two
    molecules (40 and 23 bp, 126 slots: four tiles and a ragged tail) with
    open runs of 4 (a bubble), 3 across the first tile boundary (a bubble),
    2 (not a bubble) and 2 + 2 on either side of the molecule boundary (not a
    bubble: pairs of another molecule count as closed)."""
    n_bp = [40, 23]
    rng = np.random.default_rng(12)
    X0, u0 = I.straight_helix(40)
    X1, u1 = I.straight_helix(23, origin=(8.0, 0.0, 0.0))
    X = np.concatenate([X0, X1]); u = np.concatenate([u0, u1])
    X, u = I.perturb(X, u, rng, dx=0.02, dtheta=0.05)
    opened = [5, 6, 7, 8, 15, 16, 17, 26, 27, 38, 39, 40, 41]
    X = _open_pairs(X, opened)
    gc = (np.arange(63) % 3 == 1).astype(np.int8)
    zero = np.zeros_like(X)
    kw = dict(R0=3.0, K2_gc=9.0)
    ctx = D.Context(D.dsdna_default_params(precision=prec, bubble_rule=1, **kw), n_bp, X=X, V=zero, u=u, Om=zero,
                    gc=gc)
    Fb, Fp = ctx.compute_forces()
    E, _ = ctx.energy_virial()
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    po = O.params(bubble_rule=1, gc=gc, **kw)
    r = O.forces(po, n_bp, Xs, us)
    Sb, Sp = O.force_scale(po, n_bp, Xs, us)
    eb, ep = excess(Fb, r["Fb"], Sb, prec), excess(Fp, r["Fp"], Sp, prec)
    assert eb < 1.0 and ep < 1.0, (eb, ep)
    Eo = r["energy"].sum(axis=0)[:8]
    tol = 1e-9 if prec == D.PREC_FP64 else 2e-5
    assert np.abs(E[:8] - Eo).max() < tol * np.abs(Eo).sum(), (E[:8], Eo)
    # the rule and the sequence change this configuration's energy
    Eoff = O.forces(O.params(**kw), n_bp, Xs, us)["energy"].sum(axis=0)
    assert Eoff[D.E_DIHEDRAL] - Eo[D.E_DIHEDRAL] > 1e-3 or Eo[D.E_DIHEDRAL] - Eoff[D.E_DIHEDRAL] > 1e-3
    assert abs(Eoff[D.E_HBOND] - Eo[D.E_HBOND]) > 1e-3


@pytest.mark.parametrize("prec", PRECS)
def test_profiles_sum_to_the_observables(prec):
    """dsdna_profiles: the twist increments add up to the oracle's twist and the
    centreline is the patch midpoint of each base pair (Sec. 3.1, App. B)."""
    cfg = dense_walk(300, seed=11)
    ctx = ctx_for(cfg, prec)
    cen, tw = ctx.profiles(0)
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    oo = O.observables(oparams(cfg), cfg.n_bp, Xs, us, mol=0)
    assert abs(tw.sum() - oo["tw"]) < 1e-9, (tw.sum(), oo["tw"])
    p = Xs + 0.25 * us
    assert np.abs(cen - 0.5 * (p[0::2] + p[1::2])).max() < 1e-6


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("list_build", [0, 1])
def test_open_box_list_with_shared_buckets_equals_brute_force(prec, list_build):
    """Open box: the hashed table of the cell walk (list_build 1) puts blocks
    of 8 x-cells in buckets; four overlapping 400 bp molecules occupy about
    500 blocks of 1024 buckets, so two of the 9 rows of a bead share a bucket
    for a few percent of the 3200 beads.  The chain-window build (list_build
    0) hashes (molecule, cell) of its segments instead, and the overlapping
    molecules share entries.  The list holds each pair once and exactly the
    brute-force set."""
    rng = np.random.default_rng(3)
    parts = [I.wlc_helix(400, 50.0, rng) for _ in range(4)]
    X = np.concatenate([q[0] for q in parts]); u = np.concatenate([q[1] for q in parts])
    n_bp = [400] * 4
    ctx = D.Context(D.dsdna_default_params(precision=prec, list_build=list_build), n_bp, X=X, u=u)
    assert ctx.info()["chain_list"] == (list_build == 0)
    pl = ctx.neighbor_pairs()
    got = {tuple(x) for x in pl}
    assert len(pl) == len(got), "a pair listed twice"
    skin = ctx.params.skin + 0.01
    lo = {tuple(x) for x in O.pairs(O.params(), n_bp, X, u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(O.params(), n_bp, X, u, extra=skin + 1e-4)}
    assert lo <= got <= hi and len(lo) > 1000
    assert ctx.info()["cell_table"] == 8192      # 2^13 entries = 1024 buckets for 3200 beads
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("list_build", [0, 1])
def test_open_box_list_across_hash_blocks_equals_brute_force(prec, list_build):
    """Open box, molecules spread over the hashed table's x-blocks of 8 cells:
    worm-like molecules with their origins at negative and positive x and y
    (some on block edges), one held along z through the origin (x-cells -1
    and 0, inside one block), one lying along x across many blocks.  The list
    holds each pair once and exactly the brute-force set."""
    rng = np.random.default_rng(11)
    Xs, us = [], []
    for k in range(5):
        X, u = I.wlc_helix(300, 40.0, rng, origin=(rng.uniform(-40.0, 40.0), rng.uniform(-40.0, 40.0), 0.0))
        Xs.append(X); us.append(u)
    X, u = I.straight_helix(300)
    Xs.append(X); us.append(u)
    R = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])   # a quarter turn about y: z -> x
    X, u = I.straight_helix(300, origin=(0.0, 0.0, -50.0))
    Xs.append(X @ R.T); us.append(u @ R.T)
    X = np.concatenate(Xs); u = np.concatenate(us)
    n_bp = [300] * 7
    ctx = D.Context(D.dsdna_default_params(precision=prec, list_build=list_build), n_bp, X=X, u=u)
    pl = ctx.neighbor_pairs()
    got = {tuple(x) for x in pl}
    assert len(pl) == len(got), "a pair listed twice"
    skin = ctx.params.skin + 0.01
    lo = {tuple(x) for x in O.pairs(O.params(), n_bp, X, u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(O.params(), n_bp, X, u, extra=skin + 1e-4)}
    assert lo <= got <= hi and len(lo) > 1000
    assert X[:, 0].min() < -20.0 and X[:, 0].max() > 20.0   # the molecules span many x-blocks
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("periodic", [False, True])
def test_rebuild_in_the_step_kernel_follows_the_same_trajectory(prec, periodic):
    """rebuild_mode 2 (list rebuilt inside the persistent step kernel) and 1
    (separate rebuild kernels) build the same sorted lists, so 400 steps with
    many rebuilds give bitwise the same state (open box: hashed table;
    periodic: linear table)."""
    if periodic:
        cfg = dense_walk(1200, seed=13)
        kw = dict(box=cfg.box)
    else:
        cfg = I.c4_batch(n_mol=6, lo=200, hi=600, seed=2)
        kw = {}
    out = []
    for mode in (1, 2):
        p = D.dsdna_default_params(precision=prec, rebuild_mode=mode, skin=0.1, seed=4, **kw)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether)
        ctx.step(400)
        info = ctx.info()
        assert info["rebuild_in_step"] == (mode == 2) and info["rebuilds"] > 10
        out.append(ctx.get_state())
        ctx.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
