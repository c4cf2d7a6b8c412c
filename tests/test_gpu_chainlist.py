"""Chain-window list build (list_build 0) against the cell walk (list_build 1)
and the brute-force pair search, in periodic and open boxes.

The chain-window build tests every bead pair of adjacent 16-slot segments
directly and finds the other pairs through a grid of segment bounding
spheres.  It must list the pairs of the brute-force search (up to pairs
within FP32 rounding of the list radius, which lie beyond every cutoff), so
forces, energies and trajectories equal those of the cell walk bit for bit
in both precisions (the FP64 path also checks the minimum-image shift of
every entry).  The split cases cut one walk into molecules of ragged
lengths: segments then span two molecules (they enter the segment grid bead
by bead) and 32-slot tiles hold beads of two molecules (their window pairs
take the per-pair minimum image)."""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PRECS = [D.PREC_MIXED, D.PREC_FP64]
SPLIT = np.array([397, 1203, 611, 789], np.int32)   # 3000 bp; molecule ends fall inside 16-slot segments


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


def _walk(n_bp, seed, split=False, phi=0.15):
    """Dense self-avoiding walk in a periodic box: contacts between distant
    stretches of the chain and across the box faces."""
    cfg = I.random_walk_helix(n_bp=n_bp, phi=phi, clearance=1.7, seed=seed)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, np.random.default_rng(seed), dx=0.01, dtheta=0.02)
    if split:
        assert SPLIT.sum() == n_bp
        cfg.n_bp = SPLIT.copy()
    return cfg


def _ctx(cfg, prec, list_build, **kw):
    p = D.dsdna_default_params(precision=prec, box=cfg.box, list_build=list_build, **kw)
    return D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("split", [False, True])
def test_chain_list_pairs_equal_brute_force_and_cell_walk(prec, split):
    cfg = _walk(3000, 21, split)
    got = {}
    for lb in (0, 1):
        ctx = _ctx(cfg, prec, lb)
        assert ctx.info()["chain_list"] == (1 if lb == 0 else 0)
        got[lb] = {tuple(x) for x in ctx.neighbor_pairs()}
        skin = ctx.params.skin + 0.01   # the list radius carries a 0.01 margin over the skin
        ctx.close()
    po = O.params(box=cfg.box)
    lo = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin + 1e-4)}
    for lb in (0, 1):
        assert lo <= got[lb] <= hi, lb
    assert len(lo) > 2000
    # contacts between stretches of the chain more than three segments apart,
    # the pairs the segment grid has to find (138 unsplit, 48 between parts of
    # one molecule when split)
    assert sum(1 for i, j in lo if abs(j - i) > 48) > 40


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("split", [False, True])
def test_chain_list_forces_and_trajectory_equal_the_cell_walk(prec, split):
    """Forces on the initial state, then 300 steps with a list rebuilt every
    few steps (skin 0.1): bitwise the same with either build.  Energies and
    virial are sums of FP64 atomic additions, whose order varies from run to
    run: equal to 1e-12 of the sum of the magnitudes."""
    cfg = _walk(3000, 13, split)
    out, ew = [], []
    for lb in (0, 1):
        ctx = _ctx(cfg, prec, lb, rebuild_mode=1, skin=0.1, seed=4)
        Fb, Fp = ctx.compute_forces()
        ew.append(ctx.energy_virial())
        ctx.step(300)
        info = ctx.info()
        assert info["rebuilds"] > 10 and info["chain_list"] == (lb == 0)
        out.append([Fb, Fp, *ctx.get_state()])
        ctx.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    for a, b in zip(ew[0], ew[1]):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).sum()


@pytest.mark.parametrize("prec", PRECS)
def test_chain_list_forces_match_oracle_on_split_molecules(prec):
    """Four molecules cut from one dense walk never interact with each other."""
    cfg = _walk(3000, 8, True)
    ctx = _ctx(cfg, prec, 0)
    Fb, Fp = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    po = O.params(box=cfg.box)
    r = O.forces(po, cfg.n_bp, Xs, us)
    Sb, Sp = O.force_scale(po, cfg.n_bp, Xs, us)
    rel, ab = (1e-5, 5e-4) if prec == D.PREC_MIXED else (1e-9, 1e-10)
    for F, Fo, S in ((Fb, r["Fb"], Sb), (Fp, r["Fp"], Sp)):
        assert (np.linalg.norm(F - Fo, axis=1) <= rel * S + ab).all()


def test_chain_list_sparse_box_with_halving():
    """A sparse walk (volume fraction 0.05, 20 kbp, the density of the 1 Mbp
    workload) in mixed precision with pair halving: every tile takes the
    unwrapped window, the lists equal the cell walk's, and 200 steps agree bit
    for bit."""
    cfg = I.random_walk_helix(n_bp=20000, phi=0.05, seed=3)
    out, pairs = [], []
    for lb in (0, 1):
        ctx = _ctx(cfg, D.PREC_MIXED, lb, rebuild_mode=1, skin=0.2, seed=9)
        pairs.append({tuple(x) for x in ctx.neighbor_pairs()})
        ctx.step(200)
        info = ctx.info()
        assert info["rebuilds"] > 5 and info["halved_tiles"] > 0.9 * (info["n_nt"] + 31) // 32
        out.append(ctx.get_state())
        ctx.close()
    d = pairs[0] ^ pairs[1]
    assert len(d) <= 2, d     # at most a pair within FP32 rounding of the list radius
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("pose", ["overlapping", "random"])
def test_chain_list_open_box_batch_equals_the_cell_walk(prec, pose):
    """Open box, a batch of molecules (hashed segment grid): held along z from
    the origin, so that they overlap in space and share hash entries, or in
    random orientations and places.  Pairs equal to brute force; forces and
    300 steps with a list rebuilt every few steps bitwise equal to the cell
    walk's."""
    cfg = I.c4_batch(n_mol=8, lo=150, hi=700, seed=6, random_pose=(pose == "random"))
    out, got = [], []
    for lb in (0, 1):
        p = D.dsdna_default_params(precision=prec, list_build=lb, rebuild_mode=1, skin=0.1, seed=5)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om, tether=cfg.tether)
        for m in range(len(cfg.n_bp)):
            ctx.set_external_force_torque(m, cfg.ext_f[m], cfg.ext_t[m])
        assert ctx.info()["chain_list"] == (lb == 0)
        got.append({tuple(x) for x in ctx.neighbor_pairs()})
        Fb, Fp = ctx.compute_forces()
        ctx.step(300)
        assert ctx.info()["rebuilds"] >= 4    # 5 or 6 builds in the first 300 steps
        out.append([Fb, Fp, *ctx.get_state()])
        skin = ctx.params.skin + 0.01
        ctx.close()
    po = O.params()
    lo = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin + 1e-4)}
    for g in got:
        assert lo <= g <= hi
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("periodic", [True, False])
def test_chain_list_tiny_and_ragged_molecules(prec, periodic):
    """Molecules of 1 to 33 base pairs (segments and tiles cut anywhere,
    single-nucleotide strands) in a 20 nm periodic box, just wide enough for 3
    grid cells per edge, or in an open box: pairs equal to brute force, forces
    bitwise equal to the cell walk."""
    cfg = I.ragged_batch([1, 2, 7, 9, 17, 33], seed=4, spread=0.02)
    box = (20.0, 20.0, 20.0) if periodic else None
    out, got = [], []
    for lb in (0, 1):
        kw = dict(box=box) if periodic else {}
        p = D.dsdna_default_params(precision=prec, list_build=lb, **kw)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
        assert ctx.info()["chain_list"] == (lb == 0)
        got.append({tuple(x) for x in ctx.neighbor_pairs()})
        out.append(ctx.compute_forces())
        skin = ctx.params.skin + 0.01
        ctx.close()
    po = O.params(box=box) if periodic else O.params()
    lo = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(po, cfg.n_bp, cfg.X, cfg.u, extra=skin + 1e-4)}
    for g in got:
        assert lo <= g <= hi
    assert len(lo) > 50
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("periodic", [True, False])
def test_chain_list_with_every_segment_wide(periodic):
    """Strand B of a walk moved 4 nm away from strand A: every 16-slot segment
    is wider than the grid's limit, so every bead enters the segment grid
    alone and queries it alone.  The list still equals brute force.  (The
    forces of this configuration stay finite: largest bead force 6e5 kT/nm.)"""
    cfg = I.random_walk_helix(n_bp=1500, phi=0.02, clearance=1.7, seed=18)
    X = cfg.X.copy()
    X[1::2] += np.array([4.0, 0.0, 0.0])      # odd slots: strand B
    box = cfg.box if periodic else None
    got = []
    for lb in (0, 1):
        kw = dict(box=box) if periodic else {}
        p = D.dsdna_default_params(list_build=lb, **kw)
        ctx = D.Context(p, cfg.n_bp, X=X, V=cfg.V, u=cfg.u, Om=cfg.Om)
        assert ctx.info()["chain_list"] == (lb == 0)
        got.append({tuple(x) for x in ctx.neighbor_pairs()})
        skin = ctx.params.skin + 0.01
        ctx.close()
    po = O.params(box=box) if periodic else O.params()
    lo = {tuple(x) for x in O.pairs(po, cfg.n_bp, X, cfg.u, extra=skin - 1e-4)}
    hi = {tuple(x) for x in O.pairs(po, cfg.n_bp, X, cfg.u, extra=skin + 1e-4)}
    for g in got:
        assert lo <= g <= hi
    assert len(lo) > 800
