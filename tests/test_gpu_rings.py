"""GPU parity of circular molecules (supercoiled rings, Sec. 6 / Fig. 10) and
of the permanent bubble rule (Sec. 5, rule 2) against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PRECS = [D.PREC_MIXED, D.PREC_FP64]
TOL = {D.PREC_MIXED: (1e-5, 5e-4), D.PREC_FP64: (1e-9, 1e-10)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


def excess(Fg, Fo, S, prec):
    rel, ab = TOL[prec]
    return (np.linalg.norm(Fg - Fo, axis=1) / (rel * S + ab)).max()


def _open_pairs(X, bps, shift=0.5):
    """Move the strand-B nucleotide of each listed base pair 0.5 nm further
    from its partner along their centre line (outwards from the axis)."""
    X = X.copy()
    for k in bps:
        r = X[2 * k + 1] - X[2 * k]
        X[2 * k + 1] += shift * r / np.linalg.norm(r)
    return X


def _mixed_system(seed=3):
    """Ring of 36 bp, linear 40 bp, ring of 100 bp (200 slots: several tiles),
    ring of 6 bp (the smallest): 364 slots with ragged tails."""
    rng = np.random.default_rng(seed)
    parts = [I.ring_helix(36, 3, center=(0, 0, 0)), I.straight_helix(40, origin=(20, 0, 0)),
             I.ring_helix(100, 9, center=(0, 30, 0)), I.ring_helix(6, 1, center=(30, 30, 0))]
    X = np.concatenate([p[0] for p in parts]); u = np.concatenate([p[1] for p in parts])
    X, u = I.perturb(X, u, rng, dx=0.02, dtheta=0.05)
    return [36, 40, 100, 6], [1, 0, 1, 1], X, u


def _check_static(prec, n_bp, ring, X, u, mask=None, **kw):
    zero = np.zeros_like(X)
    ctx = D.Context(D.dsdna_default_params(precision=prec, **kw), n_bp, X=X, V=zero, u=u, Om=zero, circular=ring)
    if mask is not None:
        ctx.set_bubble_mask(mask)
    Fb, Fp = ctx.compute_forces()
    E, _ = ctx.energy_virial()
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    po = O.params(ring=np.array(ring, np.int8), removed=mask, **kw)
    r = O.forces(po, n_bp, Xs, us)
    Sb, Sp = O.force_scale(po, n_bp, Xs, us)
    eb, ep = excess(Fb, r["Fb"], Sb, prec), excess(Fp, r["Fp"], Sp, prec)
    assert eb < 1.0 and ep < 1.0, (eb, ep)
    Eo = r["energy"].sum(axis=0)[:8]
    tol = 1e-9 if prec == D.PREC_FP64 else 2e-5
    assert np.abs(E[:8] - Eo).max() < tol * np.abs(Eo).sum(), (E[:8], Eo)
    return r


@pytest.mark.parametrize("prec", PRECS)
def test_ring_forces_and_energy_match_oracle(prec):
    n_bp, ring, X, u = _mixed_system()
    r = _check_static(prec, n_bp, ring, X, u, R0=3.0)
    # the closing terms matter: the same coordinates as linear molecules differ
    lin = O.forces(O.params(R0=3.0), n_bp, X, u)["energy"].sum(axis=0)
    assert abs(lin[7] - r["energy"].sum(axis=0)[7]) > 1.0


@pytest.mark.parametrize("prec", PRECS)
def test_ring_bubble_across_the_junction_with_a_mask(prec):
    """Rule 2 on rings: an open run of four pairs across the 36 bp ring's
    junction and one inside the 100 bp ring, plus a removed-term mask from an
    earlier bubble on the linear molecule."""
    n_bp, ring, X, u = _mixed_system(4)
    X = _open_pairs(X, [34, 35, 0, 1, 36 + 40 + 50, 36 + 40 + 51, 36 + 40 + 52])
    mask = np.zeros(X.shape[0], np.uint8)
    for k in range(36 + 10, 36 + 14):
        mask[2 * k] |= 1
        mask[2 * (k + 1) + 1] |= 1
    mask[2 * (36 + 12)] |= 2
    mask[2 * (36 + 12) + 1] |= 2
    r = _check_static(prec, n_bp, ring, X, u, mask=mask, R0=3.0, bubble_rule=2)
    off = O.forces(O.params(ring=np.array(ring, np.int8), R0=3.0), n_bp, X, u)["energy"].sum(axis=0)
    assert off[4] - r["energy"].sum(axis=0)[4] > 1e-3


@pytest.mark.parametrize("prec", PRECS)
def test_ring_observables_match_oracle(prec):
    n_bp, ring, X, u = _mixed_system(5)
    zero = np.zeros_like(X)
    ctx = D.Context(D.dsdna_default_params(precision=prec, R0=3.0), n_bp, X=X, V=zero, u=u, Om=zero, circular=ring)
    Xs, _, us, _ = ctx.get_state()
    po = O.params(ring=np.array(ring, np.int8), R0=3.0)
    for m in range(len(n_bp)):
        ob = ctx.observables(m, flags=D.OBS_EXT | D.OBS_DENAT | D.OBS_TW | D.OBS_LK)
        oo = O.observables(po, n_bp, Xs, us, mol=m, with_lk=True)
        for k in ("tw", "tw_ideal", "lk", "wr", "denat"):
            assert abs(ob[k] - oo[k]) < 1e-6, (m, k, ob[k], oo[k])
    assert abs(ctx.observables(2, flags=D.OBS_LK)["lk"] - 9) < 1e-6
    ctx.close()


def test_fp64_ring_trajectory_with_permanent_bubbles_matches_oracle():
    """FP64 engine and oracle, same Philox noise, 150 steps of a 36 bp ring
    and a 30 bp linear molecule at K2 = 1 kT with rule 2: positions agree and
    the removed-term masks are identical."""
    n_bp = [36, 30]
    X0, u0 = I.ring_helix(36, 3)
    X1, u1 = I.straight_helix(30, origin=(20, 0, 0))
    X = np.concatenate([X0, X1]); u = np.concatenate([u0, u1])
    X = _open_pairs(X, [34, 35, 0, 1, 36 + 10, 36 + 11, 36 + 12])
    ring = [1, 0]
    kw = dict(K2=1.0, bubble_rule=2, seed=9, R0=3.0)
    p = D.dsdna_default_params(precision=D.PREC_FP64, **kw)
    ctx = D.Context(p, n_bp, X=X, u=u, circular=ring)
    Xg, Vg, ug, Og = ctx.get_state()
    ctx.step(150)
    Xe, _, ue, _ = ctx.get_state()
    me = ctx.get_bubble_mask()
    ctx.close()
    mask = np.zeros(X.shape[0], np.uint8)
    po = O.params(ring=np.array(ring, np.int8), removed=mask, **kw)
    Xo, Vo, uo, Oo = (np.ascontiguousarray(a).copy() for a in (Xg, Vg, ug, Og))
    O.run(po, n_bp, Xo, Vo, uo, Oo, 150)
    assert np.abs(Xe - Xo).max() < 1e-9 and np.abs(ue - uo).max() < 1e-9
    assert np.array_equal(me, mask) and mask.any()


def test_ring_linking_number_is_conserved_in_mixed_precision():
    """Fig. 10 setting: a 500 bp ring wound 47 turns (Delta Lk = -3, sigma =
    -0.06) keeps Lk = 47 exactly over 20000 steps while twist turns into
    writhe."""
    N, lk = 500, 47
    X, u = I.ring_helix(N, lk)
    ctx = D.Context(D.dsdna_default_params(seed=2), [N], X=X, u=u, circular=[1])
    o0 = ctx.observables(0, flags=D.OBS_TW | D.OBS_LK)
    ctx.step(20000)
    o1 = ctx.observables(0, flags=D.OBS_TW | D.OBS_LK)
    ctx.close()
    assert abs(o0["lk"] - lk) < 1e-6 and abs(o1["lk"] - lk) < 1e-3, (o0, o1)
    assert abs(o1["tw"] + o1["wr"] - o1["lk"]) < 1e-9
    assert abs(o1["wr"]) > 1e-3


def test_permanent_rule_melts_low_k2_without_breaking():
    """Sec. 5 at K2 = 1 kT, rule 2: a 100 bp molecule denatures (most pairs
    open) within 20000 steps, with no broken backbone; at the Table 1 K2 = 6
    it stays paired."""
    out = {}
    for K2 in (1.0, 6.0):
        ctx = D.Context(D.dsdna_default_params(K2=K2, bubble_rule=2, seed=4), [100])
        ctx.step(20000)
        out[K2] = ctx.observables(0, flags=D.OBS_DENAT)["denat"]
        ctx.close()
    assert out[1.0] > 0.6 and out[6.0] < 0.1, out


def test_persistence_lengths_match_the_paper():
    """Sec. 3.1-3.2 through the GPU profiles: 128 chains of 300 bp, 2.5e5 steps;
    the tangent correlator over its first 20 bp decays with the paper's
    l_p = 143 +- 7 bp (within 35 bp: short equilibration; 148 bp after 2e6
    steps on 512 chains) and the residual twist with the paper's
    l_tau = 512 +- 18 bp (within 430-620 bp here; 509 +- 2 bp in the long
    run), at a mean twist near 35.0 deg per base pair."""
    from paper_1608_03722_gb300 import persistence as P
    r = P.measure(n_mol=128, n_bp=300, equil=200_000, every=5_000, samples=10, seed=7, groups=4)
    assert abs(r["l_p_short_bp"] - 143.0) < 35.0, r
    assert 430.0 < r["l_tau_mean_twist_bp"] < 620.0, r
    assert 34.5 < r["twist_per_bp_deg"] < 35.5, r
