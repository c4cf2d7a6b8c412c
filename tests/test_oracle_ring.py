"""Pins of the oracle's circular molecules (supercoiled rings, Sec. 6 and
Fig. 10): each strand's last nucleotide is bonded to its first, so every
bonded term of a linear chain also appears across the junction.

The pins use the linear-molecule oracle (pinned elsewhere) and closed forms:
cutting a ring at each of its N steps in turn and summing the linear
energies counts every step term N - 1 times and every bending term N - 2
times; a planar ring built with lk turns has linking number lk and no
writhe; relabelling a ring cyclically changes nothing."""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import inputs as I


def _shift(A, N, c):
    """Relabel base pairs k -> k - c (mod N): the new base pair 0 is the old c."""
    idx = np.concatenate([[2 * ((k + c) % N), 2 * ((k + c) % N) + 1] for k in range(N)])
    return A[idx]


def _ring(N, lk, seed=None, dx=0.02, dth=0.05):
    X, u = I.ring_helix(N, lk)
    if seed is not None:
        X, u = I.perturb(X, u, np.random.default_rng(seed), dx=dx, dtheta=dth)
    return X, u


def test_planar_ring_linking_twist_and_writhe():
    """App. C Eq. 17 on the closed strands: a planar ring wound lk times has
    Lk = lk (an integer), Tw = lk and Wr = 0 (planar axis)."""
    p = O.params(ring=[1])
    for N, lk in ((30, 3), (30, 2), (60, 4), (501, 47)):
        X, u = I.ring_helix(N, lk)
        ob = O.observables(p, N, X, u, with_lk=True)
        assert abs(ob["lk"] - lk) < 1e-9 and abs(ob["tw"] - lk) < 1e-9 and abs(ob["wr"]) < 1e-9, (N, lk, ob)
        assert abs(ob["tw_ideal"] - N / 10) < 1e-12


def test_planar_ring_bending_closed_form():
    """All patches lie on a regular N-gon: each of the 2N bending angles
    (every nucleotide of a ring has two neighbours) contributes
    K6 (1 - cos(2 pi / N)); the H-bonds all sit at their minimum -K2/2."""
    for N in (30, 61, 300):
        X, u = I.ring_helix(N, N // 10)
        p = O.params(ring=[1])
        E = O.forces(p, N, X, u)["energy"][0]
        assert abs(E[7] - 2 * N * p.K6 * (1 - np.cos(2 * np.pi / N))) < 1e-9 * E[7]
        assert abs(E[2] + 0.5 * p.K2 * N) < 1e-9 * N


@pytest.mark.parametrize("N,lk,seed", [(30, 3, 1), (33, 2, 2), (64, 6, 3)])
def test_ring_energy_equals_sum_over_cuts(N, lk, seed):
    """Cut the ring at step c (relabel so that c is the last base pair) for
    every c: each step term (FENE, its WCA, dihedral, Morse, planarity) is
    missing from exactly one cut and each bending term from two, the
    hydrogen bonds from none.  Sum over cuts / (N - 1), / (N - 2), / N."""
    X, u = _ring(N, lk, seed)
    Er = O.forces(O.params(ring=[1]), N, X, u)["energy"][0]
    S = np.zeros(O.NTERMS)
    for c in range(N):
        S += O.forces(O.params(), N, _shift(X, N, c), _shift(u, N, c))["energy"][0]
    for k, w in ((0, N - 1), (1, N - 1), (4, N - 1), (5, N - 1), (6, N - 1), (7, N - 2), (2, N)):
        assert abs(Er[k] - S[k] / w) < 1e-9 * max(1.0, abs(Er[k])), (k, Er[k], S[k] / w)


@pytest.mark.parametrize("N,lk,seed", [(30, 2, 11), (47, 4, 12)])
def test_ring_twist_equals_sum_over_cuts(N, lk, seed):
    """App. B on a ring: one frame per base-pair step (the last one closes
    the ring) and one twist increment per pair of consecutive frames.  A cut
    at step c drops that step's frame and so the two increments that touch
    it: summed over all N cuts every increment is counted N - 2 times."""
    X, u = _ring(N, lk, seed, dx=0.05, dth=0.1)
    tw = O.observables(O.params(ring=[1]), N, X, u)["tw"]
    S = sum(O.observables(O.params(), N, _shift(X, N, c + 1), _shift(u, N, c + 1))["tw"] for c in range(N))
    assert abs(tw - S / (N - 2)) < 1e-12 * N, (tw, S / (N - 2))
    assert abs(tw - lk) > 1e-4          # off the planar value: the identity is not trivial


@pytest.mark.parametrize("bubble_rule", [0, 1])
def test_ring_is_invariant_under_cyclic_relabelling(bubble_rule):
    """Shifting the labels by a multiple of 3 (N divisible by 3: the steric
    typing maps onto itself) permutes the forces and keeps every energy term,
    with an open run of four pairs across the junction (bubble rule on) or
    not."""
    N = 36
    X, u = _ring(N, 3, 5)
    for k in (34, 35, 0, 1):        # open run across the junction
        r = X[2 * k + 1] - X[2 * k]
        r[2] = 0.0
        X[2 * k + 1] += 0.5 * r / np.linalg.norm(r)
    p = O.params(ring=[1], R0=3.0, bubble_rule=bubble_rule)
    r0 = O.forces(p, N, X, u)
    for c in (3, 12, 33):
        rc = O.forces(p, N, _shift(X, N, c), _shift(u, N, c))
        assert np.allclose(rc["energy"][0], r0["energy"][0], rtol=1e-12, atol=1e-9)
        assert np.allclose(rc["Fb"], _shift(r0["Fb"], N, c), rtol=1e-10, atol=1e-9)
        assert np.allclose(rc["Fp"], _shift(r0["Fp"], N, c), rtol=1e-10, atol=1e-9)
    if bubble_rule:
        off = O.forces(O.params(ring=[1], R0=3.0), N, X, u)["energy"][0]
        assert off[4] != r0["energy"][0][4] and off[7] != r0["energy"][0][7]


def test_ring_forces_are_minus_energy_gradient_across_the_junction():
    N = 30
    X, u = _ring(N, 3, 7)
    p = O.params(ring=[1])
    r = O.forces(p, N, X, u)
    b, pt = O.sites(p, X, u)
    h = 1e-6
    for g in (0, 1, 2, 57, 58, 59):
        for site in (0, 1):
            for c in range(3):
                vals = []
                for sgn in (1, -1):
                    bb, pp = b.copy(), pt.copy()
                    (bb if site == 0 else pp)[g, c] += sgn * h
                    vals.append(O.forces(p, N, 0.5 * (bb + pp), (pp - bb) / p.ell)["energy"][0][:8].sum())
                fd = -(vals[0] - vals[1]) / (2 * h)
                an = (r["Fb"] if site == 0 else r["Fp"])[g, c]
                assert abs(an - fd) < 1e-6 * max(1.0, abs(fd)), (g, site, c, an, fd)


def test_ring_net_force_and_torque_vanish():
    N = 45
    X, u = _ring(N, 4, 9)
    r = O.forces(O.params(ring=[1]), N, X, u)
    F = r["F"]
    T = np.cross(X, F).sum(0) + r["T"].sum(0)
    assert np.abs(F.sum(0)).max() < 1e-9 and np.abs(T).max() < 1e-8


def test_ring_needs_six_base_pairs():
    X, u = I.ring_helix(6, 1)
    O.forces(O.params(ring=[1], R0=3.0), 6, X, u)     # a 6-gon stretches the outer backbone
    X, u = I.ring_helix(5, 1)
    with pytest.raises(O.OracleError, match="EINVAL"):
        O.forces(O.params(ring=[1], R0=3.0), 5, X, u)


def test_linking_number_is_conserved_by_langevin_dynamics():
    """Lk is topological: strands that never pass through each other keep
    it while twist and writhe exchange (a 60 bp ring wound 5 turns, i.e.
    Delta Lk = -1, over 400 steps at kT = 1)."""
    N = 60
    X, u = I.ring_helix(N, 5)
    p = O.params(ring=[1], seed=3)
    V, Om = I.maxwell(u, np.random.default_rng(4))
    X, u, V, Om = (np.ascontiguousarray(a) for a in (X, u, V, Om))
    tw0 = O.observables(p, N, X, u, with_lk=True)["tw"]
    O.run(p, N, X, V, u, Om, 400)
    ob = O.observables(p, N, X, u, with_lk=True)
    assert abs(ob["lk"] - 5) < 1e-6, ob
    assert abs(ob["tw"] + ob["wr"] - ob["lk"]) < 1e-9
    assert abs(ob["tw"] - tw0) > 1e-3      # the state moved


@pytest.mark.parametrize("N", [30, 31, 32, 33, 34, 35])
@pytest.mark.parametrize("phase", [0, 1, 2])
def test_ring_steric_beads_stay_three_apart(N, phase):
    """Sec. 2 steric typing on a ring: along each strand consecutive steric
    beads are 3 nucleotides apart, except one gap of 4 or 5 when N is not a
    multiple of 3 (read from the typed pair set: two beads of one strand
    interact only if both are steric)."""
    X, u = I.ring_helix(N, N // 10)
    p = O.params(ring=[1], steric_phase=phase)
    prs = O.pairs(p, N, X, u, extra=1e3)
    for s in (0, 1):
        st = sorted({int(g) for pr in prs if (pr[0] & 1) == s and (pr[1] & 1) == s for g in pr})
        q = np.sort([(g // 2) if s == 0 else N - 1 - g // 2 for g in st])
        gaps = np.diff(np.concatenate([q, [q[0] + N]]))
        assert gaps.min() >= 3 and (gaps > 3).sum() == (0 if N % 3 == 0 else 1), (s, gaps)
        assert q[0] == phase      # the pattern starts at the 5' end as on a linear strand
