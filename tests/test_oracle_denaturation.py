"""Pins of the Sec. 5 denaturation rules in the oracle: sequence-dependent
hydrogen-bond stiffness K2(AT) < K2(CG), and no dihedral or bending term
inside bubbles of more than two open base pairs."""
import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import inputs as I


def _E(p, N, X, u):
    return O.forces(p, N, X, u)["energy"][0]


def _perturbed(N, seed):
    X, u = I.straight_helix(N)
    return I.perturb(X, u, np.random.default_rng(seed), dx=0.03, dtheta=0.08)


def _open(X, bps, shift=0.5):
    """Move the strand-B nucleotide of each listed base pair 0.5 nm off its
    partner (radially): its patch leaves the 0.3 nm hydrogen-bond range."""
    X = X.copy()
    for k in bps:
        r = X[2 * k + 1, :2] - X[2 * k, :2]
        r /= np.linalg.norm(r)
        X[2 * k + 1, :2] += shift * r
    return X


def test_hbond_depth_per_pair_type():
    """Ideal helix: paired patches coincide (r = r0 = 0), so every bond sits at
    its depth -K2/2 with its own K2."""
    p0 = O.params()
    N = 12
    X, u = O.ideal_helix(p0, N)
    gc = np.array([1, 0, 1, 1, 0, 0, 1, 0, 0, 1, 1, 0], np.int8)
    p = O.params(gc=gc, K2_gc=9.0)
    E = _E(p, N, X, u)
    want = -0.5 * (9.0 * gc.sum() + p0.K2 * (N - gc.sum()))
    assert abs(E[2] - want) < 1e-12
    assert abs(_E(p0, N, X, u)[2] + 0.5 * p0.K2 * N) < 1e-12       # no sequence: uniform K2


def test_fully_open_molecule_has_no_dihedral_or_bending():
    """Strand B moved rigidly 3 nm away: every base pair is open, so with the
    rule on no dihedral or bending term is left; the other terms are unchanged."""
    N = 10
    X, u = _perturbed(N, 1)
    X[1::2, 0] += 3.0
    off = _E(O.params(), N, X, u)
    on = _E(O.params(bubble_rule=1), N, X, u)
    assert off[4] > 1e-3 and off[7] > 1e-6
    assert on[4] == 0.0 and on[7] == 0.0
    for k in (0, 1, 2, 3, 5, 6):
        assert on[k] == off[k]


def test_two_open_base_pairs_are_not_a_bubble():
    N = 12
    X, u = _perturbed(N, 2)
    X = _open(X, [5, 6])
    p = O.params(R0=3.0)
    assert np.array_equal(_E(O.params(R0=3.0, bubble_rule=1), N, X, u), _E(p, N, X, u))


@pytest.mark.parametrize("bubble", [(4, 5, 6), (3, 4, 5, 6), (0, 1, 2), (9, 10, 11)])
def test_bubble_removes_exactly_its_inner_terms(bubble):
    """The terms the rule removes are those whose nucleotides all lie in the
    bubble: the dihedral and bending energy of a molecule made of the
    bubble's base pairs alone."""
    N = 12
    X, u = _perturbed(N, 3)
    X = _open(X, bubble)
    p_off, p_on = O.params(R0=3.0), O.params(R0=3.0, bubble_rule=1)
    off, on = _E(p_off, N, X, u), _E(p_on, N, X, u)
    s = slice(2 * bubble[0], 2 * (bubble[-1] + 1))
    inner = _E(p_off, len(bubble), X[s], u[s])
    assert abs((off[4] - on[4]) - inner[4]) < 1e-12 and inner[4] > 0.0
    assert abs((off[7] - on[7]) - inner[7]) < 1e-12
    for k in (0, 1, 2, 3, 5, 6):
        assert on[k] == off[k]


def test_forces_with_bubble_and_sequence_are_minus_energy_gradient():
    """Away from the switching distance the masked energy is smooth: the
    oracle's site forces equal central differences of its energy."""
    N = 12
    X, u = _perturbed(N, 4)
    X = _open(X, [3, 4, 5, 6])
    gc = (np.arange(N) % 3 == 0).astype(np.int8)
    p = O.params(R0=3.0, bubble_rule=1, gc=gc, K2_gc=8.0)
    r = O.forces(p, N, X, u)
    b, pt = O.sites(p, X, u)
    h = 1e-6
    for g in (5, 6, 8, 9, 12, 13, 18):
        for site in (0, 1):
            for c in range(3):
                vals = []
                for sgn in (1, -1):
                    bb, pp = b.copy(), pt.copy()
                    (bb if site == 0 else pp)[g, c] += sgn * h
                    vals.append(_E(p, N, 0.5 * (bb + pp), (pp - bb) / p.ell)[:8].sum())
                fd = -(vals[0] - vals[1]) / (2 * h)
                an = (r["Fb"] if site == 0 else r["Fp"])[g, c]
                assert abs(an - fd) < 1e-6 * max(1.0, abs(fd)), (g, site, c, an, fd)


def _inner_mask(N, a, b):
    """Removed-term mask of a bubble over base pairs a..b (bits: 1 dihedral of
    the step to the next nucleotide, 2 bending centred on the nucleotide)."""
    m = np.zeros(2 * N, np.uint8)
    for k in range(a, b):
        m[2 * k] |= 1            # strand A step k -> k + 1
        m[2 * (k + 1) + 1] |= 1  # strand B step k + 1 -> k
    for k in range(a + 1, b):
        m[2 * k] |= 2
        m[2 * k + 1] |= 2
    return m


@pytest.mark.parametrize("bubble", [(4, 5, 6), (0, 1, 2, 3), (8, 9, 10, 11)])
def test_permanent_rule_equals_while_rule_without_history(bubble):
    """Rule 2 with an empty mask evaluates exactly what rule 1 does."""
    N = 12
    X, u = _perturbed(N, 3)
    X = _open(X, bubble)
    r1 = O.forces(O.params(R0=3.0, bubble_rule=1), N, X, u)
    r2 = O.forces(O.params(R0=3.0, bubble_rule=2), N, X, u)
    for k in ("Fb", "Fp", "energy"):
        assert np.array_equal(r1[k], r2[k])


def test_mask_removes_exactly_the_marked_terms_of_a_closed_molecule():
    """A closed duplex with the mask of a former bubble over pairs 3..6: its
    energy lacks the dihedral and bending energy of a molecule made of those
    pairs alone; the forces are minus the gradient of that energy."""
    N = 12
    X, u = _perturbed(N, 8)
    mask = _inner_mask(N, 3, 6)
    p = O.params(bubble_rule=2, removed=mask)
    on, off = _E(p, N, X, u), _E(O.params(), N, X, u)
    inner = _E(O.params(), 4, X[6:14], u[6:14])
    assert abs((off[4] - on[4]) - inner[4]) < 1e-12 and inner[4] > 0.0
    assert abs((off[7] - on[7]) - inner[7]) < 1e-12
    assert _E(O.params(bubble_rule=1, removed=mask), N, X, u)[4] == off[4]   # rule 1 ignores the mask
    r = O.forces(p, N, X, u)
    b, pt = O.sites(p, X, u)
    h = 1e-6
    for g in (6, 9, 13):
        for c in range(3):
            vals = []
            for sgn in (1, -1):
                pp = pt.copy()
                pp[g, c] += sgn * h
                vals.append(_E(p, N, 0.5 * (b + pp), (pp - b) / p.ell)[:8].sum())
            assert abs(r["Fp"][g, c] + (vals[0] - vals[1]) / (2 * h)) < 1e-6 * max(1.0, abs(r["Fp"][g, c]))


def test_run_records_bubbles_and_keeps_them_removed():
    """One step from a configuration with a bubble over pairs 3..6 records
    exactly that bubble's inner terms; after the bubble closes again (the
    original duplex) another step keeps them removed."""
    N = 12
    X0, u0 = _perturbed(N, 9)
    X = _open(X0, [3, 4, 5, 6])
    mask = np.zeros(2 * N, np.uint8)
    p = O.params(R0=3.0, bubble_rule=2, removed=mask, noise=0, dt=1e-6)
    V = np.zeros_like(X); Om = np.zeros_like(X)
    Xr, ur = X.copy(), u0.copy()
    O.run(p, N, Xr, V.copy(), ur, Om.copy(), 1)
    assert np.array_equal(mask, _inner_mask(N, 3, 6))
    Xc, uc = X0.copy(), u0.copy()
    O.run(p, N, Xc, V.copy(), uc, Om.copy(), 1)
    assert np.array_equal(mask, _inner_mask(N, 3, 6))
    free = np.zeros(2 * N, np.uint8)
    O.run(O.params(R0=3.0, bubble_rule=2, removed=free, noise=0, dt=1e-6), N, X0.copy(), V.copy(), u0.copy(),
          Om.copy(), 1)
    assert not free.any()
