"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Nothing here retypes an oracle formula: each test checks the oracle against
printed values (tests/golden/), special points of the potentials the paper
states, finite differences of the oracle's own energy, symmetry invariants,
brute force, or textbook statistical mechanics.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import inputs as I
from tests.conftest import read_golden


def test_philox_known_answers():
    for name, line in read_golden("philox_kat.txt").items():
        lhs, rhs = line.split("->")
        w = [int(x, 16) for x in lhs.split()]
        want = [int(x, 16) for x in rhs.split()]
        assert O.philox4x32_10(w[:4], w[4:6]) == want, name


def _angle(a, b):
    return math.degrees(math.acos(np.clip(a @ b / np.linalg.norm(a) / np.linalg.norm(b), -1, 1)))


def _dihedral(A, E, F, B):
    b1, b2, b3 = E - A, F - E, B - F
    n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
    return math.degrees(math.atan2(np.linalg.norm(b2) * (b1 @ n2), n1 @ n2))


def test_ideal_helix_geometry_matches_paper():
    g = read_golden("helix_geometry.txt")
    p = O.params()
    N = 40
    X, u = O.ideal_helix(p, N)
    b, pt = O.sites(p, X, u)
    A = b[0::2]; PA = pt[0::2]; B = b[1::2]; PB = pt[1::2]
    assert np.allclose(np.linalg.norm(PA[1:] - PA[:-1], axis=1), float(g["patch_rise"]), atol=1e-12)
    assert np.allclose(np.linalg.norm(A[1:] - A[:-1], axis=1), float(g["bead_spacing"]), atol=0.005)
    assert np.allclose(np.linalg.norm(b - pt, axis=1), float(g["bead_patch"]), atol=1e-12)
    # phosphates sit 0.5 nm beyond the bead, away from the patch (Fig. 1a/b)
    ph = b - 0.5 * u
    assert np.allclose(np.linalg.norm(ph[2::2] - ph[0:-2:2], axis=1), float(g["phosphate_spacing"]), atol=0.01)
    radial = np.linalg.norm(b[:, :2], axis=1).max() + 0.5  # bead radius 0.5 (unit diameter, Sec. 2)
    assert abs(2 * radial - float(g["thickness"])) < 1e-9
    assert np.allclose(PA, PB, atol=1e-12)                                   # H-bond at r0 = 0
    for k in range(N - 1):                                                   # strand A, 5'->3'
        assert abs(_dihedral(A[k], PA[k], PA[k + 1], A[k + 1]) - float(g["dihedral_min_deg"])) < 1e-9
        assert abs(_angle(PA[k] - PA[k + 1], A[k + 1] - PA[k + 1]) - float(g["planarity_deg"])) < 1e-9
    for k in range(N - 1, 0, -1):                                            # strand B runs 5'->3' downwards
        assert abs(_dihedral(B[k], PB[k], PB[k - 1], B[k - 1]) - float(g["dihedral_min_deg"])) < 1e-9
    # pitch: bead of A_k and A_{k+10} share the same azimuth
    pitch = int(g["pitch_bp"])
    assert np.allclose(A[pitch:, :2], A[:-pitch, :2], atol=1e-12)


def test_generator_helix_equals_oracle_helix():
    p = O.params()
    X0, u0 = O.ideal_helix(p, 57)
    X1, u1 = I.straight_helix(57)
    assert np.allclose(X0, X1, atol=1e-12) and np.allclose(u0, u1, atol=1e-12)


def _E(p, N, X, u, **kw):
    return O.forces(p, N, X, u, **kw)["energy"][0]


def test_ideal_helix_is_stationary_except_backbone():
    """Every bonded term sits at its minimum in the relaxed helix except FENE+WCA
    (rest length 0.4594 vs the FENE+WCA minimum near 0.46).  Steric beads of
    opposite strands within 2 bp sit 1.00-1.06 nm apart: no steric energy when
    such pairs take the ghost size 0.5, some under reading A1 (size 1), which
    unwinds the relaxed helix slightly."""
    g = read_golden("helix_geometry.txt")
    p = O.params()
    N = 30
    X, u = O.ideal_helix(p, N)
    E = _E(p, N, X, u)
    names = dict(zip(O.TERM_NAMES, E))
    assert abs(names["dihedral"]) < 1e-10 and abs(names["planar"]) < 1e-10
    assert abs(names["bend"]) < 1e-10 and abs(names["morse"]) < 1e-10
    assert abs(names["hbond"] + N * float(g["hbond_depth"])) < 1e-10
    assert names["wca"] > 1.0
    E0 = dict(zip(O.TERM_NAMES, _E(O.params(sigma_cross_steric=0.0), N, X, u)))
    assert abs(E0["wca"]) < 1e-12


def test_special_points_of_each_potential():
    p = O.params()
    # H-bond (App. A Eq. 10): depth K2/2 at r0, zero at rc and beyond (bond broken)
    X, u = O.ideal_helix(p, 1)
    for r, want in ((0.0, -p.K2 / 2), (p.rc_hb, 0.0), (p.rc_hb * 1.01, 0.0), (0.7, 0.0)):
        X2 = X.copy(); X2[1, 2] += r
        assert abs(_E(p, 1, X2, u)[2] - want) < 1e-12
    # WCA (App. A Eq. 11): zero and force-free at 2^(1/6) sigma, equal to eps at
    # sigma.  The two nucleotides of a 1 bp molecule are both steric (each is
    # the first of its strand): sigma = 1 under reading A1, sigma_cross = 0.5
    # when steric pairs across strands take the ghost size.
    for pp, sig in ((p, p.sigma_ss), (O.params(sigma_cross_steric=0.0), p.sigma_cross)):
        for r, want in ((2 ** (1 / 6) * sig, 0.0), (sig, pp.eps_ev), (2 ** (1 / 6) * sig * 1.001, 0.0)):
            u2 = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
            beads = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
            X2 = beads + 0.5 * pp.ell * u2
            assert abs(_E(pp, 1, X2, u2)[3] - want) < 1e-12, (sig, r)
    # Morse (App. A Eq. 13): zero at r0, tends to K4 when far
    for rise, want in ((p.r0_m, 0.0),):
        X, u = I.straight_helix(3)
        X[:, 2] *= rise / I.RISE
        assert abs(_E(p, 3, X, u)[5] - want) < 1e-12
    for rise in (0.30, 0.38):
        X, u = I.straight_helix(3)
        X[:, 2] *= rise / I.RISE
        assert _E(p, 3, X, u)[5] > 0.0
    # FENE (App. A Eq. 9): infinite at R0 -> error
    X, u = I.straight_helix(2)
    b, _ = O.sites(p, X, u)
    X[2:, 2] += 0.7
    with pytest.raises(O.OracleError):
        O.forces(p, 2, X, u)


def test_fene_wca_minimum_near_bond_length():
    """Sec. 2: consecutive beads are joined by FENE bonds of length d_bp = 0.46 nm;
    FENE + backbone WCA (Table 1) must have its minimum there."""
    p = O.params()
    rs = np.linspace(0.44, 0.48, 4001)
    Es = []
    X, u = I.straight_helix(2)
    for r in rs:
        X2 = np.zeros_like(X); u2 = np.zeros_like(u)
        u2[:] = (0, 0, 1)
        X2[0] = (0, 0, 0); X2[2] = (r, 0, 0)          # strand A beads r apart
        X2[1] = (0, 0, 50); X2[3] = (r, 0, 50)        # strand B far away
        E = _E(p, 2, X2, u2)
        Es.append(E[0] + E[1])
    rmin = rs[int(np.argmin(Es))]
    assert abs(rmin - 0.46) < 0.005


def _helix_with(N, twist=I.TWIST, tilt=0.0):
    """Relaxed helix with a different twist or with beads tilted along the axis."""
    axis = np.zeros((N, 3)); axis[:, 2] = I.RISE * np.arange(N)
    ang = twist * np.arange(N)
    d = np.stack([np.cos(ang), np.sin(ang), np.zeros(N)], 1)
    X = np.empty((2 * N, 3)); u = np.empty((2 * N, 3))
    for s, sg in ((0, 1.0), (1, -1.0)):
        bead = axis + sg * I.ELL * math.cos(tilt) * d
        bead[:, 2] += I.ELL * math.sin(tilt)
        X[s::2] = 0.5 * (bead + axis)
        uu = axis - bead
        u[s::2] = uu / np.linalg.norm(uu, axis=1, keepdims=True)
    return X, u


def test_dihedral_handedness_and_minimum():
    """Sec. 2: the dihedral imposes right-handedness with its minimum at 36 deg.
    A left-handed helix of the same pitch must cost energy; the right-handed
    relaxed helix sits at the minimum."""
    p = O.params()
    N = 12
    X, u = _helix_with(N, twist=I.TWIST)
    Xl, ul = _helix_with(N, twist=-I.TWIST)
    assert abs(_E(p, N, X, u)[4]) < 1e-10
    El = _E(p, N, Xl, ul)[4]
    # the maximum of K3 [1 + cos(phi - d)] is 2 K3 at phi = d = -144 deg
    Xm, um = _helix_with(N, twist=math.radians(-144.0))
    Em = _E(O.params(R0=2.0), N, Xm, um)[4]      # wide FENE so the unwound chain stays bonded
    assert El > 0.0
    assert abs(Em - 2 * (N - 1) * 2 * p.K3) < 1e-9


def test_planarity_minimum_at_ninety_degrees():
    p = O.params()
    N = 6
    X, u = _helix_with(N, tilt=0.0)
    assert abs(_E(p, N, X, u)[6]) < 1e-12
    for tilt in (0.05, -0.1):
        X, u = _helix_with(N, tilt=tilt)
        assert _E(p, N, X, u)[6] > 0.0


def _morse_energy(p, rise):
    """Morse energy (App. A Eq. 13) of a straight 2 bp duplex whose patches are
    `rise` apart along the axis: two patch-patch pairs, one per strand."""
    X, u = I.straight_helix(2)
    X[:, 2] *= rise / I.RISE
    return _E(p, 2, X, u)[5]


def test_morse_amplitude_range_and_stiffness():
    """App. A Eq. 13 with Table 1 (K4 = 30, lambda = 8, r0 = 0.34): the well is
    K4 deep (the energy of two separated patches), the energy at
    r0 + ln(2)/lambda, where the exponential has halved, is K4/4, and the
    curvature at r0 is 2 K4 lambda^2.  A Morse amplitude off by any factor, or
    a wrong range, fails one of these."""
    p = O.params(R0=10.0)          # a wide FENE bond, so the stretched backbone stays bonded
    far = _morse_energy(p, 3.0)
    assert abs(far - 2 * 30.0) < 1e-6, far                      # two pairs, each K4 away from the well
    half = _morse_energy(p, 0.34 + math.log(2.0) / 8.0)
    assert abs(half - 2 * 30.0 / 4) < 1e-9, half
    h = 1e-4
    curv = (_morse_energy(p, 0.34 + h) + _morse_energy(p, 0.34 - h) - 2 * _morse_energy(p, 0.34)) / h ** 2
    assert abs(curv / 2 - 2 * 30.0 * 64.0) < 1e-4 * 3840.0, curv


def _planar_energy(p, alpha):
    """Planarity energy (App. A Eq. 14) of one strand step whose angle E-F-B
    (vertex at patch F of nucleotide 1, between patch E of nucleotide 0 and
    bead B of nucleotide 1) is alpha; strand B sits 50 nm away as a relaxed
    helix (its angle is 90 degrees, zero energy)."""
    X, u = I.straight_helix(2)
    pe, pf = np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.0, I.RISE])
    b0 = pe + np.array([I.ELL, 0.0, 0.0])
    b1 = pf + I.ELL * np.array([math.sin(alpha), 0.0, -math.cos(alpha)])   # angle alpha to pe - pf = -z
    for g, (bead, patch) in ((0, (b0, pe)), (2, (b1, pf))):
        X[g] = 0.5 * (bead + patch)
        u[g] = (patch - bead) / np.linalg.norm(patch - bead)
    X[1::2, 0] += 50.0
    return _E(p, 2, X, u)[6]


def test_planarity_amplitude_and_form():
    """App. A Eq. 14 with Table 1 (K5 = 200, alpha0 = 90 deg): harmonic in the
    angle itself with the printed 1/2, so the energy is (K5/2)(pi/2)^2 with the
    three sites in a line (alpha = 0 or 180 deg), a quarter of that at 45 and
    135 deg (a harmonic form in cos(alpha) would give half), and the curvature
    at 90 deg is K5.  A factor K5 in place of K5/2 doubles every value."""
    p = O.params(R0=10.0)
    top = 100.0 * (math.pi / 2) ** 2
    for a in (0.0, math.pi):
        assert abs(_planar_energy(p, a) - top) < 1e-9 * top, (a, _planar_energy(p, a))
    for a in (math.pi / 4, 3 * math.pi / 4):
        assert abs(_planar_energy(p, a) - top / 4) < 1e-9 * top, (a, _planar_energy(p, a))
    assert abs(_planar_energy(p, math.pi / 2)) < 1e-12
    d = 1e-4
    curv = (_planar_energy(p, math.pi / 2 + d) + _planar_energy(p, math.pi / 2 - d)) / d ** 2
    assert abs(curv - 200.0) < 1e-6 * 200.0, curv


def test_bending_zero_straight_and_maximal_folded():
    p = O.params()
    X, u = I.straight_helix(3)
    assert abs(_E(p, 3, X, u)[7]) < 1e-12


def _site_fd(p, N, X, u, h=1e-6, idx=None, **kw):
    """Central differences of the oracle energy with respect to free site positions."""
    b, pt = O.sites(p, X, u)
    rng = np.random.default_rng(1)
    n = X.shape[0]
    if idx is None:
        idx = rng.choice(n, size=min(n, 12), replace=False)
    out = []
    for g in idx:
        for site in (0, 1):
            for c in range(3):
                vals = []
                for sgn in (1, -1):
                    bb, pp = b.copy(), pt.copy()
                    (bb if site == 0 else pp)[g, c] += sgn * h
                    X2 = 0.5 * (bb + pp)
                    u2 = (pp - bb) / p.ell                # exact sites, u need not be unit here
                    vals.append(_E(p, N, X2, u2, **kw)[:8].sum())
                out.append((g, site, c, -(vals[0] - vals[1]) / (2 * h)))
    return out


@pytest.mark.parametrize("periodic", [False, True])
def test_site_forces_are_minus_energy_gradient(periodic):
    p = O.params(box=(7.0, 7.0, 7.0)) if periodic else O.params()
    rng = np.random.default_rng(3)
    N = 14
    X, u = I.straight_helix(N)
    X, u = I.perturb(X, u, rng, dx=0.03, dtheta=0.08)
    if periodic:
        X[:, 0] += 3.2   # straddle the box face
    # bring a far part of the chain close to exercise the typed WCA pairs
    X[2 * 10:] += np.array([0.0, 0.0, 0.0])
    r = O.forces(p, N, X, u)
    for g, site, c, fd in _site_fd(p, N, X, u):
        an = (r["Fb"] if site == 0 else r["Fp"])[g, c]
        assert abs(an - fd) < 1e-6 * max(1.0, abs(fd)), (g, site, c, an, fd)


def test_pair_forces_gradient_in_compact_fold():
    """A hairpin-like fold brings same-strand steric beads and cross-strand beads into WCA range
    (a wide FENE keeps the stretched hinge bonded)."""
    p = O.params(R0=3.0)
    rng = np.random.default_rng(5)
    N = 12
    X, u = I.straight_helix(N)
    X, u = I.perturb(X, u, rng, dx=0.01, dtheta=0.02)
    # fold the top half back next to the bottom half, 1.5 nm away (closer, the
    # energy of the steric pairs grows past 10^4 kT and central differences of
    # it lose the digits this test compares)
    top = slice(2 * 6, 2 * N)
    X[top, 2] = 2 * X[2 * 6, 2] - X[top, 2]
    X[top, 0] += 1.5
    E = _E(p, N, X, u)
    assert E[3] > 0.0
    r = O.forces(p, N, X, u)
    idx = list(range(2 * 4, 2 * 8))
    for g, site, c, fd in _site_fd(p, N, X, u, idx=idx):
        an = (r["Fb"] if site == 0 else r["Fp"])[g, c]
        assert abs(an - fd) < 1e-6 * max(1.0, abs(fd)), (g, site, c, an, fd)


def test_no_net_force_or_torque_without_load():
    p = O.params()
    rng = np.random.default_rng(7)
    N = 25
    X, u = I.straight_helix(N)
    X, u = I.perturb(X, u, rng, dx=0.03, dtheta=0.08)
    r = O.forces(p, N, X, u)
    F, T = r["F"], r["T"]
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-12 * scale * len(F)
    L = (np.cross(X, F) + T).sum(0)
    assert np.abs(L).max() < 1e-11 * scale * len(F)


def test_energy_invariant_under_rigid_motion():
    p = O.params()
    rng = np.random.default_rng(8)
    N = 16
    X, u = I.perturb(*I.straight_helix(N), rng, dx=0.03, dtheta=0.08)
    E0 = _E(p, N, X, u)
    q = rng.normal(size=4); q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                  [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                  [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])
    E1 = _E(p, N, X @ R.T + np.array([3.0, -2.0, 11.0]), u @ R.T)
    assert np.allclose(E0, E1, atol=1e-10)


def test_body_force_and_torque_from_rigid_motion_fd():
    """F = -dE/dX and torque = -dE/d(rotation angle) for rotations normal to u."""
    p = O.params()
    rng = np.random.default_rng(9)
    N = 10
    X, u = I.perturb(*I.straight_helix(N), rng, dx=0.03, dtheta=0.08)
    r = O.forces(p, N, X, u)
    h = 1e-6
    for g in (0, 5, 9, 14, 19):
        for c in range(3):
            Xp = X.copy(); Xp[g, c] += h
            Xm = X.copy(); Xm[g, c] -= h
            fd = -(_E(p, N, Xp, u)[:8].sum() - _E(p, N, Xm, u)[:8].sum()) / (2 * h)
            assert abs(fd - r["F"][g, c]) < 1e-6 * max(1, abs(fd))
        for ax in np.linalg.svd(u[g][None, :])[2][1:]:   # two axes normal to u
            def rot(ang):
                u2 = u.copy()
                v = u[g]
                u2[g] = v * math.cos(ang) + np.cross(ax, v) * math.sin(ang) + ax * (ax @ v) * (1 - math.cos(ang))
                return u2
            fd = -(_E(p, N, X, rot(h))[:8].sum() - _E(p, N, X, rot(-h))[:8].sum()) / (2 * h)
            assert abs(fd - r["T"][g] @ ax) < 1e-6 * max(1, abs(fd))


@pytest.mark.parametrize("box", [None, (6.3, 5.1, 30.0)])
def test_cell_hash_equals_brute_force(box):
    p = O.params(box=box) if box else O.params()
    rng = np.random.default_rng(11)
    cfg = I.ragged_batch([9, 30, 4, 17], seed=2, spread=0.03)
    X, u = cfg.X.copy(), cfg.u.copy()
    # pack molecules close together: they must still not interact (independent systems)
    off = 0
    for m, nb in enumerate(cfg.n_bp):
        X[2 * off: 2 * (off + nb)] += rng.uniform(-0.5, 0.5, size=3)
        off += nb
    a = O.forces(p, cfg.n_bp, X, u)
    b = O.forces(p, cfg.n_bp, X, u, cells=True)
    for k in ("Fb", "Fp", "energy", "virial"):
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-12), k


def test_molecules_are_independent():
    p = O.params()
    cfg = I.ragged_batch([12, 12], seed=3, spread=0.02)
    X = cfg.X.copy()
    X[24:] = X[:24] + 0.3      # second molecule overlaps the first in space
    both = O.forces(p, cfg.n_bp, X, cfg.u)
    one = O.forces(p, 12, X[:24].copy(), cfg.u[:24].copy())
    assert np.allclose(both["Fb"][:24], one["Fb"], atol=1e-12)


def test_sampled_forces_equal_full():
    p = O.params(box=(9.0, 9.0, 9.0))
    rng = np.random.default_rng(12)
    cfg = I.ragged_batch([20, 7], seed=4, spread=0.03)
    ef = np.array([[0, 0, 2.0], [0.5, 0, 1.0]]); et = np.array([[0, 0, 3.0], [0, 1.0, 0]])
    full = O.forces(p, cfg.n_bp, cfg.X, cfg.u, ext_f=ef, ext_t=et)
    idx = rng.choice(cfg.n_nt, size=15, replace=False)
    idx = np.concatenate([idx, [38, 39, 52, 53, 0, 1]])
    Fb, Fp = O.forces_sampled(p, cfg.n_bp, cfg.X, cfg.u, idx, ext_f=ef, ext_t=et)
    assert np.allclose(Fb, full["Fb"][idx], atol=1e-12)
    assert np.allclose(Fp, full["Fp"][idx], atol=1e-12)


def test_external_load_is_pure_force_plus_couple():
    """Sec. 4.1-4.2: force f on the last base pair and a torque Gamma about the
    load axis.  Net added force is f; the couple adds no force and its torque
    about the pair centre has component |Gamma| along Gamma (two points can
    only be twisted about an axis normal to the line joining them, so the
    couple acts on their offsets projected normal to Gamma)."""
    p = O.params()
    rng = np.random.default_rng(13)
    N = 8
    X, u = I.perturb(*I.straight_helix(N), rng, dx=0.02, dtheta=0.05)
    f = np.array([[0.3, -0.2, 4.0]]); T = np.array([[0.0, 0.0, -2.5]])
    a = O.forces(p, N, X, u)
    b = O.forces(p, N, X, u, ext_f=f, ext_t=T)
    dF = b["F"] - a["F"]
    assert np.allclose(dF[:-2], 0.0, atol=1e-13)
    assert np.allclose(dF[-2:].sum(0), f[0], atol=1e-12)
    c = 0.5 * (X[-2] + X[-1])
    tq = np.cross(X[-2:] - c, dF[-2:]).sum(0) + (b["T"] - a["T"])[-2:].sum(0)
    assert abs(tq @ (T[0] / np.linalg.norm(T[0])) - np.linalg.norm(T[0])) < 1e-12
    c2 = O.forces(p, N, X, u, ext_t=T)
    assert np.allclose((c2["F"] - a["F"]).sum(0), 0.0, atol=1e-12)


def test_nve_energy_conservation_scales_as_dt_squared():
    """App. A Eq. 8 with gamma = 0 and no noise is Hamiltonian: the leapfrog
    energy error is bounded and shrinks as dt^2."""
    rng = np.random.default_rng(14)
    N = 12
    X0, u0 = I.perturb(*I.straight_helix(N), rng, dx=0.01, dtheta=0.02)
    V0, O0 = I.maxwell(u0, rng, kT=0.3)
    res = {}
    for dt in (0.002, 0.001):
        p = O.params(gamma=0.0, noise=0, dt=dt)
        X, V, u, Om = X0.copy(), V0.copy(), u0.copy(), O0.copy()
        Es = []
        nsteps = int(round(0.8 / dt))
        chunk = nsteps // 40
        for s in range(40):
            E, _ = O.energy(p, N, X, V, u, Om, s * chunk)
            Es.append(E.sum())
            O.run(p, N, X, V, u, Om, chunk, step0=s * chunk)
        Es = np.array(Es)
        res[dt] = np.abs(Es - Es[0]).max()
    ratio = res[0.002] / res[0.001]
    assert 2.5 < ratio < 6.0, res
    assert res[0.001] < 5e-3 * 0.3 * 2 * N * 2.5


@pytest.mark.slow
def test_langevin_equipartition():
    """App. A Eq. 8: at kT = 1 the mean translational kinetic energy is 3/2 kT
    and the rotational one kT (two axes normal to u) per nucleotide."""
    rng = np.random.default_rng(15)
    N = 20
    p = O.params(seed=77)
    X, u = I.straight_helix(N)
    V, Om = I.maxwell(u, rng)
    O.run(p, N, X, V, u, Om, 1000)
    kt, kr = [], []
    for s in range(150):
        O.run(p, N, X, V, u, Om, 40, step0=1000 + 40 * s)
        E, _ = O.energy(p, N, X, V, u, Om, 1000 + 40 * (s + 1))
        kt.append(E[0, 8] / (2 * N)); kr.append(E[0, 9] / (2 * N))
    assert abs(np.mean(kt) - 1.5) < 0.08, np.mean(kt)
    assert abs(np.mean(kr) - 1.0) < 0.06, np.mean(kr)


def test_noise_stream_moments():
    """One Philox4x32-10 draw per nucleotide gives six 21-bit fields (top 21 bits
    of each word, then the low 11 bits of x / z joined with bits 0-9 of y / w):
    each uniform on [0, 2^21) with mean 0 and variance 1 after centring and
    scaling by sqrt(12) 2^-21, and the six mutually uncorrelated."""
    fields = []
    for l in range(400):
        for s in range(10):
            x, y, z, w = O.philox4x32_10([l, s, 0, 0], [0, 0])
            k = [x >> 11, y >> 11, z >> 11, w >> 11, (x & 0x7FF) | ((y & 0x3FF) << 11), (z & 0x7FF) | ((w & 0x3FF) << 11)]
            fields.append([((q - 1048575.5) * 2.0 ** -21) * math.sqrt(12) for q in k])
    v = np.array(fields)
    assert v.min() > -math.sqrt(3) and v.max() < math.sqrt(3)
    assert np.abs(v.mean(0)).max() < 0.06 and np.abs(v.var(0) - 1.0).max() < 0.08
    c = np.corrcoef(v.T) - np.eye(6)
    assert np.abs(c).max() < 0.08


def test_mb_velocities_statistics():
    p = O.params(seed=5)
    N = 3000
    X, u = O.ideal_helix(p, N)
    V, Om = O.mb_velocities(p, 0, N, u, tether=1)
    assert np.all(V[:2] == 0) and np.all(Om[:2] == 0)
    assert np.abs((Om * u).sum(1)).max() < 1e-12
    M, I_ = 2.0, 0.125
    assert abs(0.5 * M * (V[2:] ** 2).sum(1).mean() - 1.5) < 0.06
    assert abs(0.5 * I_ * (Om[2:] ** 2).sum(1).mean() - 1.0) < 0.05


def test_observables_of_ideal_helix():
    """Sec. 3.2: 36 deg of twist per base-pair step; Sec. 4.1: R_z = rise * (N-1)."""
    p = O.params()
    N = 57
    X, u = O.ideal_helix(p, N)
    o = O.observables(p, N, X, u, with_lk=True)
    assert abs(o["tw"] - (N - 2) / 10.0) < 1e-12
    assert abs(o["tw"] - o["tw_ideal"]) < 1e-12
    assert abs(o["rz"] - 0.34 * (N - 1)) < 1e-12
    assert o["denat"] == 0.0
    # the closed strands link an integer number of times, about once per 10 bp (Sec. 4.2)
    assert abs(o["lk"] - round(o["lk"])) < 1e-6   # asin near +-1 limits the sum to ~sqrt(eps)
    assert abs(o["lk"] - o["tw"]) < 1.0
    # separating the strands breaks every bond
    X2 = X.copy(); X2[1::2, 0] += 1.0
    assert O.observables(p, N, X2, u)["denat"] == 1.0


def _lk_by_disk(circle_r, b):
    """a = circle of radius circle_r in the z=0 plane, counter-clockwise seen from +z; count
    signed crossings of polygon b through its disk (+1 when crossing along +z)."""
    s = 0
    n = len(b)
    for i in range(n):
        p0, p1 = b[i], b[(i + 1) % n]
        if (p0[2] > 0) == (p1[2] > 0):
            continue
        t = p0[2] / (p0[2] - p1[2])
        x = p0 + t * (p1 - p0)
        if x[0] ** 2 + x[1] ** 2 < circle_r ** 2:
            s += 1 if p1[2] > p0[2] else -1
    return s


@pytest.mark.parametrize("turns", [1, 2, 3, -2])
def test_linking_number_against_crossing_count(turns):
    """Gauss linking number of closed curves equals the signed crossing count
    through a spanning disk (App. C): pins sign and normalisation."""
    n = 400
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    a = np.stack([np.cos(t), np.sin(t), 0 * t], 1)
    # b winds |turns| times around the circle of a (a torus curve), direction by sign
    m = 2000
    s = np.linspace(0, 2 * np.pi, m, endpoint=False)
    R, r = 1.0, 0.3
    b = np.stack([(R + r * np.cos(turns * s)) * np.cos(s), (R + r * np.cos(turns * s)) * np.sin(s), r * np.sin(turns * s)], 1)
    lk = O.linking_number(a, b)
    assert abs(lk - _lk_by_disk(1.0, b)) < 1e-6, lk


def test_steric_typing_counts_from_each_five_prime_end():
    """Sec. 2 / Fig. 1d: along a strand one steric bead is followed by two ghost
    beads; ghosts never see their own strand, every bead sees the other strand.
    Reading: each strand starts (5' end) with a steric bead.  Strand B runs
    5'->3' from base pair N-1 down to 0."""
    p = O.params()
    N = 8
    X, u = I.straight_helix(N)
    prs = {tuple(x) for x in O.pairs(p, N, X, u, extra=1e3)}
    same = {(i, j) for (i, j) in prs if (i & 1) == (j & 1)}
    a_steric = [2 * k for k in (0, 3, 6)]
    b_steric = [2 * k + 1 for k in (7, 4, 1)]
    want = {(min(i, j), max(i, j)) for grp in (a_steric, b_steric) for i in grp for j in grp if i < j}
    assert same == want
    assert len(prs - same) == N * N
