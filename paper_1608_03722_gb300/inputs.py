"""Seeded synthetic inputs for the dsDNA model (arXiv:1608.03722).

This module only builds configurations: base-pair counts, coordinates,
velocities and loads.  It evaluates no interaction, integrator or observable
of the model, and both the CUDA library and the FP64 oracle take its arrays as
plain inputs.

Layout: AoS float64 arrays of shape ``(n_nt, 3)`` in slot order
``g = 2*(bp_offset + k) + s`` (s = 0 strand A nucleotide k, s = 1 its partner
on strand B).  Each nucleotide is described by its centre ``X`` (midpoint of
bead and patch) and the unit vector ``u`` from bead to patch; velocities are
``V`` (centre) and ``Om`` (angular, normal to ``u``).

Geometry of the relaxed helix (Sec. 2, Fig. 1): both patches of base pair k on
the axis with a rise of 0.34 nm, the two beads 0.5 nm off the axis on opposite
sides, turning by 36 degrees per base pair (pitch 10 bp).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RISE = 0.34          # nm per base pair (Sec. 2, Fig. 1b)
TWIST = math.pi / 5  # 36 degrees per base pair (Sec. 2)
ELL = 0.5            # bead-patch distance (Sec. 2)


@dataclass
class Config:
    """A synthetic workload: molecules, initial state and loads."""
    name: str
    n_bp: np.ndarray                 # int32 [n_mol]
    X: np.ndarray                    # [n_nt, 3]
    u: np.ndarray
    V: np.ndarray
    Om: np.ndarray
    box: tuple = (0.0, 0.0, 0.0)     # periodic edges (0 = open)
    tether: np.ndarray = None        # int32 [n_mol]
    ext_f: np.ndarray = None         # [n_mol, 3]
    ext_t: np.ndarray = None         # [n_mol, 3]
    seq: bytes = b""
    meta: dict = field(default_factory=dict)

    @property
    def n_nt(self) -> int:
        return int(self.X.shape[0])


def helix_frame(n_bp: int, origin, t, n, phase0: float = 0.0):
    """Straight helix of n_bp base pairs along unit tangent t with reference normal n."""
    t = np.asarray(t, float); n = np.asarray(n, float)
    b = np.cross(t, n)
    k = np.arange(n_bp)
    axis = np.asarray(origin, float)[None, :] + RISE * k[:, None] * t[None, :]
    ang = phase0 + TWIST * k
    d = np.cos(ang)[:, None] * n[None, :] + np.sin(ang)[:, None] * b[None, :]
    return axis, d


def place(axis: np.ndarray, d: np.ndarray):
    """Nucleotide centres and orientations from axis points and bead directions."""
    nbp = axis.shape[0]
    X = np.empty((2 * nbp, 3)); u = np.empty((2 * nbp, 3))
    X[0::2] = axis + 0.5 * ELL * d      # centre between bead (axis + ELL d) and patch (axis)
    u[0::2] = -d
    X[1::2] = axis - 0.5 * ELL * d
    u[1::2] = d
    return X, u


def straight_helix(n_bp: int, origin=(0.0, 0.0, 0.0)):
    axis, d = helix_frame(n_bp, origin, (0, 0, 1), (1, 0, 0))
    return place(axis, d)


def maxwell(u: np.ndarray, rng: np.random.Generator, kT: float = 1.0, mass: float = 1.0, ell: float = ELL,
            frozen: np.ndarray | None = None):
    """Maxwell-Boltzmann centre and angular velocities (angular normal to u)."""
    M = 2.0 * mass
    I = 0.5 * mass * ell * ell
    n = u.shape[0]
    V = rng.normal(0.0, math.sqrt(kT / M), size=(n, 3))
    w = rng.normal(0.0, math.sqrt(kT / I), size=(n, 3))
    Om = w - (w * u).sum(1, keepdims=True) * u
    if frozen is not None:
        V[frozen] = 0.0
        Om[frozen] = 0.0
    V -= V.mean(0, keepdims=True) if frozen is None else 0.0
    return V, Om


def perturb(X: np.ndarray, u: np.ndarray, rng: np.random.Generator, dx: float = 0.02, dtheta: float = 0.05):
    """Thermal-like jitter: Gaussian centre shifts and small random tilts of u."""
    X2 = X + rng.normal(0.0, dx, size=X.shape)
    r = rng.normal(0.0, dtheta, size=u.shape)
    r -= (r * u).sum(1, keepdims=True) * u
    u2 = u + r
    u2 /= np.linalg.norm(u2, axis=1, keepdims=True)
    return X2, u2


def _frozen_mask(n_bp: np.ndarray, tether: np.ndarray) -> np.ndarray:
    off = np.concatenate([[0], np.cumsum(n_bp)])
    mask = np.zeros(2 * int(off[-1]), dtype=bool)
    for m, t in enumerate(tether):
        if t:
            mask[2 * off[m]: 2 * off[m] + 2] = True
    return mask


def c1_linear(n_bp: int = 200, seed: int = 0) -> Config:
    """Linear dsDNA of n_bp (default 200 bp), ideal helix, open boundaries."""
    rng = np.random.default_rng(seed)
    X, u = straight_helix(n_bp)
    V, Om = maxwell(u, rng)
    seq = bytes(rng.choice(np.frombuffer(b"ATGC", np.uint8), size=n_bp))
    return Config("linear_%dbp" % n_bp, np.array([n_bp], np.int32), X, u, V, Om, seq=seq)


def c2_tethered(n_bp: int = 10_000, force: float = 1.0, torque: float = 0.0, seed: int = 0) -> Config:
    """Linear dsDNA along z, base pair 0 anchored, constant force f e_z and torque Gamma e_z on the last bp."""
    rng = np.random.default_rng(seed)
    X, u = straight_helix(n_bp)
    tether = np.array([1], np.int32)
    V, Om = maxwell(u, rng, frozen=_frozen_mask(np.array([n_bp]), tether))
    cfg = Config("tethered_%dbp" % n_bp, np.array([n_bp], np.int32), X, u, V, Om, tether=tether,
                 ext_f=np.array([[0.0, 0.0, force]]), ext_t=np.array([[0.0, 0.0, torque]]))
    cfg.meta.update(force=force, torque=torque)
    return cfg


def box_edge(n_nt: int, phi: float) -> float:
    """Periodic cube edge giving volume fraction phi of unit-diameter beads."""
    return (n_nt * (math.pi / 6.0) / phi) ** (1.0 / 3.0)


def _rot(axis, ang):
    a = np.asarray(axis, float); a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def c3_confined(n_bp: int = 1_000_000, phi: float = 0.05, seg_bp: int = 30, max_joint_deg: float = 20.0,
                clearance: float = 2.5, seed: int = 0) -> Config:
    """Self-avoiding helix in a periodic cube at volume fraction phi.

    The axis is a chain of straight seg_bp-long helical segments joined at
    random angles up to max_joint_deg with a continuous helical phase
    (parallel-transported reference normal).  A segment is redrawn when one of
    its sample points comes closer than ``clearance`` (periodic) to an axis
    point of any earlier, non-adjacent segment.  Coordinates stay unwrapped.
    """
    rng = np.random.default_rng(seed)
    L = box_edge(2 * n_bp, phi)
    nseg = (n_bp + seg_bp - 1) // seg_bp
    cell = clearance
    ncell = max(1, int(L // cell))
    h = L / ncell
    grid: dict = {}
    t = np.array([0.0, 0.0, 1.0]); n = np.array([1.0, 0.0, 0.0])
    start = rng.uniform(0, L, size=3)
    starts = np.empty((nseg, 3)); ts = np.empty((nseg, 3)); ns = np.empty((nseg, 3))
    sample = np.arange(0, seg_bp, 5)
    maxj = math.radians(max_joint_deg)
    pos = start.copy()
    for s in range(nseg):
        for attempt in range(200):
            if s == 0:
                t2, n2 = t, n
            else:
                ang = maxj * math.sqrt(rng.uniform()) if attempt < 100 else rng.uniform(0, math.pi / 2)
                perp = np.cross(t, rng.normal(size=3)); perp /= np.linalg.norm(perp)
                R = _rot(perp, ang)
                t2 = R @ t; n2 = R @ n
                n2 -= (n2 @ t2) * t2; n2 /= np.linalg.norm(n2)
            pts = pos[None, :] + RISE * (sample[:, None] + (1 if s else 0)) * t2[None, :]
            ok = True
            for q in pts:
                w = np.floor((q % L) / h).astype(int)
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            key = ((w[0] + dx) % ncell, (w[1] + dy) % ncell, (w[2] + dz) % ncell)
                            for (qq, seg) in grid.get(key, ()):
                                if seg >= s - 2:
                                    continue
                                dd = q - qq
                                dd -= L * np.round(dd / L)
                                if dd @ dd < clearance * clearance:
                                    ok = False
                                    break
                            if not ok:
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok or attempt == 199:
                break
        first = pos + (RISE * t2 if s else 0.0)
        starts[s] = first; ts[s] = t2; ns[s] = n2
        for q in pts:
            w = np.floor((q % L) / h).astype(int)
            grid.setdefault((w[0] % ncell, w[1] % ncell, w[2] % ncell), []).append((q.copy(), s))
        pos = first + RISE * (seg_bp - 1) * t2
        t, n = t2, n2
    k = np.arange(n_bp)
    s_of = k // seg_bp
    j = k - s_of * seg_bp
    axis = starts[s_of] + RISE * j[:, None] * ts[s_of]
    b = np.cross(ts[s_of], ns[s_of])
    ang = TWIST * k
    d = np.cos(ang)[:, None] * ns[s_of] + np.sin(ang)[:, None] * b
    X, u = place(axis, d)
    V, Om = maxwell(u, rng)
    seq = bytes(rng.choice(np.frombuffer(b"ATGC", np.uint8), size=n_bp))
    cfg = Config("confined_%dbp_phi%.2f" % (n_bp, phi), np.array([n_bp], np.int32), X, u, V, Om,
                 box=(L, L, L), seq=seq)
    cfg.meta.update(L=L, phi=phi)
    return cfg


def c4_batch(n_mol: int = 256, lo: int = 500, hi: int = 20_000, seed: int = 0) -> Config:
    """Independent linear molecules, lengths log-uniform in [lo, hi] bp, each
    anchored at bp 0 and loaded with its own force (U[0.1, 10] e_z) and torque
    (U[-5, 5] e_z) on the last base pair."""
    rng = np.random.default_rng(seed)
    n_bp = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_mol)).astype(np.int32)
    n_bp = np.clip(n_bp, lo, hi).astype(np.int32)
    Xs, us = [], []
    for nb in n_bp:
        X, u = straight_helix(int(nb))
        Xs.append(X); us.append(u)
    X = np.concatenate(Xs); u = np.concatenate(us)
    tether = np.ones(n_mol, np.int32)
    V, Om = maxwell(u, rng, frozen=_frozen_mask(n_bp, tether))
    f = rng.uniform(0.1, 10.0, size=n_mol)
    g = rng.uniform(-5.0, 5.0, size=n_mol)
    ext_f = np.zeros((n_mol, 3)); ext_f[:, 2] = f
    ext_t = np.zeros((n_mol, 3)); ext_t[:, 2] = g
    return Config("batch_%dx[%d,%d]bp" % (n_mol, lo, hi), n_bp, X, u, V, Om, tether=tether,
                  ext_f=ext_f, ext_t=ext_t)


def ragged_batch(lengths, seed: int = 0, spread: float = 0.0) -> Config:
    """Molecules of the given lengths, optionally jittered, for parity tests."""
    rng = np.random.default_rng(seed)
    Xs, us = [], []
    for nb in lengths:
        X, u = straight_helix(int(nb))
        if spread:
            X, u = perturb(X, u, rng, dx=spread, dtheta=2.5 * spread)
        Xs.append(X); us.append(u)
    X = np.concatenate(Xs); u = np.concatenate(us)
    n_bp = np.asarray(lengths, np.int32)
    V, Om = maxwell(u, rng)
    return Config("ragged_%d" % len(lengths), n_bp, X, u, V, Om)


def surrogate_points(n: int, seed: int = 0):
    """Sweep inputs (force 0.1-10, supercoiling density -0.06..0.06,
    length 500-20000 bp, kT 0.8-1.4), length log-uniform."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.1, 10.0, n)
    sig = rng.uniform(-0.06, 0.06, n)
    L = np.exp(rng.uniform(math.log(500), math.log(20000), n))
    kT = rng.uniform(0.8, 1.4, n)
    return np.stack([f, sig, L, kT], axis=1)
