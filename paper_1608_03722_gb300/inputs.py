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


def ring_helix(n_bp: int, lk: int, center=(0.0, 0.0, 0.0)):
    """Planar circular duplex of n_bp base pairs in the xy plane whose bead
    direction turns lk times about the local tangent (linking number lk of
    the two closed strands; lk = n_bp/10 is torsionally relaxed).  The axis
    points sit on a regular n_bp-gon with sides of one rise."""
    k = np.arange(n_bp)
    R = RISE / (2.0 * math.sin(math.pi / n_bp))
    th = 2.0 * math.pi * k / n_bp
    nrm = np.stack([np.cos(th), np.sin(th), np.zeros(n_bp)], axis=1)     # radial
    tan = np.stack([-np.sin(th), np.cos(th), np.zeros(n_bp)], axis=1)    # tangent, strand A direction
    b = np.cross(tan, nrm)
    axis = np.asarray(center, float)[None, :] + R * nrm
    ang = 2.0 * math.pi * lk * k / n_bp
    d = np.cos(ang)[:, None] * nrm + np.sin(ang)[:, None] * b
    return place(axis, d)


def wlc_helix(n_bp: int, lp_bp: float, rng: np.random.Generator, origin=(0.0, 0.0, 0.0), clearance: float = 2.5,
              seg: int = 10, tries: int = 100):
    """Relaxed helix (36 degrees per base pair about a parallel-transported
    frame) along a smooth worm-like axis: tangents drawn every `seg` base
    pairs with <t . t'> = exp(-seg / lp_bp), interpolated by slerp in between,
    so the bending is spread over `seg` base pairs as thermal bending of the
    duplex is.  Axis points more than 10 bp apart along the chain stay at
    least `clearance` nm apart (redrawn otherwise)."""
    nc = (n_bp + seg - 1) // seg + 1
    c = 1.0 - math.exp(-float(seg) / lp_bp)
    for _ in range(tries):
        T = np.empty((nc, 3)); T[0] = (0.0, 0.0, 1.0)
        for k in range(1, nc):
            a = rng.normal(size=3)
            a -= a.dot(T[k - 1]) * T[k - 1]
            a /= np.linalg.norm(a)
            ct = max(-1.0, 1.0 - rng.exponential(c))
            T[k] = ct * T[k - 1] + math.sqrt(1.0 - ct * ct) * a
            T[k] /= np.linalg.norm(T[k])
        t = np.empty((n_bp, 3))
        for i in range(n_bp):
            j, f = divmod(i, seg)
            f /= seg
            om = math.acos(max(-1.0, min(1.0, float(T[j].dot(T[j + 1])))))
            if om < 1e-9:
                t[i] = T[j]
            else:
                t[i] = (math.sin((1.0 - f) * om) * T[j] + math.sin(f * om) * T[j + 1]) / math.sin(om)
            t[i] /= np.linalg.norm(t[i])
        axis = np.asarray(origin, float)[None, :] + RISE * np.concatenate([[np.zeros(3)], np.cumsum(t[:-1], 0)])
        far = np.abs(np.arange(n_bp)[:, None] - np.arange(n_bp)[None, :]) > 10
        dist = np.linalg.norm(axis[:, None, :] - axis[None, :, :], axis=2)
        if (dist[far] >= clearance).all():
            break
    else:
        raise RuntimeError("no self-avoiding worm-like axis found")
    n = np.empty((n_bp, 3))
    ref = np.array([1.0, 0.0, 0.0])
    n[0] = ref - ref.dot(t[0]) * t[0]; n[0] /= np.linalg.norm(n[0])
    for k in range(1, n_bp):                  # parallel transport of the normal
        v = n[k - 1] - n[k - 1].dot(t[k]) * t[k]
        n[k] = v / np.linalg.norm(v)
    b = np.cross(t, n)
    ang = TWIST * np.arange(n_bp)
    d = np.cos(ang)[:, None] * n + np.sin(ang)[:, None] * b
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


def random_walk_helix(n_bp: int = 3000, phi: float = 0.05, seg_bp: int = 30, max_joint_deg: float = 25.0,
                clearance: float = 2.2, joint_bp: int = 5, seed: int = 0) -> Config:
    """Self-avoiding helix in a periodic cube at volume fraction phi.

    The axis is a chain of seg_bp-long helical segments; each segment turns
    the axis by a random angle up to max_joint_deg, spread evenly over its
    first joint_bp base pairs, and the reference normal is carried along by
    the same rotations so the helical phase stays continuous.  Axis points
    every 3 bp of a new segment must stay ``clearance`` (periodic) away from
    those of every earlier, non-adjacent segment; a segment that cannot be
    placed makes the walk back up a few segments.  Coordinates stay unwrapped.
    """
    rng = np.random.default_rng(seed)
    L = box_edge(2 * n_bp, phi)
    nseg = (n_bp + seg_bp - 1) // seg_bp
    maxj = math.radians(max_joint_deg)
    j = np.arange(1, seg_bp + 1)
    frac = np.minimum(j, joint_bp) / float(joint_bp)
    sample = np.arange(0, seg_bp, 3)
    c2 = clearance * clearance
    # sample points are filed in a grid of cells at least `clearance` wide (KS
    # slots per cell, a dict for the rare overflow), so every earlier point
    # closer than the clearance sits in one of the 27 cells around a new point
    nc = max(1, int(L // clearance))
    hc = L / nc
    KS = 6
    seg_of = np.full((nc ** 3, KS), -1, np.int32)
    spts = np.zeros((nc ** 3, KS, 3))
    spill: dict = {}
    offs = np.array([(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)])

    def cells_of(q):
        w = np.floor((q % L) / hc).astype(np.int64) % nc
        return (w[:, 0] * nc + w[:, 1]) * nc + w[:, 2]

    def around(q):
        w = np.floor((q % L) / hc).astype(np.int64) % nc
        v = (w[:, None, :] + offs[None, :, :]) % nc
        return (v[..., 0] * nc + v[..., 1]) * nc + v[..., 2]        # [points, 27]

    def clash(pts, s):
        idx = around(pts)
        sg = seg_of[idx]                                             # [points, 27, KS]
        ok = (sg >= 0) & (sg < s - 2)
        if ok.any():
            d = pts[:, None, None, :] - spts[idx]
            d -= L * np.round(d / L)
            if (((d * d).sum(-1) < c2) & ok).any():
                return True
        if spill:
            for i, q in enumerate(pts):
                for c in set(idx[i].tolist()):
                    for e, qq in spill.get(c, ()):
                        if e < s - 2:
                            dd = q - qq
                            dd -= L * np.round(dd / L)
                            if dd @ dd < c2:
                                return True
        return False

    def file(pts, s):
        for c, q in zip(cells_of(pts).tolist(), pts):
            free = np.flatnonzero(seg_of[c] < 0)
            if len(free):
                seg_of[c, free[0]] = s
                spts[c, free[0]] = q
            else:
                spill.setdefault(c, []).append((s, q))

    def unfile(pts, s):
        for c in cells_of(pts).tolist():
            seg_of[c][seg_of[c] == s] = -1
            if c in spill:
                spill[c] = [e for e in spill[c] if e[0] != s]

    segs = []          # accepted segments: (pts, ts, ns)
    t0 = np.array([0.0, 0.0, 1.0]); n0 = np.array([1.0, 0.0, 0.0])
    start = rng.uniform(0, L, size=3) - RISE * t0
    fails = 0
    while len(segs) < nseg:
        s = len(segs)
        if s:
            pos, t, n = segs[-1][0][-1], segs[-1][1][-1], segs[-1][2][-1]
            n = n - (n @ t) * t
            n /= np.linalg.norm(n)
        else:
            pos, t, n = start, t0, n0
        placed = False
        for attempt in range(60):
            ang = 0.0 if s == 0 else maxj * math.sqrt(rng.uniform())
            perp = np.cross(t, rng.normal(size=3)); perp /= np.linalg.norm(perp)
            K = np.array([[0, -perp[2], perp[1]], [perp[2], 0, -perp[0]], [-perp[1], perp[0], 0]])
            a = ang * frac
            Rs = np.eye(3)[None] + np.sin(a)[:, None, None] * K[None] + (1 - np.cos(a))[:, None, None] * (K @ K)[None]
            ts = Rs @ t
            ns = Rs @ n
            pts = pos[None, :] + RISE * np.cumsum(ts, axis=0)
            if not clash(pts[sample], s):
                placed = True
                break
        if placed:
            segs.append((pts, ts, ns))
            file(pts[sample], s)
            continue
        fails += 1
        if fails > 20 * nseg + 1000:
            raise RuntimeError("could not grow the self-avoiding helix")
        back = min(len(segs), 1 + int(rng.integers(0, 4)))
        for _ in range(back):
            pts_d, _, _ = segs.pop()
            unfile(pts_d[sample], len(segs))
    axis = np.concatenate([sg[0] for sg in segs])[:n_bp]
    T = np.concatenate([sg[1] for sg in segs])[:n_bp]
    Nn = np.concatenate([sg[2] for sg in segs])[:n_bp]
    Nn = Nn - (Nn * T).sum(1, keepdims=True) * T
    Nn /= np.linalg.norm(Nn, axis=1, keepdims=True)
    B = np.cross(T, Nn)
    ang = TWIST * np.arange(n_bp)
    d = np.cos(ang)[:, None] * Nn + np.sin(ang)[:, None] * B
    X, u = place(axis, d)
    V, Om = maxwell(u, rng)
    seq = bytes(rng.choice(np.frombuffer(b"ATGC", np.uint8), size=n_bp))
    cfg = Config("confined_%dbp_phi%.2f" % (n_bp, phi), np.array([n_bp], np.int32), X, u, V, Om,
                 box=(L, L, L), seq=seq)
    cfg.meta.update(L=L, phi=phi)
    return cfg


def _rotations(axis_vec, angles):
    """Rotation matrices about a fixed unit axis for an array of angles."""
    k = np.asarray(axis_vec, float)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    a = np.asarray(angles, float)
    return np.eye(3)[None] + np.sin(a)[:, None, None] * K[None] + (1 - np.cos(a))[:, None, None] * (K @ K)[None]


def c3_confined(n_bp: int = 1_000_000, phi: float = 0.05, seed: int = 0) -> Config:
    """One dsDNA molecule filling a periodic cube at volume fraction phi.

    The helix axis snakes through the box: straight rows along x on a square
    lattice of (y, z) positions, consecutive rows joined by semicircular
    U-turns, layers joined the same way in the xz plane, so the molecule is
    self-avoiding by construction and locally looks like an array of parallel
    helices.  The reference normal is parallel-transported (rotated with the
    tangent through each turn) and the helix turns by 36 degrees per base pair
    along the whole chain.  The lattice spacing is the largest that fits the
    contour length; the start phase and a global shift are random (seed).
    Coordinates stay unwrapped (they lie inside [0, L)).
    """
    rng = np.random.default_rng(seed)
    L = box_edge(2 * n_bp, phi)
    need = RISE * (n_bp + 1)
    nrow = int(math.ceil(math.sqrt(need / (L - 4.0))))
    while True:
        a = L / nrow
        x0, x1 = 0.5 * a + 1.0, L - 0.5 * a - 1.0
        total = nrow * nrow * (x1 - x0) + (nrow * nrow - 1) * math.pi * 0.5 * a
        if total >= need:
            break
        nrow += 1
    rows = []
    for jz in range(nrow):
        order = range(nrow) if jz % 2 == 0 else range(nrow - 1, -1, -1)
        for iy in order:
            rows.append(((iy + 0.5) * a, (jz + 0.5) * a))
    pts, tans, nors = [], [], []
    t = np.array([1.0, 0.0, 0.0]); n = np.array([0.0, 1.0, 0.0])
    carry = 0.0          # arc length into the next piece at which the next base pair sits
    for r, (y, z) in enumerate(rows):
        dirx = 1.0 if r % 2 == 0 else -1.0
        xs, xe = (x0, x1) if dirx > 0 else (x1, x0)
        length = x1 - x0
        sarr = np.arange(carry, length, RISE)
        p = np.stack([xs + dirx * sarr, np.full_like(sarr, y), np.full_like(sarr, z)], 1)
        pts.append(p); tans.append(np.repeat(t[None], len(sarr), 0)); nors.append(np.repeat(n[None], len(sarr), 0))
        carry = sarr[-1] + RISE - length if len(sarr) else carry - length
        if r + 1 == len(rows):
            break
        ny_, nz_ = rows[r + 1]
        off = np.array([0.0, ny_ - y, nz_ - z])
        rad = 0.5 * np.linalg.norm(off)
        w = off / np.linalg.norm(off)
        centre = np.array([xe, y, z]) + rad * w
        b = np.cross(t, w)                     # turn axis: rotates t into -t through w
        arc = math.pi * rad
        sarr = np.arange(carry, arc, RISE)
        ang = sarr / rad
        R = _rotations(b, ang)
        start = np.array([xe, y, z])
        p = centre[None] + (R @ (start - centre))
        pts.append(p); tans.append(R @ t); nors.append(R @ n)
        Rend = _rotations(b, [math.pi])[0]
        t = Rend @ t; n = Rend @ n
        carry = sarr[-1] + RISE - arc if len(sarr) else carry - arc
    axis = np.concatenate(pts)[:n_bp]
    T = np.concatenate(tans)[:n_bp]
    Nn = np.concatenate(nors)[:n_bp]
    assert len(axis) == n_bp, "box too small for the contour length"
    Nn = Nn - (Nn * T).sum(1, keepdims=True) * T
    Nn /= np.linalg.norm(Nn, axis=1, keepdims=True)
    B = np.cross(T, Nn)
    ang = rng.uniform(0, 2 * math.pi) + TWIST * np.arange(n_bp)
    d = np.cos(ang)[:, None] * Nn + np.sin(ang)[:, None] * B
    axis = axis + rng.uniform(-0.5, 0.5, size=3)
    X, u = place(axis, d)
    V, Om = maxwell(u, rng)
    seq = bytes(rng.choice(np.frombuffer(b"ATGC", np.uint8), size=n_bp))
    cfg = Config("confined_%dbp_phi%.2f" % (n_bp, phi), np.array([n_bp], np.int32), X, u, V, Om,
                 box=(L, L, L), seq=seq)
    cfg.meta.update(L=L, phi=phi, rows=nrow * nrow, spacing=a)
    return cfg


def c3_walk(n_bp: int = 1_000_000, phi: float = 0.05, seed: int = 0) -> Config:
    """One dsDNA molecule confined in a periodic cube at volume fraction phi,
    grown as a self-avoiding walk of straight 30 bp helical segments joined at
    angles of at most 30 degrees (each joint spread over 5 base pairs), with
    the helical phase continuous along the chain and axis points of
    non-adjacent segments at least 2.2 nm apart (periodic distance); random
    sequence (force-inert).  Coordinates stay unwrapped."""
    cfg = random_walk_helix(n_bp=n_bp, phi=phi, seg_bp=30, max_joint_deg=30.0, clearance=2.2, joint_bp=5, seed=seed)
    cfg.name = "confined_walk_%dbp_phi%.2f" % (n_bp, phi)
    return cfg


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (normalised Gaussian quaternion)."""
    q = rng.normal(size=4)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def c4_batch(n_mol: int = 256, lo: int = 500, hi: int = 20_000, seed: int = 0, random_pose: bool = False,
             spread: float = 200.0) -> Config:
    """Independent linear molecules, lengths log-uniform in [lo, hi] bp, each
    anchored at bp 0 and loaded with its own force (U[0.1, 10] along the
    molecule's axis) and torque (U[-5, 5] about it) on the last base pair.
    Molecules are relaxed straight helices along +z from the origin, or with
    random_pose each turned by a uniformly random rotation about its first
    base pair and moved to a uniformly random origin in a cube of edge
    `spread` nm (its load turned with it)."""
    rng = np.random.default_rng(seed)
    n_bp = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_mol)).astype(np.int32)
    n_bp = np.clip(n_bp, lo, hi).astype(np.int32)
    pose = np.random.default_rng(seed + 7919) if random_pose else None
    Xs, us, R = [], [], []
    for nb in n_bp:
        X, u = straight_helix(int(nb))
        Rm = np.eye(3)
        if pose is not None:
            Rm = random_rotation(pose)
            X = X @ Rm.T + pose.uniform(-0.5 * spread, 0.5 * spread, size=3)
            u = u @ Rm.T
        Xs.append(X); us.append(u); R.append(Rm)
    X = np.concatenate(Xs); u = np.concatenate(us)
    tether = np.ones(n_mol, np.int32)
    V, Om = maxwell(u, rng, frozen=_frozen_mask(n_bp, tether))
    f = rng.uniform(0.1, 10.0, size=n_mol)
    g = rng.uniform(-5.0, 5.0, size=n_mol)
    R = np.asarray(R)
    ext_f = f[:, None] * R[:, :, 2]     # the molecule's own axis (z before the turn)
    ext_t = g[:, None] * R[:, :, 2]
    name = "batch_%dx[%d,%d]bp%s" % (n_mol, lo, hi, "_random_pose" if random_pose else "")
    return Config(name, n_bp, X, u, V, Om, tether=tether, ext_f=ext_f, ext_t=ext_t)


def paper_array(nx: int = 40, ny: int = 40, n_bp: int = 600, spacing: float = 5.0, seed: int = 0) -> Config:
    """The paper's benchmark geometry (Sec. 6): a regular nx x ny array of
    linear n_bp dsDNA strands (40 x 40 x 600 bp = 960 kbp, 1.92e6 nucleotides;
    10 x 10 = 60 kbp).  The paper gives no spacing or box; here the relaxed
    helices stand along z on a square lattice of `spacing` nm in a periodic box
    of nx*spacing x ny*spacing x (n_bp*0.34 + spacing) nm, random start phases."""
    rng = np.random.default_rng(seed)
    Xs, us = [], []
    for ix in range(nx):
        for iy in range(ny):
            axis, d = helix_frame(n_bp, ((ix + 0.5) * spacing, (iy + 0.5) * spacing, 0.5 * spacing), (0, 0, 1), (1, 0, 0),
                                  phase0=rng.uniform(0.0, 2.0 * math.pi))
            X, u = place(axis, d)
            Xs.append(X); us.append(u)
    X = np.concatenate(Xs); u = np.concatenate(us)
    n = np.full(nx * ny, n_bp, np.int32)
    V, Om = maxwell(u, rng)
    box = (nx * spacing, ny * spacing, n_bp * RISE + spacing)
    return Config("paper_array_%dx%dx%dbp" % (nx, ny, n_bp), n, X, u, V, Om, box=box)


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
