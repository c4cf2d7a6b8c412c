"""FP64 CPU oracle for the dsDNA model of arXiv:1608.03722 (Fosado et al.).

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library: plain double-precision C (``oracle.c``) behind ctypes.  It shares
no code with the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.

Host arrays are AoS ``(n_nt, 3)`` float64, slot ``g = 2*(bp_offset + k) + s``
(s = 0 strand A, s = 1 strand B), see ``oracle.h``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
NTERMS = 10
TERM_NAMES = ["fene", "bond_wca", "hbond", "wca", "dihedral", "morse", "planar", "bend", "kin_t", "kin_r"]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "K1", "R0", "eps_bb", "sigma_bb", "K2", "r0_hb", "rc_hb", "eps_ev", "sigma_ss", "sigma_cross",
        "K3", "d_dih", "K4", "lambda_m", "r0_m", "K5", "alpha0", "K6", "mass", "ell", "kT", "gamma", "dt")] + [
        ("seed", C.c_uint64), ("noise", C.c_int), ("steric_phase", C.c_int), ("box", C.c_double * 3),
        ("bubble_rule", C.c_int), ("K2_gc", C.c_double), ("gc", C.c_void_p), ("ring", C.c_void_p),
        ("removed", C.c_void_p), ("sigma_cross_steric", C.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (plain gcc, no GPU)."""
    src = os.path.join(HERE, "oracle.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        d = P(C.c_double)
        i32 = P(C.c_int)
        i64 = P(C.c_int64)
        L.or_default_params.argtypes = [P(Params)]
        L.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.or_ideal_helix.argtypes = [P(Params), C.c_int, d, d, d]
        L.or_mb_velocities.argtypes = [P(Params), C.c_int, C.c_int, d, C.c_int, d, d]
        for fn in (L.or_forces, L.or_forces_cells):
            fn.argtypes = [P(Params), C.c_int, i32, d, d, d, d, d, d, d, d, d, d]
            fn.restype = C.c_int
        L.or_forces_sampled.argtypes = [P(Params), C.c_int, i32, d, d, d, d, C.c_int, i64, d, d, d, d]
        L.or_force_scale.argtypes = [P(Params), C.c_int, i32, d, d, d, d, d, d]
        L.or_force_scale.restype = C.c_int
        L.or_forces_sampled.restype = C.c_int
        L.or_pairs.argtypes = [P(Params), C.c_int, i32, d, d, C.c_double, C.c_int64, i64, i64]
        L.or_pairs.restype = C.c_int64
        L.or_run.argtypes = [P(Params), C.c_int, i32, d, d, d, d, d, d, i32, C.c_int64, C.c_int64, C.c_int]
        L.or_run.restype = C.c_int
        L.or_energy.argtypes = [P(Params), C.c_int, i32, d, d, d, d, d, d, i32, C.c_int64, d, d]
        L.or_energy.restype = C.c_int
        L.or_observables.argtypes = [P(Params), C.c_int, i32, d, d, C.c_int, C.c_int, d]
        L.or_observables.restype = C.c_int
        L.or_linking_number.argtypes = [C.c_int, d, C.c_int, d]
        L.or_linking_number.restype = C.c_double
        _lib = L
    return _lib


def params(**kw) -> Params:
    """Table 1 defaults, overridden by keyword (``box=(L, L, L)`` for a periodic box)."""
    p = Params()
    lib().or_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "box":
            for c in range(3):
                p.box[c] = float(v[c])
        elif k == "removed":   # bubble rule 2 mask, uint8 per nucleotide, shared (or_run updates it in place)
            if v is not None:
                assert v.dtype == np.uint8 and v.flags.c_contiguous
            p._removed_keep = v
            p.removed = None if v is None else v.ctypes.data
        elif k in ("gc", "ring"):   # G.C flag per base pair / circular flag per molecule (kept alive with p)
            arr = None if v is None else np.ascontiguousarray(np.atleast_1d(v), dtype=np.int8)
            setattr(p, "_" + k + "_keep", arr)
            setattr(p, k, None if arr is None else arr.ctypes.data)
        else:
            setattr(p, k, v)
    return p


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError({-1: "EINVAL", -4: "EFENE"}.get(rc, str(rc)))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def ideal_helix(p: Params, n_bp: int, origin=(0.0, 0.0, 0.0)):
    X = np.zeros((2 * n_bp, 3))
    u = np.zeros((2 * n_bp, 3))
    o = np.asarray(origin, dtype=np.float64)
    lib().or_ideal_helix(C.byref(p), n_bp, _d(o), _d(X), _d(u))
    return X, u


def mb_velocities(p: Params, mol: int, n_bp: int, u, tether: int = 0):
    V = np.zeros((2 * n_bp, 3))
    Om = np.zeros((2 * n_bp, 3))
    lib().or_mb_velocities(C.byref(p), mol, n_bp, _d(np.ascontiguousarray(u)), int(tether), _d(V), _d(Om))
    return V, Om


def forces(p: Params, n_bp, X, u, ext_f=None, ext_t=None, cells=False):
    """Site forces, body force/torque, per-molecule energy terms and virial."""
    nb, nbp = _i32(np.atleast_1d(n_bp))
    n = X.shape[0]
    Fb = np.zeros((n, 3)); Fp = np.zeros((n, 3)); F = np.zeros((n, 3)); T = np.zeros((n, 3))
    E = np.zeros((len(nb), NTERMS)); W = np.zeros((len(nb), 6))
    ef = None if ext_f is None else np.ascontiguousarray(ext_f, dtype=np.float64)
    et = None if ext_t is None else np.ascontiguousarray(ext_t, dtype=np.float64)
    fn = lib().or_forces_cells if cells else lib().or_forces
    _check(fn(C.byref(p), len(nb), nbp, _d(X), _d(u), _d(ef), _d(et), _d(Fb), _d(Fp), _d(F), _d(T), _d(E), _d(W)))
    return dict(Fb=Fb, Fp=Fp, F=F, T=T, energy=E, virial=W)


def forces_sampled(p: Params, n_bp, X, u, idx, ext_f=None, ext_t=None, with_scale=False):
    nb, nbp = _i32(np.atleast_1d(n_bp))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    Fb = np.zeros((len(idx), 3)); Fp = np.zeros((len(idx), 3))
    Sb = np.zeros(len(idx)); Sp = np.zeros(len(idx))
    ef = None if ext_f is None else np.ascontiguousarray(ext_f, dtype=np.float64)
    et = None if ext_t is None else np.ascontiguousarray(ext_t, dtype=np.float64)
    _check(lib().or_forces_sampled(C.byref(p), len(nb), nbp, _d(X), _d(u), _d(ef), _d(et), len(idx),
                                   idx.ctypes.data_as(C.POINTER(C.c_int64)), _d(Fb), _d(Fp), _d(Sb), _d(Sp)))
    return (Fb, Fp, Sb, Sp) if with_scale else (Fb, Fp)


def force_scale(p: Params, n_bp, X, u, ext_f=None, ext_t=None):
    """Per-site sum over terms of |term force| (condition scale of a floating-point force sum)."""
    nb, nbp = _i32(np.atleast_1d(n_bp))
    n = X.shape[0]
    Sb = np.zeros(n); Sp = np.zeros(n)
    ef = None if ext_f is None else np.ascontiguousarray(ext_f, dtype=np.float64)
    et = None if ext_t is None else np.ascontiguousarray(ext_t, dtype=np.float64)
    _check(lib().or_force_scale(C.byref(p), len(nb), nbp, _d(X), _d(u), _d(ef), _d(et), _d(Sb), _d(Sp)))
    return Sb, Sp


def pairs(p: Params, n_bp, X, u, extra=0.0):
    """Brute-force set of interacting bead pairs (i<j) within r_cut(type) + extra."""
    nb, nbp = _i32(np.atleast_1d(n_bp))
    cnt = lib().or_pairs(C.byref(p), len(nb), nbp, _d(X), _d(u), float(extra), 0, None, None)
    pi = np.zeros(max(cnt, 1), dtype=np.int64); pj = np.zeros(max(cnt, 1), dtype=np.int64)
    lib().or_pairs(C.byref(p), len(nb), nbp, _d(X), _d(u), float(extra), cnt,
                   pi.ctypes.data_as(C.POINTER(C.c_int64)), pj.ctypes.data_as(C.POINTER(C.c_int64)))
    return np.stack([pi[:cnt], pj[:cnt]], axis=1)


def run(p: Params, n_bp, X, V, u, Om, nsteps, step0=0, ext_f=None, ext_t=None, tether=None, cells=False):
    """Advance the state in place by nsteps (half-step velocities)."""
    nb, nbp = _i32(np.atleast_1d(n_bp))
    ef = None if ext_f is None else np.ascontiguousarray(ext_f, dtype=np.float64)
    et = None if ext_t is None else np.ascontiguousarray(ext_t, dtype=np.float64)
    tt = None
    if tether is not None:
        tt, tptr = _i32(np.atleast_1d(tether))
    _check(lib().or_run(C.byref(p), len(nb), nbp, _d(X), _d(V), _d(u), _d(Om), _d(ef), _d(et),
                        None if tt is None else tptr, int(step0), int(nsteps), int(bool(cells))))


def energy(p: Params, n_bp, X, V, u, Om, step, ext_f=None, ext_t=None, tether=None):
    nb, nbp = _i32(np.atleast_1d(n_bp))
    E = np.zeros((len(nb), NTERMS)); W = np.zeros((len(nb), 6))
    ef = None if ext_f is None else np.ascontiguousarray(ext_f, dtype=np.float64)
    et = None if ext_t is None else np.ascontiguousarray(ext_t, dtype=np.float64)
    tptr = None
    if tether is not None:
        tt, tptr = _i32(np.atleast_1d(tether))
    _check(lib().or_energy(C.byref(p), len(nb), nbp, _d(X), _d(V), _d(u), _d(Om), _d(ef), _d(et), tptr,
                           int(step), _d(E), _d(W)))
    return E, W


def observables(p: Params, n_bp, X, u, mol=0, with_lk=False):
    """dict(rz, denat, tw, tw_ideal, lk, wr) of molecule ``mol``."""
    nb, nbp = _i32(np.atleast_1d(n_bp))
    out = np.zeros(6)
    _check(lib().or_observables(C.byref(p), len(nb), nbp, _d(X), _d(u), int(mol), int(bool(with_lk)), _d(out)))
    return dict(rz=out[0], denat=out[1], tw=out[2], tw_ideal=out[3], lk=out[4], wr=out[5])


def linking_number(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().or_linking_number(a.shape[0], _d(a), b.shape[0], _d(b))


def sites(p: Params, X, u):
    """Bead and patch positions (Sec. 2): X -/+ (ell/2) u."""
    return X - 0.5 * p.ell * u, X + 0.5 * p.ell * u
