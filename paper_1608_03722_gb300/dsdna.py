"""Python binding of the dsDNA engine C ABI (include/dsdna.h).

Argument marshalling only: every computation runs in ``libdsdna.so``.  The
functions carry the C names (``dsdna_create``, ``dsdna_step``, ...); the
``Context`` class wraps them for convenience.  PyTorch provides the device
memory (caching allocator) and the CUDA stream.  There is no fallback: if the
library is missing or cannot load, importing this module's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

NTERMS = 10
TERM_NAMES = ["fene", "bond_wca", "hbond", "wca", "dihedral", "morse", "planar", "bend", "kin_t", "kin_r"]
(E_FENE, E_BONDWCA, E_HBOND, E_WCA, E_DIHEDRAL, E_MORSE, E_PLANAR, E_BEND, E_KIN_T, E_KIN_R) = range(NTERMS)
PREC_MIXED, PREC_FP64 = 0, 1
NOISE_OFF, NOISE_UNIFORM, NOISE_GAUSSIAN = 0, 1, 2
OBS_EXT, OBS_DENAT, OBS_TW, OBS_LK = 1, 2, 4, 8
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EFENE", -5: "ENAN", -6: "EOVERFLOW",
          -7: "ETIMEOUT", -8: "ESTATE"}

_PARAM_DOUBLES = ("K1", "R0", "eps_bb", "sigma_bb", "K2", "r0_hb", "rc_hb", "eps_ev", "sigma_ss", "sigma_cross",
                  "K3", "d_dih", "K4", "lambda_m", "r0_m", "K5", "alpha0", "K6", "mass", "ell", "kT", "gamma", "dt")


class dsdna_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in _PARAM_DOUBLES] + [
        ("seed", C.c_uint64), ("noise", C.c_int), ("steric_phase", C.c_int), ("box", C.c_double * 3),
        ("skin", C.c_double), ("precision", C.c_int), ("max_neighbors", C.c_int), ("block_threads", C.c_int),
        ("blocks_per_sm", C.c_int), ("steps_per_graph", C.c_int), ("bubble_rule", C.c_int), ("K2_gc", C.c_double),
        ("rebuild_mode", C.c_int), ("sigma_cross_steric", C.c_double), ("pair_halving", C.c_int),
        ("list_build", C.c_int)]


class dsdna_system(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("n_bp", C.POINTER(C.c_int)), ("X", C.POINTER(C.c_double)),
                ("V", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)), ("Om", C.POINTER(C.c_double)),
                ("tether", C.POINTER(C.c_int)), ("gc", C.POINTER(C.c_byte)), ("circular", C.POINTER(C.c_int))]


def _system(n_bp, X, V, u, Om, tether, gc, circular=None):
    """dsdna_system for the given arrays; returns (struct, arrays to keep alive)."""
    nb = np.ascontiguousarray(np.atleast_1d(n_bp), dtype=np.int32)
    n = 2 * int(nb.sum())
    X, V, u, Om = _f64(X, n), _f64(V, n), _f64(u, n), _f64(Om, n)
    tt = None if tether is None else np.ascontiguousarray(np.atleast_1d(tether), dtype=np.int32)
    gg = None if gc is None else np.ascontiguousarray(np.asarray(gc) != 0, dtype=np.int8)
    if gg is not None and gg.size != n // 2:
        raise ValueError(f"gc needs one flag per base pair ({n // 2}), got {gg.size}")
    cc = None if circular is None else np.ascontiguousarray(np.atleast_1d(circular), dtype=np.int32)
    if cc is not None and cc.size != nb.size:
        raise ValueError(f"circular needs one flag per molecule ({nb.size}), got {cc.size}")
    sys = dsdna_system(len(nb), nb.ctypes.data_as(C.POINTER(C.c_int)), _dp(X), _dp(V), _dp(u), _dp(Om),
                       None if tt is None else tt.ctypes.data_as(C.POINTER(C.c_int)),
                       None if gg is None else gg.ctypes.data_as(C.POINTER(C.c_byte)),
                       None if cc is None else cc.ctypes.data_as(C.POINTER(C.c_int)))
    return sys, (nb, X, V, u, Om, tt, gg, cc)


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class dsdna_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", C.c_void_p)]


class dsdna_obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rz", "denat", "tw", "tw_ideal", "lk", "wr")]


class dsdna_info(C.Structure):
    _fields_ = [("n_nt", C.c_int64), ("n_mol", C.c_int), ("step", C.c_int64), ("rebuilds", C.c_int64),
                ("grid_blocks", C.c_int), ("block_threads", C.c_int), ("max_neighbors", C.c_int),
                ("precision", C.c_int), ("skin", C.c_double), ("cell_table", C.c_int64),
                ("device_bytes", C.c_int64), ("engine_launches", C.c_int64), ("rebuild_in_step", C.c_int),
                ("halved_tiles", C.c_int64), ("chain_list", C.c_int)]


class dsdna_prof(C.Structure):
    _fields_ = [("steps", C.c_int64), ("engine_launches", C.c_int64), ("engine_ms", C.c_double),
                ("rebuild_launches", C.c_int64), ("rebuild_ms", C.c_double)]


EXPORTS = ["dsdna_default_params", "dsdna_create", "dsdna_set_external_force_torque", "dsdna_step",
           "dsdna_step_profiled", "dsdna_synchronize", "dsdna_energy_virial", "dsdna_observables", "dsdna_get_state", "dsdna_set_state",
           "dsdna_compute_forces", "dsdna_neighbor_pairs", "dsdna_get_info", "dsdna_step_counter",
           "dsdna_last_error", "dsdna_destroy", "dsdna_forces_noalloc", "dsdna_autotune", "dsdna_profiles",
           "dsdna_get_bubble_mask", "dsdna_set_bubble_mask"]

_lib = None


def load(build_if_missing: bool = True):
    """Load libdsdna.so (building it from source if absent); raise if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise RuntimeError("libdsdna.so is not built")
        _build.build()
    L = C.CDLL(_build.LIB)
    P = C.POINTER
    d = P(C.c_double)
    L.dsdna_default_params.argtypes = [P(dsdna_params)]
    L.dsdna_default_params.restype = None
    L.dsdna_create.argtypes = [P(dsdna_params), P(dsdna_system), P(dsdna_allocator), C.c_void_p, P(C.c_void_p)]
    L.dsdna_set_external_force_torque.argtypes = [C.c_void_p, C.c_int, d, d]
    L.dsdna_step.argtypes = [C.c_void_p, C.c_int64]
    L.dsdna_step_profiled.argtypes = [C.c_void_p, C.c_int64, P(dsdna_prof)]
    L.dsdna_synchronize.argtypes = [C.c_void_p]
    L.dsdna_energy_virial.argtypes = [C.c_void_p, C.c_int, d, d]
    L.dsdna_observables.argtypes = [C.c_void_p, C.c_int, C.c_uint, P(dsdna_obs)]
    L.dsdna_get_state.argtypes = [C.c_void_p, C.c_int, d, d, d, d]
    L.dsdna_profiles.argtypes = [C.c_void_p, C.c_int, d, d]
    L.dsdna_set_state.argtypes = [C.c_void_p, C.c_int, d, d, d, d]
    L.dsdna_compute_forces.argtypes = [C.c_void_p, d, d]
    L.dsdna_get_bubble_mask.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    L.dsdna_set_bubble_mask.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    L.dsdna_neighbor_pairs.argtypes = [C.c_void_p, C.c_int64, P(C.c_int64), P(C.c_int64), P(C.c_int64)]
    L.dsdna_get_info.argtypes = [C.c_void_p, P(dsdna_info)]
    L.dsdna_step_counter.argtypes = [C.c_void_p]
    L.dsdna_step_counter.restype = C.c_int64
    L.dsdna_last_error.argtypes = [C.c_void_p]
    L.dsdna_last_error.restype = C.c_char_p
    L.dsdna_destroy.argtypes = [C.c_void_p]
    L.dsdna_destroy.restype = None
    L.dsdna_forces_noalloc.argtypes = [P(dsdna_params), C.c_int, P(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    L.dsdna_forces_noalloc.restype = C.c_int
    L.dsdna_autotune.argtypes = [P(dsdna_params), P(dsdna_system), P(dsdna_allocator), C.c_void_p, C.c_int,
                                 P(dsdna_params), P(C.c_double)]
    L.dsdna_autotune.restype = C.c_int
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is C.c_int or name in ("dsdna_create",):
            fn.restype = C.c_int
    _lib = L
    return L


class DsdnaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, "expected C-contiguous float64"
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == 3 * n, f"expected {n} x 3 values"
    return a


def dsdna_default_params(**overrides) -> dsdna_params:
    """Table 1 / Sec. 2 / App. A defaults, with keyword overrides (box=(L, L, L))."""
    p = dsdna_params()
    load().dsdna_default_params(C.byref(p))
    for k, v in overrides.items():
        if k == "box":
            for c in range(3):
                p.box[c] = float(v[c])
        else:
            setattr(p, k, v)
    return p


def _check(ctx, rc):
    if rc != 0:
        raise DsdnaError(rc, load().dsdna_last_error(ctx).decode(errors="replace"))


class _TorchAllocator:
    """Routes the engine's device allocations through PyTorch's caching allocator."""

    def __init__(self, stream: int):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None
            self.live[int(p)] = int(nbytes)
            return int(p)

        def _release(ptr, user):
            if ptr and int(ptr) in self.live:
                del self.live[int(ptr)]
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_cb = ALLOC_FN(_alloc)
        self.release_cb = RELEASE_FN(_release)
        self.struct = dsdna_allocator(self.alloc_cb, self.release_cb, None)


def dsdna_create(params: dsdna_params, n_bp, X=None, V=None, u=None, Om=None, tether=None, stream=None,
                 allocator="torch", gc=None, circular=None):
    """Create a context; returns (handle, keepalive).  X/u and V/Om are (n_nt, 3) arrays or None;
    gc is one flag per base pair (1 = G.C, hydrogen-bond stiffness K2_gc) or None; circular one
    flag per molecule (1 = ring) or None."""
    L = load()
    sys, _keep = _system(n_bp, X, V, u, Om, tether, gc, circular)
    alloc = None
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if allocator == "torch":
        alloc = _TorchAllocator(stream)
    h = C.c_void_p()
    rc = L.dsdna_create(C.byref(params), C.byref(sys), C.byref(alloc.struct) if alloc else None,
                        C.c_void_p(stream), C.byref(h))
    _check(None, rc)
    return h, alloc


def dsdna_autotune(params: dsdna_params, n_bp, X=None, V=None, u=None, Om=None, tether=None, trial_steps=50,
                   stream=None, allocator="torch", gc=None, circular=None):
    """Fastest (skin, CTA size, CTAs per SM) for this system; returns (params, ns per nucleotide-step)."""
    L = load()
    sys, _keep = _system(n_bp, X, V, u, Om, tether, gc, circular)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    alloc = _TorchAllocator(stream) if allocator == "torch" else None
    best = dsdna_params()
    ns = C.c_double()
    rc = L.dsdna_autotune(C.byref(params), C.byref(sys), C.byref(alloc.struct) if alloc else None, C.c_void_p(stream),
                          int(trial_steps), C.byref(best), C.byref(ns))
    _check(None, rc)
    return best, ns.value


class Context:
    """One engine context on the current CUDA device and stream."""

    def __init__(self, params: dsdna_params, n_bp, X=None, V=None, u=None, Om=None, tether=None, stream=None,
                 allocator="torch", gc=None, circular=None):
        self.lib = load()
        self.params = params
        self.n_bp = np.ascontiguousarray(np.atleast_1d(n_bp), dtype=np.int32)
        self.n_nt = 2 * int(self.n_bp.sum())
        self.off = np.concatenate([[0], np.cumsum(self.n_bp)]).astype(np.int64)
        self.circular = np.zeros(len(self.n_bp), np.int32) if circular is None else np.asarray(circular, np.int32)
        self.h, self._alloc = dsdna_create(params, self.n_bp, X, V, u, Om, tether, stream, allocator, gc, circular)

    def _mol_len(self, mol):
        return self.n_nt if mol < 0 else 2 * int(self.n_bp[mol])

    def set_external_force_torque(self, mol, force, torque):
        f = _f64(force); t = _f64(torque)
        _check(self.h, self.lib.dsdna_set_external_force_torque(self.h, int(mol), _dp(f), _dp(t)))

    def step(self, nsteps):
        _check(self.h, self.lib.dsdna_step(self.h, int(nsteps)))

    def step_profiled(self, nsteps):
        """dsdna_step_profiled: same steps, every launch timed with CUDA events."""
        pr = dsdna_prof()
        _check(self.h, self.lib.dsdna_step_profiled(self.h, int(nsteps), C.byref(pr)))
        return {k: getattr(pr, k) for k, _ in dsdna_prof._fields_}

    def synchronize(self):
        _check(self.h, self.lib.dsdna_synchronize(self.h))

    def energy_virial(self, mol=-1):
        E = np.zeros(NTERMS); W = np.zeros(6)
        _check(self.h, self.lib.dsdna_energy_virial(self.h, int(mol), _dp(E), _dp(W)))
        return E, W

    def observables(self, mol=0, flags=OBS_EXT | OBS_DENAT | OBS_TW):
        o = dsdna_obs()
        _check(self.h, self.lib.dsdna_observables(self.h, int(mol), int(flags), C.byref(o)))
        return dict(rz=o.rz, denat=o.denat, tw=o.tw, tw_ideal=o.tw_ideal, lk=o.lk, wr=o.wr)

    def profiles(self, mol=0):
        """dsdna_profiles: (centre [N, 3], twist increments [N-2], or [N] on a ring)."""
        N = int(self.n_bp[mol])
        cen = np.zeros((N, 3)); tw = np.zeros(N if self.circular[mol] else max(0, N - 2))
        _check(self.h, self.lib.dsdna_profiles(self.h, int(mol), _dp(cen), _dp(tw)))
        return cen, tw

    def get_state(self, mol=-1, out=None):
        n = self._mol_len(mol)
        if out is None:
            out = tuple(np.zeros((n, 3)) for _ in range(4))
        _check(self.h, self.lib.dsdna_get_state(self.h, int(mol), *[_dp(a) for a in out]))
        return out

    def set_state(self, mol=-1, X=None, V=None, u=None, Om=None):
        n = self._mol_len(mol)
        arrs = [_f64(a, n) for a in (X, V, u, Om)]
        _check(self.h, self.lib.dsdna_set_state(self.h, int(mol), *[_dp(a) for a in arrs]))

    def get_bubble_mask(self, mol=-1):
        """dsdna_get_bubble_mask: uint8 per nucleotide (bit 0 dihedral, bit 1 bending removed)."""
        m = np.zeros(self._mol_len(mol), np.uint8)
        _check(self.h, self.lib.dsdna_get_bubble_mask(self.h, int(mol), m.ctypes.data_as(C.c_void_p)))
        return m

    def set_bubble_mask(self, mask, mol=-1):
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        if m is not None and m.size != self._mol_len(mol):
            raise ValueError("bubble mask needs one byte per nucleotide")
        _check(self.h, self.lib.dsdna_set_bubble_mask(self.h, int(mol), None if m is None else m.ctypes.data_as(C.c_void_p)))

    def compute_forces(self):
        Fb = np.zeros((self.n_nt, 3)); Fp = np.zeros((self.n_nt, 3))
        _check(self.h, self.lib.dsdna_compute_forces(self.h, _dp(Fb), _dp(Fp)))
        return Fb, Fp

    def neighbor_pairs(self):
        cnt = C.c_int64()
        _check(self.h, self.lib.dsdna_neighbor_pairs(self.h, 0, None, None, C.byref(cnt)))
        k = max(1, cnt.value)
        pi = np.zeros(k, np.int64); pj = np.zeros(k, np.int64)
        _check(self.h, self.lib.dsdna_neighbor_pairs(self.h, k, pi.ctypes.data_as(C.POINTER(C.c_int64)),
                                                     pj.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(cnt)))
        return np.stack([pi[:cnt.value], pj[:cnt.value]], axis=1)

    def info(self):
        i = dsdna_info()
        _check(self.h, self.lib.dsdna_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in dsdna_info._fields_}

    @property
    def step_counter(self):
        return self.lib.dsdna_step_counter(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dsdna_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
