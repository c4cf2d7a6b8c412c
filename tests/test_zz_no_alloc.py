"""The force entry point that allocates nothing (dsdna_forces_noalloc).

It serves callers that cannot call cudaMalloc (device memory wholly owned by
another pool allocator, or loops that cannot afford the synchronisation of an
allocation): its scratch lives in a fixed device array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL, ABS = 1e-5, 5e-4   # the mixed-precision force bound used by the parity tests


def _call(L, p, n_bp, X, u, Fb, Fp, stream):
    nb = np.ascontiguousarray(n_bp, dtype=np.int32)
    return L.dsdna_forces_noalloc(C.byref(p), len(nb), nb.ctypes.data_as(C.POINTER(C.c_int)), C.c_void_p(X.data_ptr()),
                                  C.c_void_p(u.data_ptr()), C.c_void_p(Fb.data_ptr()), C.c_void_p(Fp.data_ptr()),
                                  C.c_void_p(stream))


@pytest.mark.parametrize("which", ["periodic", "ragged", "bubbles", "small_box"])
def test_noalloc_forces_equal_the_context_path_on_two_calls(which):
    """Periodic box with a linear cell table, open box with the hashed table,
    a periodic box with fewer than 3 cells on one edge (the Morton table:
    molecules meet their own periodic images along z), and the Sec. 5 bubble
    rule on (open runs of 3-5 base pairs), which the no-alloc call evaluates
    in the kernel instance that has it."""
    import torch
    assert torch.cuda.is_available()
    kw = {}
    if which == "periodic":
        cfg = I.random_walk_helix(n_bp=3000, phi=0.15, clearance=1.7, seed=2)
    elif which == "small_box":
        cfg = I.ragged_batch([10, 6, 9], seed=7, spread=0.02)
        cfg.box = (5.0, 5.0, 4.0)    # 3 x 3 x 2 cells of 1.43 nm
    else:
        cfg = I.ragged_batch([700, 1, 129, 2500, 40], seed=6, spread=0.03)
    if which == "bubbles":
        for k in (10, 11, 12, 200, 201, 202, 203, 204, 900, 901, 902):
            r = cfg.X[2 * k + 1] - cfg.X[2 * k]
            cfg.X[2 * k + 1] += 0.5 * r / np.linalg.norm(r)
        kw = dict(bubble_rule=1, R0=3.0)
    assert cfg.n_nt <= 16384
    p = D.dsdna_default_params(box=cfg.box, **kw)
    ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
    Fb_ref, Fp_ref = ctx.compute_forces()
    Xs, _, us, _ = ctx.get_state()
    ctx.close()
    L = D.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    Xd = torch.tensor(cfg.X, dtype=torch.float64, device=dev).contiguous()
    ud = torch.tensor(cfg.u, dtype=torch.float64, device=dev).contiguous()
    out = []
    for call in range(2):
        Fb = torch.full((cfg.n_nt, 3), float("nan"), dtype=torch.float64, device=dev)
        Fp = torch.full((cfg.n_nt, 3), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call(L, p, cfg.n_bp, Xd, ud, Fb, Fp, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == 0, rc
        if call == 1:
            assert free_after == free_before, "the second call changed the free device memory"
        out.append((Fb.cpu().numpy(), Fp.cpu().numpy()))
    po = O.params(box=cfg.box, **kw) if cfg.box[0] > 0 else O.params(**kw)
    Sb, Sp = O.force_scale(po, cfg.n_bp, Xs, us)
    if which in ("bubbles", "small_box"):   # the context path matches the oracle here too
        ro = O.forces(po, cfg.n_bp, Xs, us)
        assert (np.linalg.norm(Fb_ref - ro["Fb"], axis=1) <= REL * Sb + ABS).all()
    if which == "small_box":     # the pairs across the short edge are there
        assert O.forces(po, cfg.n_bp, Xs, us)["energy"][:, 3].sum() > 1.0
    for Fb, Fp in out:
        assert (np.linalg.norm(Fb - Fb_ref, axis=1) <= REL * Sb + ABS).all()
        assert (np.linalg.norm(Fp - Fp_ref, axis=1) <= REL * Sp + ABS).all()
    # the second call starts from the first call's leftovers in the shared array
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_noalloc_rejects_inputs_beyond_its_fixed_scratch():
    import torch
    L = D.load()
    p = D.dsdna_default_params()
    n_bp = [8193]                     # 16386 nucleotides > DSDNA_NOALLOC_MAX_NT
    X = torch.zeros((2 * 8193, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(X)
    assert _call(L, p, n_bp, X, X, F, F, 0) == -1
    p2 = D.dsdna_default_params(box=(200.0, 200.0, 200.0))   # wider than 32 cells
    assert _call(L, p2, [100], X, X, F, F, 0) == -1
    p3 = D.dsdna_default_params(precision=D.PREC_FP64)
    assert _call(L, p3, [100], X, X, F, F, 0) == -1
    for bad in (dict(skin=-0.1), dict(skin=1.5), dict(bubble_rule=3), dict(steric_phase=3), dict(steric_phase=-1)):
        assert _call(L, D.dsdna_default_params(**bad), [100], X, X, F, F, 0) == -1, bad
