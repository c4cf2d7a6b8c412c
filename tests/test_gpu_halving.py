"""Pair halving (Newton's third law within a 32-slot tile of the step kernel):
a list pair whose nucleotides share a tile is evaluated once and the other
nucleotide takes its negative.  The pair force is antisymmetric bit for bit,
so forces and trajectories with halving equal those without it bit for bit;
the tiles must actually take the halved path."""
import numpy as np
import pytest

from paper_1608_03722_gb300 import dsdna as D
from paper_1608_03722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    yield


def _walk(n_bp=3000, seed=1):
    cfg = I.random_walk_helix(n_bp=n_bp, phi=0.15, clearance=1.7, seed=seed)
    cfg.X, cfg.u = I.perturb(cfg.X, cfg.u, np.random.default_rng(seed), dx=0.01, dtheta=0.02)
    return cfg


def _cases():
    open_cfg = I.c1_linear(400)
    open_cfg.X, open_cfg.u = I.perturb(open_cfg.X, open_cfg.u, np.random.default_rng(5), dx=0.03, dtheta=0.06)
    return {"periodic_walk": _walk(), "open_helix": open_cfg, "batch": I.ragged_batch([130, 1, 64, 257, 33, 500], seed=3)}


@pytest.mark.parametrize("name", ["periodic_walk", "open_helix", "batch"])
def test_halving_gives_the_same_forces_bit_for_bit(name):
    cfg = _cases()[name]
    out = []
    for ph in (0, 1):
        p = D.dsdna_default_params(box=cfg.box, rebuild_mode=1, pair_halving=ph)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
        out.append(ctx.compute_forces())
        info = ctx.info()
        ctx.close()
        if ph:
            assert info["halved_tiles"] > 0.9 * (info["n_nt"] + 31) // 32, info
        else:
            assert info["halved_tiles"] == 0
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_halving_gives_the_same_trajectory_bit_for_bit():
    """100 steps with skin 0.1 (a rebuild every few steps) in the periodic box."""
    cfg = _walk()
    st = []
    for ph in (0, 1):
        p = D.dsdna_default_params(box=cfg.box, rebuild_mode=1, pair_halving=ph, skin=0.1, seed=18)
        ctx = D.Context(p, cfg.n_bp, X=cfg.X, V=cfg.V, u=cfg.u, Om=cfg.Om)
        ctx.step(100)
        st.append(ctx.get_state())
        info = ctx.info()
        ctx.close()
        assert info["rebuilds"] > 5
    for a, b in zip(*st):
        assert np.array_equal(a, b)


def test_halving_is_the_default_for_large_mixed_systems():
    p = D.dsdna_default_params()
    assert p.pair_halving == 1
