"""Synthetic input generators: sizes and geometry of the benchmark workloads."""
import numpy as np

from paper_1608_03722_gb300 import inputs as I


def test_paper_array_geometry():
    """Sec. 6 benchmark: a 10 x 10 array of 600 bp strands is 60 kbp (1.2e5
    nucleotides); every nucleotide lies within the helix radius of its strand's
    axis, strands stand 5 nm apart, and all fit in the periodic box."""
    cfg = I.paper_array(10, 10, 600, spacing=5.0)
    assert cfg.n_nt == 120_000 and len(cfg.n_bp) == 100 and (cfg.n_bp == 600).all()
    X = cfg.X.reshape(100, 1200, 3)
    axes = X[:, :, :2].mean(1)
    r = np.linalg.norm(X[:, :, :2] - axes[:, None, :], axis=2)
    assert r.max() < 1.1
    d = np.linalg.norm(axes[:, None] - axes[None], axis=2) + np.eye(100) * 1e9
    assert abs(d.min() - 5.0) < 1e-6
    assert (cfg.X > 0).all() and (cfg.X < np.asarray(cfg.box)).all()
    assert abs(np.linalg.norm(cfg.u, axis=1) - 1).max() < 1e-12


def test_paper_array_full_size():
    cfg = I.paper_array(40, 40, 600)
    assert cfg.n_nt == 1_920_000 and cfg.box[0] == 200.0
