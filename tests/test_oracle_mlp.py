"""Pins of the FP64 surrogate reference (oracle/mlp.py)."""
import math

import numpy as np

from oracle import mlp as M


def _norm():
    return dict(in_mean=np.array([5.0, 0.0, 1e4, 1.1]), in_scale=np.array([3.0, 3.0, 5e3, 0.2]),
                out_mean=np.array([0.5, 0.0, 0.05]), out_scale=np.array([0.2, 0.05, 0.05]))


def test_gelu_identities():
    """GELU(z) = z Phi(z): zero at 0, odd part z/2, tends to z and 0 at the tails; derivative 1/2 at 0."""
    z = np.array([0.0, 8.0, -8.0, 1.0])
    g = M.gelu(z)
    assert g[0] == 0.0 and abs(g[1] - 8.0) < 1e-12 and abs(g[2]) < 1e-12
    assert abs(g[3] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    assert abs(M.gelu_d(np.array([0.0]))[0] - 0.5) < 1e-15
    zz = np.linspace(-3, 3, 61)
    assert np.allclose(M.gelu(zz) - M.gelu(-zz), zz, atol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = M.init_params(3) + rng.normal(0, 0.05, M.NP)
    X = np.stack([rng.uniform(0.1, 10, 24), rng.uniform(-5, 5, 24), rng.uniform(500, 2e4, 24), rng.uniform(0.8, 1.4, 24)], 1)
    T = rng.normal(0, 0.1, (24, 3)) + _norm()["out_mean"]
    loss, g = M.loss_and_grad(p, X, T, _norm())
    idx = rng.choice(M.NP, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (M.loss_and_grad(pp, X, T, _norm())[0] - M.loss_and_grad(pm, X, T, _norm())[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_linear_limit_has_closed_form_gradient():
    """With W1, W2 zero the hidden layers are constant (GELU(0) = 0): the output is b3
    and the gradient of b3 is 2 mean(o - t_n) per output."""
    p = np.zeros(M.NP)
    d = M.unpack(p)
    d["b3"] = np.array([0.3, -0.2, 0.1])
    p = M.pack(d)
    X = np.ones((5, 4))
    T = np.tile([[0.5, 0.0, 0.05]], (5, 1))
    n = _norm()
    loss, g = M.loss_and_grad(p, X, T, n)
    tn = (T - n["out_mean"]) / n["out_scale"]
    want = 2.0 * (d["b3"][None, :] - tn).mean(0) / 3.0
    assert np.allclose(M.unpack(g)["b3"], want, atol=1e-15)
    assert np.allclose(M.unpack(g)["W2"], 0.0) and np.allclose(M.unpack(g)["W1"], 0.0)


def test_bf16_rounding():
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1.0 + 2 ** -9) == 1.0               # ties to even
    assert M.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    assert abs(M.bf16(math.pi) - math.pi) < 2 ** -8 * math.pi
