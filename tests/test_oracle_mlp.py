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


def test_bf16_operand_mode_rounds_each_contraction_operand():
    """operands="bf16" (the kernels' contract: BF16 operands, exact sums) on a
    network wired as a chain through unit 0 -- W1 = e0 e0^T, W2 = identity,
    W3 = e0^T, zero biases, inputs not normalised -- so its output and the
    gradient of W2[0][0] follow in closed form from GELU and BF16 rounding:
    o0 = bf16(gelu(bf16(gelu(bf16(x0))))) and
    dW2[0][0] = bf16(bf16(do0) gelu'(z2_0)) bf16(h1_0), where exact arithmetic
    has no bf16().  One row, input pi and target 0."""
    d = M.unpack(np.zeros(M.NP))
    d["W1"][0, 0] = 1.0
    d["W2"] = np.eye(M.NH)
    d["W3"][0, 0] = 1.0
    p = M.pack(d)
    n = dict(in_mean=np.zeros(4), in_scale=np.ones(4), out_mean=np.zeros(3), out_scale=np.ones(3))
    X = np.array([[math.pi, 0.0, 0.0, 0.0]])
    T = np.zeros((1, 3))
    h1 = M.gelu(M.bf16(math.pi))
    z2 = M.bf16(h1)
    o0 = M.bf16(M.gelu(z2))
    y, _ = M.forward(p, X, n, operands="bf16")
    assert y[0, 0] == o0 and y[0, 0] != M.gelu(M.gelu(math.pi))
    _, g = M.loss_and_grad(p, X, T, n, operands="bf16")
    do0 = 2.0 * o0 / 3.0
    want = M.bf16(M.bf16(do0) * M.gelu_d(z2)) * M.bf16(h1)
    assert M.unpack(g)["W2"][0, 0] == want
    # exact arithmetic keeps every operand
    _, ge = M.loss_and_grad(p, X, T, n)
    he = M.gelu(math.pi); oe = M.gelu(M.gelu(math.pi))
    assert abs(M.unpack(ge)["W2"][0, 0] - 2.0 * oe / 3.0 * M.gelu_d(he) * he) < 1e-15


def test_first_adam_step_has_closed_form():
    """From zero moments the bias-corrected first step is lr g / (|g| + eps),
    i.e. lr sign(g) for |g| >> eps, plus lr wd p on the weights only."""
    rng = np.random.default_rng(4)
    p = rng.normal(0, 1, M.NP)
    g = rng.normal(0, 1, M.NP)
    lr, wd = 1e-2, 0.1
    p1, m1, v1 = M.adam_step(p, np.zeros(M.NP), np.zeros(M.NP), g, 1, lr, weight_decay=wd)
    w = M.weight_mask()
    want = p - lr * (g / (np.abs(g) + 1e-8) + wd * w * p)
    assert np.allclose(p1, want, rtol=0, atol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    d = M.unpack(w)
    assert d["W2"].all() and not d["b2"].any() and d["W3"].all() and not d["b3"].any()
    assert w.sum() == 64 * 4 + 64 * 64 + 3 * 64


def test_adam_moments_follow_their_recurrences():
    """Constant gradient: after t steps m = (1 - beta1^t) g and v = (1 - beta2^t) g^2,
    so the bias-corrected step stays lr g / (|g| + eps) every step."""
    g = np.linspace(-2, 2, M.NP) + 0.01
    p = np.zeros(M.NP); m = np.zeros(M.NP); v = np.zeros(M.NP)
    for t in range(1, 6):
        p_prev = p
        p, m, v = M.adam_step(p, m, v, g, t, 1e-3)
        assert np.allclose(m, (1 - 0.9 ** t) * g) and np.allclose(v, (1 - 0.999 ** t) * g * g)
        assert np.allclose(p_prev - p, 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
