"""Pins for the FP64 count-predictor oracle."""
import numpy as np

from oracle import mlp


def small_net(seed=0, d_in=5, width=7):
    rng = np.random.default_rng(seed)
    n = mlp.layout(d_in, width)["total"]
    p = rng.standard_normal(n) * 0.4
    X = rng.standard_normal((9, d_in))
    y = rng.standard_normal(9)
    return p, X, y, d_in, width


def test_gradient_matches_finite_differences():
    p, X, y, d_in, width = small_net()
    mean, scale = X.mean(0), X.std(0) + 0.5
    loss, g = mlp.loss_and_grad(p, X, y, mean, scale, d_in, width, round_weights=False)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = mlp.loss_and_grad(p + e, X, y, mean, scale, d_in, width, round_weights=False)
        lm, _ = mlp.loss_and_grad(p - e, X, y, mean, scale, d_in, width, round_weights=False)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-6 * max(1.0, abs(g[k]))


def test_gelu_derivative_and_values():
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    assert np.allclose((mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), mlp.gelu_grad(x), atol=1e-8)
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu(10.0) - 10.0) < 1e-12


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 rounds to 1 (tie, to even), 1 + 3*2^-8 to 1 + 2^-6
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3.14159265])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == 1 + 2 ** -7
    assert r[4] == -2.5 and abs(r[5] - 3.140625) < 1e-12


def test_linear_special_case():
    # a network whose hidden layers see only tiny inputs acts almost linearly:
    # gelu(z) ~ z/2 near 0, so out ~ W3 (W2 (W1 x)/2)/2 + b3
    d_in, width = 3, 4
    o = mlp.layout(d_in, width)
    p = np.zeros(o["total"])
    rng = np.random.default_rng(2)
    W1 = rng.standard_normal((width, d_in)) * 1e-4
    W2 = rng.standard_normal((width, width))
    W3 = rng.standard_normal(width)
    p[o["W1"][0]:o["W1"][1]] = W1.ravel()
    p[o["W2"][0]:o["W2"][1]] = W2.ravel()
    p[o["W3"][0]:o["W3"][1]] = W3
    x = rng.standard_normal((2, d_in))
    out, _ = mlp.forward(p, x, 0.0, 1.0, d_in, width, round_weights=False)
    lin = (W3 @ (W2 @ (W1 @ x.T) / 2) / 2)
    assert np.allclose(out, lin, rtol=1e-3)


def test_adam_first_step_is_lr_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 5.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-6)
