"""The eigenvalue-count predictor in FP64 (test infrastructure).

d_in -> width -> width -> 1, GELU (tanh form) after the hidden layers, inputs
standardised by (x - mean)/scale, mean-squared-error loss, Adam.  The weights
used in the products are rounded to bfloat16 (round to nearest even), as in the
network under test; the arithmetic is FP64, so comparisons measure the FP32
accumulation of the GPU kernels.

Parameter vector layout: W1 (width x d_in, row-major), b1, W2, b2, W3 (1 x width), b3.
"""
import numpy as np

C_GELU = np.sqrt(2.0 / np.pi)


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(d_in, width):
    o = {}
    k = 0
    for name, size in (("W1", width * d_in), ("b1", width), ("W2", width * width), ("b2", width),
                       ("W3", width), ("b3", 1)):
        o[name] = (k, k + size)
        k += size
    o["total"] = k
    return o


def unpack(params, d_in, width, round_weights=True):
    o = layout(d_in, width)
    p = np.asarray(params, dtype=np.float64)
    get = lambda n: p[o[n][0]:o[n][1]]
    r = bf16_round if round_weights else (lambda a: np.asarray(a, dtype=np.float64))
    W1 = r(get("W1")).reshape(width, d_in)
    W2 = r(get("W2")).reshape(width, width)
    W3 = r(get("W3")).reshape(1, width)
    return W1, get("b1"), W2, get("b2"), W3, get("b3")


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    th = np.tanh(C_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * C_GELU * (1.0 + 3 * 0.044715 * x * x)


def forward(params, X, mean, scale, d_in, width, round_weights=True):
    W1, b1, W2, b2, W3, b3 = unpack(params, d_in, width, round_weights)
    x0 = (np.asarray(X, dtype=np.float64) - mean) / scale
    z1 = x0 @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    out = (h2 @ W3.T + b3)[:, 0]
    return out, (x0, z1, h1, z2, h2)


def loss_and_grad(params, X, y, mean, scale, d_in, width, round_weights=True):
    """(1/B) sum (net(x_b) - y_b)^2 and its gradient (the layout above)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, d_in, width, round_weights)
    out, (x0, z1, h1, z2, h2) = forward(params, X, mean, scale, d_in, width, round_weights)
    B = len(y)
    r = out - np.asarray(y, dtype=np.float64)
    loss = np.mean(r * r)
    dout = (2.0 * r / B)[:, None]
    gW3 = dout.T @ h2
    gb3 = dout.sum(0)
    d2 = (dout @ W3) * gelu_grad(z2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * gelu_grad(z1)
    gW1 = d1.T @ x0
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(params, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
