"""FP64 reference of the learned surrogate's network (test infrastructure only).

A multilayer perceptron 3 -> 64 -> 64 -> 64 -> 1 with SiLU activations, written out in plain numpy:
forward pass, the training loss, and its gradient by backpropagation (reverse-mode chain rule,
one layer at a time).  The CUDA training kernels' gradients are checked against it; it is pinned
by central finite differences (tests/test_oracle_mlp.py).

Parameter vector layout (8,641 values, row-major):
    W1[64,3], b1[64], W2[64,64], b2[64], W3[64,64], b3[64], W4[1,64] (64), b4[1]
Inputs z[B,3] are the normalised (ln alpha, ln beta, logit u); the output y[B] is logit(x)/OUT_SCALE.
Loss per sample: LOSS_X * (sigmoid(OUT_SCALE*y) - x)^2 + LOSS_LOGIT * (y - t)^2 with t the clipped
logit target divided by OUT_SCALE, averaged over the batch.
"""

from __future__ import annotations

import numpy as np

H = 64
N_PARAMS = 3 * H + H + 2 * (H * H + H) + H + 1
OUT_SCALE = 20.0
LOSS_X = 100.0
LOSS_LOGIT = 1e-3


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (N_PARAMS,)
    o = 0
    out = []
    for shape in ((H, 3), (H,), (H, H), (H,), (H, H), (H,), (1, H), (1,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in parts])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, z):
    """Returns y[B] and the cache of pre-activations and activations."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    a1 = z @ W1.T + b1
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = silu(a2)
    a3 = h2 @ W3.T + b3
    h3 = silu(a3)
    y = (h3 @ W4.T + b4)[:, 0]
    return y, (z, a1, h1, a2, h2, a3, h3)


def loss_and_dy(y, x, t):
    s = 1.0 / (1.0 + np.exp(-OUT_SCALE * y))
    B = y.shape[0]
    loss = np.mean(LOSS_X * (s - x) ** 2 + LOSS_LOGIT * (y - t) ** 2)
    dy = (2.0 * LOSS_X * (s - x) * s * (1.0 - s) * OUT_SCALE + 2.0 * LOSS_LOGIT * (y - t)) / B
    return loss, dy


def backward(p, cache, dy):
    """Gradient of the loss with respect to the parameter vector, given dL/dy."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    z, a1, h1, a2, h2, a3, h3 = cache
    dW4 = dy[None, :] @ h3
    db4 = np.array([dy.sum()])
    dh3 = dy[:, None] * W4[0][None, :]
    da3 = dh3 * silu_grad(a3)
    dW3 = da3.T @ h2
    db3 = da3.sum(0)
    dh2 = da3 @ W3
    da2 = dh2 * silu_grad(a2)
    dW2 = da2.T @ h1
    db2 = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * silu_grad(a1)
    dW1 = da1.T @ z
    db1 = da1.sum(0)
    return pack([dW1, db1, dW2, db2, dW3, db3, dW4, db4])


def loss_grad(p, z, x, t):
    y, cache = forward(p, z)
    loss, dy = loss_and_dy(y, x, t)
    return loss, backward(p, cache, dy)


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H, 3), (H, H), (H, H), (1, H)):
        b = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-b, b, size=(fan_out, fan_in)))
        parts.append(rng.uniform(-b, b, size=(fan_out,)))
    return pack(parts)
