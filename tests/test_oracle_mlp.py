"""Pins for the FP64 reference network of the learned surrogate: the forward pass against closed
forms (a network with a single active path through chosen weight positions, evaluated by hand, and
the affine map the network reduces to where every pre-activation is far from zero),
backpropagation against central finite differences of the loss on every bias and a spread of
weights, and the activation's derivative against its closed form."""

import math

import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 8641  # 3*64+64 + 2*(64*64+64) + 64+1


def test_silu_derivative_closed_form():
    z = np.linspace(-30, 30, 2001)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=1e-7, atol=1e-9)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu(40.0) - 40.0) < 1e-12


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = mlp.init_params(3)
    B = 37
    z = rng.uniform(-1, 1, size=(B, 3))
    x = rng.uniform(0.01, 0.99, size=B)
    t = np.log(x / (1 - x)) / mlp.OUT_SCALE
    loss, g = mlp.loss_grad(p, z, x, t)
    # every bias and a spread of weights in each layer
    H = mlp.H
    o_b1 = 3 * H
    o_b2 = o_b1 + H + H * H
    o_b3 = o_b2 + H + H * H
    biases = np.concatenate([np.arange(o_b1, o_b1 + H), np.arange(o_b2, o_b2 + H),
                             np.arange(o_b3, o_b3 + H), [mlp.N_PARAMS - 1]])
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=np.float64))
    assert np.array_equal(np.concatenate([b1, b2, b3, b4]), biases)  # the offsets above
    idx = np.unique(np.concatenate([np.arange(0, mlp.N_PARAMS, 97), biases]))
    assert idx.size > 193 + 80
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_grad(p + e, z, x, t)
        lm, _ = mlp.loss_grad(p - e, z, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_pack_roundtrip():
    p = mlp.init_params(1)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def _params(W1, b1, W2, b2, W3, b3, W4, b4):
    return mlp.pack([W1, b1, W2, b2, W3, b3, W4, b4])


def _silu(v: float) -> float:
    return v / (1.0 + math.exp(-v))


def test_forward_single_path_by_hand():
    """Only input 1 -> hidden unit 5 -> unit 7 -> unit 2 -> output carries a signal; every other
    unit sees a zero pre-activation (SiLU(0) = 0) or a bias alone.  A transposed weight matrix, a
    wrong input column, a dropped bias or another activation changes the result."""
    H = mlp.H
    W1 = np.zeros((H, 3)); b1 = np.zeros(H)
    W2 = np.zeros((H, H)); b2 = np.zeros(H)
    W3 = np.zeros((H, H)); b3 = np.zeros(H)
    W4 = np.zeros((1, H)); b4 = np.zeros(1)
    W1[5, 1], b1[5] = 1.5, -0.25
    W2[7, 5], b2[7] = -2.0, 0.5
    W3[2, 7], b3[2] = 3.0, -0.75
    W4[0, 2], b4[0] = 0.8, 0.125
    b2[11] = 1.25  # a unit fed by its bias alone, which the output does not read
    p = _params(W1, b1, W2, b2, W3, b3, W4, b4)
    zs = np.array([[0.3, -0.7, 0.9], [-1.0, 0.4, 0.0], [0.5, 1.0, -0.5]])
    y, cache = mlp.forward(p, zs)
    for r, (z0, z1, z2) in enumerate(zs):
        h1 = _silu(1.5 * z1 - 0.25)
        h2 = _silu(-2.0 * h1 + 0.5)
        h3 = _silu(3.0 * h2 - 0.75)
        assert abs(y[r] - (0.8 * h3 + 0.125)) <= 1e-15
        assert abs(cache[4][r, 11] - _silu(1.25)) <= 1e-15  # h2 of the bias-only unit
        assert np.count_nonzero(cache[2][r]) == 1  # h1: unit 5 only


def test_forward_reduces_to_its_affine_map():
    """With positive weights and inputs and biases of +40 every pre-activation exceeds 40, where
    SiLU(v) = v to binary64 precision: the network is then the affine map W4 W3 W2 W1 z + c,
    computed here by composing the matrices first (another association of the products).  With
    biases of -60 every hidden unit is off and the output is b4."""
    H = mlp.H
    rng = np.random.default_rng(11)
    W1 = rng.uniform(0.1, 1.0, (H, 3)); W2 = rng.uniform(0.0, 0.05, (H, H))
    W3 = rng.uniform(0.0, 0.05, (H, H)); W4 = rng.uniform(-1.0, 1.0, (1, H))
    b1 = np.full(H, 40.0); b2 = np.full(H, 40.0); b3 = np.full(H, 40.0); b4 = np.array([0.3])
    z = rng.uniform(0.0, 1.0, (25, 3))
    y, cache = mlp.forward(_params(W1, b1, W2, b2, W3, b3, W4, b4), z)
    assert min(cache[1].min(), cache[3].min(), cache[5].min()) >= 40.0
    M = W4 @ W3 @ W2 @ W1
    c = W4 @ (W3 @ (W2 @ b1 + b2) + b3) + b4
    np.testing.assert_allclose(y, (z @ M.T)[:, 0] + c[0], rtol=1e-12)
    off = _params(W1, np.full(H, -60.0), W2, np.full(H, -60.0), W3, np.full(H, -60.0), W4, b4)
    y0, _ = mlp.forward(off, z)
    np.testing.assert_allclose(y0, 0.3, atol=1e-20 + 64 * 60 * math.exp(-50))
