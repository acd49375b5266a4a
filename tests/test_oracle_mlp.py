"""Pins for the FP64 reference network of the learned surrogate: backpropagation against central
finite differences of the loss, and the activation's derivative against its closed form."""

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
    idx = np.unique(np.concatenate([np.arange(0, mlp.N_PARAMS, 97), np.arange(mlp.N_PARAMS - 70, mlp.N_PARAMS)]))
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
