"""The surrogate network as the tensor-core kernels compute it, in binary64 with their rounding
points (test infrastructure: the GPU tests compare the kernels with it element by element).

Rounding points of the training kernels: inputs z, the weights of the three hidden layers, the
layer-1 and layer-2 activations and the back-propagated layer gradients dZ are BF16 (round to
nearest even); accumulation, biases, the layer-3 activations, the output layer, the loss and the
bias gradients are FP32.  The inference kernels (evaluation, certification, the trial kernel)
carry inputs and layer-1/2 activations as FP32 values split into hi = bf16(v) and
lo = bf16(v - hi) (split=True).  SiLU is z(1 + tanh(z/2))/2 with the hardware tanh, whose error (about 2^-11
relative) the comparison cannot reproduce: element-wise bounds are drawn instead from repeated
emulations with tanh perturbed by a relative 2^-10 (which also moves the BF16 roundings it can
flip), see bounds().
"""

import numpy as np

from oracle import mlp as ref


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def split(v):
    """hi + lo of the inference kernels: the FP32 value v as bf16(v) + bf16(v - bf16(v))."""
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    hi = bf16(v)
    return hi + bf16(v - hi)


def emulate(p, z, x=None, t=None, tanh_err=0.0, rng=None, split_ops=False):
    """y (and, with x and t, the loss and the gradient) of the kernels' arithmetic; split_ops:
    the inference kernels' hi + lo operands."""
    W1, b1, W2, b2, W3, b3, W4, b4 = ref.unpack(p)

    def tanh(v):
        r = np.tanh(v)
        if tanh_err:
            r = r * (1.0 + tanh_err * rng.uniform(-1.0, 1.0, size=r.shape))
        return r

    def silu(a):
        return 0.5 * a * (1.0 + tanh(0.5 * a))

    def silu_grad(a):
        s = 0.5 * (1.0 + tanh(0.5 * a))
        return s * (1.0 + a * (1.0 - s))

    act = split if split_ops else bf16
    zq, W1q, W2q, W3q = act(z), bf16(W1), bf16(W2), bf16(W3)
    a1 = zq @ W1q.T + b1
    h1 = act(silu(a1))
    a2 = h1 @ W2q.T + b2
    h2 = act(silu(a2))
    a3 = h2 @ W3q.T + b3
    h3 = silu(a3)
    y = h3 @ W4[0] + b4[0]
    if x is None:
        return y
    B = y.shape[0]
    s = 1.0 / (1.0 + np.exp(-ref.OUT_SCALE * y))
    dx, dt = s - x, y - t
    loss = float(np.mean(ref.LOSS_X * dx ** 2 + ref.LOSS_LOGIT * dt ** 2))
    dy = (2.0 * ref.LOSS_X * dx * s * (1.0 - s) * ref.OUT_SCALE + 2.0 * ref.LOSS_LOGIT * dt) / B
    dW4 = (dy @ h3)[None, :]
    db4 = np.array([dy.sum()])
    dz3 = dy[:, None] * W4[0][None, :] * silu_grad(a3)
    db3, dz3q = dz3.sum(0), bf16(dz3)
    dW3 = dz3q.T @ h2
    dz2 = (dz3q @ W3q) * silu_grad(a2)
    db2, dz2q = dz2.sum(0), bf16(dz2)
    dW2 = dz2q.T @ h1
    dz1 = (dz2q @ W2q) * silu_grad(a1)
    db1, dz1q = dz1.sum(0), bf16(dz1)
    dW1 = dz1q.T @ zq
    return y, loss, ref.pack([dW1, db1, dW2, db2, dW3, db3, dW4, db4])


def bounds(p, z, x=None, t=None, samples=30, seed=0):
    """The emulation and element-wise bounds: twice the largest deviation over `samples`
    emulations with tanh perturbed by 2^-10, plus a floor for FP32 accumulation (1e-5 of |y|; for
    the gradient 2e-4 of the largest entry of each parameter block).  Without x: the inference
    kernels' forward pass; with x and t: the training kernels' forward and backward passes."""
    rng = np.random.default_rng(seed)
    base = emulate(p, z, x, t, split_ops=x is None)
    if x is None:
        dev = np.zeros_like(base)
        for _ in range(samples):
            dev = np.maximum(dev, np.abs(emulate(p, z, tanh_err=2.0 ** -10, rng=rng,
                                                 split_ops=True) - base))
        return base, 2.0 * dev + 1e-5 * (1.0 + np.abs(base))
    y0, _, g0 = base
    dev = np.zeros_like(g0)
    for _ in range(samples):
        dev = np.maximum(dev, np.abs(emulate(p, z, x, t, 2.0 ** -10, rng)[2] - g0))
    floor = np.concatenate([np.full(a.size, 2e-4 * np.abs(a).max())
                            for a in ref.unpack(g0)])
    return base, 2.0 * dev + floor


def scaled_params(seed: int, scale: float = 3.0) -> np.ndarray:
    """Initial parameters with weights scaled up, so that activations and outputs are O(1) as in a
    trained network (the plain initialisation leaves |y| near 0.02)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = ref.unpack(ref.init_params(seed))
    return ref.pack([W1 * scale, b1, W2 * scale, b2, W3 * scale, b3, W4 * scale, b4])
