"""FP64 oracle of the surrogate MLP (forward and backward).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network: x -> z1 = x W1^T + b1 -> a1 = silu(z1) -> z2 = a1 W2^T + b2 ->
a2 = silu(z2) -> y = a2 W3^T + b3, silu(z) = z / (1 + e^-z), loss = mean of
(y - t)^2 over all n x 40 entries.  With rounding=True every operand the GPU
stores in BF16 (inputs, weights, hidden activations, back-propagated
gradients) is rounded the same way here (FP64 -> FP32 -> BF16, round to
nearest even), and everything else is FP64.  Shapes use the padded layout:
W1 [256][16], W2 [256][256], W3 [48][256]; inputs [n][16], targets [n][48]
with the padded columns zero.
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to BF16 (via FP32), round to nearest even; returns float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, rounding=True):
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    x0 = r(x)
    z1 = x0 @ r(W1).T + b1
    a1 = r(silu(z1))
    z2 = a1 @ r(W2).T + b2
    a2 = r(silu(z2))
    y = a2 @ r(W3).T + b3
    return dict(x0=x0, z1=z1, a1=a1, z2=z2, a2=a2, y=y)


def loss_and_grads(params, x, t, n_valid_cols=40, rounding=True):
    """Loss and gradients (gW1, gb1, gW2, gb2, gW3, gb3)."""
    W1, b1, W2, b2, W3, b3 = params
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    f = forward(params, x, rounding)
    n = x.shape[0]
    mask = np.zeros(f["y"].shape[1])
    mask[:n_valid_cols] = 1.0
    d = (f["y"] - t) * mask
    loss = float(np.sum(d * d) / (n * n_valid_cols))
    dy = 2.0 * d / (n * n_valid_cols)
    dy16 = r(dy)
    gW3 = dy16.T @ f["a2"]
    gb3 = dy.sum(axis=0)
    dz2 = r((dy16 @ r(W3)) * dsilu(f["z2"]))
    gW2 = dz2.T @ f["a1"]
    gb2 = dz2.sum(axis=0)
    dz1 = r((dz2 @ r(W2)) * dsilu(f["z1"]))
    gW1 = dz1.T @ f["x0"]
    gb1 = dz1.sum(axis=0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def init_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = np.zeros((256, 16)); W1[:, :4] = rng.uniform(-1, 1, (256, 4)) * scale * np.sqrt(6 / 260)
    W2 = rng.uniform(-1, 1, (256, 256)) * scale * np.sqrt(6 / 512)
    W3 = np.zeros((48, 256)); W3[:40] = rng.uniform(-1, 1, (40, 256)) * scale * np.sqrt(6 / 296)
    b1 = rng.uniform(-0.1, 0.1, 256); b2 = rng.uniform(-0.1, 0.1, 256)
    b3 = np.zeros(48); b3[:40] = rng.uniform(-0.1, 0.1, 40)
    return [W1, b1, W2, b2, W3, b3]
