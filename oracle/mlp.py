"""FP64 reference of the walk cost model (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; its load-balancing cost q_i is the number of
interactions of a particle's last force computation (Sec. 6.1).  The CUDA library predicts
log(1 + cost) with a 6 -> 32 -> 32 -> 1 ReLU network whose weights and activations are
stored in BF16 with FP32 sums.  This module restates that network in numpy FP64 -- forward,
mean-squared-error loss and the analytic gradient -- with the BF16 rounding emulated
(round to nearest even on the FP32 bit pattern), so that the GPU kernels' forward pass and
gradient can be checked value by value.  With ``bf16=False`` it is the plain FP64 network,
whose gradient is pinned by finite differences in tests/test_oracle_mlp.py.

Parameter layout (1313 values): W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3.
"""
from __future__ import annotations

import numpy as np

F, H = 6, 32
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def forward(p, x, bf16_storage=True):
    """Returns prediction (n,) and the activations needed by the gradient."""
    w = unpack(p)
    r = bf16 if bf16_storage else (lambda v: np.asarray(v, dtype=np.float64))
    W1, W2, W3 = r(w["W1"]), r(w["W2"]), r(w["W3"])
    x0 = r(x)
    z1 = x0 @ W1.T + w["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + w["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ W3 + w["b3"][0]
    return y, (x0, h1, h2, W1, W2, W3)


def loss_and_grad(p, x, t, bf16_storage=True):
    """Mean squared error and its gradient with respect to the parameters."""
    n = x.shape[0]
    y, (x0, h1, h2, W1, W2, W3) = forward(p, x, bf16_storage)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = {}
    g["W3"] = dy @ h2
    g["b3"] = np.array([dy.sum()])
    d2 = np.where(h2 > 0, dy[:, None] * W3[None, :], 0.0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = np.where(h1 > 0, d2 @ W2, 0.0)
    g["W1"] = d1.T @ x0
    g["b1"] = d1.sum(axis=0)
    grad = np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])
    return loss, grad
