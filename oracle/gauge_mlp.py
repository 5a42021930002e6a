"""FP64 reference of the learned face-gauge predictor network (test infrastructure only).

The network is 48 -> 64 -> 64 -> 16 with ReLU, trained with the mean squared error on
three targets.  Parameters are one flat FP32 vector laid out
W1[64][48] b1[64] W2[64][64] b2[64] W3[16][64] b3[16].  With ``quantize=True`` the
reference rounds to bfloat16 exactly where the tensor-core kernels hold BF16 operands
(inputs, weights, the two hidden activations, and the back-propagated dOut, dZ2, dZ1);
every product and sum is FP64.  With ``quantize=False`` it is the plain network, whose
gradient the tests pin by central finite differences.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUTP, OUT = 48, 64, 16, 3
O_W1 = 0
O_B1 = O_W1 + HID * IN
O_W2 = O_B1 + HID
O_B2 = O_W2 + HID * HID
O_W3 = O_B2 + HID
O_B3 = O_W3 + OUTP * HID
NPARAMS = O_B3 + OUTP


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[O_W1:O_B1].reshape(HID, IN), p[O_B1:O_W2], p[O_W2:O_B2].reshape(HID, HID), p[O_B2:O_W3],
            p[O_W3:O_B3].reshape(OUTP, HID), p[O_B3:NPARAMS])


def forward(p, X, quantize=True):
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Xq = q(np.asarray(X)[:, :IN])
    h1 = q(np.maximum(Xq @ q(W1).T + b1, 0.0))
    h2 = q(np.maximum(h1 @ q(W2).T + b2, 0.0))
    out = h2 @ q(W3).T + b3
    return out, (Xq, h1, h2)


def loss_and_grad(p, X, Y, quantize=True):
    """Mean squared error over the first three outputs and its gradient (flat, FP64)."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    out, (Xq, h1, h2) = forward(p, X, quantize)
    n = out.shape[0]
    err = np.zeros_like(out)
    err[:, :OUT] = out[:, :OUT] - np.asarray(Y)[:, :OUT]
    loss = float((err ** 2).sum() / (OUT * n))
    dout = q(2.0 * err / (OUT * n))
    dz2 = q((dout @ q(W3)) * (h2 > 0))
    dz1 = q((dz2 @ q(W2)) * (h1 > 0))
    g = np.zeros(NPARAMS)
    g[O_W1:O_B1] = (dz1.T @ Xq).ravel()
    g[O_B1:O_W2] = dz1.sum(0)
    g[O_W2:O_B2] = (dz2.T @ h1).ravel()
    g[O_B2:O_W3] = dz2.sum(0)
    g[O_W3:O_B3] = (dout.T @ h2).ravel()
    g[O_B3:NPARAMS] = dout.sum(0)
    return loss, g


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAMS)
    p[O_W1:O_B1] = rng.uniform(-0.3, 0.3, HID * IN)
    p[O_B1:O_W2] = rng.uniform(-0.1, 0.1, HID)
    p[O_W2:O_B2] = rng.uniform(-0.2, 0.2, HID * HID)
    p[O_B2:O_W3] = rng.uniform(-0.1, 0.1, HID)
    p[O_W3:O_B3] = rng.uniform(-0.2, 0.2, OUTP * HID)
    p[O_B3:NPARAMS] = rng.uniform(-0.1, 0.1, OUTP)
    return p
