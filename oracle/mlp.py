"""Oracle of the warm-start network: forward pass, MSE loss, gradients, Adam.

TEST INFRASTRUCTURE ONLY (imported by tests/).

Network (parameter vector layout W1[in][hid], b1, W2[hid][hid], b2,
W3[hid][out], b3, row-major, W[k][j] taking input k to output j):
    H1 = tanh(x W1 + b1),  H2 = tanh(H1 W2 + b2),  Y = H2 W3 + b3,
    L  = 1/(2B) sum (Y - T)^2.
The gradients are the chain rule written out in FP64 (numpy matmuls):
    dY = (Y - T)/B, dW3 = H2^T dY, db3 = sum_b dY,
    dZ2 = (dY W3^T) (1 - H2^2), dW2 = H1^T dZ2, db2 = sum_b dZ2,
    dZ1 = (dZ2 W2^T) (1 - H1^2), dW1 = x^T dZ1, db1 = sum_b dZ1.
With ``bf16=True`` the operands of the three hidden-width products (H1, W2,
H2, W3, dY, dZ2) are first rounded to bfloat16 (round to nearest even of the
FP32 value), the precision in which a tensor-core implementation multiplies
them; everything else stays FP64.
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
Pinned in tests/test_oracle_mlp.py by central finite differences of the loss,
a network with zero hidden weights (Y = b3, closed-form gradients) and the
first Adam step (-lr sign(g) up to eps).
"""
from __future__ import annotations

import numpy as np


def unpack(params, in_dim: int, hid: int, out_dim: int):
    p = np.asarray(params, dtype=np.float64)
    shapes = [(in_dim, hid), (hid,), (hid, hid), (hid,), (hid, out_dim), (out_dim,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    if o != p.size:
        raise ValueError("parameter vector has the wrong length")
    return out


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(params, x, in_dim, hid, out_dim, bf16: bool = False):
    W1, b1, W2, b2, W3, b3 = unpack(params, in_dim, hid, out_dim)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    H1 = np.tanh(x @ W1 + b1)
    H2 = np.tanh(q(H1) @ q(W2) + b2)
    Y = q(H2) @ q(W3) + b3
    return H1, H2, Y


def loss_and_grad(params, x, T, in_dim, hid, out_dim, bf16: bool = False):
    W1, b1, W2, b2, W3, b3 = unpack(params, in_dim, hid, out_dim)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = x.shape[0]
    H1, H2, Y = forward(params, x, in_dim, hid, out_dim, bf16)
    L = 0.5 * np.sum((Y - T) ** 2) / B
    dY = (Y - T) / B
    dW3 = q(H2).T @ q(dY)
    db3 = dY.sum(axis=0)
    dZ2 = (q(dY) @ q(W3).T) * (1.0 - H2 ** 2)
    dW2 = q(H1).T @ q(dZ2)
    db2 = dZ2.sum(axis=0)
    dZ1 = (q(dZ2) @ q(W2).T) * (1.0 - H1 ** 2)
    dW1 = x.T @ dZ1
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([a.reshape(-1) for a in (dW1, db1, dW2, db2, dW3, db3)])
    return L, g


def adam(w, g, m, v, lr: float, t: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v
