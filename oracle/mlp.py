"""FP64 oracle of the learned low-rank DtN correction's network.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).
The network is not in the paper; this file fixes what the CUDA kernels must
compute so that their gradients can be checked:

    x = 2 (b - 1)
    a1 = relu(x W0 + c0),  a2 = relu(a1 W1 + c1),  y = a2 W2 + c2
    U = y[:, :m r] as [m][r],  V = y[:, m r:] as [m][r]
    L = mean over boxes and entries of (U V^T - (T - T0) / s)^2

Weights enter the products rounded to BF16 (round to nearest even), as in
the kernels; everything else is FP64.  The backward pass is written out by
the chain rule and pinned by central finite differences (``bf16=False``).

With ``act_bf16=True`` every product's other operand is rounded to BF16 too,
at the points where the tensor-core kernels round it (the products then run
with BF16 operands and FP32 accumulation):

    forward:  x, a1, a2 before the layer products; U, V before U V^T
    backward: g E (the scaled residual, g = 2 / #entries) before E V and
              E^T U; dy, d2, d1 before the weight-gradient and the
              back-propagation products

Bias gradients are column sums of the unrounded dy, d2, d1.  The rounded
variant is the unrounded one (pinned by finite differences) with the
rounding inserted; its pin is the bound on what the roundings may change:
each moves its operand by at most 2^-9 relative, so loss and gradient stay
within a small multiple of that of the unrounded values.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), as FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray, dims):
    """Split the flat parameter vector W0, c0, W1, c1, W2, c2."""
    out, off = [], 0
    for l in range(3):
        nw = dims[l] * dims[l + 1]
        out.append(theta[off:off + nw].reshape(dims[l], dims[l + 1]))
        off += nw
        out.append(theta[off:off + dims[l + 1]])
        off += dims[l + 1]
    return out


def loss_and_grad(theta, dims, m, r, b, dT, scale, bf16=True, act_bf16=False):
    """(loss, flat gradient) for a batch b [B][n_in], dT = T - T0 [B][m][m]."""
    W0, c0, W1, c1, W2, c2 = unpack(np.asarray(theta, dtype=np.float64), dims)
    ident = lambda w: np.asarray(w, dtype=np.float64)
    q = bf16_round if bf16 else ident
    qa = bf16_round if act_bf16 else ident
    Q0, Q1, Q2 = q(W0), q(W1), q(W2)
    B = b.shape[0]
    x = qa(2.0 * (b - 1.0))
    z1 = x @ Q0 + c0
    a1 = qa(np.maximum(z1, 0.0))
    z2 = a1 @ Q1 + c1
    a2 = qa(np.maximum(z2, 0.0))
    y = a2 @ Q2 + c2
    U = qa(y[:, :m * r]).reshape(B, m, r)
    V = qa(y[:, m * r:]).reshape(B, m, r)
    E = U @ V.transpose(0, 2, 1) - dT / scale
    L = (E ** 2).mean()
    G = qa((2.0 / E.size) * E)
    dU = G @ V
    dV = G.transpose(0, 2, 1) @ U
    dy = np.concatenate([dU.reshape(B, -1), dV.reshape(B, -1)], axis=1)
    gc2 = dy.sum(axis=0)
    dy = qa(dy)
    gW2 = a2.T @ dy
    d2 = (dy @ Q2.T) * (z2 > 0)
    gc1 = d2.sum(axis=0)
    d2 = qa(d2)
    gW1 = a1.T @ d2
    d1 = (d2 @ Q1.T) * (z1 > 0)
    gc0 = d1.sum(axis=0)
    d1 = qa(d1)
    gW0 = x.T @ d1
    grad = np.concatenate([gW0.ravel(), gc0, gW1.ravel(), gc1, gW2.ravel(), gc2])
    return L, grad


def forward(theta, dims, m, r, b, act_bf16=False):
    """y [B][2 m r] of the forward pass (BF16 weights; with act_bf16 the
    layer inputs rounded as in loss_and_grad)."""
    W0, c0, W1, c1, W2, c2 = unpack(np.asarray(theta, dtype=np.float64), dims)
    qa = bf16_round if act_bf16 else (lambda w: np.asarray(w, dtype=np.float64))
    a1 = qa(np.maximum(qa(2.0 * (b - 1.0)) @ bf16_round(W0) + c0, 0.0))
    a2 = qa(np.maximum(a1 @ bf16_round(W1) + c1, 0.0))
    return a2 @ bf16_round(W2) + c2
