"""Learned r_max oracle -- TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Plain numpy restatements of what the CUDA path computes for the learned r_max:
per-source features (loops over the out-edges of each source) and the forward and
backward pass of the 16-64-64-1 network with BF16 weights and activations.  The
oracle accumulates in FP64 (the CUDA path in FP32) at the same rounding points:
inputs (f - mu)/sigma in FP32 then BF16, weights BF16, hidden activations BF16 after
ReLU, output unrounded.  Gradients of 0.5 mean (y - t)^2 treat the BF16 rounding as
the identity (the CUDA kernels apply them to FP32 master weights).
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 16
HID = 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + HID * N_FEATURES
OFF_W2 = OFF_B1 + HID
OFF_B2 = OFF_W2 + HID * HID
OFF_W3 = OFF_B2 + HID
OFF_B3 = OFF_W3 + HID
N_PARAMS = OFF_B3 + 1


def bf16(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even), as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def features(row_ptr, col, sources, alpha, rmax_rule):
    """The 16 features of each source (definitions in include/fora.h), float32 [S, 16]."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    m = int(row_ptr[-1])
    deg = np.diff(row_ptr)
    indeg = np.bincount(col, minlength=n)
    out = np.zeros((len(sources), N_FEATURES), dtype=np.float32)
    for k, s in enumerate(sources):
        d = int(deg[s])
        inc = (1.0 - alpha) / float(d)
        sum_out = sum_in = f1 = f1_edges = 0
        for e in range(row_ptr[s], row_ptr[s + 1]):
            u = int(col[e])
            du = int(deg[u])
            sum_out += du
            sum_in += int(indeg[u])
            if inc > rmax_rule * float(du):
                f1 += 1
                f1_edges += du
        out[k, :8] = [math.log1p(d), math.log1p(int(indeg[s])), math.log1p(sum_out),
                      math.log1p(sum_in), math.log1p(f1), math.log1p(f1_edges),
                      math.log(rmax_rule * m), math.log(m / n)]
    return out


def _layers(params):
    p = np.asarray(params, dtype=np.float32)
    w = bf16(p).astype(np.float64)
    W1 = w[OFF_W1:OFF_B1].reshape(HID, N_FEATURES)
    b1 = w[OFF_B1:OFF_W2]
    W2 = w[OFF_W2:OFF_B2].reshape(HID, HID)
    b2 = w[OFF_B2:OFF_W3]
    W3 = w[OFF_W3:OFF_B3]
    b3 = w[OFF_B3]
    return W1, b1, W2, b2, W3, b3


def forward(params, norm, X, rounding=True):
    """y [S] and the activations needed by the backward pass."""
    X = np.asarray(X, dtype=np.float32)
    norm = np.asarray(norm, dtype=np.float32)
    mu, sigma = norm[:N_FEATURES], norm[N_FEATURES:]
    rnd = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    if rounding:
        W1, b1, W2, b2, W3, b3 = _layers(params)
    else:
        p = np.asarray(params, dtype=np.float64)
        W1, b1 = p[OFF_W1:OFF_B1].reshape(HID, N_FEATURES), p[OFF_B1:OFF_W2]
        W2, b2 = p[OFF_W2:OFF_B2].reshape(HID, HID), p[OFF_B2:OFF_W3]
        W3, b3 = p[OFF_W3:OFF_B3], p[OFF_B3]
    x = np.asarray(rnd((X - mu) / sigma), dtype=np.float64)      # FP32 normalisation
    z1 = x @ W1.T + b1
    h1 = np.asarray(rnd(np.maximum(z1, 0.0).astype(np.float32) if rounding
                        else np.maximum(z1, 0.0)), dtype=np.float64)
    z2 = h1 @ W2.T + b2
    h2 = np.asarray(rnd(np.maximum(z2, 0.0).astype(np.float32) if rounding
                        else np.maximum(z2, 0.0)), dtype=np.float64)
    y = h2 @ W3 + b3
    return y, (x, z1, h1, z2, h2, (W1, b1, W2, b2, W3, b3))


def gradient(params, norm, X, T, rounding=True):
    """(grad [N_PARAMS], loss) of 0.5 mean (y - t)^2, FP64."""
    y, (x, z1, h1, z2, h2, (W1, b1, W2, b2, W3, b3)) = forward(params, norm, X, rounding)
    T = np.asarray(T, dtype=np.float64)
    S = len(T)
    err = y - T
    loss = 0.5 * np.mean(err * err)
    dy = err / S
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = dy @ h2
    g[OFF_B3] = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)
    g[OFF_W2:OFF_B2] = (dz2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g[OFF_W1:OFF_B1] = (dz1.T @ x).ravel()
    g[OFF_B1:OFF_W2] = dz1.sum(0)
    return g, loss
