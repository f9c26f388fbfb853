"""CPU reference of the BF16 MLP surrogate kernels (TEST INFRASTRUCTURE ONLY).

The surrogate is not in the paper; this module restates the network the
CUDA kernels compute — Linear layers with GELU(x) = x/2 (1 + erf(x/sqrt2)),
BF16 operands, FP32 accumulation on the GPU — in plain numpy float64, with
BF16 rounding (round to nearest even) applied at exactly the points where the
kernels store BF16 values.  Sums are FP64 here, so GPU results differ by the
FP32 accumulation error, bounded per element by K * 2^-24 * sum_k |a_k b_k|.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits_to_f64(bits) -> np.ndarray:
    """Decode raw bfloat16 bit patterns (uint16) to float64."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def gemm(A, B):
    """C = A B^T in float64 (A [M, K], B [N, K], values already BF16)."""
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64).T


def gemm_error_bound(A, B, K):
    """Bound of the FP32-accumulation error of each C element."""
    return K * 2.0 ** -24 * (np.abs(A) @ np.abs(B).T) + 1e-30


def features(phases, ldx):
    """[sin phi, cos phi, 1, 0 ...] rounded to bf16 (rows of length ldx)."""
    phases = np.asarray(phases, np.float64)
    B, P = phases.shape
    X = np.zeros((B, ldx))
    X[:, :P] = np.sin(phases)
    X[:, P:2 * P] = np.cos(phases)
    X[:, 2 * P] = 1.0
    return bf16(X)


def forward(X, Ws, bs):
    """Layer-by-layer forward.  Returns (inputs of each layer, pre-activations
    of the hidden layers, final fp64 output)."""
    ins, pres = [X], []
    h = X
    for l, (W, b) in enumerate(zip(Ws, bs)):
        pre = gemm(h, W) + b
        if l + 1 < len(Ws):
            pres.append(pre)
            h = bf16(gelu(pre))
            ins.append(h)
        else:
            return ins, pres, pre
    raise ValueError("no layers")


def mse(pred, target):
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(w, m, v, g, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return w, m, v
