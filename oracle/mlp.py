"""FP64 oracle of the learned gain surrogate (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY.  A camera's 3x36x64 thumbnail (box means of its
uncorrected RGB, /255 - 0.5) goes through Linear(6912, 256) - ReLU -
Linear(256, 256) - ReLU - Linear(256, 3) and predicts the camera's three
log-gains; the labels are the log-gains of the per-camera gain fit (one
block).  The GPU stores operands in BF16 and accumulates in FP32; this
oracle computes in float64 and, when ``bf16`` is set, rounds to BF16 at the
same storage points (the input, the weights as used, the hidden activations
and their gradients).  With ``acc32`` the sums whose results are rounded to
BF16 are accumulated in float32 first, so that a BF16 rounding decision is
taken in the kernel's precision (FP32 accumulation, BF16 storage); the
remaining difference to the GPU is the order of the FP32 additions.
Weight layout: W1 [256, 6912], W2 [256, 256], W3 [3, 256] (out x in).
"""
from __future__ import annotations

from typing import Dict

import numpy as np

D_IN, D_H, D_OUT = 3 * 36 * 64, 256, 3


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) via float32."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def thumb_features(sums: np.ndarray, W: int, H: int) -> np.ndarray:
    """[3, 36, 64] cell sums -> 6912 features: cell mean / 255 - 0.5."""
    th, tw = sums.shape[1], sums.shape[2]
    cw = np.array([(i + 1) * W // tw - i * W // tw for i in range(tw)], np.float64)
    chh = np.array([(j + 1) * H // th - j * H // th for j in range(th)], np.float64)
    area = chh[:, None] * cw[None, :]
    return (sums.astype(np.float64) / area[None] / 255.0 - 0.5).reshape(-1)


def _mm(a, b, acc32):
    """a @ b, accumulated in float32 when acc32 (operands are BF16 values).
    acc32 == "split" sums the two halves of the inner dimension separately
    and then adds them: another valid float32 summation order, used to
    measure how far two FP32 orders drift apart through the BF16 rounding
    decisions (the noise floor a GPU result is compared against)."""
    if acc32 == "split":
        a32, b32 = np.asarray(a, np.float32), np.asarray(b, np.float32)
        h = a32.shape[-1] // 2
        return (a32[..., :h] @ b32[:h] + a32[..., h:] @ b32[h:]).astype(np.float64)
    if acc32:
        return (np.asarray(a, np.float32) @ np.asarray(b, np.float32)).astype(np.float64)
    return a @ b


def _add(z, bias, acc32):
    return (z.astype(np.float32) + np.asarray(bias, np.float32)).astype(np.float64) if acc32 else z + bias


def _rounder(bf16: bool):
    return bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))


def dense_relu(h: np.ndarray, W: np.ndarray, b: np.ndarray, bf16: bool = True, acc32: bool = False):
    """One hidden layer: pre-activation z = h W^T + b and the stored
    activation relu(z) (rounded to BF16 when ``bf16``).  W as used (already
    BF16-rounded when the network stores BF16 weights)."""
    z = _add(_mm(h, np.asarray(W).T, acc32), b, acc32)
    return z, _rounder(bf16)(np.maximum(z, 0.0))


def output_layer(h2: np.ndarray, W3: np.ndarray, b3: np.ndarray, acc32: bool = False) -> np.ndarray:
    """The linear output layer y = h2 W3^T + b3 (three log-gains per row)."""
    return _add(_mm(h2, np.asarray(W3).T, acc32), b3, acc32)


def output_grad(y: np.ndarray, t: np.ndarray, acc32: bool = False) -> np.ndarray:
    """dL/dy of L = mean over the batch and the three outputs of (y - t)^2."""
    N = t.shape[0]
    if acc32:
        return (np.float32(2.0) * (np.asarray(y, np.float32) - np.asarray(t, np.float32)) /
                np.float32(N * D_OUT)).astype(np.float64)
    return 2.0 * (y - t) / (N * D_OUT)


def hidden_grad(dz_next: np.ndarray, W_next: np.ndarray, active: np.ndarray, bf16: bool = True,
                acc32: bool = False) -> np.ndarray:
    """dL/dz of a hidden layer from the next layer's dL/dz and weights (as
    used): (dz_next W_next) where the ReLU was active, else 0 (stored BF16)."""
    return _rounder(bf16)(_mm(dz_next, W_next, acc32) * active)


def weight_grads(dz: np.ndarray, h_in: np.ndarray):
    """dL/dW = dz^T h_in and dL/db = sum of dz over the batch (FP64)."""
    return dz.T @ h_in, dz.sum(0)


def forward(P: Dict[str, np.ndarray], X: np.ndarray, bf16: bool = True, acc32: bool = False):
    r = _rounder(bf16)
    x = r(X)
    z1, h1 = dense_relu(x, r(P["W1"]), P["b1"], bf16, acc32)
    z2, h2 = dense_relu(h1, r(P["W2"]), P["b2"], bf16, acc32)
    y = output_layer(h2, r(P["W3"]), P["b3"], acc32)
    return y, {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y}


def mse(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def backward(P: Dict[str, np.ndarray], cache, t: np.ndarray, bf16: bool = True, acc32: bool = False):
    """Gradients of mean((y - t)^2) over the batch and the three outputs."""
    r = _rounder(bf16)
    dy = output_grad(cache["y"], t, acc32)
    g = {}
    g["W3"], g["b3"] = weight_grads(dy, cache["h2"])
    dh2 = hidden_grad(dy, r(P["W3"]), cache["z2"] > 0, bf16, acc32)
    g["W2"], g["b2"] = weight_grads(dh2, cache["h1"])
    dh1 = hidden_grad(dh2, r(P["W2"]), cache["z1"] > 0, bf16, acc32)
    g["W1"], g["b1"] = weight_grads(dh1, cache["x"])
    return g


def adam_step(P, G, state, lr: float, t: int, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the FP32 master weights, in FP64."""
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * G[k]
        v[...] = b2 * v + (1 - b2) * G[k] * G[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P


def regauge(logg: np.ndarray, groups) -> np.ndarray:
    """Subtract each chain's mean log-gain (per channel): the common scale of
    a chain is unobservable, so predictions are compared in the gauge of the
    labels (sum of log-gains zero over the chain)."""
    out = np.array(logg, np.float64, copy=True)
    groups = np.asarray(groups)
    for g in np.unique(groups):
        m = groups == g
        out[m] -= out[m].mean(0, keepdims=True)
    return out


def gain_error(pred_log: np.ndarray, label_log: np.ndarray) -> np.ndarray:
    """max over channels of |exp(pred - label) - 1| per camera."""
    return np.abs(np.exp(pred_log - label_log) - 1.0).max(-1)
