"""Seam gradient-continuity cost, Eq. (gradientcost) of Sec. "Quantitative".

TEST INFRASTRUCTURE ONLY.  For adjacent images I- (left) and I+ (right) the
last two columns of I- and the first two of I+ are compared row by row:
    d+_i = || (I+_{1,i} - I+_{0,i}) - (I+_{0,i} - I-_{0,i}) ||
    d-_i = || (I-_{-1,i} - I-_{0,i}) - (I-_{0,i} - I+_{0,i}) ||
    cost = (1/N) sum_i (d+_i + d-_i) / 2
with || . || the Euclidean norm over (r, g, b) and N the number of rows,
after an 8x8 box down-sampling of both images (the paper's factor eight).
Readings: the printed indices are garbled; N is the row count; the norm is
Euclidean; the down-sampling is a box mean.
"""
import numpy as np


def downsample(rgb: np.ndarray, f: int = 8) -> np.ndarray:
    H, W, _ = rgb.shape
    H2, W2 = H // f, W // f
    a = rgb[: H2 * f, : W2 * f].astype(np.float64)
    return a.reshape(H2, f, W2, f, 3).mean(axis=(1, 3))


def seam_cost(left: np.ndarray, right: np.ndarray, f: int = 8) -> float:
    L = downsample(left, f) if f > 1 else left.astype(np.float64)
    R = downsample(right, f) if f > 1 else right.astype(np.float64)
    n = min(L.shape[0], R.shape[0])
    L, R = L[:n], R[:n]
    Lm1, L0 = L[:, -2], L[:, -1]
    R0, R1 = R[:, 0], R[:, 1]
    dp = np.linalg.norm((R1 - R0) - (R0 - L0), axis=-1)
    dm = np.linalg.norm((Lm1 - L0) - (L0 - R0), axis=-1)
    return float(np.mean(0.5 * (dp + dm)))


def interior_cost(img: np.ndarray, f: int = 8) -> float:
    """The reference value: the cost of a cut through the middle of one image."""
    W = img.shape[1]
    c = (W // 2) // f * f
    return seam_cost(img[:, :c], img[:, c:], f)
