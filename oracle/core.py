"""Oracle of one frame set of the exposure / white-balance correction.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Per-pixel work runs in
``rt_oracle.c``; the fits, smoothing and quantisation are written here in
numpy float64, step by step in the order of Sec. "White balance and exposure
correction":

  1. measured spectra: band statistics on both sides of every seam, with the
     moving pixels removed (object removal, Fig. "thresholded difference");
  2. a shared spectrum per seam and a map per channel that takes each side's
     band onto it -- either the per-camera gain fit (log least squares over
     the seams, one gain per camera, channel and block) or the paper's affine
     map f_c(x) = a_c x + b_c per seam side (first two moments matched to the
     equal-weight mixture of the two bands);
  3. exponential smoothing E <- (1 - alpha) E_prev + alpha E_new, alpha=0.05;
  4. Q16 quantisation and per-pixel application along the convex ramp.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import lib

NV12, MONO16 = 0, 1
FIT_GLOBAL, FIT_SEAM_AFFINE, FIT_QUANTILE_AFFINE, FIT_MATRIX = 0, 1, 2, 3
MATRIX_RIDGE = 0.25             # added to band covariances (half an LSB of noise, squared)
QUANTILES = 32                  # levels (i + 1/2) / QUANTILES of the quantile fit
SCHED_CURRENT, SCHED_LAGGED = 0, 1
LINEAR, RING = 0, 1
THUMB_W, THUMB_H = 64, 36


@dataclasses.dataclass
class Params:
    strip_width: int = 32          # S: width of the narrow band at each seam
    num_blocks: int = 1            # B: vertical blocks of the band
    fit_mode: int = FIT_GLOBAL
    schedule: int = SCHED_CURRENT
    topology: int = LINEAR
    motion_threshold: int = 24     # |Y_t - Y_{t-1}| above this marks a moving pixel
    min_valid: int = 64            # a band side with fewer valid pixels is ignored
    color_matrix: int = 0          # 0 BT.709, 1 BT.601
    alpha: float = 0.05            # exponential smoothing weight
    lam: float = 1e-6              # ridge term of the gain fit
    gain_min: float = 0.25
    gain_max: float = 4.0
    blend_blocks: bool = False     # convex blending of adjacent block maps


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


_C = None


def _c():
    global _C
    if _C is None:
        L = lib()
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.orc_color_coeffs.argtypes = [i32, vp]
        L.orc_convert_nv12.argtypes = [vp, i64, vp, i64, i32, i32, i32, vp, i64]
        L.orc_convert_mono16.argtypes = [vp, i64, i32, i32, i32, vp, i64]
        L.orc_luma_mono16.argtypes = [vp, i64, i32, i32, i32, vp, i64]
        L.orc_strip_stats.argtypes = [vp, i64, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp, vp, vp, vp]
        L.orc_frame_stats.argtypes = [vp, i64, i32, i32, vp, vp, vp]
        L.orc_thumbnail.argtypes = [vp, i64, i32, i32, i32, i32, vp]
        L.orc_ramp_q16.argtypes = [i32, i32]
        L.orc_ramp_q16.restype = ctypes.c_int32
        L.orc_apply.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp, i64]
        L.orc_crop.argtypes = [vp, i64, i32, i32, i32, i32, i32, vp]
        L.orc_strip_joint.argtypes = [vp, i64, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp]
        L.orc_apply_matrix.argtypes = [vp, i64, i32, i32, i32, vp, vp, i64]
        _C = L
    return _C


# ----------------------------------------------------------------------------
# Per-pixel steps (thin wrappers over the C loops)
# ----------------------------------------------------------------------------

def color_coeffs(matrix: int = 0) -> np.ndarray:
    out = np.zeros(5, np.int32)
    _c().orc_color_coeffs(matrix, _p(out))
    return out


def convert(cam, fr: Dict[str, np.ndarray], matrix: int = 0):
    """Decoded frame -> (RGB [H, W, 3] uint8, luma [H, W] uint8)."""
    W, H = cam.width, cam.height
    rgb = np.zeros((H, W, 3), np.uint8)
    if cam.fmt == NV12:
        y = np.ascontiguousarray(fr["y"], dtype=np.uint8)
        uv = np.ascontiguousarray(fr["uv"], dtype=np.uint8)
        _c().orc_convert_nv12(_p(y), y.shape[1], _p(uv), uv.shape[1], W, H, matrix, _p(rgb), 3 * W)
        luma = np.ascontiguousarray(y[:, :W])
    else:
        ir = np.ascontiguousarray(fr["ir"]).view(np.uint16)
        _c().orc_convert_mono16(_p(ir), ir.shape[1], W, H, cam.bit_depth, _p(rgb), 3 * W)
        luma = np.zeros((H, W), np.uint8)
        _c().orc_luma_mono16(_p(ir), ir.shape[1], W, H, cam.bit_depth, _p(luma), W)
    return rgb, luma


def strip_stats(rgb: np.ndarray, luma: np.ndarray, prev_luma: Optional[np.ndarray],
                S: int, B: int, T: int) -> Dict[str, np.ndarray]:
    H, W, _ = rgb.shape
    n = np.zeros((2, B, 3), np.uint32)
    s = np.zeros((2, B, 3), np.uint64)
    ss = np.zeros((2, B, 3), np.uint64)
    h = np.zeros((2, B, 3, 256), np.uint32)
    prev_ptr = None if prev_luma is None else _p(prev_luma)
    _c().orc_strip_stats(_p(rgb), 3 * W, _p(luma), W, prev_ptr, W, W, H, S, B, T,
                         _p(n), _p(s), _p(ss), _p(h))
    return {"n": n, "sum": s, "sumsq": ss, "hist": h}


def strip_joint(rgb: np.ndarray, luma: np.ndarray, prev_luma: Optional[np.ndarray],
                S: int, B: int, T: int) -> np.ndarray:
    """Joint band statistics [2, B, 10] = {n, sums R G B, RR RG RB GG GB BB}
    over pixels neither moving nor saturated in any channel."""
    H, W, _ = rgb.shape
    out = np.zeros((2, B, 10), np.uint64)
    prev_ptr = None if prev_luma is None else _p(prev_luma)
    _c().orc_strip_joint(_p(rgb), 3 * W, _p(luma), W, prev_ptr, W, W, H, S, B, T, _p(out))
    return out


def frame_stats(rgb: np.ndarray) -> Dict[str, np.ndarray]:
    H, W, _ = rgb.shape
    h = np.zeros((3, 256), np.uint32)
    s = np.zeros(3, np.uint64)
    ss = np.zeros(3, np.uint64)
    _c().orc_frame_stats(_p(rgb), 3 * W, W, H, _p(h), _p(s), _p(ss))
    return {"hist": h, "sum": s, "sumsq": ss}


def thumbnail(rgb: np.ndarray, tw: int = THUMB_W, th: int = THUMB_H) -> np.ndarray:
    H, W, _ = rgb.shape
    out = np.zeros((3, th, tw), np.uint32)
    _c().orc_thumbnail(_p(rgb), 3 * W, W, H, tw, th, _p(out))
    return out


def ramp_q16(x: int, W: int) -> int:
    return int(_c().orc_ramp_q16(x, W))


def apply(rgb: np.ndarray, q16_cam: np.ndarray, B: int, fit_mode: int) -> np.ndarray:
    """q16_cam: int32 [2, B, 3, 2] = {a_q, b_q} of one camera.  Per-seam-side
    affine maps (the paper's and the quantile fit's) are applied along the
    convex ramp; per-camera gains on the whole image."""
    H, W, _ = rgb.shape
    q = np.ascontiguousarray(q16_cam, dtype=np.int32)
    assert q.shape == (2, B, 3, 2)
    out = np.zeros_like(rgb)
    ramp_mode = 0 if fit_mode == FIT_GLOBAL else FIT_SEAM_AFFINE
    _c().orc_apply(_p(rgb), 3 * W, W, H, B, ramp_mode, _p(q), _p(out), 3 * W)
    return out


def crop(rgb: np.ndarray, rect: Sequence[int], S: int) -> np.ndarray:
    """rect = (x0, y0, w, h) -> float64 [3, S, S] in [0, 1]."""
    H, W, _ = rgb.shape
    x0, y0, w, h = [int(v) for v in rect]
    out = np.zeros((3, S, S), np.float64)
    _c().orc_crop(_p(rgb), 3 * W, x0, y0, w, h, S, _p(out))
    return out


# ----------------------------------------------------------------------------
# Seams, fits, smoothing, quantisation (FP64)
# ----------------------------------------------------------------------------

def block_rows(j: int, H: int, B: int) -> int:
    """Rows of block j: floor((j+1) H / B) - floor(j H / B)."""
    return (j + 1) * H // B - j * H // B


def chains(cams) -> Dict[int, List[int]]:
    """Cameras of each seam chain, ordered by position."""
    out: Dict[int, List[int]] = {}
    for k, c in enumerate(cams):
        out.setdefault(c.group, []).append(k)
    for g in out:
        out[g].sort(key=lambda k: cams[k].position)
    return out


def seams(cams, topology: int):
    """(group, left camera, right camera) for every seam: the right band of
    the left camera meets the left band of the right camera.  A ring adds the
    seam from the last camera back to the first (arrays of up to 360 deg)."""
    out = []
    for g, members in chains(cams).items():
        for i in range(len(members) - 1):
            out.append((g, members[i], members[i + 1]))
        if topology == RING and len(members) >= 2:
            out.append((g, members[-1], members[0]))
    return out


def fit_global(cams, n: np.ndarray, s: np.ndarray, p: Params) -> np.ndarray:
    """Per-camera gains from the band means.

    n, s: band counts and sums [K, 2, B, 3].  Unknowns x_k = log g_k of each
    chain (per channel, per block).  Every valid seam (left camera k, right
    camera m) asks g_k mu^R_k = g_m mu^L_m, i.e. x_k - x_m = r with
    r = log mu^L_m - log mu^R_k, weighted by the valid fraction of the band;
    the gauge (the common scale is unobservable) fixes sum_k x_k = 0:
        (L_w + lam I + 1 1^T / K_g) x = B^T W r,    g = clamp(exp(x)).
    Returns maps [K, 2, B, 3, 2] with (a, b) = (g, 0) on both sides."""
    K, B, S = len(cams), p.num_blocks, p.strip_width
    g = np.ones((K, B, 3), np.float64)
    ch = chains(cams)
    sm = seams(cams, p.topology)
    for grp, members in ch.items():
        Kg = len(members)
        idx = {k: i for i, k in enumerate(members)}
        for j in range(B):
            for c in range(3):
                M = p.lam * np.eye(Kg) + np.ones((Kg, Kg)) / Kg
                rhs = np.zeros(Kg)
                for (gg, kl, kr) in sm:
                    if gg != grp or kl == kr:
                        continue
                    nR, nL = float(n[kl, 1, j, c]), float(n[kr, 0, j, c])
                    if nR < p.min_valid or nL < p.min_valid:
                        continue
                    muR = max(float(s[kl, 1, j, c]) / nR, 1.0)
                    muL = max(float(s[kr, 0, j, c]) / nL, 1.0)
                    r = math.log(muL) - math.log(muR)
                    rows = min(block_rows(j, cams[kl].height, B), block_rows(j, cams[kr].height, B))
                    w = min(nR, nL) / (S * rows)
                    a, b = idx[kl], idx[kr]
                    M[a, a] += w
                    M[b, b] += w
                    M[a, b] -= w
                    M[b, a] -= w
                    rhs[a] += w * r
                    rhs[b] -= w * r
                Lc = np.linalg.cholesky(M)
                x = np.linalg.solve(Lc.T, np.linalg.solve(Lc, rhs))
                for k in members:
                    g[k, j, c] = min(max(math.exp(x[idx[k]]), p.gain_min), p.gain_max)
    maps = np.zeros((K, 2, B, 3, 2), np.float64)
    maps[:, 0, :, :, 0] = g
    maps[:, 1, :, :, 0] = g
    return maps


def fit_affine(cams, n: np.ndarray, s: np.ndarray, ss: np.ndarray, p: Params) -> np.ndarray:
    """The paper's per-seam affine maps f_c(x) = a_c x + b_c.

    For each valid seam, block and channel the shared spectrum is the
    equal-weight mixture of the two band distributions: mean
    mu_s = (mu_L + mu_R)/2, variance (var_L + var_R)/2 + ((mu_L - mu_R)/2)^2.
    Each side's map matches its band's first two moments to it:
    a = sd_s / sd_side (1 if sd_side < 0.5), clamped; b = mu_s - a mu_side.
    Sides without a valid seam keep the identity (1, 0)."""
    K, B = len(cams), p.num_blocks
    maps = np.zeros((K, 2, B, 3, 2), np.float64)
    maps[..., 0] = 1.0
    for (_, kl, kr) in seams(cams, p.topology):
        if kl == kr:
            continue
        for j in range(B):
            for c in range(3):
                nR, nL = float(n[kl, 1, j, c]), float(n[kr, 0, j, c])
                if nR < p.min_valid or nL < p.min_valid:
                    continue
                muR = float(s[kl, 1, j, c]) / nR
                muL = float(s[kr, 0, j, c]) / nL
                vR = max(float(ss[kl, 1, j, c]) / nR - muR * muR, 0.0)
                vL = max(float(ss[kr, 0, j, c]) / nL - muL * muL, 0.0)
                mus = 0.5 * (muL + muR)
                vs = 0.5 * (vL + vR) + (0.5 * (muL - muR)) ** 2
                for (k, side, mu, v) in ((kl, 1, muR, vR), (kr, 0, muL, vL)):
                    sd = math.sqrt(v)
                    a = math.sqrt(vs) / sd if sd >= 0.5 else 1.0
                    a = min(max(a, p.gain_min), p.gain_max)
                    maps[k, side, j, c, 0] = a
                    maps[k, side, j, c, 1] = mus - a * mu
    return maps


def quantile_levels_hit(cdf_num: np.ndarray, den: int, Q: int = QUANTILES) -> np.ndarray:
    """For i < Q, the smallest value v with cdf(v) >= (2i + 1) / (2Q), where
    cdf(v) = cdf_num[v] / den; decided on integers: 2 Q cdf_num[v] >= (2i + 1) den."""
    out = np.zeros(Q, np.int64)
    for i in range(Q):
        v = 0
        while 2 * Q * int(cdf_num[v]) < (2 * i + 1) * den:
            v += 1
        out[i] = v
    return out


def fit_quantile_affine(cams, hist: np.ndarray, n: np.ndarray, p: Params) -> np.ndarray:
    """A variant of the paper's affine maps (its future work asks for better
    matching of the spectra): each side's f_c(x) = a x + b is the least-squares
    line through the pairs (its band's quantiles, the shared spectrum's
    quantiles) at the levels (i + 1/2) / 32.  The shared spectrum is the
    equal-weight mixture of the two bands (CDF the mean of the two CDFs).
    a = cov(x, y) / var(x) from exact integer sums (1 if var(x) = 0),
    clamped; b = mean(y) - a mean(x).  Sides without a valid seam keep the
    identity.  hist: band histograms [K, 2, B, 3, 256]."""
    K, B, Q = len(cams), p.num_blocks, QUANTILES
    maps = np.zeros((K, 2, B, 3, 2), np.float64)
    maps[..., 0] = 1.0
    for (_, kl, kr) in seams(cams, p.topology):
        if kl == kr:
            continue
        for j in range(B):
            for c in range(3):
                nR, nL = int(n[kl, 1, j, c]), int(n[kr, 0, j, c])
                if nR < p.min_valid or nL < p.min_valid:
                    continue
                cR = np.cumsum(hist[kl, 1, j, c].astype(np.int64))
                cL = np.cumsum(hist[kr, 0, j, c].astype(np.int64))
                xR = quantile_levels_hit(cR, nR)
                xL = quantile_levels_hit(cL, nL)
                # mixture: (cR / nR + cL / nL) / 2 >= (2i+1)/(2Q)  <=>  Q (cR nL + cL nR) >= (2i+1) nR nL
                ys = np.zeros(Q, np.int64)
                for i in range(Q):
                    v = 0
                    while Q * (int(cR[v]) * nL + int(cL[v]) * nR) < (2 * i + 1) * nR * nL:
                        v += 1
                    ys[i] = v
                for (k, side, xs) in ((kl, 1, xR), (kr, 0, xL)):
                    sx, sy = int(xs.sum()), int(ys.sum())
                    sxx, sxy = int((xs * xs).sum()), int((xs * ys).sum())
                    den = Q * sxx - sx * sx
                    num = Q * sxy - sx * sy
                    a = num / den if den != 0 else 1.0
                    a = min(max(a, p.gain_min), p.gain_max)
                    maps[k, side, j, c, 0] = a
                    maps[k, side, j, c, 1] = (sy - a * sx) / Q
    return maps


def smooth(E_prev: Optional[np.ndarray], E_new: np.ndarray, alpha: float) -> np.ndarray:
    """E_blend = (1 - alpha) E_prev + alpha E_new (Eq. of the exponential
    smoothing); the first estimate initialises E."""
    if E_prev is None:
        return E_new.copy()
    return (1.0 - alpha) * E_prev + alpha * E_new


def round_half_away(v: float) -> int:
    """Nearest integer, halves away from zero, exact for any double."""
    a = abs(v)
    r = math.floor(a)
    if a - r >= 0.5:
        r += 1
    return int(r) if v >= 0 else -int(r)


def _sym_fn(A: np.ndarray, f) -> np.ndarray:
    lam, V = np.linalg.eigh(A)
    return (V * f(lam)) @ V.T


def joint_moments(q: np.ndarray):
    """(mean [3], covariance [3, 3] + MATRIX_RIDGE I) of joint band statistics."""
    n = float(q[0])
    mu = np.array([float(q[1]), float(q[2]), float(q[3])]) / n
    S = np.array([[q[4], q[5], q[6]], [q[5], q[7], q[8]], [q[6], q[8], q[9]]], np.float64) / n
    return mu, S - np.outer(mu, mu) + MATRIX_RIDGE * np.eye(3)


def fit_matrix(cams, joint: np.ndarray, p: Params) -> np.ndarray:
    """3 x 3 cross-channel maps (the paper's future work: linear maps
    combining the three channels), the multichannel form of the paper's
    moment matching: the shared spectrum is the equal-weight mixture of the
    two bands (mean mu_s = (mu_L + mu_R)/2, covariance (S_L + S_R)/2 +
    d d^T / 4, d = mu_L - mu_R); each side's M is the symmetric positive
    definite map with M S M^T = S_s,
        M = S^-1/2 (S^1/2 S_s S^1/2)^1/2 S^-1/2,
    its eigenvalues clamped to [gain_min, gain_max], b = mu_s - M mu.  With
    diagonal covariances M_cc = sqrt(S_s,cc / S_cc), the per-channel rule.
    Covariances carry a ridge of 0.25.  joint: [K, 2, B, 10]; returns maps
    [K, 2, B, 12] = {M row-major, b}; sides without a valid seam: identity."""
    K, B = len(cams), p.num_blocks
    maps = np.zeros((K, 2, B, 12), np.float64)
    maps[..., 0] = maps[..., 4] = maps[..., 8] = 1.0
    for (_, kl, kr) in seams(cams, p.topology):
        if kl == kr:
            continue
        for j in range(B):
            qR, qL = joint[kl, 1, j], joint[kr, 0, j]
            if int(qR[0]) < p.min_valid or int(qL[0]) < p.min_valid:
                continue
            muR, SR = joint_moments(qR)
            muL, SL = joint_moments(qL)
            d = muL - muR
            mus = 0.5 * (muL + muR)
            Ss = 0.5 * (SL + SR) + 0.25 * np.outer(d, d)
            for (k, side, mu, S) in ((kl, 1, muR, SR), (kr, 0, muL, SL)):
                h = _sym_fn(S, np.sqrt)
                hi = _sym_fn(S, lambda l: 1.0 / np.sqrt(l))
                M = hi @ _sym_fn(h @ Ss @ h, np.sqrt) @ hi
                M = _sym_fn(0.5 * (M + M.T), lambda l: np.clip(l, p.gain_min, p.gain_max))
                maps[k, side, j, :9] = M.reshape(9)
                maps[k, side, j, 9:] = mus - M @ mu
    return maps


def apply_matrix(rgb: np.ndarray, q16_cam: np.ndarray, B: int) -> np.ndarray:
    """q16_cam: int32 [2, B, 12] of one camera (orc_apply_matrix)."""
    H, W, _ = rgb.shape
    q = np.ascontiguousarray(q16_cam, dtype=np.int32)
    assert q.shape == (2, B, 12)
    out = np.zeros_like(rgb)
    _c().orc_apply_matrix(_p(rgb), 3 * W, W, H, B, _p(q), _p(out), 3 * W)
    return out


def blend_rows(q16_cam: np.ndarray, H: int, B: int) -> np.ndarray:
    """Per-row maps of one camera from its block maps by convex combination of
    adjacent blocks (the paper's future work proposes it for the transition
    between the vertical blocks).  Reading: between the centres of two
    consecutive blocks the Q16 maps are interpolated linearly, above the
    first centre and below the last the edge block's map holds.  With doubled
    centres C_j = r0_j + r1_j - 1 (rows [r0_j, r1_j) of block j) and Y = 2 y:
      w = floor(65536 (Y - C_{j-1}) / (C_j - C_{j-1}))  for C_{j-1} <= Y < C_j,
      m(y) = m_{j-1} + floor((m_j - m_{j-1}) w / 65536),
    in integers, for every value of the table.  q16_cam: [2, B, ...] ->
    [2, H, ...] ([2, B, 3, 2] affine maps, [2, B, 12] 3 x 3 maps)."""
    q = np.asarray(q16_cam, np.int64)
    C = [(j * H) // B + ((j + 1) * H) // B - 1 for j in range(B)]
    out = np.zeros((2, H) + q.shape[2:], np.int64)
    for y in range(H):
        Y = 2 * y
        if Y <= C[0]:
            out[:, y] = q[:, 0]
        elif Y >= C[B - 1]:
            out[:, y] = q[:, B - 1]
        else:
            j = next(jj for jj in range(1, B) if Y < C[jj])
            w = (65536 * (Y - C[j - 1])) // (C[j] - C[j - 1])
            out[:, y] = q[:, j - 1] + ((q[:, j] - q[:, j - 1]) * w) // 65536
    return out.astype(np.int32)


def quantise(maps: np.ndarray) -> np.ndarray:
    """Q16 table: a_q = round(65536 a), b_q = round(65536 b)."""
    flat = maps.reshape(-1)
    out = np.array([round_half_away(65536.0 * float(v)) for v in flat], np.int64)
    assert np.all(np.abs(out) < 2 ** 31)
    return out.astype(np.int32).reshape(maps.shape)


def identity_maps(K: int, B: int, fit_mode: int = FIT_GLOBAL) -> np.ndarray:
    if fit_mode == FIT_MATRIX:
        m = np.zeros((K, 2, B, 12), np.float64)
        m[..., 0] = m[..., 4] = m[..., 8] = 1.0
        return m
    m = np.zeros((K, 2, B, 3, 2), np.float64)
    m[..., 0] = 1.0
    return m


# ----------------------------------------------------------------------------
# Frame-set orchestration
# ----------------------------------------------------------------------------

class ArrayOracle:
    """Runs the correction over a sequence of frame sets, keeping the state
    the method carries between frames (smoothed maps, previous luma)."""

    def __init__(self, cams, params: Params, threads: int = 1):
        self.cams = list(cams)
        self.p = params
        self.threads = max(1, int(threads))
        self.E: Optional[np.ndarray] = None
        self.prev_luma: Optional[List[np.ndarray]] = None

    def reset(self):
        self.E = None
        self.prev_luma = None

    def _map(self, fn, items):
        if self.threads == 1:
            return [fn(i) for i in items]
        with ThreadPoolExecutor(self.threads) as ex:
            return list(ex.map(fn, items))

    def step(self, frames: Sequence[Dict[str, np.ndarray]], crops: Sequence = (), crop_size: int = 0,
             q16_override: Optional[np.ndarray] = None, want_frame_stats: bool = True,
             want_thumbs: bool = False) -> Dict[str, object]:
        p, cams, K, B = self.p, self.cams, len(self.cams), self.p.num_blocks
        first = self.prev_luma is None

        def per_cam_stats(k):
            rgb, luma = convert(cams[k], frames[k], p.color_matrix)
            st = strip_stats(rgb, luma, None if first else self.prev_luma[k],
                             p.strip_width, B, p.motion_threshold)
            fs = frame_stats(rgb) if want_frame_stats else None
            th = thumbnail(rgb) if want_thumbs else None
            if p.fit_mode == FIT_MATRIX:
                st["joint"] = strip_joint(rgb, luma, None if first else self.prev_luma[k],
                                          p.strip_width, B, p.motion_threshold)
            return rgb, luma, st, fs, th

        res = self._map(per_cam_stats, range(K))
        rgb = [r[0] for r in res]
        n = np.stack([r[2]["n"] for r in res])
        s = np.stack([r[2]["sum"] for r in res])
        ss = np.stack([r[2]["sumsq"] for r in res])
        if p.fit_mode == FIT_GLOBAL:
            maps_new = fit_global(cams, n, s, p)
        elif p.fit_mode == FIT_QUANTILE_AFFINE:
            maps_new = fit_quantile_affine(cams, np.stack([r[2]["hist"] for r in res]), n, p)
        elif p.fit_mode == FIT_MATRIX:
            joint = np.stack([r[2]["joint"] for r in res])
            maps_new = fit_matrix(cams, joint, p)
        else:
            maps_new = fit_affine(cams, n, s, ss, p)
        E_prev = self.E
        self.E = smooth(E_prev, maps_new, p.alpha)
        if p.schedule == SCHED_CURRENT:
            maps_used = self.E
        else:  # lagged: this frame set is corrected with the previous estimate
            maps_used = E_prev if E_prev is not None else identity_maps(K, B, p.fit_mode)
        q16 = quantise(maps_used)
        q_apply = q16 if q16_override is None else np.asarray(q16_override, np.int32)

        def per_cam_apply(k):
            q, nb = q_apply[k], B
            if p.blend_blocks and B > 1:
                q, nb = blend_rows(q, cams[k].height, B), cams[k].height
            if p.fit_mode == FIT_MATRIX:
                return apply_matrix(rgb[k], q, nb)
            return apply(rgb[k], q, nb, p.fit_mode)

        corrected = self._map(per_cam_apply, range(K))
        out_crops = None
        if crops:
            out_crops = np.stack([crop(corrected[c[0]], c[1:], crop_size) for c in crops])
        self.prev_luma = [r[1] for r in res]
        return {
            "rgb": rgb, "corrected": corrected,
            "strip_n": n, "strip_sum": s, "strip_sumsq": ss,
            "strip_hist": np.stack([r[2]["hist"] for r in res]),
            "frame_hist": np.stack([r[3]["hist"] for r in res]) if want_frame_stats else None,
            "frame_sum": np.stack([r[3]["sum"] for r in res]) if want_frame_stats else None,
            "frame_sumsq": np.stack([r[3]["sumsq"] for r in res]) if want_frame_stats else None,
            "thumbs": np.stack([r[4] for r in res]) if want_thumbs else None,
            "strip_joint": joint if p.fit_mode == FIT_MATRIX else None,
            "maps_new": maps_new, "maps": maps_used, "E": self.E, "q16": q16,
            "crops": out_crops,
        }
