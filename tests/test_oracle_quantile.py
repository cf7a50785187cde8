"""Pins of the oracle's quantile-LS affine fit (a variant of the paper's
affine maps, Sec. "White balance and exposure correction"; its future work
asks for better matching of the spectra): quantiles against exact rational
brute force, the line against numpy's polyfit, identity for equal bands,
and the least-squares property that both sides' fitted quantile means equal
the shared spectrum's."""
from fractions import Fraction

import numpy as np

from oracle import core


class _Cam:
    def __init__(self, pos):
        self.width, self.height, self.group, self.position = 64, 32, 0, pos


def _quantiles_bruteforce(hist, Q=32):
    n = int(hist.sum())
    cdf = np.cumsum(hist.astype(np.int64))
    out = []
    for i in range(Q):
        q = Fraction(2 * i + 1, 2 * Q)
        out.append(next(v for v in range(256) if Fraction(int(cdf[v]), n) >= q))
    return np.array(out)


def _mixture_bruteforce(hR, hL, Q=32):
    nR, nL = int(hR.sum()), int(hL.sum())
    cR, cL = np.cumsum(hR.astype(np.int64)), np.cumsum(hL.astype(np.int64))
    out = []
    for i in range(Q):
        q = Fraction(2 * i + 1, 2 * Q)
        out.append(next(v for v in range(256)
                        if (Fraction(int(cR[v]), nR) + Fraction(int(cL[v]), nL)) / 2 >= q))
    return np.array(out)


def _random_hist(rng, lo, hi, n):
    v = np.clip(rng.normal((lo + hi) / 2, (hi - lo) / 6, n).round(), 1, 254).astype(np.int64)
    return np.bincount(v, minlength=256).astype(np.uint32)


def _fit(hR, hL, p=None):
    """maps of a two-camera chain whose seam bands carry hR (left camera's
    right band) and hL (right camera's left band)."""
    p = p or core.Params(fit_mode=core.FIT_QUANTILE_AFFINE, min_valid=1, gain_min=0.01, gain_max=100.0)
    hist = np.zeros((2, 2, 1, 3, 256), np.uint32)
    n = np.zeros((2, 2, 1, 3), np.uint32)
    hist[0, 1, 0, :] = hR
    hist[1, 0, 0, :] = hL
    n[0, 1, 0, :] = hR.sum()
    n[1, 0, 0, :] = hL.sum()
    return core.fit_quantile_affine([_Cam(0), _Cam(1)], hist, n, p)


def test_quantiles_match_rational_brute_force():
    rng = np.random.default_rng(8)
    for _ in range(20):
        h = _random_hist(rng, rng.integers(1, 120), rng.integers(130, 255), int(rng.integers(64, 5000)))
        cdf = np.cumsum(h.astype(np.int64))
        assert np.array_equal(core.quantile_levels_hit(cdf, int(h.sum())), _quantiles_bruteforce(h))


def test_lines_match_polyfit_and_mixture():
    rng = np.random.default_rng(9)
    for _ in range(10):
        hR = _random_hist(rng, 40, 200, 3000)
        hL = _random_hist(rng, 60, 240, 2500)
        m = _fit(hR, hL)
        ys = _mixture_bruteforce(hR, hL)
        for hist, (k, side) in ((hR, (0, 1)), (hL, (1, 0))):
            xs = _quantiles_bruteforce(hist)
            a, b = np.polyfit(xs.astype(np.float64), ys.astype(np.float64), 1)
            assert abs(m[k, side, 0, 0, 0] - a) < 1e-12 * max(1, abs(a))
            assert abs(m[k, side, 0, 0, 1] - b) < 1e-9 * max(1, abs(b))
            # least squares: the fitted line passes through the means
            fitted = m[k, side, 0, 0, 0] * xs + m[k, side, 0, 0, 1]
            assert abs(fitted.mean() - ys.mean()) < 1e-9


def test_equal_bands_give_the_identity():
    rng = np.random.default_rng(10)
    h = _random_hist(rng, 30, 220, 4000)
    m = _fit(h, h)
    assert np.allclose(m[0, 1, 0, :, 0], 1.0, atol=0) and np.allclose(m[0, 1, 0, :, 1], 0.0, atol=1e-12)
    assert np.allclose(m[1, 0, 0, :, 0], 1.0, atol=0) and np.allclose(m[1, 0, 0, :, 1], 0.0, atol=1e-12)


def test_sides_without_a_valid_seam_keep_the_identity():
    rng = np.random.default_rng(11)
    hR = _random_hist(rng, 30, 220, 30)
    hL = _random_hist(rng, 30, 220, 4000)
    p = core.Params(fit_mode=core.FIT_QUANTILE_AFFINE, min_valid=64)
    m = _fit(hR, hL, p)
    assert (m[..., 0] == 1.0).all() and (m[..., 1] == 0.0).all()
