"""Pins of the oracle's fits (per-camera gains and the paper's seam affine
maps), exponential smoothing and Q16 quantisation.

Sec. "White balance and exposure correction": a shared spectrum per seam
from the two bands, per-channel affine maps f_c(x) = a_c x + b_c, adjacent
cameras only; Eq. of the exponential smoothing with alpha = 0.05.
Pins: the closed-form solution on a chain, the gauge, exact recovery of
known camera gains on a mirror-symmetric scene, a balanced array giving
unit gains, a camera with no valid seam keeping the identity, a consistent
ring equal to the chain, the mixture moments computed from pooled samples,
the geometric approach of the smoothing and round-half-away-from-zero.
"""
import math

import numpy as np
import pytest

from paper_1910_03517_gb300 import synth


def _chain_stats(mu_R, mu_L, K, B=1, n=32 * 480):
    nn = np.full((K, 2, B, 3), n, np.uint32)
    s = np.zeros((K, 2, B, 3), np.uint64)
    for k in range(K):
        s[k, 1] = np.uint64(round(mu_R[k] * n))
        s[k, 0] = np.uint64(round(mu_L[k] * n))
    return nn, s


def _cams(K, group=0, H=480):
    return [synth.Camera(640, H, group=group, position=k) for k in range(K)]


@pytest.mark.parametrize("lam,tol", [(0.0, 1e-9), (1e-6, 1e-5)])
def test_chain_closed_form(orc, lam, tol):
    K = 5
    rng = np.random.default_rng(0)
    mu_R = rng.uniform(40, 200, K)
    mu_L = rng.uniform(40, 200, K)
    n, s = _chain_stats(mu_R, mu_L, K)
    mu_R = s[:, 1, 0, 0].astype(float) / n[:, 1, 0, 0]
    mu_L = s[:, 0, 0, 0].astype(float) / n[:, 0, 0, 0]
    p = orc.Params(lam=lam, gain_min=1e-9, gain_max=1e9)
    maps = orc.fit_global(_cams(K), n, s, p)
    x = np.log(maps[:, 0, 0, 0, 0])
    r = [math.log(mu_L[k + 1]) - math.log(mu_R[k]) for k in range(K - 1)]
    xr = np.zeros(K)
    for k in range(1, K):
        xr[k] = xr[k - 1] - r[k - 1]
    xr -= xr.mean()
    assert np.abs(x - xr).max() < tol
    assert abs(x.sum()) < 1e-12 + (0 if lam == 0 else 1e-5)
    assert (maps[:, 0] == maps[:, 1]).all() and (maps[..., 1] == 0).all()


def test_gauge_sum_zero_on_real_stats(orc):
    wl = synth.tower12(frames=1)
    wl.cams = wl.cams[:5]
    fr = [{k: v.numpy() for k, v in f.items()} for f in synth.frame_set(wl, 0)]
    o = orc.ArrayOracle(wl.cams, orc.Params(num_blocks=4))
    r = o.step(fr, want_frame_stats=False)
    x = np.log(r["maps_new"][:, 0, :, :, 0])
    inside = (r["maps_new"][..., 0] > 0.25) & (r["maps_new"][..., 0] < 4.0)
    assert inside.all()
    assert np.abs(x.sum(0)).max() < 1e-12


def test_recovers_known_gains_on_mirror_scene(orc):
    wl = synth.Workload("mirror", _cams(4), frames=1, seed=9, mirror_seams=True, noise_sigma=0.0)
    d = 0.6 + 0.35 * np.random.default_rng(4).random((4, 3))     # no clipping
    import torch
    gains = torch.tensor(d)
    rgbs = [synth.camera_rgb8(wl, k, 0, gains=gains).permute(1, 2, 0).contiguous().numpy() for k in range(4)]
    assert max(int(r.max()) for r in rgbs) < 255
    n = np.stack([orc.strip_stats(r, np.zeros(r.shape[:2], np.uint8), None, 32, 1, 24)["n"] for r in rgbs])
    s = np.stack([orc.strip_stats(r, np.zeros(r.shape[:2], np.uint8), None, 32, 1, 24)["sum"] for r in rgbs])
    maps = orc.fit_global(wl.cams, n, s, orc.Params())
    g = maps[:, 0, 0, :, 0]
    want = 1.0 / d
    want /= np.exp(np.log(want).mean(0))          # gauge: geometric mean 1
    assert np.abs(g / want - 1).max() < 5e-3


def test_balanced_array_gives_unit_gains_and_identity_output(orc):
    wl = synth.Workload("flat", _cams(3, H=64), frames=1, seed=1, noise_sigma=0.0)
    rgb = np.full((64, 640, 3), 90, np.uint8)
    rgb[:, :, 1] = 140
    st = orc.strip_stats(rgb, np.zeros((64, 640), np.uint8), None, 32, 2, 24)
    n = np.stack([st["n"]] * 3)
    s = np.stack([st["sum"]] * 3)
    maps = orc.fit_global(wl.cams, n, s, orc.Params(num_blocks=2))
    assert (maps[..., 0] == 1.0).all()
    q = orc.quantise(maps)
    assert (q[..., 0] == 65536).all() and (q[..., 1] == 0).all()
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, size=(64, 640, 3), dtype=np.uint8)
    assert (orc.apply(img, q[0], 2, 0) == img).all()


def test_camera_without_valid_seam_keeps_identity(orc):
    K = 4
    mu_R = np.array([80.0, 120, 60, 100])
    mu_L = np.array([90.0, 70, 150, 110])
    n, s = _chain_stats(mu_R, mu_L, K)
    n[2] = 10                                     # both bands of camera 2 below min_valid
    maps = orc.fit_global(_cams(K), n, s, orc.Params())
    assert abs(maps[2, 0, 0, 0, 0] - 1.0) < 1e-5
    affine = orc.fit_affine(_cams(K), n, s, s * 0 + 10**6, orc.Params())
    assert (affine[2, :, 0, 0] == [1.0, 0.0]).all()
    assert (affine[1, 1, 0, 0] == [1.0, 0.0]).all() and (affine[3, 0, 0, 0] == [1.0, 0.0]).all()


def test_consistent_ring_equals_chain(orc):
    K = 5
    rng = np.random.default_rng(7)
    x_true = rng.normal(0, 0.2, K)
    x_true -= x_true.mean()
    mu = 100.0
    # camera k sees radiance mu at its seams; its bands read mu / g_k
    n = np.full((K, 2, 1, 3), 4096, np.uint32)
    s = np.zeros((K, 2, 1, 3), np.uint64)
    for k in range(K):
        s[k] = np.uint64(round(4096 * mu * math.exp(-x_true[k])))
    lin = orc.fit_global(_cams(K), n, s, orc.Params(topology=orc.LINEAR))
    ring = orc.fit_global(_cams(K), n, s, orc.Params(topology=orc.RING))
    assert np.abs(np.log(lin[:, 0, 0, 0, 0]) - x_true).max() < 1e-4
    assert np.abs(lin - ring).max() < 1e-5


def test_affine_matches_pooled_mixture_moments(orc):
    rng = np.random.default_rng(11)
    xR = rng.integers(20, 101, size=4000)                 # camera 0, right band
    xL = 2 * rng.integers(20, 101, size=4000) - 10        # camera 1, left band: an affine image
    cams = _cams(2)
    n = np.zeros((2, 2, 1, 3), np.uint32)
    s = np.zeros((2, 2, 1, 3), np.uint64)
    ss = np.zeros((2, 2, 1, 3), np.uint64)
    for (k, side, v) in ((0, 1, xR), (1, 0, xL)):
        n[k, side] = v.size
        s[k, side] = v.sum()
        ss[k, side] = (v.astype(np.int64) ** 2).sum()
    m = orc.fit_affine(cams, n, s, ss, orc.Params(fit_mode=orc.FIT_SEAM_AFFINE))
    pooled = np.concatenate([xR, xL]).astype(float)       # equal counts: equal-weight mixture
    for (k, side, v) in ((0, 1, xR), (1, 0, xL)):
        a, b = m[k, side, 0, 0]
        y = a * v + b
        assert abs(y.mean() - pooled.mean()) < 1e-9
        assert abs(y.std() - pooled.std()) < 1e-9
    # the outer sides of a two-camera chain keep the identity
    assert (m[0, 0, 0, 0] == [1, 0]).all() and (m[1, 1, 0, 0] == [1, 0]).all()


def test_smoothing_static_and_step(orc):
    A = np.full((2, 2, 1, 3, 2), 1.3)
    Bv = np.full((2, 2, 1, 3, 2), 0.7)
    E = orc.smooth(None, A, 0.05)
    assert (E == A).all()
    for t in range(1, 60):
        E = orc.smooth(E, A, 0.05)
    assert np.abs(E - A).max() < 1e-14
    E = A.copy()
    for t in range(1, 80):
        E = orc.smooth(E, Bv, 0.05)
        assert np.abs(E - (Bv + 0.95 ** t * (A - Bv))).max() < 1e-12


def test_round_half_away_from_zero(orc):
    cases = {0.5: 1, -0.5: -1, 1.5: 2, 2.5: 3, -2.5: -3, 0.49999999999999994: 0,
             -0.49999999999999994: 0, 65535.5: 65536, 1e6 + 0.4999: 1000000, 3.0: 3}
    for v, want in cases.items():
        assert orc.round_half_away(v) == want, v
    q = orc.quantise(np.array([1.0, 0.25, 4.0, -1.5 / 65536, 0.5 / 65536]))
    assert list(q) == [65536, 16384, 262144, -2, 1]
