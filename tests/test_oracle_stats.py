"""Pins of the oracle's measured spectra (band statistics at the seams, with
object removal) and of the whole-frame statistics and thumbnails.

Sec. "White balance and exposure correction": intensity distributions in
narrow bands on each side of a seam; the band split vertically into blocks;
moving pixels (thresholded frame difference) removed from the spectra.
Pins: histogram mass and moments, brute force by an independent numpy
masking on small frames, block partition, the motion threshold's effect on
a static noisy sequence and on an object that jumps into the band.
"""
import numpy as np
import pytest

from paper_1910_03517_gb300 import synth
from conftest import np_frames


def _brute_strip(rgb, luma, prev, S, B, T):
    H, W, _ = rgb.shape
    n = np.zeros((2, B, 3), np.int64)
    s = np.zeros((2, B, 3), np.int64)
    ss = np.zeros((2, B, 3), np.int64)
    h = np.zeros((2, B, 3, 256), np.int64)
    rows = np.arange(H)
    # block of each row: the largest j with floor(j H / B) <= y
    starts = np.array([(j * H) // B for j in range(B)])
    blk = np.searchsorted(starts, rows, side="right") - 1
    for side, cols in ((0, slice(0, S)), (1, slice(W - S, W))):
        band = rgb[:, cols, :].astype(np.int64)
        still = np.ones(band.shape[:2], bool) if prev is None else \
            np.abs(luma[:, cols].astype(int) - prev[:, cols].astype(int)) <= T
        for c in range(3):
            v = band[..., c]
            ok = still & (v > 0) & (v < 255)
            for j in range(B):
                m = ok & (blk[:, None] == j)
                vals = v[m]
                n[side, j, c] = vals.size
                s[side, j, c] = vals.sum()
                ss[side, j, c] = (vals * vals).sum()
                h[side, j, c] = np.bincount(vals, minlength=256)
    return n, s, ss, h


@pytest.mark.parametrize("W,H,S,B", [(64, 38, 8, 3), (96, 40, 16, 16), (40, 30, 4, 7)])
def test_strip_stats_brute_force(orc, W, H, S, B):
    rng = np.random.default_rng(W * H + B)
    rgb = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
    rgb[rng.random((H, W)) < 0.1] = 255          # saturated patches
    luma = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    prev = np.clip(luma.astype(int) + rng.integers(-40, 41, size=(H, W)), 0, 255).astype(np.uint8)
    for p in (None, prev):
        got = orc.strip_stats(rgb, luma, p, S, B, 24)
        n, s, ss, h = _brute_strip(rgb, luma, p, S, B, 24)
        assert (got["n"] == n).all() and (got["sum"] == s).all()
        assert (got["sumsq"] == ss).all() and (got["hist"] == h).all()


def test_strip_moments_and_mass(orc):
    wl = synth.tower12(frames=2)
    wl.cams = wl.cams[:3]
    wl.glare_cams = (1,)
    fr = np_frames(synth.frame_set(wl, 0))
    for k in range(3):
        rgb, luma = orc.convert(wl.cams[k], fr[k])
        st = orc.strip_stats(rgb, luma, None, 32, 16, 24)
        h = st["hist"].astype(np.int64)
        b = np.arange(256)
        assert (h.sum(-1) == st["n"]).all()
        assert ((h * b).sum(-1) == st["sum"].astype(np.int64)).all()
        assert ((h * b * b).sum(-1) == st["sumsq"].astype(np.int64)).all()
        assert (h[..., 0] == 0).all() and (h[..., 255] == 0).all()
        # without saturation or motion every band pixel is counted once
        if k != 1:
            assert (st["n"].sum(1) <= 32 * 1080).all()


def test_blocks_partition_rows(orc):
    for H in (1080, 2160, 480, 37):
        for B in (1, 16, 64):
            assert sum(orc.block_rows(j, H, B) for j in range(B)) == H
            assert max(orc.block_rows(j, H, B) for j in range(B)) - \
                min(orc.block_rows(j, H, B) for j in range(B)) <= 1
    # unsaturated, unmasked: each band pixel lands in exactly one block
    rgb = np.full((37, 20, 3), 100, np.uint8)
    luma = np.zeros((37, 20), np.uint8)
    st = orc.strip_stats(rgb, luma, None, 5, 16, 24)
    assert (st["n"].sum(1) == 5 * 37).all()
    assert [int(st["n"][0, j, 0]) for j in range(16)] == [5 * orc.block_rows(j, 37, 16) for j in range(16)]


def test_static_noisy_sequence_is_almost_never_masked(orc):
    wl = synth.small_pair()
    f0 = np_frames(synth.frame_set(wl, 0))
    f1 = np_frames(synth.frame_set(wl, 1))    # same scene and gains, fresh noise
    for k in range(2):
        rgb0, l0 = orc.convert(wl.cams[k], f0[k])
        rgb1, l1 = orc.convert(wl.cams[k], f1[k])
        a = orc.strip_stats(rgb1, l1, None, 32, 1, 24)
        b = orc.strip_stats(rgb1, l1, l0, 32, 1, 24)
        masked = 1.0 - b["n"].sum() / a["n"].sum()
        assert masked < 1e-3


def test_object_jumping_into_band_is_removed(orc):
    rng = np.random.default_rng(3)
    W, H, S = 64, 40, 16
    base = rng.integers(60, 120, size=(H, W, 3), dtype=np.uint8)
    luma0 = rng.integers(60, 120, size=(H, W), dtype=np.uint8)
    rgb1, luma1 = base.copy(), luma0.copy()
    obj = (slice(10, 22), slice(W - 12, W))            # inside the right band
    rgb1[obj] = 240
    luma1[obj] = np.minimum(luma0[obj].astype(int) + 100, 255).astype(np.uint8)
    with_obj = orc.strip_stats(rgb1, luma1, luma0, S, 1, 24)
    ref = orc.strip_stats(base, luma0, None, S, 1, 24)
    # removing the object's pixels restores the right band's spectrum minus the covered pixels
    keep = np.ones((H, W), bool)
    keep[obj] = False
    n_ref = (keep[:, W - S:]).sum()
    assert (with_obj["n"][1, 0] == n_ref).all()
    sums = base[:, W - S:][keep[:, W - S:]].astype(np.int64).sum(0)
    assert (with_obj["sum"][1, 0] == sums).all()
    assert (with_obj["hist"][0] == ref["hist"][0]).all()   # left band untouched


def test_frame_stats_brute_force_and_mass(orc):
    rng = np.random.default_rng(5)
    rgb = rng.integers(0, 256, size=(30, 50, 3), dtype=np.uint8)
    fs = orc.frame_stats(rgb)
    for c in range(3):
        v = rgb[..., c].reshape(-1).astype(np.int64)
        assert (fs["hist"][c] == np.bincount(v, minlength=256)).all()
        assert fs["sum"][c] == v.sum() and fs["sumsq"][c] == (v * v).sum()
        assert fs["hist"][c].sum() == 30 * 50


def test_thumbnail_cells(orc):
    rng = np.random.default_rng(6)
    for (W, H) in ((640, 480), (130, 75), (64, 36)):
        rgb = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
        th = orc.thumbnail(rgb)
        assert th.shape == (3, 36, 64)
        assert (th.sum((1, 2)) == rgb.reshape(-1, 3).astype(np.int64).sum(0)).all()
        const = np.full((H, W, 3), 7, np.uint8)
        tc = orc.thumbnail(const)
        for j in (0, 17, 35):
            for i in (0, 31, 63):
                area = ((i + 1) * W // 64 - i * W // 64) * ((j + 1) * H // 36 - j * H // 36)
                assert tc[1, j, i] == 7 * area
        # brute force one cell
        i, j = 5, 3
        x0, x1 = i * W // 64, (i + 1) * W // 64
        y0, y1 = j * H // 36, (j + 1) * H // 36
        assert th[2, j, i] == rgb[y0:y1, x0:x1, 2].astype(np.int64).sum()
