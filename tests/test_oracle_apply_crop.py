"""Pins of the oracle's per-pixel application of the Q16 maps and of the
detector-input crop resample.

Sec. "White balance and exposure correction": the map is applied from the
middle of the image towards the common border as a convex combination of
the identity (centre) and f_c (border).  Sec. "Detection": the detector
takes square inputs of fixed size, so windows are cut and resized.
Pins: the identity map, pure gains and offsets in closed form, the ramp's
end points and monotonicity, and the resample against torch's bilinear
interpolation in float64 (align_corners=False), a library special case.
"""
import numpy as np
import pytest
import torch


def _q16(a, b, B=1):
    q = np.zeros((2, B, 3, 2), np.int32)
    q[..., 0] = a
    q[..., 1] = b
    return q


@pytest.fixture(scope="module")
def img():
    return np.random.default_rng(0).integers(0, 256, size=(24, 80, 3), dtype=np.uint8)


@pytest.mark.parametrize("mode", [0, 1])
def test_identity(orc, img, mode):
    assert (orc.apply(img, _q16(65536, 0), 1, mode) == img).all()


def test_pure_gain_and_offset_closed_forms(orc, img):
    v = img.astype(np.int64)
    assert (orc.apply(img, _q16(2 * 65536, 0), 1, 0) == np.minimum(2 * v, 255)).all()
    assert (orc.apply(img, _q16(32768, 0), 1, 0) == (v + 1) // 2).all()     # v/2, halves up
    assert (orc.apply(img, _q16(65536, 10 * 65536), 1, 0) == np.minimum(v + 10, 255)).all()
    assert (orc.apply(img, _q16(65536, -300 * 65536), 1, 0) == 0).all()


def test_ramp_end_points_and_shape(orc):
    for W in (640, 2048, 1920, 8):
        w = np.array([orc.ramp_q16(x, W) for x in range(W)])
        assert w[0] == 65536 and w[-1] == 65536
        assert (np.diff(w[: W // 2]) < 0).all() and (np.diff(w[W // 2:]) > 0).all()
        assert w.min() > 0 and w.max() <= 65536
        assert (w[: W // 2] == w[W // 2:][::-1]).all()           # symmetric about the centre


def test_seam_mode_full_map_at_borders_identity_near_centre(orc, img):
    q = _q16(int(1.5 * 65536), 7 * 65536)
    g = orc.apply(img, q, 1, 0)
    s = orc.apply(img, q, 1, 1)
    W = img.shape[1]
    assert (s[:, 0] == g[:, 0]).all() and (s[:, W - 1] == g[:, W - 1]).all()
    centre = s[:, W // 2 - 1: W // 2 + 1].astype(int) - img[:, W // 2 - 1: W // 2 + 1]
    assert np.abs(centre).max() <= 1 + int(np.ceil((0.5 * 255 + 7) / (W // 2)))
    # between centre and border the effect grows monotonically (positive map)
    flat = np.full((4, W, 3), 100, np.uint8)
    o = orc.apply(flat, q, 1, 1)[0, :, 0].astype(int)
    assert (np.diff(o[: W // 2]) <= 0).all() and (np.diff(o[W // 2:]) >= 0).all()


def test_monotone_in_value(orc):
    ramp = np.tile(np.arange(256, dtype=np.uint8)[None, :, None], (2, 1, 3))
    for a, b in ((0.3, 20.0), (1.7, -40.0), (1.0, 0.0), (3.9, 100.0)):
        o = orc.apply(ramp, _q16(int(a * 65536), int(b * 65536)), 1, 0)[0, :, 0].astype(int)
        assert (np.diff(o) >= 0).all()


def test_blocks_use_their_own_rows(orc):
    H, W, B = 37, 16, 5
    img = np.full((H, W, 3), 100, np.uint8)
    q = np.zeros((2, B, 3, 2), np.int32)
    for j in range(B):
        q[:, j, :, 0] = 65536
        q[:, j, :, 1] = (j + 1) * 65536
    o = orc.apply(img, q, B, 0)
    for y in range(H):
        j = max(jj for jj in range(B) if jj * H // B <= y)
        assert (o[y] == 100 + j + 1).all()


def _torch_crop(rgb, rect, S):
    x0, y0, w, h = rect
    src = torch.from_numpy(rgb[y0:y0 + h, x0:x0 + w].astype(np.float64)).permute(2, 0, 1)[None]
    out = torch.nn.functional.interpolate(src, size=(S, S), mode="bilinear", align_corners=False)
    return (out[0] / 255.0).numpy()


@pytest.mark.parametrize("rect,S", [((0, 0, 80, 24), 16), ((5, 3, 40, 17), 32), ((10, 2, 9, 9), 9),
                                    ((70, 10, 10, 14), 7), ((1, 1, 3, 5), 12)])
def test_crop_matches_torch_bilinear(orc, img, rect, S):
    got = orc.crop(img, rect, S)
    ref = _torch_crop(img, rect, S)
    assert np.abs(got - ref).max() < 1e-12


def test_identity_crop_is_exact(orc, img):
    got = orc.crop(img, (3, 4, 16, 16), 16)
    assert (got == img[4:20, 3:19].transpose(2, 0, 1) / 255.0).all()
