"""Pins of the oracle's colour conversion (decoded NV12 / mono frames -> RGB).

The paper leaves the decoder's colour matrix unstated (Sec. "System": H.264
1920x1080 streams decoded by NVDEC); the reading is ITU-R BT.709 limited
range in Q8 integers.  The pins below do not re-type the oracle's formula:
they compare it with the real-valued matrix of the standard, closed-form
points of the range, and structural facts of 4:2:0 chroma.
"""
import numpy as np
import pytest

from paper_1910_03517_gb300 import synth


def _all_triples_frame():
    """A 4096x4096 NV12 frame holding every (Y, U, V) triple exactly once:
    each 2x2 block has one (U, V) pair and four Y values."""
    W = H = 4096
    bx = np.arange(W // 2)
    by = np.arange(H // 2)
    b = by[:, None] * (W // 2) + bx[None, :]               # block index
    pair = b // 64
    U = (pair // 256).astype(np.uint8)
    V = (pair % 256).astype(np.uint8)
    ybase = 4 * (b % 64)
    y = np.zeros((H, W), np.uint8)
    y[0::2, 0::2] = ybase
    y[0::2, 1::2] = ybase + 1
    y[1::2, 0::2] = ybase + 2
    y[1::2, 1::2] = ybase + 3
    uv = np.zeros((H // 2, W), np.uint8)
    uv[:, 0::2] = U
    uv[:, 1::2] = V
    return y, uv


@pytest.mark.parametrize("matrix,kr,kb", [(0, 0.2126, 0.0722), (1, 0.299, 0.114)])
def test_all_triples_within_one_of_real_matrix(orc, matrix, kr, kb):
    y, uv = _all_triples_frame()
    cam = synth.Camera(4096, 4096)
    rgb, _ = orc.convert(cam, {"y": y, "uv": uv}, matrix)
    Yf = y.astype(np.float64)
    Uf = np.repeat(np.repeat(uv[:, 0::2], 2, 0), 2, 1).astype(np.float64)
    Vf = np.repeat(np.repeat(uv[:, 1::2], 2, 0), 2, 1).astype(np.float64)
    kg = 1 - kr - kb
    yp = (Yf - 16) * 255 / 219
    cb = (Uf - 128) * 255 / 224
    cr = (Vf - 128) * 255 / 224
    ref = np.stack([yp + 2 * (1 - kr) * cr,
                    yp - 2 * (1 - kb) * kb / kg * cb - 2 * (1 - kr) * kr / kg * cr,
                    yp + 2 * (1 - kb) * cb], -1)
    ref = np.clip(ref, 0, 255)
    err = np.abs(rgb.astype(np.float64) - ref)
    # Q8 coefficients and a floor-with-half-offset round: the integer result
    # is within one level of the exact matrix everywhere.
    assert err.max() <= 1.0 + 1e-9
    # and within half a level plus the coefficient quantisation for most triples
    assert np.mean(err <= 0.75) > 0.97


# The published 8-bit integer forms of the two limited-range matrices
# (coefficients scaled by 256): luma 298, then Cr->R, Cb->G, Cr->G, Cb->B.
Q8 = {0: (298, 459, 55, 136, 541),      # ITU-R BT.709
      1: (298, 409, 100, 208, 516)}     # ITU-R BT.601


@pytest.mark.parametrize("matrix,kr,kb", [(0, 0.2126, 0.0722), (1, 0.299, 0.114)])
def test_q8_integers_exact(orc, matrix, kr, kb):
    """The oracle's integers are exactly the standard's Q8 matrix, and that
    matrix follows from the luma weights (Kr, Kb) of the standard: 255/219
    scales limited-range luma, 255/224 chroma, and the RGB rows are
    R = Y' + 2(1-Kr) Cr', G = Y' - 2(1-Kb)Kb/Kg Cb' - 2(1-Kr)Kr/Kg Cr',
    B = Y' + 2(1-Kb) Cb' (Kg = 1 - Kr - Kb)."""
    kg = 1.0 - kr - kb
    sy, sc = 256 * 255 / 219, 256 * 255 / 224
    derived = (round(sy), round(sc * 2 * (1 - kr)), round(sc * 2 * (1 - kb) * kb / kg),
               round(sc * 2 * (1 - kr) * kr / kg), round(sc * 2 * (1 - kb)))
    assert derived == Q8[matrix]
    assert tuple(int(v) for v in orc.color_coeffs(matrix)) == Q8[matrix]


@pytest.mark.parametrize("matrix", [0, 1])
def test_all_triples_exact_with_published_integers(orc, matrix):
    """Every (Y, U, V) triple converts exactly as the published Q8 matrix
    gives: v = clamp(floor(N / 256), 0, 255), N = 298 C + ... + 128 (C = Y - 16,
    D = U - 128, E = V - 128).  A coefficient off by one (e.g. 460 for 459)
    changes some triple's output and fails here."""
    cy, crv, cgu, cgv, cbu = Q8[matrix]
    y, uv = _all_triples_frame()
    rgb, _ = orc.convert(synth.Camera(4096, 4096), {"y": y, "uv": uv}, matrix)
    C = y.astype(np.int64) - 16
    D = np.repeat(np.repeat(uv[:, 0::2], 2, 0), 2, 1).astype(np.int64) - 128
    E = np.repeat(np.repeat(uv[:, 1::2], 2, 0), 2, 1).astype(np.int64) - 128
    want = np.stack([(cy * C + crv * E + 128) // 256,
                     (cy * C - cgu * D - cgv * E + 128) // 256,
                     (cy * C + cbu * D + 128) // 256], -1)
    assert np.array_equal(rgb, np.clip(want, 0, 255).astype(np.uint8))


def test_range_end_points(orc):
    cam = synth.Camera(2, 2)
    for Y, want in [(235, 255), (16, 0), (255, 255), (0, 0)]:
        y = np.full((2, 2), Y, np.uint8)
        uv = np.array([[128, 128]], np.uint8)
        rgb, luma = orc.convert(cam, {"y": y, "uv": uv})
        assert (rgb == want).all(), (Y, rgb)
        assert (luma == Y).all()


def test_chroma_shared_by_2x2_block(orc):
    rng = np.random.default_rng(0)
    W, H = 64, 32
    y = np.full((H, W), 120, np.uint8)
    uv = rng.integers(16, 241, size=(H // 2, W), dtype=np.uint8)
    rgb, _ = orc.convert(synth.Camera(W, H), {"y": y, "uv": uv})
    blocks = rgb.reshape(H // 2, 2, W // 2, 2, 3)
    assert (blocks == blocks[:, :1, :, :1, :]).all()        # 4 pixels of a block agree
    # with constant luma, red depends on V only and blue on U only
    V = uv[:, 1::2].reshape(-1)
    U = uv[:, 0::2].reshape(-1)
    R = blocks[:, 0, :, 0, 0].reshape(-1)
    Bc = blocks[:, 0, :, 0, 2].reshape(-1)
    for v in np.unique(V):
        assert len(np.unique(R[V == v])) == 1
    for u in np.unique(U):
        assert len(np.unique(Bc[U == u])) == 1


def test_pitch_is_respected(orc):
    rng = np.random.default_rng(1)
    W, H, P = 48, 16, 64
    y = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    uv = rng.integers(0, 256, size=(H // 2, W), dtype=np.uint8)
    yp = np.full((H, P), 7, np.uint8)
    yp[:, :W] = y
    uvp = np.full((H // 2, P), 9, np.uint8)
    uvp[:, :W] = uv
    a, _ = orc.convert(synth.Camera(W, H), {"y": y, "uv": uv})
    b, _ = orc.convert(synth.Camera(W, H, y_pitch=P, uv_pitch=P), {"y": yp, "uv": uvp})
    assert (a == b).all()


def test_mono16_to_gray(orc):
    cam = synth.Camera(4, 2, fmt=synth.MONO16, bit_depth=12)
    ir = np.array([[0, 15, 16, 4095], [4080, 2048, 65535 >> 1, 31]], np.uint16).view(np.int16)
    rgb, luma = orc.convert(cam, {"ir": ir})
    want = np.array([[0, 0, 1, 255], [255, 128, 255, 1]], np.uint8)
    assert (rgb == want[..., None]).all()
    assert (luma == want).all()
