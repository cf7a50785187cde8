"""Pins of the oracle's convex blending of adjacent block maps: the block
centres carry the block maps exactly, the edges hold, rows between two
centres are monotone and between the two maps, equal blocks give the block
map everywhere, and the apply with B = H rows equals the apply with blocks
when every block has one row."""
import numpy as np

from oracle import core


def _q(vals_a, vals_b=None):
    B = len(vals_a)
    q = np.zeros((2, B, 3, 2), np.int32)
    for j, v in enumerate(vals_a):
        q[:, j, :, 0] = v
        q[:, j, :, 1] = 0 if vals_b is None else vals_b[j]
    return q


def test_centres_edges_and_monotone():
    H, B = 100, 4                        # blocks of 25 rows, centres 12, 37, 62, 87
    q = _q([60000, 70000, 65536, 80000], [-1000, 500, 0, 2000])
    r = core.blend_rows(q, H, B)
    for j, c in enumerate((12, 37, 62, 87)):
        assert np.array_equal(r[:, c], q[:, j])          # centre rows (C_j even)
    assert (r[:, :12] == q[:, :1]).all() and (r[:, 88:] == q[:, 3:]).all()
    for j in range(1, B):
        seg = r[0, (12 + 25 * (j - 1)):(12 + 25 * j) + 1, 0, 0].astype(np.int64)
        lo, hi = sorted((int(q[0, j - 1, 0, 0]), int(q[0, j, 0, 0])))
        assert (seg >= lo).all() and (seg <= hi).all()
        d = np.diff(seg)
        assert (d >= 0).all() or (d <= 0).all()


def test_equal_blocks_and_one_row_blocks():
    q = _q([70000] * 5, [300] * 5)
    r = core.blend_rows(q, 37, 5)
    assert (r == q[:, :1]).all()
    # one row per block: blending changes nothing
    rng = np.random.default_rng(3)
    q2 = rng.integers(40000, 90000, (2, 8, 3, 2)).astype(np.int32)
    assert np.array_equal(core.blend_rows(q2, 8, 8), q2)


def test_odd_heights():
    H, B = 1079, 16
    q = np.random.default_rng(4).integers(30000, 100000, (2, B, 3, 2)).astype(np.int32)
    r = core.blend_rows(q, H, B)
    C = [(j * H) // B + ((j + 1) * H) // B - 1 for j in range(B)]
    for j in range(B):
        if C[j] % 2 == 0:
            assert np.array_equal(r[:, C[j] // 2], q[:, j])
