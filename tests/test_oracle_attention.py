"""Pins of the difference-attention oracle (Sec. "Attention mechanisms", the
difference approach): brute-force window sums, the threshold's edge, mass
conservation, a static scene and a moving block."""
import numpy as np

from oracle import attention as at


class _Cam:
    def __init__(self, w, h):
        self.width, self.height = w, h


def test_window_sums_equal_brute_force():
    rng = np.random.default_rng(3)
    for (W, H, window) in [(300, 200, 64), (256, 256, 128), (97, 61, 32), (40, 30, 64)]:
        on = rng.random((H, W)) < 0.2
        cc = at.cell_counts(on, window // 2)
        assert cc.sum() == on.sum()                       # mass
        for (i, j, x0, y0, w, h) in at.window_rects(W, H, window):
            ny, nx = cc.shape
            via_cells = cc[j:min(j + 2, ny), i:min(i + 2, nx)].sum()
            assert via_cells == on[y0:y0 + h, x0:x0 + w].sum(), (W, H, window, i, j)
            assert x0 + w <= W and y0 + h <= H


def test_windows_cover_the_frame_at_half_stride():
    rects = at.window_rects(1024, 512, 256)
    xs = sorted({r[2] for r in rects})
    ys = sorted({r[3] for r in rects})
    assert xs == list(range(0, 1024 - 128, 128)) and ys == list(range(0, 512 - 128, 128))
    assert all(r[4] == 256 and r[5] == 256 for r in rects)


def test_threshold_edge():
    prev = np.full((4, 4), 100, np.uint8)
    cur = prev.copy()
    cur[0, 0] = 124          # |d| = T: not on
    cur[0, 1] = 125          # T + 1: on
    cur[1, 0] = 76           # |d| = T downwards: not on
    cur[1, 1] = 75
    on = at.change_map(cur, prev, 24)
    assert on.sum() == 2 and on[0, 1] and on[1, 1]


def test_static_scene_proposes_nothing():
    rng = np.random.default_rng(4)
    lum = [rng.integers(0, 256, (120, 200), dtype=np.uint8)]
    props, counts = at.proposals([_Cam(200, 120)], lum, lum, window=64, min_on=1)
    assert props == [] and counts[0].sum() == 0


def test_moving_block_is_proposed():
    H, W = 300, 400
    prev = np.full((H, W), 80, np.uint8)
    cur = prev.copy()
    prev[100:140, 50:110] = 220          # a bright block ...
    cur[100:140, 60:120] = 220           # ... moved 10 px to the right
    props, counts = at.proposals([_Cam(W, H)], [prev], [cur], window=128, min_on=200)
    on = at.change_map(cur, prev, 24)
    assert on.sum() == 2 * 40 * 10 and counts[0].sum() == on.sum()
    assert props, "the block's windows are proposed"
    for (k, x0, y0, w, h) in props:
        assert on[y0:y0 + h, x0:x0 + w].sum() >= 200
    # every window holding at least min_on on-pixels is proposed, in order
    want = [(0, x0, y0, w, h) for (_, _, x0, y0, w, h) in at.window_rects(W, H, 128)
            if on[y0:y0 + h, x0:x0 + w].sum() >= 200]
    assert props == want


def test_cap_keeps_the_first_in_order():
    rng = np.random.default_rng(5)
    prev = rng.integers(0, 256, (256, 256), dtype=np.uint8)
    cur = (prev.astype(np.int16) + 128) % 256
    full, _ = at.proposals([_Cam(256, 256)], [prev], [cur.astype(np.uint8)], window=64, min_on=1, cap=1000)
    capped, _ = at.proposals([_Cam(256, 256)], [prev], [cur.astype(np.uint8)], window=64, min_on=1, cap=5)
    assert len(full) == 49 and capped == full[:5]
