"""Host-side logic of bench.py (no GPU): the timed region's graph plan covers
exactly the requested frame sets, and the crops' algorithmic bytes count
every output value once and every source pixel the bilinear taps touch
once (checked against a brute-force enumeration of the taps)."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("K", [1, 5, 6, 20, 600, 1200, 1201, 1206, 24000, 24001, 100003])
def test_graph_plan_covers_exactly_K(K):
    L, launches, singles = bench.graph_plan(K)
    assert L * launches + singles == K
    assert L >= 1 and launches >= 1 and 0 <= singles < 6
    if K <= bench.MAX_GRAPH_SETS:
        assert (L, launches, singles) == (K, 1, 0)
    else:
        assert L % 6 == 0 and L <= bench.MAX_GRAPH_SETS     # relaunchable back to back


def _taps(x0, w, S):
    """Source columns the half-pixel-centred bilinear resample of a window of
    width w to S outputs reads (clamped inside the window)."""
    cols = set()
    for o in range(S):
        sx = min(max(x0 + (o + 0.5) * w / S - 0.5, x0), x0 + w - 1)
        i = int(np.floor(sx))
        cols.add(i)
        cols.add(min(i + 1, x0 + w - 1))
    return len(cols)


@pytest.mark.parametrize("w,h,S", [(512, 512, 512), (1024, 300, 512), (256, 700, 512), (700, 700, 640), (3, 5, 4)])
def test_crop_bytes_match_brute_force(w, h, S):
    got = bench.crop_alg_bytes([(0, 7, 11, w, h)], S)
    assert got == 6 * S * S + 3 * _taps(7, w, S) * _taps(11, h, S)
