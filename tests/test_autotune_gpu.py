"""The launch-shape autotuner (rt_autotune, include/rt.h): it times
candidate shapes on the caller's frame sets, keeps the sequence state, caches
its choice in a JSON file, and no shape changes any result."""
import json

import numpy as np
import pytest
import torch

from paper_1910_03517_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1910_03517_gb300 import build, rt as rtmod
    build.build()
    rtmod.load()
    return rtmod


def _setup():
    wl = synth.small_pair()
    wl.n_crops, wl.crop_side, wl.crop_out = 5, (16, 200), 40
    frames = [synth.frame_set(wl, t, device="cuda") for t in range(8)]
    crops = [synth.crop_list(wl, t) for t in range(8)]
    return wl, frames, crops


def _outputs(arr, K):
    maps, q16 = arr.get_gains()
    imgs = [arr.get_corrected(k).clone() for k in range(K)]
    return maps, q16, imgs, arr.get_crops().clone(), arr.get_stats()["frame_hist"].copy()


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for x, y in zip(a[2], b[2]):
        assert torch.equal(x, y)
    assert torch.equal(a[3], b[3])
    assert np.array_equal(a[4], b[4])


@pytest.mark.parametrize("kw", [{}, {"fit_mode": 1, "num_blocks": 16, "schedule": 1}])
def test_autotune_keeps_state_and_caches(rt, tmp_path, kw):
    """Also the seam maps under the lagged schedule: the frame set after the
    tuning applies the restored Q16 slot through its coefficient table, which
    the tuning's own frame sets had overwritten."""
    wl, frames, crops = _setup()
    K = len(wl.cams)
    cache = str(tmp_path / "tuning.json")
    a = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    b = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    a.submit_frames(frames[0], 0, crops[0])
    b.submit_frames(frames[0], 0, crops[0])
    before = a.get_gains()
    ring = list(range(1, 7))
    t = a.autotune([frames[i] for i in ring], [crops[i] for i in ring], cache_path=cache)
    assert t["from_cache"] == 0 and t["candidates"] >= 10 and t["step_us"] > 0
    assert 64 <= t["pass_b_threads"] <= 512 and t["pass_b_ctas_per_sm"] in (1, 2)
    assert a.get_tuning()["pass_b_threads"] == t["pass_b_threads"]
    # the smoothing state and the last Q16 table are those of frame set 0 again
    after = a.get_gains()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    # the sequence continues exactly as on an untuned array
    for i in (1, 2, 3):
        a.submit_frames(frames[i], i, crops[i])
        b.submit_frames(frames[i], i, crops[i])
        _same(_outputs(a, K), _outputs(b, K))
    # a cache hit applies the same shape without timing
    c = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    t2 = c.autotune([frames[i] for i in ring], [crops[i] for i in ring], cache_path=cache)
    assert t2["from_cache"] == 1 and t2["candidates"] == 0
    for k in ("pass_b_threads", "pass_b_ctas_per_sm", "pass_a_rows", "pass_a_threads", "crop_threads", "crop_grid"):
        assert t2[k] == t[k], k
    doc = json.load(open(cache))
    assert len(doc) == 1 and list(doc.values())[0]["pass_b_threads"] == t["pass_b_threads"]
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize("kw", [{}, {"fit_mode": 1, "num_blocks": 16, "schedule": 1}])
def test_every_shape_gives_the_same_results(rt, kw):
    wl, frames, crops = _setup()
    K = len(wl.cams)
    a = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    b = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    b.set_tuning(pass_b_threads=64, pass_b_ctas_per_sm=1, pass_a_rows=8, pass_a_threads=256, crop_threads=128,
                 crop_grid=1)
    for i in range(4):
        a.submit_frames(frames[i], i, crops[i])
        b.submit_frames(frames[i], i, crops[i])
        _same(_outputs(a, K), _outputs(b, K))
    a.close()
    b.close()


def test_invalid_shapes_are_rejected(rt):
    wl, _, _ = _setup()
    a = rt.CameraArray(wl.cams)
    for bad in ({"pass_b_threads": 100}, {"pass_b_threads": 1024}, {"pass_b_ctas_per_sm": 3}, {"pass_a_rows": 4},
                {"pass_a_threads": 96}, {"crop_threads": 64}, {"crop_grid": 0}):
        with pytest.raises(rt.RtError) as ei:
            a.set_tuning(**bad)
        assert ei.value.status == rt.RT_ERR_INVALID, bad
    with pytest.raises(rt.RtError):
        a.autotune([synth.frame_set(wl, 0, device="cuda")] * 4)   # not a multiple of 6
    a.close()
