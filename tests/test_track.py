"""Detection post-processing and tracking (Sec. "AI-based video tracking"):
the library's tracker (host code, no GPU needed) against the oracle on
random scenes, and the GPU NMS (marked gpu) against the oracle's greedy NMS."""
import numpy as np
import pytest

from oracle import track as otrack


def _f32(rows):
    """The boxes as the library sees them (float32 coordinates and scores)."""
    return [tuple(float(np.float32(v)) for v in r[:5]) + (int(r[5]),) for r in rows]


def _scene(rng, n_obj, frames, classes=3):
    """Boxes of n_obj objects moving a few pixels per frame; objects appear
    and disappear; jittered detections; spurious boxes now and then."""
    pos = rng.uniform(0, 1000, (n_obj, 2))
    size = rng.uniform(20, 80, (n_obj, 2))
    vel = rng.uniform(-6, 6, (n_obj, 2))
    cls = rng.integers(0, classes, n_obj)
    life = np.stack([rng.integers(0, frames // 2, n_obj), rng.integers(frames // 2, frames + 1, n_obj)], 1)
    out = []
    for f in range(frames):
        rows = []
        for i in range(n_obj):
            if not (life[i, 0] <= f < life[i, 1]) or rng.random() < 0.1:
                continue
            c = pos[i] + vel[i] * f + rng.normal(0, 1.0, 2)
            rows.append((c[0], c[1], c[0] + size[i, 0], c[1] + size[i, 1], rng.uniform(0.7, 1.0), int(cls[i])))
        if rng.random() < 0.3:
            c = rng.uniform(0, 1000, 2)
            rows.append((c[0], c[1], c[0] + 30, c[1] + 30, 0.8, int(rng.integers(0, classes))))
        out.append(rows)
    return out


def test_tracker_matches_the_oracle():
    from paper_1910_03517_gb300 import build, rt
    build.build()
    for seed in range(4):
        rng = np.random.default_rng(seed)
        lib, ref = rt.Tracker(), otrack.Tracker()
        for f, rows in enumerate(_scene(rng, 12, 40)):
            rows = _f32(rows)
            assert lib.update(rows, f) == ref.update(rows, f), (seed, f)
        objs = lib.objects()
        assert len(objs) == len(ref.objects)
        for o, r in zip(objs, ref.objects):
            assert o["id"] == r["id"] and o["cls"] == r["cls"] and o["frame"] == r["frame"]
            assert o["history"] == len(r["history"])
        lib.close()


def test_tracker_rejects_bad_parameters():
    from paper_1910_03517_gb300 import build, rt
    build.build()
    for bad in ((0.0, 0.05, 0.001), (1.5, 0.05, 0.001), (0.99, 1.0, 0.001), (0.99, 0.05, -1.0)):
        with pytest.raises(rt.RtError):
            rt.Tracker(*bad)


@pytest.mark.gpu
def test_gpu_nms_matches_the_oracle():
    from paper_1910_03517_gb300 import build, rt
    build.build()
    rng = np.random.default_rng(7)
    for n in (1, 17, 300, 2000, 4096):
        while True:
            rows = []
            for _ in range(n):
                c = rng.uniform(0, 600, 2)
                s = rng.uniform(10, 60, 2)
                rows.append((c[0], c[1], c[0] + s[0], c[1] + s[1], rng.uniform(0.3, 1.0), int(rng.integers(0, 4))))
            rows = _f32(rows)
            # no same-category pair with an IoU within 1e-5 of the tolerance
            # (the GPU decides in float32, the oracle in float64)
            b = np.array(rows, np.float64)
            ix = np.clip(np.minimum(b[:, None, 2], b[None, :, 2]) - np.maximum(b[:, None, 0], b[None, :, 0]), 0, None)
            iy = np.clip(np.minimum(b[:, None, 3], b[None, :, 3]) - np.maximum(b[:, None, 1], b[None, :, 1]), 0, None)
            inter = ix * iy
            area = (b[:, 2] - b[:, 0]) * (b[:, 3] - b[:, 1])
            iou = inter / (area[:, None] + area[None, :] - inter)
            same = b[:, None, 5] == b[None, :, 5]
            if not (same & (np.abs(iou - 0.45) < 1e-5)).any():
                break
        assert rt.nms(rows, 0.65, 0.45) == otrack.nms(rows, 0.65, 0.45), n
    # equal scores keep the earlier box
    same = _f32([(0, 0, 10, 10, 0.9, 0), (1, 0, 11, 10, 0.9, 0)])
    assert rt.nms(same, 0.5, 0.45) == [0]
    with pytest.raises(rt.RtError):
        rt.nms(_f32([(0, 0, 1, 1, 0.9, 40000)]))
