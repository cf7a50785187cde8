"""The learned surrogate inside the frame-set pipeline, through the C ABI.

- Training on the array's own generated frame sets (rt_surrogate_train)
  lowers the loss and predicts held-out arrays' gains far better than no
  correction (rt_surrogate_evaluate).
- A checkpoint (rt_surrogate_save / rt_surrogate_load: FP32 weights, both
  Adam moments, step and call counts) resumes training bit for bit.
- Surrogate mode with tolerance 0 never trusts a prediction: every frame set
  is corrected with the plain fit, so maps, Q16 tables and images equal the
  plain pipeline's exactly (the fit, smoothing and quantisation run on the
  same operands).
- The fallback switches on and off with the judgement: with an unreachable
  tolerance the prediction is applied (the fit runs every judge_every-th
  frame set) and the smoothed maps follow the prediction the handle's network
  makes from the thumbnails of frame set t - 1 (mode 1) or t - 2 (mode 2);
  tolerance 0 turns the fallback on at the next judgement, a large one off
  again.
"""
import os
import tempfile

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


def _cams(n=16, w=256, h=144):
    return [synth.Camera(w, h, position=i) for i in range(n)]


def _array(rt, cams, **kw):
    return rt.CameraArray(cams, flags=rt.RT_FLAG_THUMBNAILS | rt.RT_FLAG_FRAME_STATS, **kw)


def test_train_and_evaluate(rt):
    cams = _cams()
    arr = _array(rt, cams)
    losses = []
    for ep in range(6):
        losses.append(arr.surrogate_train(16 * 160, batch=256, lr=1e-3 * 0.5 ** ep, seed=1))
    assert len(losses[0]) == 16 * 160 // 256
    assert np.isfinite(np.concatenate(losses)).all()
    assert np.mean(losses[-1]) < 0.5 * np.mean(losses[0][:3]), (losses[0][:3], losses[-1][-3:])
    err, err_id = arr.surrogate_evaluate(16 * 24, seed=2)
    assert err.shape == (24, 16)
    assert np.median(err) < 0.5 * np.median(err_id), (np.median(err), np.median(err_id))
    arr.close()


def test_checkpoint_resumes_bit_for_bit(rt):
    cams = _cams(8, 256, 144)
    n, seed = 8 * 64, 5
    a = _array(rt, cams)
    a.surrogate_train(n, 128, 1e-3, seed)
    a.surrogate_train(n, 128, 5e-4, seed)
    want = a.surrogate_params()
    a.close()
    b = _array(rt, cams)
    b.surrogate_train(n, 128, 1e-3, seed)
    first = b.surrogate_params()
    path = os.path.join(tempfile.gettempdir(), "rt_sg_%d.bin" % os.getpid())
    b.surrogate_save(path)
    b.close()
    c = _array(rt, cams)
    c.surrogate_load(path)
    assert np.array_equal(c.surrogate_params(), first)
    c.surrogate_train(n, 128, 5e-4, seed)
    got = c.surrogate_params()
    c.close()
    os.remove(path)
    assert not np.array_equal(got, first)          # the second pass changed the weights
    assert np.array_equal(got, want)               # ... exactly as uninterrupted training did
    # a file that is not a checkpoint is refused
    bad = os.path.join(tempfile.gettempdir(), "rt_sg_bad_%d.bin" % os.getpid())
    open(bad, "wb").write(b"not a checkpoint")
    d = _array(rt, cams)
    with pytest.raises(rt.RtError):
        d.surrogate_load(bad)
    d.close()
    os.remove(bad)


def _sequence(cams, frames, seed=41):
    wl = synth.Workload("surrogate pipeline", cams, frames=frames, seed=seed, gain_walk=0.01, moving_object=True)
    return [synth.frame_set(wl, t, device="cuda") for t in range(frames)]


@pytest.mark.parametrize("mode", [1, 2])
def test_tolerance_zero_is_the_plain_pipeline(rt, mode):
    cams = _cams(8, 256, 144)
    seq = _sequence(cams, 10)
    plain = _array(rt, cams)
    sur = _array(rt, cams, surrogate_mode=mode, judge_every=3, fallback_tol=0.0)
    sur.surrogate_train(8 * 64, 128, 1e-3, seed=7)
    for t, fs in enumerate(seq):
        plain.submit_frames(fs, t)
        sur.submit_frames(fs, t)
        mp, qp = plain.get_gains()
        ms, qs = sur.get_gains()
        assert np.array_equal(mp, ms), t
        assert np.array_equal(qp, qs), t
        for k in range(len(cams)):
            assert torch.equal(plain.get_corrected(k), sur.get_corrected(k)), (t, k)
    r = sur.surrogate_report()
    assert r["frame_sets"] == 10 and r["plain"] == 10 and r["predicted"] == 0
    # every frame set from `mode` on has a prediction to judge (and fails)
    assert r["judged"] == 10 - mode and r["judged_failed"] == 10 - mode and r["fallback"] == 1
    plain.close()
    sur.close()


def _expected_step(E_prev, g, alpha=0.05):
    """The solve's smoothing of the gain maps (b stays 0)."""
    e = E_prev.copy()
    e[..., 0] = (1 - alpha) * E_prev[..., 0] + alpha * g[..., 0]
    e[..., 1] = (1 - alpha) * E_prev[..., 1]
    return e


def test_fallback_switches_on_and_off(rt):
    cams = _cams(8, 256, 144)
    seq = _sequence(cams, 18)
    arr = _array(rt, cams, surrogate_mode=1, judge_every=3, fallback_tol=1e9)
    arr.surrogate_train(8 * 64, 128, 1e-3, seed=9)
    E_prev = None
    for t, fs in enumerate(seq):
        if t == 9:
            arr.surrogate_set_tolerance(0.0)       # next judgement (t = 9) fails: fallback on
        if t == 12:
            arr.surrogate_set_tolerance(1e9)       # next judgement (t = 12) passes: fallback off
        pred = arr.surrogate_predict()[0] if t > 0 else None   # from frame set t-1's thumbnails
        arr.submit_frames(fs, t)
        E, q = arr.get_gains()
        if t in (2, 4, 5, 13, 14):                 # prediction applied without a judgement
            assert np.abs(E - _expected_step(E_prev, pred)).max() <= 1e-12 * np.abs(E).max(), t
        if t in (10, 11):                          # fallback: the fit's gains, not the prediction
            assert np.abs(E - _expected_step(E_prev, pred)).max() > 1e-9, t
        want_q = np.where(65536 * E >= 0, np.floor(65536 * E + 0.5), -np.floor(-65536 * E + 0.5))
        assert np.array_equal(q, want_q.astype(np.int32)), t
        E_prev = E
        r = arr.surrogate_report()
        if t == 8:
            # 0: first (plain); 1: judged, passes; then judged at 3 and 6
            assert (r["plain"], r["predicted"], r["judged"], r["judged_failed"], r["fallback"]) == (1, 8, 3, 0, 0), r
        if t == 11:
            # 9: judged, fails; 10, 11: fallback (judged every frame set, fail)
            assert (r["plain"], r["judged"], r["judged_failed"], r["fallback"]) == (4, 6, 3, 1), r
        if t == 17:
            # 12: judged, passes; 13, 14 predicted; 15 judged, passes; 16, 17
            assert (r["plain"], r["predicted"], r["judged"], r["judged_failed"], r["fallback"]) == (4, 14, 8, 3, 0), r
    arr.close()


def test_lag_two_predicts_from_two_frame_sets_back(rt):
    """Mode 2: frame set t gets the prediction made from frame set t-2's
    thumbnails (frame sets 0 and 1 the fit's gains)."""
    cams = _cams(8, 256, 144)
    seq = _sequence(cams, 9)
    arr = _array(rt, cams, surrogate_mode=2, judge_every=4, fallback_tol=1e9)
    arr.surrogate_train(8 * 64, 128, 1e-3, seed=13)
    preds, E_prev = {}, None
    for t, fs in enumerate(seq):
        arr.submit_frames(fs, t)
        E, _ = arr.get_gains()
        preds[t] = arr.surrogate_predict()[0]           # from frame set t's thumbnails
        if t in (3, 5, 6, 7):                           # predicted, not judged (judged: 2 and 4 and 8)
            assert np.abs(E - _expected_step(E_prev, preds[t - 2])).max() <= 1e-12 * np.abs(E).max(), t
        E_prev = E
    r = arr.surrogate_report()
    # 0, 1: plain (no prediction yet); 2: judged, passes; 4, 8: judged
    assert (r["plain"], r["predicted"], r["judged"], r["judged_failed"]) == (2, 7, 3, 0), r
    arr.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_surrogate_mode_captured_ring_matches_single_submits(rt, mode):
    cams = _cams(8, 256, 144)
    seq = _sequence(cams, 12)
    outs = []
    for captured in (False, True):
        arr = _array(rt, cams, surrogate_mode=mode, judge_every=4, fallback_tol=1e9)
        arr.surrogate_train(8 * 64, 128, 1e-3, seed=11)
        arr.submit_frames(seq[0], 0)
        if captured:
            arr.capture_sequence(seq[1:7])
            arr.launch_sequence()
            for t in range(7, 12):
                arr.submit_frames(seq[t], t)
        else:
            for t in range(1, 12):
                arr.submit_frames(seq[t], t)
        outs.append((arr.get_gains(), arr.surrogate_report()))
        arr.close()
    (m0, q0), r0 = outs[0]
    (m1, q1), r1 = outs[1]
    assert np.array_equal(m0, m1) and np.array_equal(q0, q1)
    assert r0 == r1
