"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point the headers declare; configurations that break a
stated rule are rejected before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_1910_03517_gb300 import build, rt
    build.build()
    return rt.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(rt_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    from paper_1910_03517_gb300 import rt
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(L, name), name
    assert set(rt.EXPORTS) | set(rt.MLP_EXPORTS) <= declared


def test_defaults(L):
    from paper_1910_03517_gb300 import rt
    p = rt.default_params()
    assert (p.strip_width, p.num_blocks, p.motion_threshold, p.min_valid) == (32, 1, 24, 64)
    assert p.alpha == 0.05 and p.lambda_ == 1e-6 and (p.gain_min, p.gain_max) == (0.25, 4.0)
    assert (p.surrogate_mode, p.judge_every, p.fallback_tol) == (0, 8, 0.02)


def test_surrogate_calls_refuse_a_null_handle(L):
    from paper_1910_03517_gb300 import rt
    rt._load_mlp(L)
    assert L.rt_surrogate_train(None, 256, 256, 1e-3, 0) == rt.RT_ERR_INVALID
    assert L.rt_surrogate_save(None, b"x") == rt.RT_ERR_INVALID
    assert L.rt_surrogate_load(None, b"x") == rt.RT_ERR_INVALID
    assert L.rt_surrogate_set_tolerance(None, 0.0) == rt.RT_ERR_INVALID
    assert L.rt_surrogate_evaluate(None, 16, 0, None, None, 0, None) == rt.RT_ERR_INVALID


def _config(L, cams, **kw):
    from paper_1910_03517_gb300 import rt
    p = rt.default_params()
    arr = (rt.CameraDesc * len(cams))(*cams)
    p.num_cameras = len(cams)
    p.cams = ctypes.cast(arr, ctypes.POINTER(rt.CameraDesc))
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    st = L.rt_array_config(ctypes.byref(p), None, ctypes.byref(h))
    return st, L.rt_last_error(None).decode()


@pytest.mark.parametrize("cam,kw,needle", [
    ((641, 480, 0, 8, 656, 656, 0, 0), {}, "even"),
    ((640, 480, 0, 8, 650, 640, 0, 0), {}, "y_pitch"),
    ((640, 480, 0, 8, 640, 600, 0, 0), {}, "uv_pitch"),
    ((40, 480, 0, 8, 48, 48, 0, 0), {}, "strip_width"),
    ((640, 480, 1, 20, 1280, 0, 0, 0), {}, "bit_depth"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"num_blocks": 65}, "num_blocks"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"strip_width": 24}, "strip_width"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"alpha": 0.0}, "alpha"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"fit_mode": 7}, "fit_mode"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"fit_mode": 4}, "fit_mode"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"gain_max": 17.0}, "gain_max"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"max_crops": 4, "crop_size": 0}, "crop_size"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 3}, "surrogate_mode"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 1}, "surrogate"),                 # no thumbnails
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 1, "flags": 3, "num_blocks": 4}, "surrogate"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 1, "flags": 3, "schedule": 1}, "surrogate"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 1, "flags": 3, "judge_every": 0}, "judge_every"),
    ((640, 480, 0, 8, 640, 640, 0, 0), {"surrogate_mode": 1, "flags": 3, "fallback_tol": -1.0}, "fallback_tol"),
])
def test_invalid_configs_are_rejected(L, cam, kw, needle):
    from paper_1910_03517_gb300 import rt
    st, msg = _config(L, [rt.CameraDesc(*cam)], **kw)
    assert st == rt.RT_ERR_INVALID
    assert needle in msg


def test_zero_cameras_and_duplicate_positions(L):
    from paper_1910_03517_gb300 import rt
    st, _ = _config(L, [], )
    assert st == rt.RT_ERR_INVALID
    c = rt.CameraDesc(640, 480, 0, 8, 640, 640, 0, 3)
    st, msg = _config(L, [c, c])
    assert st == rt.RT_ERR_INVALID and "position" in msg


def test_null_handle_calls_are_invalid(L):
    from paper_1910_03517_gb300 import rt
    assert L.rt_sync(None, 0) == rt.RT_ERR_INVALID
    assert L.rt_get_gains(None, None, None, 0, 0) == rt.RT_ERR_INVALID
    L.rt_destroy(None)


@pytest.mark.parametrize("fit_mode", [0, 1, 2, 3])
def test_every_fit_mode_passes_validation(L, fit_mode):
    """The four fits are accepted by the checks made before any device
    work (without a GPU the call then fails on the device, not on them)."""
    from paper_1910_03517_gb300 import rt
    p = rt.default_params()
    cams = (rt.CameraDesc * 2)(rt.CameraDesc(640, 480, 0, 8, 640, 640, 0, 0),
                               rt.CameraDesc(640, 480, 0, 8, 640, 640, 0, 1))
    p.num_cameras = 2
    p.cams = ctypes.cast(cams, ctypes.POINTER(rt.CameraDesc))
    p.fit_mode = fit_mode
    p.num_blocks = 1 if fit_mode == 0 else 16
    h = ctypes.c_void_p()
    st = L.rt_array_config(ctypes.byref(p), None, ctypes.byref(h))
    if st == rt.RT_OK:
        L.rt_destroy(h)
    else:
        assert st != rt.RT_ERR_INVALID, L.rt_last_error(None).decode()
