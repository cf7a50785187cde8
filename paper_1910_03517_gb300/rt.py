"""Thin ctypes binding of librt.so (include/rt.h): argument marshalling only.

Every step of the correction runs in the library's CUDA kernels; torch only
provides device buffers (tensor data pointers) and the caller's stream.
Loading fails loudly when librt.so is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt.so")

RT_OK, RT_ERR_INVALID, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_NOT_READY, RT_ERR_TIMEOUT, RT_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
RT_NV12, RT_MONO16 = 0, 1
RT_LINEAR, RT_RING = 0, 1
RT_FIT_GLOBAL, RT_FIT_SEAM_AFFINE, RT_FIT_QUANTILE_AFFINE, RT_FIT_MATRIX = 0, 1, 2, 3
RT_SCHED_CURRENT, RT_SCHED_LAGGED = 0, 1
RT_BT709, RT_BT601 = 0, 1
RT_FLAG_FRAME_STATS = 1
RT_FLAG_THUMBNAILS = 2
RT_FLAG_SEAM_COST = 4
RT_FLAG_ATTENTION = 8
RT_FLAG_BLEND_BLOCKS = 16
RT_CROPS_FROM_PROPOSALS = -1
RT_PROFILE_ALL = 1
RT_PROFILE_PASS_B = 2
RT_MAX_CAMERAS = 32

# every symbol include/rt.h declares (checked by the tests)
EXPORTS = ["rt_default_params", "rt_array_config", "rt_submit_frames", "rt_submit_frames_host",
           "rt_get_gains", "rt_get_corrected", "rt_copy_corrected", "rt_get_crops", "rt_get_stats",
           "rt_copy_out", "rt_sync", "rt_save_state", "rt_load_state", "rt_last_error", "rt_destroy",
           "rt_stream_wait", "rt_capture_sequence", "rt_launch_sequence", "rt_profile", "rt_get_profile",
           "rt_get_thumb_features", "rt_autotune", "rt_get_tuning", "rt_set_tuning", "rt_get_seam_costs", "rt_get_proposals"]

c_i32, c_i64, c_dbl, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


class CameraDesc(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("format", c_i32), ("bit_depth", c_i32),
                ("y_pitch", c_i32), ("uv_pitch", c_i32), ("group", c_i32), ("position", c_i32)]


class ArrayParams(ctypes.Structure):
    _fields_ = [("num_cameras", c_i32), ("cams", ctypes.POINTER(CameraDesc)), ("topology", c_i32),
                ("strip_width", c_i32), ("num_blocks", c_i32), ("fit_mode", c_i32), ("schedule", c_i32),
                ("motion_threshold", c_i32), ("min_valid", c_i32), ("color_matrix", c_i32),
                ("alpha", c_dbl), ("lambda_", c_dbl), ("gain_min", c_dbl), ("gain_max", c_dbl),
                ("max_crops", c_i32), ("crop_size", c_i32), ("flags", c_i32),
                ("attn_window", c_i32), ("attn_min_on", c_i32), ("attn_max", c_i32),
                ("surrogate_mode", c_i32), ("judge_every", c_i32), ("fallback_tol", c_dbl)]


class SurrogateReport(ctypes.Structure):
    _fields_ = [("frame_sets", c_i64), ("predicted", c_i64), ("plain", c_i64), ("judged", c_i64),
                ("judged_failed", c_i64), ("fallback", c_i32), ("last_error", c_dbl), ("max_error", c_dbl),
                ("tolerance", c_dbl)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Crop(ctypes.Structure):
    _fields_ = [("cam", c_i32), ("x0", c_i32), ("y0", c_i32), ("w", c_i32), ("h", c_i32)]


class ProfileReport(ctypes.Structure):
    _fields_ = [("frame_sets", c_i32), ("pass_a_ms", c_dbl), ("solve_ms", c_dbl), ("pass_b_ms", c_dbl),
                ("crops_ms", c_dbl)]


class Tuning(ctypes.Structure):
    _fields_ = [("pass_b_threads", c_i32), ("pass_b_ctas_per_sm", c_i32), ("pass_a_rows", c_i32),
                ("pass_a_threads", c_i32), ("crop_threads", c_i32), ("crop_grid", c_i32), ("step_us", c_dbl),
                ("from_cache", c_i32), ("candidates", c_i32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class StatsView(ctypes.Structure):
    _fields_ = [("strip_hist", c_vp), ("strip_n", c_vp), ("strip_sum", c_vp), ("strip_sumsq", c_vp),
                ("frame_hist", c_vp), ("thumbs", c_vp), ("num_cameras", c_i32), ("num_blocks", c_i32),
                ("strip_joint", c_vp)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librt.so not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    L.rt_default_params.argtypes = [ctypes.POINTER(ArrayParams)]
    L.rt_default_params.restype = None
    L.rt_array_config.argtypes = [ctypes.POINTER(ArrayParams), c_vp, ctypes.POINTER(c_vp)]
    L.rt_submit_frames.argtypes = [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_i64, ctypes.POINTER(Crop), c_i32]
    L.rt_submit_frames_host.argtypes = [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_i64,
                                        ctypes.POINTER(Crop), c_i32, ctypes.POINTER(c_vp), c_i64]
    L.rt_get_gains.argtypes = [c_vp, c_vp, c_vp, c_sz, c_i32]
    L.rt_get_corrected.argtypes = [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_i32), c_i32]
    L.rt_copy_corrected.argtypes = [c_vp, c_i32, c_vp, c_i64, c_i32]
    L.rt_get_crops.argtypes = [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_i32), c_i32]
    L.rt_get_stats.argtypes = [c_vp, ctypes.POINTER(StatsView), c_i32]
    L.rt_copy_out.argtypes = [c_vp, c_vp, c_vp, c_sz, c_i32]
    L.rt_sync.argtypes = [c_vp, c_i32]
    L.rt_save_state.argtypes = [c_vp, c_vp, ctypes.POINTER(c_sz)]
    L.rt_load_state.argtypes = [c_vp, c_vp, c_sz]
    L.rt_last_error.argtypes = [c_vp]
    L.rt_last_error.restype = ctypes.c_char_p
    L.rt_stream_wait.argtypes = [c_vp, c_vp]
    L.rt_capture_sequence.argtypes = [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp),
                                      ctypes.POINTER(Crop), ctypes.POINTER(c_i32)]
    L.rt_launch_sequence.argtypes = [c_vp]
    L.rt_profile.argtypes = [c_vp, c_i32]
    L.rt_get_profile.argtypes = [c_vp, ctypes.POINTER(ProfileReport), c_i32]
    L.rt_get_thumb_features.argtypes = [c_vp, c_vp, c_i32]
    L.rt_get_seam_costs.argtypes = [c_vp, c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(c_i32), c_i32]
    L.rt_get_proposals.argtypes = [c_vp, c_vp, c_i32, ctypes.POINTER(c_i32), c_i32]
    L.rt_autotune.argtypes = [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), ctypes.POINTER(Crop),
                              ctypes.POINTER(c_i32), ctypes.c_char_p, ctypes.POINTER(Tuning)]
    L.rt_get_tuning.argtypes = [c_vp, ctypes.POINTER(Tuning)]
    L.rt_set_tuning.argtypes = [c_vp, ctypes.POINTER(Tuning)]
    L.rt_destroy.argtypes = [c_vp]
    L.rt_destroy.restype = None
    L.rt_check_solve_math.argtypes = [c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]
    L.rt_check_solve_math.restype = c_i32
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is ctypes.c_int:   # default restype: rt_status
            fn.restype = c_i32
    _lib = L
    return L


def check_solve_math(a: np.ndarray, b: np.ndarray, x: np.ndarray):
    """(ln(a/b), e^x) from the gain solve's device routines (include/rt_check.h)."""
    L = load()
    a = np.ascontiguousarray(a, np.uint64)
    b = np.ascontiguousarray(b, np.uint64)
    x = np.ascontiguousarray(x, np.float64)
    n = len(a)
    assert len(b) == n and len(x) == n
    lr = np.zeros(n, np.float64)
    ex = np.zeros(n, np.float64)
    st = L.rt_check_solve_math(n, a.ctypes.data, b.ctypes.data, lr.ctypes.data, x.ctypes.data, ex.ctypes.data)
    if st != RT_OK:
        raise RtError(st, "rt_check_solve_math")
    return lr, ex


class Box(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("x1", ctypes.c_float), ("y1", ctypes.c_float),
                ("score", ctypes.c_float), ("cls", c_i32)]


TRACK_EXPORTS = ["rt_nms", "rt_tracker_create", "rt_tracker_update", "rt_tracker_objects", "rt_tracker_destroy"]


def _load_track(L):
    if getattr(L, "_track_ready", False):
        return
    L.rt_nms.argtypes = [c_vp, c_i32, ctypes.c_float, ctypes.c_float, c_vp, c_vp]
    L.rt_nms.restype = c_i32
    L.rt_tracker_create.argtypes = [ctypes.POINTER(c_vp), c_dbl, c_dbl, c_dbl]
    L.rt_tracker_create.restype = c_i32
    L.rt_tracker_update.argtypes = [c_vp, c_vp, c_i32, c_i64, c_vp]
    L.rt_tracker_update.restype = c_i32
    L.rt_tracker_objects.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(c_i32)]
    L.rt_tracker_objects.restype = c_i32
    L.rt_tracker_destroy.argtypes = [c_vp]
    L.rt_tracker_destroy.restype = None
    L._track_ready = True


def _boxes(rows):
    """rows of (x0, y0, x1, y1, score, cls) -> a ctypes array of rt_box."""
    return (Box * max(1, len(rows)))(*[Box(float(r[0]), float(r[1]), float(r[2]), float(r[3]), float(r[4]),
                                           int(r[5])) for r in rows])


def nms(rows, score_min: float = 0.65, iou_max: float = 0.45, stream=None) -> List[int]:
    """Indices of the boxes greedy per-category NMS keeps (rt_nms, on the GPU)."""
    L = load()
    _load_track(L)
    n = len(rows)
    keep = np.zeros(max(1, n), np.int32)
    st = L.rt_nms(ctypes.cast(_boxes(rows), c_vp), n, score_min, iou_max, keep.ctypes.data,
                  None if stream is None else stream.cuda_stream)
    if st != RT_OK:
        raise RtError(st, "rt_nms")
    return [i for i in range(n) if keep[i]]


class Tracker:
    """The paper's per-category assignment tracker (rt_tracker_*, host code)."""

    def __init__(self, a: float = 0.99, tol_iou: float = 0.05, tol_new: float = 0.001):
        self.L = load()
        _load_track(self.L)
        h = c_vp()
        st = self.L.rt_tracker_create(ctypes.byref(h), a, tol_iou, tol_new)
        if st != RT_OK:
            raise RtError(st, "rt_tracker_create")
        self.h = h

    def update(self, rows, frame: int) -> List[int]:
        n = len(rows)
        out = np.zeros(max(1, n), np.int32)
        st = self.L.rt_tracker_update(self.h, ctypes.cast(_boxes(rows), c_vp), n, int(frame), out.ctypes.data)
        if st != RT_OK:
            raise RtError(st, "rt_tracker_update")
        return [int(x) for x in out[:n]]

    def objects(self):
        n = c_i32(0)
        self.L.rt_tracker_objects(self.h, None, None, None, None, None, 0, ctypes.byref(n))
        m = n.value
        ids, cls, hist = (np.zeros(max(1, m), np.int32) for _ in range(3))
        frames = np.zeros(max(1, m), np.int64)
        boxes = (Box * max(1, m))()
        st = self.L.rt_tracker_objects(self.h, ids.ctypes.data, cls.ctypes.data, ctypes.cast(boxes, c_vp),
                                       frames.ctypes.data, hist.ctypes.data, m, ctypes.byref(n))
        if st != RT_OK:
            raise RtError(st, "rt_tracker_objects")
        return [{"id": int(ids[i]), "cls": int(cls[i]), "frame": int(frames[i]), "history": int(hist[i]),
                 "box": (boxes[i].x0, boxes[i].y0, boxes[i].x1, boxes[i].y1)} for i in range(m)]

    def close(self):
        if self.h:
            self.L.rt_tracker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("rt status %d: %s" % (status, msg))
        self.status = status


def _check(L, h, st):
    if st != RT_OK:
        msg = L.rt_last_error(h)
        raise RtError(st, msg.decode() if msg else "")


def default_params() -> ArrayParams:
    p = ArrayParams()
    load().rt_default_params(ctypes.byref(p))
    return p


def camera_desc(cam) -> CameraDesc:
    """From any object with width/height/fmt/bit_depth/y_pitch/uv_pitch/group/position."""
    return CameraDesc(cam.width, cam.height, cam.fmt, getattr(cam, "bit_depth", 8), cam.y_pitch,
                      getattr(cam, "uv_pitch", 0), getattr(cam, "group", 0), getattr(cam, "position", 0))


class CameraArray:
    """One configured camera array (a handle of librt.so)."""

    def __init__(self, cams, stream=None, **kw):
        import torch
        self.L = load()
        self.cams = list(cams)
        self.K = len(self.cams)
        p = default_params()
        self._descs = (CameraDesc * self.K)(*[camera_desc(c) for c in self.cams])
        p.num_cameras = self.K
        p.cams = ctypes.cast(self._descs, ctypes.POINTER(CameraDesc))
        for k, v in kw.items():
            setattr(p, "lambda_" if k == "lam" else k, v)
        self.p = p
        self.B = p.num_blocks
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = c_vp()
        st = self.L.rt_array_config(ctypes.byref(p), c_vp(sp), ctypes.byref(self.h))
        if st != RT_OK:
            raise RtError(st, self.L.rt_last_error(None).decode())
        self._keep: List[object] = []

    # -- submission ------------------------------------------------------
    def _planes(self, frames):
        y = (c_vp * self.K)()
        uv = (c_vp * self.K)()
        for k, f in enumerate(frames):
            if "ir" in f:
                y[k] = f["ir"].data_ptr()
                uv[k] = None
            else:
                y[k] = f["y"].data_ptr()
                uv[k] = f["uv"].data_ptr()
        return y, uv

    @staticmethod
    def _crops(crops):
        """crops: a list of (cam, x0, y0, w, h), or RT_CROPS_FROM_PROPOSALS."""
        if isinstance(crops, int):
            return (Crop * 1)(), int(crops)
        n = len(crops)
        arr = (Crop * max(1, n))(*[Crop(*map(int, c)) for c in crops])
        return arr, n

    def submit_frames(self, frames: Sequence[Dict[str, object]], frame_index: int, crops=()):
        y, uv = self._planes(frames)
        arr, n = self._crops(crops)
        st = self.L.rt_submit_frames(self.h, y, uv, int(frame_index), arr, n)
        _check(self.L, self.h, st)
        self._keep = (self._keep + [frames])[-3:]

    def submit_frames_host(self, frames, frame_index: int, crops=(), rgb_out=None, rgb_out_pitch=0):
        y, uv = self._planes(frames)
        arr, n = self._crops(crops)
        outp = None
        if rgb_out is not None:
            outp = (c_vp * self.K)(*[t.data_ptr() for t in rgb_out])
        st = self.L.rt_submit_frames_host(self.h, y, uv, int(frame_index), arr, n, outp, int(rgb_out_pitch))
        _check(self.L, self.h, st)
        self._keep = (self._keep + [(frames, rgb_out)])[-3:]

    # -- results ---------------------------------------------------------
    def get_gains(self, timeout_ms: int = 60000):
        """(maps FP64, maps Q16): [K, 2, B, 3, 2] = (a, b) per channel, or
        [K, 2, B, 12] = (M row-major, b) for the 3 x 3 maps."""
        shape = (self.K, 2, self.B, 12) if self.p.fit_mode == RT_FIT_MATRIX else (self.K, 2, self.B, 3, 2)
        maps = np.zeros(shape, np.float64)
        q = np.zeros(shape, np.int32)
        st = self.L.rt_get_gains(self.h, maps.ctypes.data, q.ctypes.data, maps.size, timeout_ms)
        _check(self.L, self.h, st)
        return maps, q

    def get_corrected(self, cam: int, timeout_ms: int = 60000):
        """Corrected RGB24 of camera cam as a device tensor [H, W, 3] (a copy)."""
        import torch
        c = self.cams[cam]
        out = torch.empty((c.height, c.width, 3), dtype=torch.uint8, device="cuda")
        st = self.L.rt_copy_corrected(self.h, cam, out.data_ptr(), 3 * c.width, timeout_ms)
        _check(self.L, self.h, st)
        return out

    def copy_out(self, dst_ptr: int, src_ptr: int, nbytes: int, timeout_ms: int = 60000):
        st = self.L.rt_copy_out(self.h, c_vp(dst_ptr), c_vp(src_ptr), nbytes, timeout_ms)
        _check(self.L, self.h, st)

    def get_crops(self, timeout_ms: int = 60000):
        import torch
        ptr, n = c_vp(), c_i32()
        st = self.L.rt_get_crops(self.h, ctypes.byref(ptr), ctypes.byref(n), timeout_ms)
        _check(self.L, self.h, st)
        S = self.p.crop_size
        out = torch.empty((n.value, 3, S, S), dtype=torch.float16, device="cuda")
        if n.value:
            self.copy_out(out.data_ptr(), ptr.value, out.numel() * 2, timeout_ms)
        return out

    def get_stats(self, timeout_ms: int = 60000) -> Dict[str, np.ndarray]:
        v = StatsView()
        st = self.L.rt_get_stats(self.h, ctypes.byref(v), timeout_ms)
        _check(self.L, self.h, st)
        K, B = self.K, self.B
        out = {}
        for name, ptr, shape, dt in (("strip_hist", v.strip_hist, (K, 2, B, 3, 256), np.uint32),
                                     ("strip_n", v.strip_n, (K, 2, B, 3), np.uint32),
                                     ("strip_sum", v.strip_sum, (K, 2, B, 3), np.uint64),
                                     ("strip_sumsq", v.strip_sumsq, (K, 2, B, 3), np.uint64),
                                     ("frame_hist", v.frame_hist, (K, 3, 256), np.uint32),
                                     ("thumbs", v.thumbs, (K, 3, 36, 64), np.uint32),
                                     ("strip_joint", v.strip_joint, (K, 2, B, 10), np.uint64)):
            if not ptr:
                out[name] = None
                continue
            a = np.zeros(shape, dt)
            self.copy_out(a.ctypes.data, ptr, a.nbytes, timeout_ms)
            out[name] = a
        return out

    def stream_wait(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self.L, self.h, self.L.rt_stream_wait(self.h, c_vp(sp)))

    def _sequence_args(self, frame_sets, crops_per_set):
        n = len(frame_sets)
        y = (c_vp * (n * self.K))()
        uv = (c_vp * (n * self.K))()
        for i, fs in enumerate(frame_sets):
            yi, uvi = self._planes(fs)
            for k in range(self.K):
                y[i * self.K + k] = yi[k]
                uv[i * self.K + k] = uvi[k]
        cr_p, nc_p = None, None
        if crops_per_set is not None:
            M = max(1, self.p.max_crops)
            flat = []
            counts = []
            for cl in crops_per_set:
                if isinstance(cl, int):            # RT_CROPS_FROM_PROPOSALS
                    counts.append(int(cl))
                    flat += [Crop()] * M
                    continue
                counts.append(len(cl))
                flat += [Crop(*map(int, c)) for c in cl] + [Crop()] * (M - len(cl))
            cr_p = (Crop * len(flat))(*flat)
            nc_p = (c_i32 * n)(*counts)
        return n, y, uv, cr_p, nc_p

    def capture_sequence(self, frame_sets, crops_per_set=None):
        """Capture a graph over these frame sets (any number; relaunchable while
        the frame sets submitted since the capture are a multiple of 6)."""
        n, y, uv, cr_p, nc_p = self._sequence_args(frame_sets, crops_per_set)
        st = self.L.rt_capture_sequence(self.h, n, y, uv, cr_p, nc_p)
        _check(self.L, self.h, st)
        self._captured = frame_sets

    def autotune(self, frame_sets, crops_per_set=None, cache_path=None) -> Dict[str, float]:
        """Pick the launch shapes by timing them on these frame sets (len a
        multiple of 6); cache_path: JSON cache file (read, and written on a miss)."""
        n, y, uv, cr_p, nc_p = self._sequence_args(frame_sets, crops_per_set)
        t = Tuning()
        path = cache_path.encode() if cache_path else None
        _check(self.L, self.h, self.L.rt_autotune(self.h, n, y, uv, cr_p, nc_p, path, ctypes.byref(t)))
        self._captured = frame_sets
        return t.as_dict()

    def proposals(self, timeout_ms: int = 60000):
        """[(cam, x0, y0, w, h)] attention windows of the last frame set (RT_FLAG_ATTENTION)."""
        n = c_i32(0)
        cap = max(1, self.p.attn_max)
        buf = (Crop * cap)()
        _check(self.L, self.h, self.L.rt_get_proposals(self.h, buf, cap, ctypes.byref(n), timeout_ms))
        return [(c.cam, c.x0, c.y0, c.w, c.h) for c in buf[:min(n.value, cap)]]

    def seam_costs(self, timeout_ms: int = 60000):
        """[(left camera, right camera, cost)] of the last frame set (RT_FLAG_SEAM_COST)."""
        n = c_i32(0)
        _check(self.L, self.h, self.L.rt_get_seam_costs(self.h, None, None, None, 0, ctypes.byref(n), timeout_ms))
        m = n.value
        lc = np.zeros(max(m, 1), np.int32)
        rc = np.zeros(max(m, 1), np.int32)
        co = np.zeros(max(m, 1), np.float64)
        _check(self.L, self.h, self.L.rt_get_seam_costs(self.h, lc.ctypes.data, rc.ctypes.data, co.ctypes.data, m,
                                                        ctypes.byref(n), timeout_ms))
        return [(int(lc[i]), int(rc[i]), float(co[i])) for i in range(m)]

    def get_tuning(self) -> Dict[str, float]:
        t = Tuning()
        _check(self.L, self.h, self.L.rt_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        _check(self.L, self.h, self.L.rt_get_tuning(self.h, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(self.L, self.h, self.L.rt_set_tuning(self.h, ctypes.byref(t)))

    def launch_sequence(self):
        _check(self.L, self.h, self.L.rt_launch_sequence(self.h))

    def profile(self, enable, pass_b_only: bool = False):
        """Start (enable true: clears what was collected) or stop collecting."""
        mode = (RT_PROFILE_PASS_B if pass_b_only else RT_PROFILE_ALL) if enable else 0
        _check(self.L, self.h, self.L.rt_profile(self.h, mode))

    def get_profile(self, timeout_ms: int = 60000) -> Dict[str, float]:
        r = ProfileReport()
        _check(self.L, self.h, self.L.rt_get_profile(self.h, ctypes.byref(r), timeout_ms))
        return {"frame_sets": r.frame_sets, "pass_a_ms": r.pass_a_ms, "solve_ms": r.solve_ms,
                "pass_b_ms": r.pass_b_ms, "crops_ms": r.crops_ms}

    def surrogate_predict(self, net: Optional["GainMLP"] = None, timeout_ms: int = 60000):
        """(maps [K,2,1,3,2] predicted by the network -- net, or the handle's
        own when None -- and the judge's error against the fit)."""
        _load_mlp(self.L)
        maps = np.zeros((self.K, 2, self.B, 3, 2), np.float64)
        err = np.zeros(1, np.float64)
        _check(self.L, self.h, self.L.rt_surrogate_predict(self.h, net.h if net is not None else None,
                                                           maps.ctypes.data, err.ctypes.data, timeout_ms))
        return maps, float(err[0])

    # -- the array's own surrogate network (rt_surrogate.h) ---------------
    def surrogate_train(self, n_samples: int, batch: int = 256, lr: float = 1e-3, seed: int = 0):
        """One pass of training over n_samples generated samples; returns the step losses."""
        _load_mlp(self.L)
        _check(self.L, self.h, self.L.rt_surrogate_train(self.h, int(n_samples), int(batch), float(lr), int(seed)))
        n = c_i64(0)
        _check(self.L, self.h, self.L.rt_surrogate_losses(self.h, None, 0, ctypes.byref(n)))
        out = np.zeros(max(1, n.value), np.float32)
        _check(self.L, self.h, self.L.rt_surrogate_losses(self.h, out.ctypes.data, n.value, ctypes.byref(n)))
        return out[: n.value]

    def surrogate_evaluate(self, n_samples: int, seed: int):
        """Per-camera held-out gain error [sets, K] of the handle's network, and
        the same error of leaving the cameras uncorrected."""
        _load_mlp(self.L)
        n = c_i64(0)
        cap = -(-int(n_samples) // self.K) * self.K
        out = np.zeros(cap, np.float64)
        out0 = np.zeros(cap, np.float64)
        _check(self.L, self.h, self.L.rt_surrogate_evaluate(self.h, int(n_samples), int(seed), out.ctypes.data,
                                                             out0.ctypes.data, cap, ctypes.byref(n)))
        return out[: n.value].reshape(-1, self.K), out0[: n.value].reshape(-1, self.K)

    def surrogate_save(self, path: str):
        _load_mlp(self.L)
        _check(self.L, self.h, self.L.rt_surrogate_save(self.h, path.encode()))

    def surrogate_load(self, path: str):
        _load_mlp(self.L)
        _check(self.L, self.h, self.L.rt_surrogate_load(self.h, path.encode()))

    def surrogate_params(self) -> np.ndarray:
        _load_mlp(self.L)
        a = np.zeros(MLP_PARAMS, np.float32)
        _check(self.L, self.h, self.L.rt_surrogate_get_params(self.h, a.ctypes.data, a.size))
        return a

    def surrogate_set_tolerance(self, tol: float):
        _load_mlp(self.L)
        _check(self.L, self.h, self.L.rt_surrogate_set_tolerance(self.h, float(tol)))

    def surrogate_report(self, timeout_ms: int = 60000) -> Dict[str, float]:
        _load_mlp(self.L)
        r = SurrogateReport()
        _check(self.L, self.h, self.L.rt_surrogate_get_report(self.h, ctypes.byref(r), timeout_ms))
        return r.as_dict()

    def thumb_features(self, timeout_ms: int = 60000):
        """BF16 device tensor [K, 6912] of the last frame set's thumbnail features."""
        import torch
        x = torch.empty((self.K, 6912), dtype=torch.bfloat16, device="cuda")
        _check(self.L, self.h, self.L.rt_get_thumb_features(self.h, x.data_ptr(), timeout_ms))
        return x

    def sync(self, timeout_ms: int = 60000):
        _check(self.L, self.h, self.L.rt_sync(self.h, timeout_ms))

    def save_state(self) -> bytes:
        n = c_sz(0)
        _check(self.L, self.h, self.L.rt_save_state(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.L, self.h, self.L.rt_save_state(self.h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self.L, self.h, self.L.rt_load_state(self.h, buf, len(blob)))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.rt_destroy(self.h)
            self.h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned gain surrogate (include/rt_surrogate.h)
# ---------------------------------------------------------------------------

MLP_INPUTS = 6912
MLP_PARAMS = 1836291
MLP_EXPORTS = ["rt_mlp_create", "rt_mlp_set_params", "rt_mlp_get_params", "rt_mlp_forward", "rt_mlp_gradients",
               "rt_mlp_train_step", "rt_mlp_last_error", "rt_mlp_destroy", "rt_surrogate_predict",
               "rt_surrogate_train", "rt_surrogate_losses", "rt_surrogate_evaluate", "rt_surrogate_save",
               "rt_surrogate_load", "rt_surrogate_get_params", "rt_surrogate_set_tolerance", "rt_surrogate_get_report"]


def _load_mlp(L):
    if getattr(L, "_mlp_ready", False):
        return
    L.rt_mlp_create.argtypes = [ctypes.POINTER(c_vp), c_vp]
    L.rt_mlp_set_params.argtypes = [c_vp, c_vp, c_sz]
    L.rt_mlp_get_params.argtypes = [c_vp, c_vp, c_sz]
    L.rt_mlp_forward.argtypes = [c_vp, c_vp, c_i32, c_vp]
    L.rt_mlp_gradients.argtypes = [c_vp, c_vp, c_vp, c_i32, c_vp, c_vp]
    L.rt_mlp_train_step.argtypes = [c_vp, c_vp, c_vp, c_i32, c_dbl, c_vp]
    L.rt_mlp_last_error.argtypes = [c_vp]
    L.rt_mlp_last_error.restype = ctypes.c_char_p
    L.rt_mlp_destroy.argtypes = [c_vp]
    L.rt_mlp_destroy.restype = None
    L.rt_mlp_check_activations.argtypes = [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]
    L.rt_surrogate_train.argtypes = [c_vp, c_i64, c_i32, c_dbl, ctypes.c_uint64]
    L.rt_surrogate_losses.argtypes = [c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]
    L.rt_surrogate_evaluate.argtypes = [c_vp, c_i64, ctypes.c_uint64, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]
    L.rt_surrogate_save.argtypes = [c_vp, ctypes.c_char_p]
    L.rt_surrogate_load.argtypes = [c_vp, ctypes.c_char_p]
    L.rt_surrogate_get_params.argtypes = [c_vp, c_vp, c_sz]
    L.rt_surrogate_set_tolerance.argtypes = [c_vp, c_dbl]
    L.rt_surrogate_get_report.argtypes = [c_vp, ctypes.POINTER(SurrogateReport), c_i32]
    for name in MLP_EXPORTS:
        fn = getattr(L, name)
        if fn.restype is ctypes.c_int:
            fn.restype = c_i32
    L.rt_surrogate_predict.argtypes = [c_vp, c_vp, c_vp, c_vp, c_i32]
    L.rt_surrogate_predict.restype = c_i32
    for n in MLP_EXPORTS[:-3]:
        getattr(L, n).restype = c_i32
    L._mlp_ready = True


def param_offsets():
    """(name, offset, shape) of each tensor in the flat parameter vector."""
    out, off = [], 0
    for name, shape in (("W1", (256, MLP_INPUTS)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
                        ("W3", (3, 256)), ("b3", (3,))):
        n = int(np.prod(shape))
        out.append((name, off, shape))
        off += n
    assert off == MLP_PARAMS
    return out


class GainMLP:
    """The surrogate network (a handle of librt.so's rt_mlp)."""

    def __init__(self, stream=None):
        import torch
        self.L = load()
        _load_mlp(self.L)
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = c_vp()
        st = self.L.rt_mlp_create(ctypes.byref(self.h), c_vp(sp))
        if st != RT_OK:
            raise RtError(st, "rt_mlp_create failed")

    def _chk(self, st):
        if st != RT_OK:
            raise RtError(st, self.L.rt_mlp_last_error(self.h).decode())

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, np.float32)
        self._chk(self.L.rt_mlp_set_params(self.h, a.ctypes.data, a.size))

    def get_params(self) -> np.ndarray:
        a = np.zeros(MLP_PARAMS, np.float32)
        self._chk(self.L.rt_mlp_get_params(self.h, a.ctypes.data, a.size))
        return a

    def forward(self, x):
        import torch
        n = x.shape[0]
        y = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        self._chk(self.L.rt_mlp_forward(self.h, x.data_ptr(), n, y.data_ptr()))
        return y

    def gradients(self, x, t):
        n = x.shape[0]
        g = np.zeros(MLP_PARAMS, np.float32)
        loss = np.zeros(1, np.float32)
        self._chk(self.L.rt_mlp_gradients(self.h, x.data_ptr(), t.data_ptr(), n, g.ctypes.data, loss.ctypes.data))
        return g, float(loss[0])

    def activations(self, n: int) -> Dict[str, np.ndarray]:
        """The last gradients() call's intermediate values (rt_check.h), BF16
        as float64: h1, h2, dz2 [n, 256]; dz1 [n, 256]; y [n, 3] (FP32)."""
        u = lambda shape: np.zeros(shape, np.uint16)
        h1, h2, dz2, dz1t = u((n, 256)), u((n, 256)), u((n, 256)), u((256, 256))
        y = np.zeros((n, 3), np.float32)
        self._chk(self.L.rt_mlp_check_activations(self.h, n, h1.ctypes.data, h2.ctypes.data, dz2.ctypes.data,
                                                  dz1t.ctypes.data, y.ctypes.data))
        f = lambda a: (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return {"h1": f(h1), "h2": f(h2), "dz2": f(dz2), "dz1": f(np.ascontiguousarray(dz1t[:, :n].T)),
                "y": y.astype(np.float64)}

    def train_step(self, x, t, lr: float) -> float:
        loss = np.zeros(1, np.float32)
        self._chk(self.L.rt_mlp_train_step(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], float(lr),
                                           loss.ctypes.data))
        return float(loss[0])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.rt_mlp_destroy(self.h)
            self.h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
