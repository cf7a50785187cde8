"""The allocation-free gain fit (rt_fit_gains_noalloc) against the handle
path, through the C ABI.

It exists for callers that cannot call cudaMalloc (their device memory is
owned by another allocator or reserved up front), so it keeps its working
memory in a fixed array inside the library.  Checked here: two calls in a
row on different frame sets give the maps of the handle path's first frame
set within the tolerance the parity tests use (1e-6 relative for FP64
maps, exact Q16), so the second call is not disturbed by what the first
left in the shared array, and the second call leaves the device's free
memory unchanged.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1910_03517_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_path_twice():
    from paper_1910_03517_gb300 import build, rt
    build.build()
    L = rt.load()
    L.rt_fit_gains_noalloc.argtypes = [ctypes.POINTER(rt.CameraDesc), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.rt_fit_gains_noalloc.restype = ctypes.c_int32
    cams = [synth.Camera(1920, 1080, position=i) for i in range(5)]
    cams.append(synth.Camera(640, 512, fmt=synth.MONO16, bit_depth=12, group=1, position=0))
    cams.append(synth.Camera(640, 512, fmt=synth.MONO16, bit_depth=12, group=1, position=1))
    wl = synth.Workload("no-alloc check", cams, frames=2, seed=31, glare_cams=(2,))
    K, B = len(cams), 4
    descs = (rt.CameraDesc * K)(*[rt.camera_desc(c) for c in cams])
    stream = torch.cuda.current_stream()
    for t in range(2):
        fs = synth.frame_set(wl, t, device="cuda")
        ref = rt.CameraArray(cams, num_blocks=B, topology=rt.RT_RING)
        ref.submit_frames(fs, 0)
        m_ref, q_ref = ref.get_gains()
        ref.close()
        y = (ctypes.c_void_p * K)(*[(f["ir"] if "ir" in f else f["y"]).data_ptr() for f in fs])
        uv = (ctypes.c_void_p * K)(*[(f["uv"].data_ptr() if "uv" in f else None) for f in fs])
        maps = torch.full((K, 2, B, 3, 2), -7.0, dtype=torch.float64, device="cuda")
        q16 = torch.full((K, 2, B, 3, 2), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = L.rt_fit_gains_noalloc(descs, K, y, uv, 32, B, rt.RT_RING, maps.data_ptr(), q16.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == rt.RT_OK
        torch.cuda.synchronize()
        if t == 1:
            # the second call takes no device memory (the first may load the module)
            assert torch.cuda.mem_get_info()[0] == free0
        m = maps.cpu().numpy()
        q = q16.cpu().numpy()
        assert (np.abs(m - m_ref) <= 1e-6 * np.abs(m_ref) + 1e-9).all(), (t, np.abs(m - m_ref).max())
        assert np.array_equal(q, q_ref), t
    # beyond the stated limits the call refuses before doing anything
    big = (rt.CameraDesc * 17)(*([rt.camera_desc(cams[0])] * 17))
    assert L.rt_fit_gains_noalloc(big, 17, y, uv, 32, B, 0, maps.data_ptr(), q16.data_ptr(), None) == rt.RT_ERR_INVALID
    assert L.rt_fit_gains_noalloc(descs, K, y, uv, 32, 5, 0, maps.data_ptr(), q16.data_ptr(), None) == rt.RT_ERR_INVALID
