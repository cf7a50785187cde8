"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (written here, per output):
  - band and frame statistics, histograms, the Q16 table and the corrected
    8-bit images: bit-exact;
  - the FP64 maps (gains, or affine a and b): |gpu - oracle| <= 1e-6 |oracle|
    + 1e-9 (the same formulas in FP64; only summation order and libm ulps
    differ);
  - FP16 crops: within 1e-3 absolute of the oracle's FP64 resample.
The Q16 table is compared exactly except where the oracle's 65536*E lies
within 1e-6 of a rounding tie (there both roundings are correct); the
oracle then applies the GPU's table so the 8-bit output is still compared
bit for bit.
"""
import numpy as np
import pytest
import torch

from conftest import np_frames
from paper_1910_03517_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1910_03517_gb300 import build, rt as rtmod
    build.build()
    rtmod.load()
    return rtmod


def _params_for_oracle(orc, **kw):
    m = dict(kw)
    if "lam" in m:
        m["lam"] = m.pop("lam")
    keep = {k: v for k, v in m.items() if k in orc.Params.__dataclass_fields__}
    return orc.Params(**keep)


def _check_q16(q_gpu, q_orc, E):
    diff = q_gpu.astype(np.int64) - q_orc.astype(np.int64)
    if not (diff == 0).all():
        v = 65536.0 * E
        near_tie = np.abs(np.abs(v - np.floor(v)) - 0.5) < 1e-6 * np.maximum(1.0, np.abs(v))
        bad = (diff != 0) & ~(near_tie & (np.abs(diff) <= 1))
        assert not bad.any(), (np.argwhere(bad)[:5], q_gpu[bad][:5], q_orc[bad][:5])


def _check_matrix_maps(maps, E, rtol, t):
    """3 x 3 maps compared norm-wise per map: |dM| <= rtol max|M|, and the
    offsets |db| <= rtol (|b| + 255 max|M|) (b = mu_s - M mu inherits M's
    error times a mean of up to 255)."""
    scale = np.abs(E[..., :9]).max(axis=-1, keepdims=True)
    dM = np.abs(maps[..., :9] - E[..., :9])
    db = np.abs(maps[..., 9:] - E[..., 9:])
    assert (dM <= rtol * scale).all(), (t, (dM / scale).max())
    assert (db <= rtol * (np.abs(E[..., 9:]) + 255 * scale)).all(), (t, db.max())


def run_sequence(rt, orc, wl, frames, crops_per_frame=0, crop_size=0, device_inputs=True,
                 stats=True, check_images=True, thumbs=False, maps_rtol=1e-6, blend=False, **kw):
    """Submit `frames` frame sets to the GPU and the oracle, compare each."""
    from oracle import mlp as omlp
    p = _params_for_oracle(orc, **kw)
    p.blend_blocks = blend
    flags = (rt.RT_FLAG_FRAME_STATS if stats else 0) | (rt.RT_FLAG_THUMBNAILS if thumbs else 0) | \
        (rt.RT_FLAG_BLEND_BLOCKS if blend else 0)
    arr = rt.CameraArray(wl.cams, max_crops=max(crops_per_frame, 0), crop_size=max(crop_size, 0),
                         flags=flags, **kw)
    o = orc.ArrayOracle(wl.cams, p)
    K = len(wl.cams)
    results = []
    for t in range(frames):
        fs = synth.frame_set(wl, t, device="cuda")
        crops = synth.crop_list(wl, t, crops_per_frame) if crops_per_frame else []
        if device_inputs:
            arr.submit_frames(fs, t, crops)
        else:
            host = [{k: v.cpu().pin_memory() for k, v in f.items()} for f in fs]
            arr.submit_frames_host(host, t, crops)
        maps, q16 = arr.get_gains()
        st = arr.get_stats()
        r = o.step(np_frames(fs), crops=crops, crop_size=crop_size, q16_override=q16,
                   want_frame_stats=stats, want_thumbs=thumbs)
        if thumbs:
            assert np.array_equal(st["thumbs"], r["thumbs"]), t
            feat = arr.thumb_features().float().cpu().numpy()
            for k, c in enumerate(wl.cams):
                ref = omlp.bf16_round(omlp.thumb_features(r["thumbs"][k], c.width, c.height))
                assert np.array_equal(feat[k], ref.astype(np.float32)), (t, k)
        # statistics: bit-exact
        assert np.array_equal(st["strip_n"], r["strip_n"]), t
        assert np.array_equal(st["strip_sum"], r["strip_sum"]), t
        assert np.array_equal(st["strip_sumsq"], r["strip_sumsq"]), t
        assert np.array_equal(st["strip_hist"], r["strip_hist"]), t
        if r.get("strip_joint") is not None:
            assert np.array_equal(st["strip_joint"], r["strip_joint"]), t
        if stats:
            assert np.array_equal(st["frame_hist"], r["frame_hist"]), t
        # FP64 maps
        E = r["E"]
        if maps.shape[-1] == 12:
            _check_matrix_maps(maps, E, maps_rtol, t)
        else:
            assert (np.abs(maps - E) <= maps_rtol * np.abs(E) + 1e-3 * maps_rtol).all(), (t, np.abs(maps - E).max())
        _check_q16(q16, r["q16"], r["maps"])
        if check_images:
            for k in range(K):
                got = arr.get_corrected(k).cpu().numpy()
                ref = r["corrected"][k]
                if not np.array_equal(got, ref):
                    bad = np.argwhere(got != ref)
                    raise AssertionError("frame %d cam %d: %d bytes differ, first %s got %s want %s" % (
                        t, k, len(bad), bad[:3].tolist(), got[tuple(bad[0])], ref[tuple(bad[0])]))
        if crops:
            cr = arr.get_crops().float().cpu().numpy()
            assert cr.shape == r["crops"].shape
            assert np.abs(cr - r["crops"]).max() < 1e-3, (t, np.abs(cr - r["crops"]).max())
        results.append((maps, q16))
    arr.close()
    return results


# ---------------------------------------------------------------------------

def _all_triples(W=4096):
    H = W
    b = np.arange(H // 2)[:, None] * (W // 2) + np.arange(W // 2)[None, :]
    pair = b // 64
    y = np.zeros((H, W), np.uint8)
    base = 4 * (b % 64)
    y[0::2, 0::2] = base
    y[0::2, 1::2] = base + 1
    y[1::2, 0::2] = base + 2
    y[1::2, 1::2] = base + 3
    uv = np.zeros((H // 2, W), np.uint8)
    uv[:, 0::2] = (pair // 256).astype(np.uint8)
    uv[:, 1::2] = (pair % 256).astype(np.uint8)
    return y, uv


@pytest.mark.parametrize("matrix", [0, 1])
def test_conversion_every_yuv_triple(rt, orc, matrix):
    y, uv = _all_triples()
    cam = synth.Camera(4096, 4096)
    arr = rt.CameraArray([cam], color_matrix=matrix)
    fr = [{"y": torch.from_numpy(y).cuda(), "uv": torch.from_numpy(uv).cuda()}]
    arr.submit_frames(fr, 0)
    got = arr.get_corrected(0).cpu().numpy()          # one camera: no seam, identity gains
    maps, q16 = arr.get_gains()
    assert (q16[..., 0] == 65536).all() and (q16[..., 1] == 0).all()
    ref, _ = orc.convert(cam, {"y": y, "uv": uv}, matrix)
    assert np.array_equal(got, ref)
    st = arr.get_stats()
    assert np.array_equal(st["frame_hist"][0], orc.frame_stats(ref)["hist"])
    arr.close()


def test_small_pair_global(rt, orc):
    run_sequence(rt, orc, synth.small_pair(), 8)


def test_small_pair_seam_affine_16_blocks(rt, orc):
    run_sequence(rt, orc, synth.small_pair(), 8, fit_mode=1, num_blocks=16)


@pytest.mark.parametrize("kw", [{"num_blocks": 16}, {"fit_mode": 1, "num_blocks": 16},
                                {"fit_mode": 2, "num_blocks": 7, "schedule": 1}])
def test_blended_block_maps(rt, orc, kw):
    """Convex blending of adjacent block maps: per-row maps in exact Q16
    integers, images bit-exact to the oracle; also cameras of several heights
    (the per-row table has the tallest camera's rows)."""
    run_sequence(rt, orc, synth.small_pair(), 4, blend=True, **kw)
    cams = [synth.Camera(200, 120, position=0, y_pitch=208, uv_pitch=208),
            synth.Camera(220, 90, position=1, y_pitch=224, uv_pitch=224),
            synth.Camera(96, 40, fmt=synth.MONO16, bit_depth=10, group=1, position=0, y_pitch=192),
            synth.Camera(96, 64, fmt=synth.MONO16, bit_depth=10, group=1, position=1, y_pitch=192)]
    wl = synth.Workload("blend ragged", cams, frames=3, seed=41)
    run_sequence(rt, orc, wl, 3, blend=True, strip_width=16, min_valid=8, **kw)


def test_quantile_affine_fit(rt, orc):
    """The quantile-LS affine maps: maps within the FP64 bar (the kernel does
    the oracle's arithmetic operation for operation), images bit-exact."""
    run_sequence(rt, orc, synth.small_pair(), 6, fit_mode=2, num_blocks=16)
    wl = synth.small_pair()
    wl.cams = [synth.Camera(640, 480, position=i) for i in range(3)]
    wl.moving_object = True
    run_sequence(rt, orc, wl, 4, fit_mode=2, num_blocks=4, topology=1, schedule=1, maps_rtol=1e-12)


def _matrix_residual(rt, wl, frames, **kw):
    """max over maps of |M S M - S_s| / |S_s| for the GPU's unsmoothed maps of
    the last frame set (alpha = 1), S and S_s from the GPU's own joint
    moments (bit-exact to the oracle's): the defining equation, checked
    without the oracle's eigen-decompositions."""
    from oracle import core as oc
    arr = rt.CameraArray(wl.cams, fit_mode=3, alpha=1.0, gain_min=1e-3, gain_max=16.0, **kw)
    for t in range(frames):
        arr.submit_frames(synth.frame_set(wl, t, device="cuda"), t, [])
    maps, _ = arr.get_gains()
    joint = arr.get_stats()["strip_joint"]
    arr.close()
    worst, checked = 0.0, 0
    for (_, kl, kr) in oc.seams(wl.cams, kw.get("topology", 0)):
        for j in range(joint.shape[2]):
            muR, SR = oc.joint_moments(joint[kl, 1, j])
            muL, SL = oc.joint_moments(joint[kr, 0, j])
            d = muL - muR
            Ss = 0.5 * (SL + SR) + 0.25 * np.outer(d, d)
            for (k, side, S) in ((kl, 1, SR), (kr, 0, SL)):
                M = maps[k, side, j, :9].reshape(3, 3)
                ev = np.linalg.eigvalsh(M)
                if ev.min() <= 1.001e-3 or ev.max() >= 16.0 * (1 - 1e-9):
                    continue   # the eigenvalue clamp acted: M no longer solves the equation
                worst = max(worst, np.abs(M @ S @ M - Ss).max() / np.abs(Ss).max())
                checked += 1
    assert checked > 0
    return worst


def test_matrix_maps(rt, orc):
    """3 x 3 cross-channel maps: joint band moments bit-exact, the FP64 maps
    (FP32 seed refined by FP64 Newton steps) within the FP64 bar of the
    oracle's eigen-decompositions (the oracle's own evaluation loses up to
    ~1e-8 on ill-conditioned bands), images bit-exact; a ring under the
    lagged schedule with a moving object, blended block maps; and the
    defining equation M S M = S_s to 1e-12."""
    run_sequence(rt, orc, synth.small_pair(), 6, fit_mode=3, num_blocks=16)
    wl = synth.small_pair()
    wl.cams = [synth.Camera(640, 480, position=i) for i in range(3)]
    wl.moving_object = True
    run_sequence(rt, orc, wl, 4, fit_mode=3, num_blocks=4, topology=1, schedule=1)
    run_sequence(rt, orc, synth.small_pair(), 3, fit_mode=3, num_blocks=8, blend=True)
    assert _matrix_residual(rt, wl, 2, num_blocks=4, topology=1) < 1e-12


def test_matrix_maps_clamped_and_mono(rt, orc):
    """Tight gain limits make the eigenvalue clamp act (the divided-difference
    path); mono cameras give rank-one band covariances (two equal
    eigenvalues from the ridge); ragged widths."""
    run_sequence(rt, orc, synth.small_pair(), 4, fit_mode=3, num_blocks=4, gain_min=0.97, gain_max=1.02)
    cams = [synth.Camera(200, 120, position=0, y_pitch=208, uv_pitch=208),
            synth.Camera(220, 90, position=1, y_pitch=224, uv_pitch=224),
            synth.Camera(96, 40, fmt=synth.MONO16, bit_depth=10, group=1, position=0, y_pitch=192),
            synth.Camera(96, 64, fmt=synth.MONO16, bit_depth=10, group=1, position=1, y_pitch=192)]
    wl = synth.Workload("matrix ragged", cams, frames=3, seed=43)
    run_sequence(rt, orc, wl, 3, fit_mode=3, num_blocks=2, strip_width=16, min_valid=8)
    assert _matrix_residual(rt, wl, 2, num_blocks=2, strip_width=16, min_valid=8) < 1e-12


def test_seam_affine_64_blocks_ring_lagged(rt, orc):
    wl = synth.small_pair()
    wl.cams = [synth.Camera(640, 480, position=i) for i in range(3)]
    wl.moving_object = True
    run_sequence(rt, orc, wl, 5, fit_mode=1, num_blocks=64, topology=1, schedule=1)


@pytest.mark.parametrize("kw", [{}, {"topology": 1}, {"lam": 1e-2, "num_blocks": 4},
                                {"gain_min": 0.97, "gain_max": 1.02, "topology": 1}])
def test_global_fit_accuracy(rt, orc, kw):
    """The table-driven logarithm / exponential and the continuant solve stay
    within 1e-9 of the oracle's FP64 Cholesky solve (1e-6 is the parity bar):
    a 12-camera chain and ring, a larger ridge term, clamped gains."""
    wl = synth.tower12(frames=4)
    wl.cams = [synth.Camera(256, 144, position=i) for i in range(12)]
    wl.moving_object = True
    run_sequence(rt, orc, wl, 4, maps_rtol=1e-9, **kw)


def test_global_blocks_lagged_moving_object(rt, orc):
    wl = synth.small_pair()
    wl.moving_object = True
    run_sequence(rt, orc, wl, 6, num_blocks=16, schedule=1)


def test_ragged_widths_uneven_groups_and_ir(rt, orc):
    cams = [
        synth.Camera(72, 38, group=0, position=0, y_pitch=80, uv_pitch=80),
        synth.Camera(100, 38, group=0, position=1, y_pitch=112, uv_pitch=112),
        synth.Camera(66, 40, group=0, position=2, y_pitch=80, uv_pitch=96),
        synth.Camera(90, 20, fmt=synth.MONO16, bit_depth=12, group=1, position=0, y_pitch=192),
        synth.Camera(64, 20, fmt=synth.MONO16, bit_depth=10, group=1, position=1),
        synth.Camera(34, 6, group=2, position=0, y_pitch=48, uv_pitch=48),
    ]
    wl = synth.Workload("ragged", cams, frames=4, seed=12, glare_cams=(1,))
    for kw in ({}, {"fit_mode": 1, "num_blocks": 3}, {"num_blocks": 5, "topology": 1}, {"fit_mode": 2, "num_blocks": 2}):
        run_sequence(rt, orc, wl, 4, strip_width=16, min_valid=8, crops_per_frame=0, **kw)


def test_crops_edges_and_sizes(rt, orc):
    wl = synth.small_pair()
    wl.n_crops, wl.crop_side, wl.crop_out = 12, (1, 480), 48
    run_sequence(rt, orc, wl, 3, crops_per_frame=12, crop_size=48)
    wl.crop_side = (40, 64)
    run_sequence(rt, orc, wl, 2, crops_per_frame=9, crop_size=97)


def test_host_input_path_matches(rt, orc):
    run_sequence(rt, orc, synth.small_pair(), 3, device_inputs=False, crops_per_frame=4, crop_size=32)


def test_host_outputs_pipelined(rt):
    wl = synth.small_pair()
    a = rt.CameraArray(wl.cams)
    b = rt.CameraArray(wl.cams)
    outs = []
    for t in range(4):
        fs = synth.frame_set(wl, t, device="cuda")
        host = [{k: v.cpu().pin_memory() for k, v in f.items()} for f in fs]
        o = [torch.empty((c.height, 3 * c.width), dtype=torch.uint8).pin_memory() for c in wl.cams]
        a.submit_frames_host(host, t, rgb_out=o, rgb_out_pitch=3 * 640)
        b.submit_frames(fs, t)
        a.sync()
        for k in range(2):
            assert torch.equal(o[k].view(480, 640, 3), b.get_corrected(k).cpu())
        outs.append(o)
    a.close()
    b.close()


@pytest.mark.parametrize("fit_mode", [1, 3])
def test_state_save_and_resume(rt, orc, fit_mode):
    wl = synth.small_pair()
    a = rt.CameraArray(wl.cams, fit_mode=fit_mode, num_blocks=4)
    for t in range(3):
        a.submit_frames(synth.frame_set(wl, t, device="cuda"), t)
    blob = a.save_state()
    b = rt.CameraArray(wl.cams, fit_mode=fit_mode, num_blocks=4)
    b.load_state(blob)
    for t in range(3, 6):
        fs = synth.frame_set(wl, t, device="cuda")
        a.submit_frames(fs, t)
        b.submit_frames(fs, t)
        ma, qa = a.get_gains()
        mb, qb = b.get_gains()
        assert np.array_equal(ma, mb) and np.array_equal(qa, qb)
        assert torch.equal(a.get_corrected(1), b.get_corrected(1))
    a.close()
    b.close()


def test_get_times_out_instead_of_hanging(rt):
    wl = synth.small_pair()
    s = torch.cuda.Stream()
    a = rt.CameraArray(wl.cams, stream=s)
    fs = synth.frame_set(wl, 0, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(400_000_000)      # finite busy kernel ahead of the submit on the caller's stream
    a.submit_frames(fs, 0)
    with pytest.raises(rt.RtError) as ei:
        a.get_gains(timeout_ms=1)
    assert ei.value.status == rt.RT_ERR_TIMEOUT
    a.get_gains(timeout_ms=60000)
    a.close()


def test_tower12_full_size(rt, orc):
    """12 x 2048 x 1080 with glare and drifting gains, the benchmark's launch shape."""
    run_sequence(rt, orc, synth.tower12(frames=3), 3)


@pytest.mark.parametrize("fit_mode", [1, 2, 3])
def test_tower12_full_size_seam_fits(rt, orc, fit_mode):
    """The seam fits at full size, 16 blocks, the benchmark's launch shape:
    the paper's affine maps, the quantile-LS maps and the 3 x 3 maps."""
    run_sequence(rt, orc, synth.tower12(frames=2), 2, fit_mode=fit_mode, num_blocks=16)


def test_uneven_array_full_size_with_crops(rt, orc):
    wl = synth.uneven_array(frames=2)
    run_sequence(rt, orc, wl, 2, crops_per_frame=8, crop_size=512, num_blocks=16)


@pytest.mark.parametrize("kw", [{}, {"fit_mode": 1, "num_blocks": 16, "schedule": 1},
                                {"fit_mode": 2, "num_blocks": 8}, {"fit_mode": 3, "num_blocks": 8, "schedule": 1}])
def test_captured_ring_matches_single_submits(rt, kw):
    wl = synth.small_pair()
    wl.n_crops, wl.crop_side, wl.crop_out = 5, (16, 200), 40
    ring = 6
    frames = [synth.frame_set(wl, t, device="cuda") for t in range(ring)]
    crops = [synth.crop_list(wl, t) for t in range(ring)]
    a = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    b = rt.CameraArray(wl.cams, max_crops=5, crop_size=40, **kw)
    a.submit_frames(frames[0], 0, crops[0])
    a.profile(True)
    order = [(1 + j) % ring for j in range(ring)]
    a.capture_sequence([frames[i] for i in order], [crops[i] for i in order])
    a.profile(False)
    for t in range(0, 1 + 2 * ring):
        b.submit_frames(frames[t % ring], t, crops[t % ring])
    a.launch_sequence()
    a.launch_sequence()
    ma, qa = a.get_gains()
    mb, qb = b.get_gains()
    assert np.array_equal(ma, mb) and np.array_equal(qa, qb)
    for k in range(2):
        assert torch.equal(a.get_corrected(k), b.get_corrected(k))
    assert torch.equal(a.get_crops(), b.get_crops())
    sa, sb = a.get_stats(), b.get_stats()
    for name in ("strip_hist", "strip_n", "strip_sum", "frame_hist", "strip_joint"):
        assert (sa[name] is None and sb[name] is None) or np.array_equal(sa[name], sb[name]), name
    prof = a.get_profile()
    assert prof["frame_sets"] == ring
    assert prof["pass_b_ms"] > 0 and prof["pass_a_ms"] > 0 and prof["solve_ms"] > 0 and prof["crops_ms"] > 0
    # a single submit in between breaks the ring's slot alignment
    a.submit_frames(frames[1], 13, crops[1])
    with pytest.raises(rt.RtError) as ei:
        a.launch_sequence()
    assert ei.value.status == rt.RT_ERR_STATE
    # events around pass B only: the other passes report nothing
    a.profile(True, pass_b_only=True)
    order = [(14 + j) % ring for j in range(ring)]
    a.capture_sequence([frames[i] for i in order], [crops[i] for i in order])
    a.profile(False)
    a.launch_sequence()
    prof = a.get_profile()
    assert prof["frame_sets"] == ring
    assert prof["pass_b_ms"] > 0 and prof["crops_ms"] > 0
    assert prof["pass_a_ms"] == 0 and prof["solve_ms"] == 0
    assert a.L.rt_profile(a.h, 3) == rt.RT_ERR_INVALID     # unknown mode
    a.close()
    b.close()


@pytest.mark.parametrize("topology", [0, 1])
def test_seam_costs(rt, orc, topology):
    """Eq. (gradientcost) per seam of the corrected output against the
    oracle's FP64 cost of the oracle's own corrected images."""
    from oracle import seamcost
    cams = [synth.Camera(200, 100, position=0, y_pitch=208, uv_pitch=208),
            synth.Camera(210, 120, position=1, y_pitch=224, uv_pitch=224),
            synth.Camera(256, 96, position=2),
            synth.Camera(160, 64, group=1, position=0), synth.Camera(176, 72, group=1, position=1)]
    wl = synth.Workload("seam cost", cams, frames=3, seed=23, glare_cams=(1,))
    p = _params_for_oracle(orc, topology=topology)
    arr = rt.CameraArray(wl.cams, flags=rt.RT_FLAG_SEAM_COST, topology=topology)
    o = orc.ArrayOracle(wl.cams, p)
    for t in range(3):
        fs = synth.frame_set(wl, t, device="cuda")
        arr.submit_frames(fs, t)
        maps, q16 = arr.get_gains()
        r = o.step(np_frames(fs), q16_override=q16, want_frame_stats=False)
        got = {(l, rr): c for l, rr, c in arr.seam_costs()}
        want = {(l, rr): seamcost.seam_cost(r["corrected"][l], r["corrected"][rr]) for _, l, rr in
                orc.seams(wl.cams, topology)}
        assert set(got) == set(want)
        for key, v in want.items():
            assert abs(got[key] - v) <= 1e-12 * max(1.0, abs(v)), (t, key, got[key], v)
    arr.close()


def test_attention_proposals_and_their_crops(rt, orc):
    """Difference attention (Sec. "Attention mechanisms"): the proposal list
    equals the oracle's exactly, frame set by frame set, and the crops of the
    proposals equal the oracle's crops of its corrected images."""
    from oracle import attention as oat
    cams = [synth.Camera(640, 480, position=0), synth.Camera(650, 480, position=1, y_pitch=656, uv_pitch=656),
            synth.Camera(300, 200, fmt=synth.MONO16, bit_depth=12, group=1, y_pitch=608)]
    wl = synth.Workload("attention", cams, frames=5, seed=31, moving_object=True)
    kw = dict(attn_window=128, attn_min_on=150, attn_max=12)
    arr = rt.CameraArray(wl.cams, flags=rt.RT_FLAG_ATTENTION | rt.RT_FLAG_FRAME_STATS, max_crops=8, crop_size=48,
                         **kw)
    p = _params_for_oracle(orc)
    o = orc.ArrayOracle(wl.cams, p)
    prev = None
    seen = 0
    for t in range(5):
        fs = synth.frame_set(wl, t, device="cuda")
        arr.submit_frames(fs, t, rt.RT_CROPS_FROM_PROPOSALS)
        lum = [orc.convert(c, f)[1] for c, f in zip(wl.cams, np_frames(fs))]
        want = [] if prev is None else oat.proposals(wl.cams, prev, lum, 24, 128, 150, 12)[0]
        got = arr.proposals()
        assert got == want, (t, got[:4], want[:4])
        seen += len(got)
        maps, q16 = arr.get_gains()
        crops = want[:8]
        r = o.step(np_frames(fs), crops=crops, crop_size=48, q16_override=q16, want_frame_stats=False)
        cr = arr.get_crops().float().cpu().numpy()
        assert cr.shape[0] == len(crops)
        if crops:
            assert np.abs(cr - r["crops"]).max() < 1e-3, t
        prev = lum
    assert seen > 0, "the moving object was proposed"
    arr.close()


def test_attention_in_a_captured_ring(rt):
    wl = synth.small_pair()
    wl.moving_object = True
    ring = 6
    frames = [synth.frame_set(wl, t, device="cuda") for t in range(ring + 1)]
    kw = dict(flags=rt.RT_FLAG_ATTENTION | rt.RT_FLAG_FRAME_STATS, max_crops=4, crop_size=32, attn_window=128,
              attn_min_on=150, attn_max=8)
    a = rt.CameraArray(wl.cams, **kw)
    b = rt.CameraArray(wl.cams, **kw)
    a.submit_frames(frames[0], 0)
    order = [1 + j for j in range(ring)]
    a.capture_sequence([frames[i] for i in order], [rt.RT_CROPS_FROM_PROPOSALS] * ring)
    b.submit_frames(frames[0], 0)
    for i in order:
        b.submit_frames(frames[i], i, rt.RT_CROPS_FROM_PROPOSALS)
    a.launch_sequence()
    assert a.proposals() == b.proposals()
    assert torch.equal(a.get_crops(), b.get_crops())
    a.close()
    b.close()


def test_thumbnails_and_features(rt, orc):
    run_sequence(rt, orc, synth.small_pair(), 2, thumbs=True)
    cams = [synth.Camera(72, 38, position=0, y_pitch=80, uv_pitch=80),
            synth.Camera(130, 76, position=1, y_pitch=144, uv_pitch=144),
            synth.Camera(90, 40, fmt=synth.MONO16, bit_depth=12, group=1, y_pitch=192)]
    wl = synth.Workload("ragged thumbs", cams, frames=2, seed=21)
    run_sequence(rt, orc, wl, 2, thumbs=True, strip_width=16, min_valid=8)
    # seam maps beside the thumbnails (with and without frame statistics)
    run_sequence(rt, orc, wl, 2, thumbs=True, strip_width=16, min_valid=8, fit_mode=1, num_blocks=3)
    run_sequence(rt, orc, wl, 2, thumbs=True, stats=False, strip_width=16, min_valid=8, fit_mode=3, num_blocks=2)
    run_sequence(rt, orc, synth.tower12(frames=1), 1, thumbs=True, stats=False)


@pytest.mark.parametrize("kw", [{}, {"fit_mode": 1, "num_blocks": 16}])
def test_thumbnails_wide_cameras(rt, orc, kw):
    """Cameras at least 16 x 64 columns wide sum a unit's thumbnail values in
    registers (two cells at most per unit): the per-camera gains with frame
    statistics and the seam maps' table variant, at full size."""
    run_sequence(rt, orc, synth.tower12(frames=1), 1, thumbs=True, **kw)
