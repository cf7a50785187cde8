"""Pins of the oracle's 3 x 3 cross-channel maps (the paper's future work:
linear maps that combine the three colour channels, Sec. "Conclusion"):
joint band statistics against a numpy brute force, the moment-matching
identity M S M^T = S_s with S_s the covariance of the pooled pixels, the
pooled mean, symmetry and the eigenvalue clamp, the per-channel closed form
for diagonal covariances, identity for equal bands, and the apply against the
pinned affine apply (diagonal M) and against channel permutations; and the
whole fit against the definition evaluated with 40 significant digits."""
import numpy as np
import pytest

from oracle import core


class _Cam:
    def __init__(self, pos, W=64, H=32):
        self.width, self.height, self.group, self.position = W, H, 0, pos


def _joint_of(pix):
    """{n, sums, second moments} of an [n, 3] pixel list, by numpy."""
    pix = pix.astype(np.int64)
    P = pix.T @ pix
    return np.array([len(pix), *pix.sum(0), P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]],
                    np.uint64)


def _fit(pR, pL, p=None):
    """maps of a two-camera chain: pR = pixels of the left camera's right
    band, pL = pixels of the right camera's left band."""
    p = p or core.Params(fit_mode=core.FIT_MATRIX, min_valid=1, gain_min=0.01, gain_max=100.0)
    joint = np.zeros((2, 2, 1, 10), np.uint64)
    joint[0, 1, 0] = _joint_of(pR)
    joint[1, 0, 0] = _joint_of(pL)
    return core.fit_matrix([_Cam(0), _Cam(1)], joint, p)


def _Mb(maps, k, side):
    return maps[k, side, 0, :9].reshape(3, 3), maps[k, side, 0, 9:]


def _cov(pix):
    return np.cov(pix.astype(np.float64).T, bias=True) + core.MATRIX_RIDGE * np.eye(3)


def _band(rng, n, mean, mix):
    base = rng.normal(0, 1, (n, 3)) @ mix + mean
    return np.clip(base.round(), 1, 254).astype(np.int64)


def test_joint_stats_match_numpy():
    rng = np.random.default_rng(31)
    H, W, S, B, T = 37, 96, 16, 3, 6
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    rgb[rng.random((H, W)) < 0.1, 1] = 255
    rgb[rng.random((H, W)) < 0.1, 2] = 0
    luma = rng.integers(0, 256, (H, W), dtype=np.uint8)
    prev = np.clip(luma.astype(np.int64) + rng.integers(-12, 13, (H, W)), 0, 255).astype(np.uint8)
    for pl in (None, prev):
        got = core.strip_joint(rgb, luma, pl, S, B, T)
        for side, x0 in ((0, 0), (1, W - S)):
            for j in range(B):
                y0, y1 = j * H // B, (j + 1) * H // B
                blk = rgb[y0:y1, x0:x0 + S].reshape(-1, 3)
                ok = np.all((blk > 0) & (blk < 255), axis=1)
                if pl is not None:
                    d = np.abs(luma[y0:y1, x0:x0 + S].astype(int) - pl[y0:y1, x0:x0 + S].astype(int))
                    ok &= d.reshape(-1) <= T
                assert np.array_equal(got[side, j], _joint_of(blk[ok])), (side, j)


def test_moment_matching_to_pooled_pixels():
    """With equal pixel counts the equal-weight mixture is the pooled sample:
    each side's map sends its band's mean to the pooled mean and its
    covariance (plus ridge) to the pooled covariance (plus ridge)."""
    rng = np.random.default_rng(32)
    for _ in range(10):
        n = 4000
        pR = _band(rng, n, rng.uniform(60, 190, 3), rng.uniform(-12, 12, (3, 3)) + 14 * np.eye(3))
        pL = _band(rng, n, rng.uniform(60, 190, 3), rng.uniform(-12, 12, (3, 3)) + 14 * np.eye(3))
        m = _fit(pR, pL)
        pooled = np.concatenate([pR, pL])
        Ss, mus = _cov(pooled), pooled.mean(0)
        for pix, (k, side) in ((pR, (0, 1)), (pL, (1, 0))):
            M, b = _Mb(m, k, side)
            S = _cov(pix)
            assert np.allclose(M @ S @ M.T, Ss, rtol=1e-9, atol=1e-9 * np.abs(Ss).max())
            assert np.allclose(M @ pix.mean(0) + b, mus, rtol=0, atol=1e-9)
            assert np.allclose(M, M.T, atol=1e-12)
            assert np.linalg.eigvalsh(M).min() > 0


def test_diagonal_covariances_give_per_channel_rule():
    """Uncorrelated channels and means differing in one channel: M is diagonal
    with M_cc = sqrt((v_s + r) / (v_c + r)), v_s the mixture variance."""
    n = 8
    pR = np.array([[10, 20, 30], [14, 20, 30], [10, 24, 30], [10, 20, 36],
                   [14, 24, 30], [14, 20, 36], [10, 24, 36], [14, 24, 36]])
    pL = pR * np.array([3, 1, 2]) + np.array([5, 0, -33])  # means differ in R only
    m = _fit(pR, pL)
    r = core.MATRIX_RIDGE
    vR = pR.var(0)
    vL = pL.var(0)
    d = pL.mean(0) - pR.mean(0)
    vs = (vR + vL) / 2 + d * d / 4
    for (k, side, v) in ((0, 1, vR), (1, 0, vL)):
        M, b = _Mb(m, k, side)
        assert np.allclose(M, np.diag(np.sqrt((vs + r) / (v + r))), rtol=0, atol=1e-12)
    assert n == len(pR)


def test_identical_bands_give_identity_and_clamp_holds():
    rng = np.random.default_rng(33)
    p = _band(rng, 3000, np.array([100, 120, 90]), rng.uniform(-10, 10, (3, 3)) + 15 * np.eye(3))
    m = _fit(p, p)
    for (k, side) in ((0, 1), (1, 0)):
        M, b = _Mb(m, k, side)
        assert np.allclose(M, np.eye(3), atol=1e-12) and np.allclose(b, 0, atol=1e-9)
    # a 4x contrast difference against gain limits [0.8, 1.25]
    lo = _band(rng, 3000, np.array([128, 128, 128]), 4 * np.eye(3))
    hi = _band(rng, 3000, np.array([128, 128, 128]), 16 * np.eye(3))
    par = core.Params(fit_mode=core.FIT_MATRIX, min_valid=1, gain_min=0.8, gain_max=1.25)
    m = _fit(lo, hi, par)
    for (k, side) in ((0, 1), (1, 0)):
        ev = np.linalg.eigvalsh(_Mb(m, k, side)[0])
        assert ev.min() >= 0.8 - 1e-12 and ev.max() <= 1.25 + 1e-12
    assert np.allclose(np.linalg.eigvalsh(_Mb(m, 0, 1)[0]), 1.25)
    assert np.allclose(np.linalg.eigvalsh(_Mb(m, 1, 0)[0]), 0.8)


def test_too_few_pixels_keep_identity():
    rng = np.random.default_rng(34)
    pR = _band(rng, 50, np.array([80, 90, 100]), 10 * np.eye(3))
    pL = _band(rng, 500, np.array([120, 90, 100]), 10 * np.eye(3))
    m = _fit(pR, pL, core.Params(fit_mode=core.FIT_MATRIX, min_valid=64))
    ident = core.identity_maps(2, 1, core.FIT_MATRIX)
    assert np.array_equal(m, ident)


def test_diagonal_apply_equals_affine_apply():
    rng = np.random.default_rng(35)
    H, W, B = 23, 70, 3
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    aff = np.zeros((2, B, 3, 2), np.int32)
    aff[..., 0] = rng.integers(40000, 90000, (2, B, 3))
    aff[..., 1] = rng.integers(-40 * 65536, 40 * 65536, (2, B, 3))
    mat = np.zeros((2, B, 12), np.int32)
    for c in range(3):
        mat[..., 4 * c] = aff[..., c, 0]
        mat[..., 9 + c] = aff[..., c, 1]
    assert np.array_equal(core.apply_matrix(rgb, mat, B), core.apply(rgb, aff, B, core.FIT_SEAM_AFFINE))


def test_permutation_at_border_columns():
    """At the outer columns the ramp weight is 1 and the map is applied whole:
    a cyclic permutation (R' = G, G' = B, B' = R) and a grey projection."""
    rng = np.random.default_rng(36)
    H, W = 9, 40
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    perm = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]])
    q = np.zeros((2, 1, 12), np.int32)
    q[:, 0, :9] = 65536 * perm.reshape(9)
    out = core.apply_matrix(rgb, q, 1)
    for x in (0, W - 1):
        assert np.array_equal(out[:, x], rgb[:, x][:, [1, 2, 0]])
    # a grey projection with an offset
    grey = np.zeros((2, 1, 12), np.int32)
    grey[:, 0, :9] = 21845
    grey[:, 0, 9:] = -3 * 65536
    out = core.apply_matrix(rgb, grey, 1)
    for x in (0, W - 1):
        v = rgb[:, x].astype(np.int64)
        want = np.clip((21845 * v.sum(1, keepdims=True) - 3 * 65536 + 32768) // 65536, 0, 255)
        assert np.array_equal(out[:, x], np.broadcast_to(want, v.shape))


def test_step_runs_matrix_mode_and_blending():
    """Lagged schedule: the first frame set uses the identity 3 x 3 maps and
    leaves the images unchanged; blending of block maps runs on 12-value maps."""
    from paper_1910_03517_gb300 import synth
    from conftest import np_frames
    wl = synth.small_pair()
    p = core.Params(fit_mode=core.FIT_MATRIX, num_blocks=2, schedule=core.SCHED_LAGGED)
    o = core.ArrayOracle(wl.cams, p)
    r0 = o.step(np_frames(synth.frame_set(wl, 0)))
    assert np.array_equal(r0["maps"], core.identity_maps(2, 2, core.FIT_MATRIX))
    for k in range(2):
        assert np.array_equal(r0["corrected"][k], r0["rgb"][k])
    r1 = o.step(np_frames(synth.frame_set(wl, 1)))
    assert r1["strip_joint"].shape == (2, 2, 2, 10)
    assert np.array_equal(r1["maps"], r0["E"])
    q = core.quantise(r1["maps"])
    rows = core.blend_rows(q[0], wl.cams[0].height, 2)
    assert rows.shape == (2, wl.cams[0].height, 12)
    assert np.array_equal(rows[:, 0], q[0][:, 0]) and np.array_equal(rows[:, -1], q[0][:, 1])
    p.blend_blocks = True
    o2 = core.ArrayOracle(wl.cams, p)
    o2.step(np_frames(synth.frame_set(wl, 0)))
    r2 = o2.step(np_frames(synth.frame_set(wl, 1)))
    assert np.array_equal(r2["maps"], r1["maps"])


def test_matches_a_40_digit_evaluation():
    """The oracle's FP64 eigen-decomposition route against the same
    definition evaluated with 40 significant digits (mpmath), on generic,
    luma-dominated and mono-like (rank one plus ridge) bands, with and
    without an active eigenvalue clamp: within the FP64 parity bar."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def fn(A, f):
        E, Q = mp.eigsy(A)
        return Q * mp.diag([f(e) for e in E]) * Q.T

    rng = np.random.default_rng(37)
    for trial in range(12):
        n = 2000
        if trial % 3 == 0:
            mix1, mix2 = rng.uniform(-12, 12, (3, 3)) + 14 * np.eye(3), rng.uniform(-12, 12, (3, 3)) + 14 * np.eye(3)
            pR = _band(rng, n, rng.uniform(60, 190, 3), mix1)
            pL = _band(rng, n, rng.uniform(60, 190, 3), mix2)
        elif trial % 3 == 1:
            pR = _band(rng, n, rng.uniform(60, 190, 3), np.ones((3, 3)) * rng.uniform(5, 30) + np.eye(3))
            pL = _band(rng, n, rng.uniform(60, 190, 3), np.ones((3, 3)) * rng.uniform(5, 30) + np.eye(3))
        else:
            g1, g2 = rng.normal(0, rng.uniform(3, 30), (n, 1)), rng.normal(0, rng.uniform(3, 30), (n, 1))
            pR = np.clip((np.repeat(g1, 3, 1) + rng.uniform(50, 200)).round(), 1, 254).astype(np.int64)
            pL = np.clip((np.repeat(g2, 3, 1) + rng.uniform(50, 200)).round(), 1, 254).astype(np.int64)
        gmin, gmax = (0.25, 4.0) if trial < 6 else (0.97, 1.02)
        m = _fit(pR, pL, core.Params(fit_mode=core.FIT_MATRIX, min_valid=1, gain_min=gmin, gain_max=gmax))
        # the definition in 40 digits, from the exact integer moments
        qR, qL = _joint_of(pR), _joint_of(pL)

        def moments(q):
            nn = mp.mpf(int(q[0]))
            mu = [mp.mpf(int(q[1 + i])) / nn for i in range(3)]
            idx = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
            S = mp.matrix(3, 3)
            for i in range(3):
                for j in range(3):
                    S[i, j] = mp.mpf(int(q[idx[(min(i, j), max(i, j))]])) / nn - mu[i] * mu[j] + \
                        (mp.mpf(core.MATRIX_RIDGE) if i == j else 0)
            return mu, S

        muR, SR = moments(qR)
        muL, SL = moments(qL)
        d = [muL[i] - muR[i] for i in range(3)]
        Ss = (SL + SR) * mp.mpf(0.5) + mp.matrix([[d[i] * d[j] / 4 for j in range(3)] for i in range(3)])
        for (k, side, S) in ((0, 1, SR), (1, 0, SL)):
            h, hi = fn(S, mp.sqrt), fn(S, lambda x: 1 / mp.sqrt(x))
            M = hi * fn(h * Ss * h, mp.sqrt) * hi
            M = fn((M + M.T) * mp.mpf(0.5), lambda x: min(max(x, mp.mpf(gmin)), mp.mpf(gmax)))
            want = np.array([[float(M[i, j]) for j in range(3)] for i in range(3)])
            got = m[k, side, 0, :9].reshape(3, 3)
            assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), (trial, np.abs(got - want).max())
