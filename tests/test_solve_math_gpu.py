"""The gain solve's table-driven logarithm and exponential (include/rt_check.h)
against their error bounds.

The per-camera gain fit (Sec. "White balance and exposure correction") needs
ln of a ratio of band sums and the exponential of the solved log-gains; the
kernels evaluate both with Tang's table-driven methods.  The references here
are the host C library's log / exp in double precision (errors below one ulp),
evaluated in Python; the bounds are the methods' own.  Logarithm: each of the
two FP32 tails u^2/2 - u^3/3 + ... (|u| <= 1/256, so at most 7.7e-6) carries
up to ~6 FP32 roundings, 6 x 2^-24 x 7.7e-6 = 2.8e-12, and their difference
one more: under 1e-11 absolute.  Exponential: the FP32 tail (at most 1.5e-5)
and the FP32 copy of r give ~6e-12 relative: under 1e-11.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ref_log_ratio(a, b):
    # ln a - ln b with each log taken on the exact integer (Python ints)
    return np.array([math.log(int(p)) - math.log(int(q)) for p, q in zip(a, b)])


def test_log_ratio_random_and_edges():
    from paper_1910_03517_gb300 import rt
    rng = np.random.default_rng(5)
    n = 20000
    # band-sum products span 1 .. 2^62; mix magnitudes
    e = rng.integers(0, 62, size=(2, n))
    a = (rng.random(n) * 2.0 ** e[0]).astype(np.uint64) + 1
    b = (rng.random(n) * 2.0 ** e[1]).astype(np.uint64) + 1
    # table boundaries (1 + i/128) 2^k, their neighbours, powers of two, equal pairs
    edge = []
    for i in range(129):
        for k in (10, 30, 52, 61):
            v = int(round((1 + i / 128) * 2 ** k))
            edge += [v - 1, v, v + 1]
    edge = np.array(edge, np.uint64)
    a = np.concatenate([a, edge, np.array([1, 2, 1 << 62, 12345], np.uint64)])
    b = np.concatenate([b, edge[::-1], np.array([1, 1, 1, 12345], np.uint64)])
    x = np.zeros(len(a))
    got, _ = rt.check_solve_math(a, b, x)
    ref = _ref_log_ratio(a, b)
    err = np.abs(got - ref)
    assert err.max() < 1e-11, (err.max(), np.argmax(err))
    assert got[-1] == 0.0 and got[-4] == 0.0            # ln 1, ln(a/a)


def test_exp_random_and_edges():
    from paper_1910_03517_gb300 import rt
    rng = np.random.default_rng(6)
    x = np.concatenate([rng.uniform(-5, 5, 20000), rng.uniform(-700, 700, 2000),
                        np.arange(-64, 65) * math.log(2) / 64,      # table points j ln2/64
                        np.array([0.0, -700.0, 700.0, 1e-300, -1e-300])])
    a = np.ones(len(x), np.uint64)
    _, got = rt.check_solve_math(a, a, x)
    ref = np.exp(x)
    rel = np.abs(got / ref - 1.0)
    assert rel.max() < 1e-11, (rel.max(), x[np.argmax(rel)])
    assert got[-5] == 1.0


def test_invalid_inputs_are_rejected():
    from paper_1910_03517_gb300 import rt
    with pytest.raises(rt.RtError):
        rt.check_solve_math(np.array([0], np.uint64), np.array([1], np.uint64), np.zeros(1))
    with pytest.raises(rt.RtError):
        rt.check_solve_math(np.array([1], np.uint64), np.array([1], np.uint64), np.array([800.0]))
