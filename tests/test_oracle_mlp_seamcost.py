"""Pins of the FP64 surrogate oracle (forward, backward, Adam, features,
gauge) and of the seam-cost metric, Eq. (gradientcost).

Pins: backward against central finite differences of the float64 loss,
forward against torch's float64 linear layers, BF16 rounding against
torch's float32 -> bfloat16 conversion, Adam's first step in closed form,
and the seam cost of images whose gradient continues across the seam (0)
or jumps by a known step (the step).
"""
import numpy as np
import pytest
import torch

from oracle import mlp, seamcost


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, scale / np.sqrt(mlp.D_IN), (mlp.D_H, mlp.D_IN)),
        "b1": rng.normal(0, 0.05, mlp.D_H),
        "W2": rng.normal(0, scale / np.sqrt(mlp.D_H), (mlp.D_H, mlp.D_H)),
        "b2": rng.normal(0, 0.05, mlp.D_H),
        "W3": rng.normal(0, scale / np.sqrt(mlp.D_H), (mlp.D_OUT, mlp.D_H)),
        "b3": rng.normal(0, 0.05, mlp.D_OUT),
    }


def test_forward_matches_torch_float64():
    P = _params()
    X = np.random.default_rng(1).uniform(-0.5, 0.5, (8, mlp.D_IN))
    y, _ = mlp.forward(P, X, bf16=False)
    t = {k: torch.from_numpy(v) for k, v in P.items()}
    h = torch.relu(torch.nn.functional.linear(torch.from_numpy(X), t["W1"], t["b1"]))
    h = torch.relu(torch.nn.functional.linear(h, t["W2"], t["b2"]))
    ref = torch.nn.functional.linear(h, t["W3"], t["b3"]).numpy()
    assert np.abs(y - ref).max() < 1e-12


def test_backward_matches_finite_differences():
    P = _params(2, scale=2.0)
    rng = np.random.default_rng(3)
    X = rng.uniform(-0.5, 0.5, (6, mlp.D_IN))
    T = rng.normal(0, 0.3, (6, 3))
    y, cache = mlp.forward(P, X, bf16=False)
    G = mlp.backward(P, cache, T, bf16=False)
    eps = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        gflat = G[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.mse(mlp.forward(P, X, bf16=False)[0], T)
            flat[idx] = old - eps
            lm = mlp.mse(mlp.forward(P, X, bf16=False)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gflat[idx]) <= 1e-6 * max(1e-3, abs(gflat).max()), (name, idx, fd, gflat[idx])


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(4).normal(0, 3, 10000).astype(np.float32)
    x[:4] = [1.00390625, 1.01171875, -2.00390625, 3.0]       # exact ties
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert (mlp.bf16_round(x) == ref).all()


def test_adam_first_step_closed_form():
    P = {"w": np.array([1.0, -2.0, 0.5])}
    G = {"w": np.array([0.3, -4.0, 1e-3])}
    st = {}
    out = mlp.adam_step(dict(P), G, st, lr=0.01, t=1)
    step = 0.01 * G["w"] / (np.abs(G["w"]) + 1e-8)
    assert np.abs(out["w"] - (P["w"] - step)).max() < 1e-15


def test_features_and_gauge():
    sums = np.zeros((3, 36, 64), np.uint32)
    W, H = 130, 75
    for j in range(36):
        for i in range(64):
            area = ((i + 1) * W // 64 - i * W // 64) * ((j + 1) * H // 36 - j * H // 36)
            sums[:, j, i] = 51 * area
    f = mlp.thumb_features(sums, W, H)
    assert f.shape == (6912,) and np.abs(f - (0.2 - 0.5)).max() < 1e-15
    lg = np.random.default_rng(5).normal(0, 1, (6, 3))
    r = mlp.regauge(lg, [0, 0, 0, 1, 1, 1])
    assert np.abs(r[:3].sum(0)).max() < 1e-14 and np.abs(r[3:].sum(0)).max() < 1e-14
    assert np.abs((r - lg)[:3] - (r - lg)[0]).max() < 1e-14


def test_seam_cost_continuing_gradient_is_zero_and_step_is_measured():
    H, W = 64, 48
    x = np.arange(2 * W, dtype=np.float64)
    img = np.zeros((H, 2 * W, 3))
    img[..., 0] = 2.0 * x
    img[..., 1] = 100 + 0.5 * x
    img[..., 2] = 50
    left, right = img[:, :W], img[:, W:]
    assert seamcost.seam_cost(left, right, f=1) == pytest.approx(0.0, abs=1e-12)
    right2 = right.copy()
    right2[..., 1] += 12.0
    # d+ = |(0) - (12)| = 12 in green, d- = |0 - (-12)| = 12: cost 12
    assert seamcost.seam_cost(left, right2, f=1) == pytest.approx(12.0, abs=1e-12)
    assert seamcost.interior_cost(img, f=8) == pytest.approx(0.0, abs=1e-9)
