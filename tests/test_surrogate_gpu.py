"""GPU parity of the learned gain surrogate's tensor-core kernels against the
FP64 oracle (oracle/mlp.py) on identical BF16 operands.

Bars: forward outputs and every parameter gradient within 1e-3 of the
oracle relative to the tensor's norm; the batch loss within 1e-3 relative.
The GPU accumulates in FP32 and stores hidden activations and their
gradients in BF16; the oracle rounds at the same points and accumulates the
sums it rounds in float32 (acc32), so that both sides take each BF16
rounding decision in the kernel's precision.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    from paper_1910_03517_gb300 import build, rt as rtmod
    build.build()
    rtmod.load()
    return rtmod


def _flat_to_dict(rt, flat):
    return {name: flat[off:off + int(np.prod(shape))].reshape(shape).astype(np.float64)
            for name, off, shape in rt.param_offsets()}


def _random_params(rt, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    flat = np.zeros(rt.MLP_PARAMS, np.float32)
    for name, off, shape in rt.param_offsets():
        fan_in = shape[-1] if len(shape) == 2 else 16
        n = int(np.prod(shape))
        flat[off:off + n] = rng.normal(0, scale / np.sqrt(fan_in), n)
    return flat


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, (n, omlp.D_IN)).astype(np.float32)
    x = omlp.bf16_round(x).astype(np.float32)
    t = rng.normal(0, 0.3, (n, 3)).astype(np.float32)
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    return x, t, xt, torch.from_numpy(t).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [1, 16, 128, 200, 256])
def test_forward_matches_oracle(rt, n):
    net = rt.GainMLP()
    flat = _random_params(rt, 1, scale=2.0)
    net.set_params(flat)
    x, t, xt, tt = _inputs(n, n)
    y = net.forward(xt).cpu().numpy()
    ref, _ = omlp.forward(_flat_to_dict(rt, flat), x.astype(np.float64), bf16=True, acc32=True)
    assert _rel(y, ref) < 1e-3, _rel(y, ref)
    net.close()


@pytest.mark.parametrize("n", [256, 96])
def test_gradients_match_oracle(rt, n):
    net = rt.GainMLP()
    flat = _random_params(rt, 2, scale=2.0)
    net.set_params(flat)
    x, t, xt, tt = _inputs(n, 7 + n)
    g, loss = net.gradients(xt, tt)
    P = _flat_to_dict(rt, flat)
    y, cache = omlp.forward(P, x.astype(np.float64), bf16=True, acc32=True)
    G = omlp.backward(P, cache, t.astype(np.float64), bf16=True, acc32=True)
    assert abs(loss - omlp.mse(y, t)) <= 1e-3 * omlp.mse(y, t)
    gd = _flat_to_dict(rt, g)
    errs = {name: _rel(gd[name], G[name]) for name in G}
    assert max(errs.values()) < 1e-3, errs
    net.close()


def test_adam_step_matches_oracle(rt):
    net = rt.GainMLP()
    flat = _random_params(rt, 3)
    net.set_params(flat)
    x, t, xt, tt = _inputs(256, 11)
    net.train_step(xt, tt, 1e-3)
    after = net.get_params()
    P = _flat_to_dict(rt, flat)
    y, cache = omlp.forward(P, x.astype(np.float64), bf16=True, acc32=True)
    G = omlp.backward(P, cache, t.astype(np.float64), bf16=True, acc32=True)
    ref = omlp.adam_step(dict(P), G, {}, lr=1e-3, t=1)
    got = _flat_to_dict(rt, after)
    for name in P:
        step_ref = ref[name] - P[name]
        step_got = got[name] - P[name]
        # the first Adam step is lr * sign(g) except where |g| is tiny: compare the step
        assert _rel(step_got, step_ref) < 2e-2, name
    net.close()


def test_training_fits_a_linear_teacher(rt):
    net = rt.GainMLP()
    net.set_params(_random_params(rt, 4))
    rng = np.random.default_rng(5)
    A = rng.normal(0, 0.05, (omlp.D_IN, 3))
    losses = []
    for step in range(150):
        x = omlp.bf16_round(rng.uniform(-0.5, 0.5, (256, omlp.D_IN))).astype(np.float32)
        t = (x.astype(np.float64) @ A).astype(np.float32)
        losses.append(net.train_step(torch.from_numpy(x).to(torch.bfloat16).cuda(), torch.from_numpy(t).cuda(), 1e-3))
    assert np.mean(losses[-10:]) < 0.2 * np.mean(losses[:3]), (losses[:3], losses[-10:])
    net.close()
