"""GPU parity of the learned gain surrogate's tensor-core kernels against the
FP64 oracle (oracle/mlp.py) on identical BF16 operands.

Primary pin (bit-exact): on sparse dyadic inputs every sum of the forward
and backward pass is exactly representable in FP32, which the test proves
by checking that the oracle's float32 and float64 paths agree bit for bit;
there any correct implementation must reproduce the oracle's output, loss
and every gradient exactly, whatever order it adds in.

Random inputs, layer by layer: the tensor cores add in their own order, so
a BF16 activation or gradient the GPU stores can round the other way than
the oracle's where the exact value sits near a BF16 rounding boundary, and
whole-network comparisons would compound those decisions through the layers.
So each layer's step is checked on the GPU's own operands (its stored BF16
activations, ReLU masks and incoming gradients, read back through
rt_check.h): every stored activation, every masked gradient and every
parameter gradient within 1e-3 of the oracle relative to the tensor's norm
(the bar for gradients on identical BF16 operands), the loss within 1e-4.
The forward of the whole network against the oracle's own activations stays
within 1e-3 relative to the output's norm.  Adam steps are checked on the
GPU's own gradients to FP32 rounding.
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
def test_layers_match_oracle_on_identical_operands(rt, n):
    net = rt.GainMLP()
    flat = _random_params(rt, 2, scale=2.0)
    net.set_params(flat)
    x, t, xt, tt = _inputs(n, 7 + n)
    g, loss = net.gradients(xt, tt)
    a = net.activations(n)
    P = _flat_to_dict(rt, flat)
    W1, W2, W3 = (omlp.bf16_round(P[k]) for k in ("W1", "W2", "W3"))
    x64 = omlp.bf16_round(x)
    errs = {}
    # forward: each layer from the GPU's own input to it
    _, h1 = omlp.dense_relu(x64, W1, P["b1"])
    errs["h1"] = _rel(a["h1"], h1)
    _, h2 = omlp.dense_relu(a["h1"], W2, P["b2"])
    errs["h2"] = _rel(a["h2"], h2)
    y = omlp.output_layer(a["h2"], W3, P["b3"])
    errs["y"] = _rel(a["y"], y)
    assert abs(loss - omlp.mse(a["y"], t)) <= 1e-4 * omlp.mse(a["y"], t)
    # backward: each step from the GPU's outputs, stored activations and masks
    gd = _flat_to_dict(rt, g)
    dy = omlp.output_grad(a["y"], t.astype(np.float64))
    dW3, db3 = omlp.weight_grads(dy, a["h2"])
    errs["W3"], errs["b3"] = _rel(gd["W3"], dW3), _rel(gd["b3"], db3)
    dz2 = omlp.hidden_grad(dy, W3, a["h2"] > 0)
    errs["dz2"] = _rel(a["dz2"], dz2)
    dW2, db2 = omlp.weight_grads(a["dz2"], a["h1"])
    errs["W2"], errs["b2"] = _rel(gd["W2"], dW2), _rel(gd["b2"], db2)
    dz1 = omlp.hidden_grad(a["dz2"], W2, a["h1"] > 0)
    errs["dz1"] = _rel(a["dz1"], dz1)
    dW1, db1 = omlp.weight_grads(a["dz1"], x64)
    errs["W1"], errs["b1"] = _rel(gd["W1"], dW1), _rel(gd["b1"], db1)
    assert max(errs.values()) <= 1e-3, errs
    # the activations really are the network's (not a zero read-back)
    assert np.linalg.norm(a["h1"]) > 0 and np.linalg.norm(a["dz1"]) > 0
    net.close()


def _exact_case(rt, n, seed):
    """Sparse dyadic parameters and inputs whose every sum is exact in FP32."""
    rng = np.random.default_rng(seed)
    flat = np.zeros(rt.MLP_PARAMS, np.float32)
    for name, off, shape in rt.param_offsets():
        m = int(np.prod(shape))
        if len(shape) == 2:
            v = rng.choice([-1.0, 0.0, 1.0], size=m, p=[0.25, 0.5, 0.25]) / 16.0
        else:
            v = rng.integers(-2, 3, size=m) / 256.0
        flat[off:off + m] = v
    x = (rng.choice([-1.0, 0.0, 1.0], size=(n, omlp.D_IN), p=[0.03, 0.94, 0.03]) / 16.0).astype(np.float32)
    return flat, x


@pytest.mark.parametrize("n", [1, 2, 3])
def test_forward_and_gradients_bit_exact_on_exact_arithmetic(rt, n):
    flat, x = _exact_case(rt, n, 100 + n)
    P = _flat_to_dict(rt, flat)
    y32, c32 = omlp.forward(P, x.astype(np.float64), bf16=True, acc32=True)
    y64, c64 = omlp.forward(P, x.astype(np.float64), bf16=True, acc32=False)
    assert np.array_equal(y32, y64)                      # the forward sums are exact
    # targets that make dy = 2 (y - t) / (3 n) a small dyadic number
    k = np.random.default_rng(n).integers(-2, 3, size=(n, 3))
    t = (y64 - 3 * n * k * 2.0 ** -14).astype(np.float32)
    assert np.array_equal(t.astype(np.float64), y64 - 3 * n * k * 2.0 ** -14)
    G32 = omlp.backward(P, c32, t.astype(np.float64), bf16=True, acc32=True)
    G64 = omlp.backward(P, c64, t.astype(np.float64), bf16=True, acc32=False)
    for name in G64:
        assert np.array_equal(G32[name], G64[name]), name   # the backward sums are exact too
    net = rt.GainMLP()
    net.set_params(flat)
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    y = net.forward(xt).cpu().numpy().astype(np.float64)
    assert np.array_equal(y, y64)
    g, loss = net.gradients(xt, torch.from_numpy(t).cuda())
    gd = _flat_to_dict(rt, g)
    for name in G64:
        assert np.array_equal(gd[name], G64[name]), (name, np.abs(gd[name] - G64[name]).max())
    net.close()
    net.close()


def test_adam_steps_match_oracle_on_gpu_gradients(rt):
    """Two Adam steps: the oracle's update (FP64) of the GPU's FP32 master
    weights with the GPU's own gradient matches the GPU's update to FP32
    rounding (the moments carry over from the first step to the second)."""
    net = rt.GainMLP()
    flat = _random_params(rt, 3)
    net.set_params(flat)
    P = _flat_to_dict(rt, flat)
    state = {}
    for step, seed in ((1, 11), (2, 12)):
        x, t, xt, tt = _inputs(256, seed)
        G, _ = net.gradients(xt, tt)
        net.train_step(xt, tt, 1e-3)
        got = _flat_to_dict(rt, net.get_params())
        ref = omlp.adam_step({k: v.copy() for k, v in P.items()}, _flat_to_dict(rt, G), state, lr=1e-3, t=step)
        for name in P:
            step_ref = ref[name] - P[name]
            assert np.abs(step_ref).max() > 1e-5, name            # the step moved the weights
            err = np.abs(got[name] - ref[name]).max()
            assert err <= 2e-8 + 2e-7 * np.abs(ref[name]).max(), (step, name, err)
        P = got
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


def test_trained_surrogate_beats_no_correction(rt):
    """Train on arrays labelled by the per-camera gain fit, then predict the
    gains of unseen arrays: the re-gauged prediction error must be well below
    the error of leaving the cameras uncorrected (identity gains)."""
    from paper_1910_03517_gb300 import surrogate as sg
    Xtr, Ytr = sg.make_dataset(160, seed=1, n_cams=16, width=256, height=144)
    Xte, Yte = sg.make_dataset(24, seed=2, n_cams=16, width=256, height=144)
    net = rt.GainMLP()
    net.set_params(sg.init_params(0))
    losses = sg.train(net, Xtr, Ytr, epochs=6, lr=1e-3)
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5])
    pred = sg.regauge(sg.predict(net, Xte), 16)
    lab = Yte.cpu().numpy()
    err = sg.gain_error(pred, lab)
    err_id = sg.gain_error(np.zeros_like(lab), lab)
    assert np.median(err) < 0.5 * np.median(err_id), (np.median(err), np.median(err_id))
    # inference + judge through the handle: re-gauged clamped gains and the
    # largest relative deviation from the fit of the same frame set
    wl = sg.training_workload(16, 256, 144, seed=77)
    arr = rt.CameraArray(wl.cams, flags=rt.RT_FLAG_THUMBNAILS)
    arr.submit_frames(synth_frames(wl), 0)
    fit, _ = arr.get_gains()
    pmaps, perr = arr.surrogate_predict(net)
    y = net.forward(arr.thumb_features()).cpu().numpy().astype(np.float64)
    want = np.clip(np.exp(y - y.mean(0, keepdims=True)), 0.25, 4.0)
    assert np.abs(pmaps[:, 0, 0, :, 0] - want).max() < 1e-9
    assert (pmaps[:, 1] == pmaps[:, 0]).all() and (pmaps[..., 1] == 0).all()
    assert abs(perr - np.abs(want / fit[:, 0, 0, :, 0] - 1).max()) < 1e-9
    arr.close()
    net.close()


def synth_frames(wl):
    from paper_1910_03517_gb300 import synth
    return synth.frame_set(wl, 0, device="cuda")
