"""Training data and training loop of the learned gain surrogate.

The surrogate (include/rt_surrogate.h) predicts a camera's three log-gains
from its own 64x36 thumbnail.  Its labels come from the library's per-camera
gain fit (one block) run on synthetic arrays whose cameras carry random
exposure / white-balance gains and a random illuminant common to the array;
the features are the library's thumbnail features of the same frame sets.
A chain's common scale is unobservable, so predictions are compared after
re-gauging (subtracting the chain's mean log-gain), as the labels are.

Everything runs through the C ABI (librt.so); torch only holds buffers.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
import torch

from . import rt, synth


def training_workload(n_cams: int = 16, width: int = 512, height: int = 288, seed: int = 0) -> synth.Workload:
    cams = [synth.Camera(width, height, position=i) for i in range(n_cams)]
    return synth.Workload("surrogate training array", cams, frames=1, seed=seed)


def _array_gains(rng: np.random.Generator, n_cams: int) -> torch.Tensor:
    illum = rng.uniform(0.8, 1.25, size=(1, 3))
    d = rng.uniform(0.6, 1.5, size=(n_cams, 3)) * illum
    return torch.from_numpy(np.clip(d, 0.45, 1.9))


def make_dataset(n_arrays: int, seed: int = 0, n_cams: int = 16, width: int = 512, height: int = 288,
                 device="cuda") -> Tuple[torch.Tensor, torch.Tensor]:
    """(features BF16 [n_arrays*n_cams, 6912], labels FP32 [.., 3]) on the device."""
    wl = training_workload(n_cams, width, height, seed)
    arr = rt.CameraArray(wl.cams, flags=rt.RT_FLAG_THUMBNAILS)
    rng = np.random.default_rng(seed)
    xs: List[torch.Tensor] = []
    ys: List[torch.Tensor] = []
    for a in range(n_arrays):
        wl.seed = seed * 100003 + a             # a new panorama per array
        d = _array_gains(rng, n_cams)
        frames = []
        for k, cam in enumerate(wl.cams):
            y, uv = synth.encode_nv12(synth.camera_rgb8(wl, k, 0, device, gains=d), cam.y_pitch, cam.uv_pitch)
            frames.append({"y": y, "uv": uv})
        arr.submit_frames(frames, 0)            # frame index 0: no smoothing, the fit of this array
        maps, _ = arr.get_gains()
        x = arr.thumb_features()
        logg = np.log(maps[:, 0, 0, :, 0])      # per camera, gauge: sum over the chain is zero
        xs.append(x.clone())
        ys.append(torch.from_numpy(logg.astype(np.float32)).to(device))
    arr.close()
    return torch.cat(xs), torch.cat(ys)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial parameters (drawn here and passed in as an input)."""
    rng = np.random.default_rng(seed)
    flat = np.zeros(rt.MLP_PARAMS, np.float32)
    for name, off, shape in rt.param_offsets():
        n = int(np.prod(shape))
        if len(shape) == 2:
            flat[off:off + n] = rng.normal(0, math.sqrt(2.0 / shape[1]), n) * (0.5 if name == "W3" else 1.0)
    return flat


def regauge(pred: np.ndarray, n_cams: int) -> np.ndarray:
    """Subtract each array's mean predicted log-gain (per channel)."""
    p = pred.reshape(-1, n_cams, 3)
    return (p - p.mean(1, keepdims=True)).reshape(-1, 3)


def gain_error(pred_log: np.ndarray, label_log: np.ndarray) -> np.ndarray:
    """Per camera: max over channels of |exp(pred - label) - 1|."""
    return np.abs(np.exp(pred_log - label_log) - 1.0).max(-1)


def train(net: rt.GainMLP, X: torch.Tensor, Y: torch.Tensor, epochs: int = 4, batch: int = 256,
          lr: float = 1e-3, seed: int = 0) -> List[float]:
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        lr_ep = lr * (0.5 ** ep)
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            losses.append(net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr_ep))
    return losses


def predict(net: rt.GainMLP, X: torch.Tensor, batch: int = 256) -> np.ndarray:
    out = []
    for i in range(0, X.shape[0], batch):
        out.append(net.forward(X[i:i + batch].contiguous()).cpu().numpy())
    return np.concatenate(out)
