"""Seeded synthetic camera-array frames shaped like a remote-tower array.

This module paints scenes; it holds no step of the correction method.  A
continuous panorama (sky above a ground band, smooth gradients, low-frequency
sinusoids) is sliced into adjacent cameras that share a seam but no overlap
(the setting of Sec. "White balance and exposure correction").  Each camera
scales its linear RGB by its own per-channel gain ``d[k, c]``, adds Gaussian
noise, rounds to 8 bit and encodes NV12 (BT.709 limited range, chroma the mean
of each 2x2 block) or 12-bit mono in 16-bit words for infrared cameras.

Both sides of every parity test (the CUDA path and the CPU oracle) consume the
bytes made here; neither side's arithmetic lives here.  Everything runs as
torch tensor ops on the requested device, so the benchmark can fill a ring of
frame sets on the GPU while the tests build small cases on the CPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import torch

NV12 = 0
MONO16 = 1


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fmt: int = NV12
    bit_depth: int = 8
    group: int = 0
    position: int = 0
    y_pitch: int = 0       # bytes per row of the Y plane (NV12) or of the mono plane
    uv_pitch: int = 0      # bytes per row of the interleaved UV plane (NV12)

    def __post_init__(self):
        if self.y_pitch == 0:
            self.y_pitch = self.width * (2 if self.fmt == MONO16 else 1)
        if self.uv_pitch == 0 and self.fmt == NV12:
            self.uv_pitch = self.width


@dataclasses.dataclass
class Workload:
    """A named array of cameras plus the scene options used to fill it."""
    name: str
    cams: List[Camera]
    frames: int
    seed: int
    glare_cams: Sequence[int] = ()
    gain_walk: float = 0.0          # per-frame random-walk step of the camera gains
    noise_sigma: float = 4.0
    mirror_seams: bool = False      # scene symmetric about every seam
    moving_object: bool = False     # bright block crossing a seam
    n_crops: int = 0
    crop_side: Sequence[int] = (0, 0)
    crop_out: int = 0

    @property
    def pixels(self) -> int:
        return sum(c.width * c.height for c in self.cams)


# ----------------------------------------------------------------------------
# Workloads with the shapes of the remote-tower arrays the benchmarks use.
# ----------------------------------------------------------------------------

def small_pair(seed: int = 1) -> Workload:
    """2 cameras of 640x480 NV12, 8 frames."""
    cams = [Camera(640, 480, position=i) for i in range(2)]
    return Workload("2x640x480 nv12, 8 frames", cams, frames=8, seed=seed)


def tower12(seed: int = 2, frames: int = 300) -> Workload:
    """12 cameras of 2048x1080 NV12 (26.5 MP per frame set), drifting gains,
    sun glare saturating part of cameras 3 and 8."""
    cams = [Camera(2048, 1080, position=i) for i in range(12)]
    return Workload("12x2048x1080 nv12", cams, frames=frames, seed=seed,
                    glare_cams=(3, 8), gain_walk=0.01)


def uneven_array(seed: int = 3, frames: int = 120) -> Workload:
    """4x3840x2160 + 6x2560x1440 + 6x1920x1080 NV12 and 2x640x512 12-bit IR,
    one seam chain per resolution class, 64 crops per frame set -> 512^2."""
    cams: List[Camera] = []
    for g, (w, h, n) in enumerate([(3840, 2160, 4), (2560, 1440, 6), (1920, 1080, 6)]):
        cams += [Camera(w, h, group=g, position=i) for i in range(n)]
    cams += [Camera(640, 512, fmt=MONO16, bit_depth=12, group=3, position=i) for i in range(2)]
    return Workload("uneven 4x4K+6x1440p+6x1080p+2xIR", cams, frames=frames, seed=seed,
                    n_crops=64, crop_side=(256, 1024), crop_out=512)


def stress24(seed: int = 5, frames: int = 60) -> Workload:
    """24 cameras of 3840x2160 NV12 (199 MP per frame set), 128 crops -> 640^2."""
    cams = [Camera(3840, 2160, position=i) for i in range(24)]
    return Workload("24x3840x2160 nv12", cams, frames=frames, seed=seed,
                    n_crops=128, crop_side=(320, 1280), crop_out=640)


# ----------------------------------------------------------------------------
# Scene painting
# ----------------------------------------------------------------------------

def _phases(seed: int, group: int) -> torch.Tensor:
    g = torch.Generator().manual_seed(1000003 * seed + 7919 * group + 17)
    return torch.rand(16, generator=g, dtype=torch.float64)


def initial_gains(wl: Workload) -> torch.Tensor:
    """Per-camera per-channel exposure/white-balance gains d[k, c] ~ U[0.6, 1.5]."""
    g = torch.Generator().manual_seed(wl.seed * 31 + 5)
    return 0.6 + 0.9 * torch.rand(len(wl.cams), 3, generator=g, dtype=torch.float64)


def gains_at(wl: Workload, frame: int) -> torch.Tensor:
    """Gains after ``frame`` random-walk steps of +-gain_walk, kept in [0.6, 1.5]."""
    d = initial_gains(wl)
    if wl.gain_walk > 0.0:
        g = torch.Generator().manual_seed(wl.seed * 131 + 11)
        for _ in range(frame):
            step = torch.where(torch.rand(d.shape, generator=g, dtype=torch.float64) < 0.5, -1.0, 1.0)
            d = (d + wl.gain_walk * step).clamp(0.6, 1.5)
    return d


def _panorama(u: torch.Tensor, vn: torch.Tensor, ph: torch.Tensor) -> torch.Tensor:
    """Radiance in [0, 255] of the three channels at panorama column u (pixels)
    and normalised row vn in [0, 1).  u: [1, W], vn: [H, 1] -> [3, H, W]."""
    p = [float(x) for x in ph]
    horizon = 0.40 + 0.03 * torch.sin(2 * math.pi * u / (2900.0 + 900 * p[0]) + 6.28 * p[1])
    sky = vn < horizon
    t = (vn / 0.4).clamp(max=1.0)
    wave = torch.sin(2 * math.pi * u / (1700.0 + 600 * p[2]) + 6.28 * p[3]) * \
        torch.cos(2 * math.pi * vn * (3.0 + p[4]) + 6.28 * p[5])
    slow = torch.sin(2 * math.pi * u / (5300.0 + 1500 * p[6]) + 6.28 * p[7])
    out = []
    sky_c = (110.0 + 20 * p[8], 150.0 + 15 * p[9], 205.0 + 10 * p[10])
    gnd_c = (95.0 + 20 * p[11], 105.0 + 15 * p[12], 70.0 + 15 * p[13])
    for c in range(3):
        s = sky_c[c] + 35.0 * t + 12.0 * slow
        gr = gnd_c[c] + 25.0 * wave + 20.0 * (vn - 0.4) + 10.0 * slow
        out.append(torch.where(sky, s, gr))
    return torch.stack(out, 0)


def _group_layout(wl: Workload):
    """Panorama column offset of each camera inside its seam chain."""
    offs, seams = {}, {}
    for g in sorted({c.group for c in wl.cams}):
        members = sorted([k for k, c in enumerate(wl.cams) if c.group == g],
                         key=lambda k: wl.cams[k].position)
        x = 0
        s = []
        for k in members:
            offs[k] = x
            x += wl.cams[k].width
            s.append(x)
        seams[g] = s[:-1]
    return offs, seams


def camera_rgb(wl: Workload, k: int, frame: int, device="cpu",
               gains: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Linear RGB (float32, [3, H, W], before noise/rounding) seen by camera k."""
    cam = wl.cams[k]
    offs, seams = _group_layout(wl)
    x = torch.arange(cam.width, device=device, dtype=torch.float32).view(1, -1) + offs[k]
    vn = (torch.arange(cam.height, device=device, dtype=torch.float32).view(-1, 1) + 0.5) / cam.height
    u = x
    if wl.mirror_seams and seams[cam.group]:
        # distance to the nearest seam of the chain: mirror symmetric about every seam
        s = torch.tensor(seams[cam.group], device=device, dtype=torch.float32).view(-1, 1, 1)
        u = (x.unsqueeze(0) + 0.5 - s).abs().min(0).values
    rgb = _panorama(u, vn, _phases(wl.seed, cam.group).to(device))
    if wl.moving_object:
        # a bright vehicle-sized block moving 6 px per frame along the ground
        ox = 6.0 * frame + 0.5 * (wl.cams[0].width) - 100.0
        oy0 = 0.62
        inside = ((x >= ox) & (x < ox + 120.0)) & ((vn >= oy0) & (vn < oy0 + 0.10))
        rgb = torch.where(inside.unsqueeze(0), torch.tensor([235.0, 232.0, 220.0], device=device).view(3, 1, 1), rgb)
    d = gains if gains is not None else gains_at(wl, frame)
    rgb = rgb * d[k].to(device=device, dtype=torch.float32).view(3, 1, 1)
    return rgb


def _noise(wl: Workload, k: int, frame: int, shape, device) -> torch.Tensor:
    if wl.noise_sigma <= 0:
        return torch.zeros(shape, device=device)
    g = torch.Generator(device=device).manual_seed((wl.seed * 1_000_003 + frame) * 1009 + k)
    return wl.noise_sigma * torch.randn(shape, generator=g, device=device)


def camera_rgb8(wl: Workload, k: int, frame: int, device="cpu", gains=None) -> torch.Tensor:
    """The camera's 8-bit RGB image [3, H, W] (uint8) after gain, noise and glare."""
    cam = wl.cams[k]
    rgb = camera_rgb(wl, k, frame, device, gains)
    rgb = rgb + _noise(wl, k, frame, rgb.shape, device)
    if k in wl.glare_cams:
        yy = torch.arange(cam.height, device=device, dtype=torch.float32).view(-1, 1)
        xx = torch.arange(cam.width, device=device, dtype=torch.float32).view(1, -1)
        r = 0.12 * cam.height
        disc = (xx - 0.6 * cam.width) ** 2 + (yy - 0.25 * cam.height) ** 2 < r * r
        rgb = torch.where(disc.unsqueeze(0), torch.full_like(rgb, 300.0), rgb)
    return rgb.round().clamp(0, 255).to(torch.uint8)


_KR, _KB = 0.2126, 0.0722  # BT.709 luma weights used by the camera's encoder


def encode_nv12(rgb8: torch.Tensor, y_pitch: int, uv_pitch: int):
    """BT.709 limited-range encoder of an 8-bit RGB image (what a camera's
    H.264 pipeline hands the decoder).  Returns (Y [H, y_pitch], UV [H/2, uv_pitch])."""
    _, H, W = rgb8.shape
    f = rgb8.to(torch.float32) / 255.0
    kg = 1.0 - _KR - _KB
    yn = _KR * f[0] + kg * f[1] + _KB * f[2]
    Y = (16.0 + 219.0 * yn).round().clamp(0, 255).to(torch.uint8)
    m = f.view(3, H // 2, 2, W // 2, 2).mean(dim=(2, 4))
    ym = _KR * m[0] + kg * m[1] + _KB * m[2]
    cb = (128.0 + 224.0 * (m[2] - ym) / (2 * (1 - _KB))).round().clamp(0, 255).to(torch.uint8)
    cr = (128.0 + 224.0 * (m[0] - ym) / (2 * (1 - _KR))).round().clamp(0, 255).to(torch.uint8)
    yplane = torch.zeros(H, y_pitch, dtype=torch.uint8, device=rgb8.device)
    yplane[:, :W] = Y
    uv = torch.zeros(H // 2, uv_pitch, dtype=torch.uint8, device=rgb8.device)
    uv[:, 0:W:2] = cb
    uv[:, 1:W:2] = cr
    return yplane, uv


def encode_mono(rgb8: torch.Tensor, bit_depth: int, pitch_bytes: int) -> torch.Tensor:
    """Infrared-like mono image: luminance scaled to ``bit_depth`` bits, stored
    in 16-bit words (as int16 storage; values never exceed 2^15 - 1)."""
    _, H, W = rgb8.shape
    f = rgb8.to(torch.float32)
    lum = _KR * f[0] + (1 - _KR - _KB) * f[1] + _KB * f[2]
    top = (1 << bit_depth) - 1
    v = (lum / 255.0 * top).round().clamp(0, top).to(torch.int16)
    plane = torch.zeros(H, pitch_bytes // 2, dtype=torch.int16, device=rgb8.device)
    plane[:, :W] = v
    return plane


def frame_set(wl: Workload, frame: int, device="cpu") -> List[Dict[str, torch.Tensor]]:
    """All cameras of one frame set, encoded.  Each entry holds either
    ``y``/``uv`` (NV12) or ``ir`` (mono16) tensors on ``device``."""
    out = []
    d = gains_at(wl, frame)
    for k, cam in enumerate(wl.cams):
        rgb8 = camera_rgb8(wl, k, frame, device, d)
        if cam.fmt == NV12:
            y, uv = encode_nv12(rgb8, cam.y_pitch, cam.uv_pitch)
            out.append({"y": y, "uv": uv})
        else:
            out.append({"ir": encode_mono(rgb8, cam.bit_depth, cam.y_pitch)})
    return out


def crop_list(wl: Workload, frame: int, n: Optional[int] = None):
    """Random square attention windows (cam, x0, y0, w, h) inside their camera."""
    n = wl.n_crops if n is None else n
    g = torch.Generator().manual_seed(wl.seed * 7 + frame * 7919 + 3)
    out = []
    lo, hi = wl.crop_side
    for _ in range(n):
        k = int(torch.randint(len(wl.cams), (1,), generator=g))
        cam = wl.cams[k]
        side = int(torch.randint(lo, hi + 1, (1,), generator=g))
        side = max(2, min(side, cam.width, cam.height))
        x0 = int(torch.randint(0, cam.width - side + 1, (1,), generator=g))
        y0 = int(torch.randint(0, cam.height - side + 1, (1,), generator=g))
        out.append((k, x0, y0, side, side))
    return out
