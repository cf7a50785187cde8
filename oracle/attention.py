"""Difference attention: where to look for moving objects (Sec. "Attention
mechanisms", the difference approach and Fig. "thresholded difference").

TEST INFRASTRUCTURE ONLY.  Plain numpy restatement:

  1. the change map of a camera: on-pixels where the absolute difference of
     the luma of two consecutive frame sets exceeds T;
  2. a window slides across the change map; a window is proposed for a
     detection when its number of on-pixels reaches min_on.

Readings (the paper gives no numbers): the luma is the NV12 Y plane (the
8-bit value of a mono camera), T is the motion threshold of the band
statistics (24), windows are squares of side `window` (256) at stride
window / 2 -- 2 x 2 blocks of square cells of side window / 2, the cells
covering the frame with the last row and column of cells partial, windows
clipped to the frame -- and min_on is 1 % of a window's area (655).
Proposals are listed camera by camera, window row by window row, left to
right, and cut at `cap`.  The first frame set of a sequence has no previous
frame and proposes nothing.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def change_map(cur: np.ndarray, prev: np.ndarray, T: int) -> np.ndarray:
    """|cur - prev| > T per pixel (bool [H, W])."""
    return np.abs(cur.astype(np.int16) - prev.astype(np.int16)) > T


def cell_counts(on: np.ndarray, cell: int) -> np.ndarray:
    """On-pixels per cell [ceil(H / cell), ceil(W / cell)]."""
    H, W = on.shape
    ny, nx = -(-H // cell), -(-W // cell)
    out = np.zeros((ny, nx), np.int64)
    for j in range(ny):
        for i in range(nx):
            out[j, i] = int(on[j * cell:(j + 1) * cell, i * cell:(i + 1) * cell].sum())
    return out


def window_rects(W: int, H: int, window: int) -> List[Tuple[int, int, int, int, int, int]]:
    """(cell column, cell row, x0, y0, w, h) of every window of a W x H frame,
    row by row; a window covers cells (i, j) .. (i + 1, j + 1) where they exist."""
    c = window // 2
    nx, ny = -(-W // c), -(-H // c)
    out = []
    for j in range(max(ny - 1, 1)):
        for i in range(max(nx - 1, 1)):
            x0, y0 = i * c, j * c
            out.append((i, j, x0, y0, min(window, W - x0), min(window, H - y0)))
    return out


def proposals(cams, prev_lumas: Sequence[np.ndarray], cur_lumas: Sequence[np.ndarray], T: int = 24,
              window: int = 256, min_on: int = 655, cap: int = 256):
    """(list of (cam, x0, y0, w, h), per-camera cell counts)."""
    c = window // 2
    props, counts = [], []
    for k, cam in enumerate(cams):
        cc = cell_counts(change_map(cur_lumas[k], prev_lumas[k], T), c)
        counts.append(cc)
        ny, nx = cc.shape
        for (i, j, x0, y0, w, h) in window_rects(cam.width, cam.height, window):
            n = int(cc[j:min(j + 2, ny), i:min(i + 2, nx)].sum())
            if n >= min_on and len(props) < cap:
                props.append((k, x0, y0, w, h))
    return props, counts
