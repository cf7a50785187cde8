"""Detection post-processing and tracking (Sec. "AI-based video tracking").

TEST INFRASTRUCTURE ONLY.  Plain restatement of the paper's rules:

* detections below a confidence tolerance are dropped (tol_detect = 0.65);
* greedy non-maximum suppression per category: repeatedly keep the
  remaining detection of highest probability and suppress the detections of
  its category whose IoU with it exceeds tol_NMS (0.45 inside a detection,
  0.3 between attention mechanisms);
* per category, detections d are assigned one-to-one to existing objects o
  by the linear sum assignment of C(d, o) = 1 - IoU(B_d, B_o) a^(f_d - f_o),
  a = 0.99 (B_o, f_o: the object's last box and frame);
* an assigned detection joins its object if 1 - C(d, o) > tol_IoU = 0.05;
  otherwise, and for unassigned detections, it starts a new object if
  1 - min_o C(d, o) < tol'_IoU = 0.001 over the objects of its category.

Readings: IoU of boxes (x0, y0, x1, y1) with area (x1 - x0)(y1 - y0) and
IoU 0 when the union is empty; ties of probability keep the earlier box;
a rejected detection that overlaps an object is dropped (neither joins nor
starts one).  The assignment itself is scipy's linear_sum_assignment (a
library step), pinned against brute force in the tests.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
from scipy.optimize import linear_sum_assignment


def iou(a, b) -> float:
    ix = max(0.0, min(a[2], b[2]) - max(a[0], b[0]))
    iy = max(0.0, min(a[3], b[3]) - max(a[1], b[1]))
    inter = ix * iy
    union = (a[2] - a[0]) * (a[3] - a[1]) + (b[2] - b[0]) * (b[3] - b[1]) - inter
    return inter / union if union > 0 else 0.0


def nms(boxes: Sequence[Tuple[float, float, float, float, float, int]], score_min: float, iou_max: float) -> List[int]:
    """Indices of the kept boxes (x0, y0, x1, y1, score, cls), in input order."""
    alive = [b[4] >= score_min for b in boxes]
    keep = []
    while True:
        best = -1
        for i, b in enumerate(boxes):
            if alive[i] and (best < 0 or b[4] > boxes[best][4]):
                best = i
        if best < 0:
            break
        keep.append(best)
        alive[best] = False
        for j, b in enumerate(boxes):
            if alive[j] and b[5] == boxes[best][5] and iou(b, boxes[best]) > iou_max:
                alive[j] = False
    return sorted(keep)


class Tracker:
    def __init__(self, a: float = 0.99, tol_iou: float = 0.05, tol_new: float = 0.001):
        self.a, self.tol_iou, self.tol_new = a, tol_iou, tol_new
        self.objects: List[Dict] = []     # {"id", "cls", "box", "frame", "history"}

    def update(self, dets: Sequence[Tuple[float, float, float, float, float, int]], frame: int) -> List[int]:
        """Object id each detection joined or started, -1 if dropped."""
        out = [-1] * len(dets)
        for cls in sorted({d[5] for d in dets}):
            di = [i for i, d in enumerate(dets) if d[5] == cls]
            oi = [j for j, o in enumerate(self.objects) if o["cls"] == cls]
            C = np.ones((len(di), len(oi)))
            for r, i in enumerate(di):
                for c, j in enumerate(oi):
                    o = self.objects[j]
                    C[r, c] = 1.0 - iou(dets[i], o["box"]) * self.a ** (frame - o["frame"])
            assigned = {}
            if len(di) and len(oi):
                rows, cols = linear_sum_assignment(C)
                assigned = {int(r): int(c) for r, c in zip(rows, cols)}
            joined = []
            for r, i in enumerate(di):
                if r in assigned and 1.0 - C[r, assigned[r]] > self.tol_iou:
                    joined.append((i, oi[assigned[r]]))
                elif len(oi) == 0 or 1.0 - C[r].min() < self.tol_new:
                    new_id = len(self.objects)
                    self.objects.append({"id": new_id, "cls": cls, "box": tuple(dets[i][:4]), "frame": frame,
                                         "history": [(frame, tuple(dets[i][:4]))]})
                    out[i] = new_id
            for i, j in joined:
                o = self.objects[j]
                o["box"], o["frame"] = tuple(dets[i][:4]), frame
                o["history"].append((frame, tuple(dets[i][:4])))
                out[i] = o["id"]
        return out
