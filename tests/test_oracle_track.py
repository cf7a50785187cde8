"""Pins of the tracking oracle (Sec. "AI-based video tracking"): IoU closed
forms, greedy NMS on hand-made cases, the assignment against brute force
over permutations, and the tracker's joining / starting rules."""
import itertools

import numpy as np

from oracle import track


def test_iou_closed_forms():
    assert track.iou((0, 0, 2, 2), (0, 0, 2, 2)) == 1.0
    assert track.iou((0, 0, 2, 2), (2, 2, 4, 4)) == 0.0
    assert abs(track.iou((0, 0, 2, 2), (1, 0, 3, 2)) - 2 / 6) < 1e-15
    assert track.iou((0, 0, 0, 0), (0, 0, 0, 0)) == 0.0


def test_nms_hand_cases():
    boxes = [(0, 0, 10, 10, 0.9, 0), (1, 1, 11, 11, 0.8, 0),     # overlaps the first (IoU 0.68): suppressed
             (1, 1, 11, 11, 0.85, 1),                           # same place, other category: kept
             (50, 50, 60, 60, 0.7, 0),                          # far away: kept
             (0, 0, 10, 10, 0.5, 0)]                            # below the confidence tolerance
    assert track.nms(boxes, 0.65, 0.45) == [0, 2, 3]
    # chained suppression: the middle box is suppressed, so it cannot suppress the third
    chain = [(0, 0, 10, 10, 0.9, 0), (6, 0, 16, 10, 0.8, 0), (12, 0, 22, 10, 0.7, 0)]
    assert track.nms(chain, 0.0, 0.2) == [0, 2]


def test_assignment_matches_brute_force():
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(2)
    for m, n in [(3, 3), (4, 2), (2, 5), (5, 5)]:
        C = rng.random((m, n))
        r, c = linear_sum_assignment(C)
        best = min(sum(C[i, p[i]] for i in range(m)) for p in itertools.permutations(range(n), m)) if m <= n else \
            min(sum(C[p[j], j] for j in range(n)) for p in itertools.permutations(range(m), n))
        assert abs(C[r, c].sum() - best) < 1e-12


def test_tracker_rules():
    t = track.Tracker()
    ids = t.update([(0, 0, 10, 10, 0.9, 0), (100, 100, 110, 110, 0.9, 1)], 0)
    assert ids == [0, 1]                                     # first detections start objects
    ids = t.update([(1, 0, 11, 10, 0.9, 0)], 1)               # moved by 1 px: IoU 0.82 > 0.05 -> joins 0
    assert ids == [0] and t.objects[0]["frame"] == 1 and len(t.objects[0]["history"]) == 2
    ids = t.update([(300, 300, 310, 310, 0.9, 0)], 2)         # no overlap with any object -> new
    assert ids == [2]
    # overlaps object 0 a little (discounted IoU between 0.001 and 0.05): neither joins nor starts
    ids = t.update([(10.5, 0, 20.5, 10, 0.9, 0)], 3)
    assert ids == [-1] and len(t.objects) == 3
    # the discount: the same box 300 frames later no longer joins (0.82 * 0.99^300 < 0.05)
    t2 = track.Tracker()
    t2.update([(0, 0, 10, 10, 0.9, 0)], 0)
    assert t2.update([(1, 0, 11, 10, 0.9, 0)], 300) == [-1]
