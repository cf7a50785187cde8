/*
 * rt_track.h -- detection post-processing and tracking of librt.so
 * (Sec. "AI-based video tracking").  The detector itself (YOLO with trained
 * weights) is not part of the library: detections come from the caller.
 */
#ifndef RT_TRACK_H
#define RT_TRACK_H

#include <stdint.h>

#include "rt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* An axis-aligned box (x0, y0) - (x1, y1) with its probability and category. */
typedef struct {
    float x0, y0, x1, y1;
    float score;
    int32_t cls;        /* 0 .. 32767 */
} rt_box;

/* Greedy non-maximum suppression on the device: boxes with score < score_min
 * are dropped; then, per category, the remaining box of highest probability
 * is kept and the boxes of its category whose IoU (area of intersection over
 * area of union, 0 for an empty union) with it exceeds iou_max are
 * suppressed, until none remains; equal probabilities keep the earlier box.
 * boxes: n boxes in host or device memory (1 <= n <= 4096); keep: n int32 in
 * host memory, 1 for a kept box, 0 otherwise.  Runs on cuda_stream (NULL:
 * the default stream) and returns when done; allocates nothing (calls from
 * several threads run one at a time).  RT_ERR_INVALID for a bad n, a
 * NULL pointer or (boxes in host memory) a category outside 0..32767; the
 * category of a box in device memory is taken modulo 32768.  RT_ERR_CUDA on
 * a CUDA error. */
rt_status rt_nms(const rt_box *boxes, int32_t n, float score_min, float iou_max, int32_t *keep, void *cuda_stream);

typedef struct rt_tracker rt_tracker;

/* A tracker of objects across frames with the paper's rules: per category,
 * detections d are assigned one-to-one to existing objects o by the linear
 * sum assignment (Hungarian method) of C(d, o) = 1 - IoU(B_d, B_o) a^(f_d - f_o)
 * (B_o, f_o: the object's last box and frame); an assigned detection joins
 * its object if 1 - C(d, o) > tol_iou; otherwise, and for unassigned
 * detections, it starts a new object if 1 - min_o C(d, o) < tol_new over the
 * objects of its category (or there are none); else it is dropped.  The
 * paper's values: a = 0.99, tol_iou = 0.05, tol_new = 0.001.  Host code. */
rt_status rt_tracker_create(rt_tracker **out, double a, double tol_iou, double tol_new);

/* Process the detections of frame `frame` (host array of n boxes, usually
 * the boxes rt_nms kept): object_of[i] (host, n int32) receives the id of
 * the object detection i joined or started, -1 if it was dropped.  Object
 * ids count up from 0 in order of creation. */
rt_status rt_tracker_update(rt_tracker *t, const rt_box *dets, int32_t n, int64_t frame, int32_t *object_of);

/* The objects so far: for i < min(cap, count), id[i], cls[i], their last box
 * (score of the detection that set it), last frame and number of
 * detections in their history (any output may be NULL); *n = count. */
rt_status rt_tracker_objects(rt_tracker *t, int32_t *id, int32_t *cls, rt_box *last, int64_t *last_frame,
                             int32_t *history, int32_t cap, int32_t *n);

void rt_tracker_destroy(rt_tracker *t);

#ifdef __cplusplus
}
#endif

#endif /* RT_TRACK_H */
