/*
 * rt_surrogate.h -- learned gain surrogate of librt.so.
 *
 * No counterpart in the paper: its correction (Sec. "White balance and
 * exposure correction") always fits the maps from the band statistics.  The
 * surrogate is a small MLP that predicts a camera's three log-gains from its
 * own 64x36 thumbnail, trained on frame sets that the per-camera gain fit
 * (rt.h, RT_FIT_GLOBAL, one block) labels; that fit stays the fallback and
 * the judge of the prediction's error.
 *
 * Network: x (6912 = 3 x 36 x 64 thumbnail cell means / 255 - 0.5, BF16,
 * channel-major) -> Linear(6912, 256) -> ReLU -> Linear(256, 256) -> ReLU ->
 * Linear(256, 3).  Operands BF16, accumulation FP32 on the tensor cores,
 * FP32 master weights, Adam.  Parameter vector layout (1,836,291 FP32):
 *   W1 [256][6912], b1 [256], W2 [256][256], b2 [256], W3 [3][256], b3 [3]
 * (weights out x in).  Loss: mean over the batch and the three outputs of
 * (y - t)^2.
 *
 * All pointers may be host or device memory unless stated.  Calls are
 * synchronous with respect to the handle's stream (they return when done).
 */
#ifndef RT_SURROGATE_H
#define RT_SURROGATE_H

#include "rt.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RT_MLP_INPUTS 6912
#define RT_MLP_PARAMS 1836291

typedef struct rt_mlp rt_mlp;

/* Allocate a network on the current device (parameters zero; set them with
 * rt_mlp_set_params).  cuda_stream: stream the network's work runs on. */
rt_status rt_mlp_create(rt_mlp **out, void *cuda_stream);

/* Copy n = RT_MLP_PARAMS FP32 parameters in / out (layout above).
 * rt_mlp_set_params also clears the optimiser state. */
rt_status rt_mlp_set_params(rt_mlp *m, const float *params, size_t n);
rt_status rt_mlp_get_params(rt_mlp *m, float *params, size_t n);

/* y[n][3] = network(x[n][6912]) for 1 <= n <= 256 rows of BF16 inputs. */
rt_status rt_mlp_forward(rt_mlp *m, const void *x_bf16, int32_t n, float *y);

/* Gradients of the loss over the batch (x[n][6912] BF16, targets t[n][3]
 * FP32, 1 <= n <= 256) into grads (RT_MLP_PARAMS FP32, may be NULL) and the
 * loss into *loss (may be NULL); parameters unchanged. */
rt_status rt_mlp_gradients(rt_mlp *m, const void *x_bf16, const float *t, int32_t n, float *grads, float *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the batch; *loss (may be NULL) receives the batch loss before the step. */
rt_status rt_mlp_train_step(rt_mlp *m, const void *x_bf16, const float *t, int32_t n, double lr, float *loss);

/* Surrogate inference and its judge for the last frame set of an array
 * (rt.h handle with per-camera gains, one block, RT_FLAG_THUMBNAILS): the
 * thumbnail features of every camera go through the network m (NULL: the
 * handle's own network, see rt_surrogate_train); the
 * predicted log-gains are re-gauged per seam chain (the chain's mean
 * log-gain per channel subtracted, as the fit's gauge does) and turned into
 * gains clamped like the fit's.  Writes maps_fp64 (may be NULL; layout of
 * rt_get_gains, (g, 0) on both sides) and *max_error (may be NULL): the
 * largest |g_pred / g_fit - 1| over cameras and channels against the
 * per-camera gain fit of the same frame set (before smoothing).  A caller
 * uses the prediction while *max_error stays below its tolerance and the
 * plain fit otherwise. */
rt_status rt_surrogate_predict(rt_handle *h, rt_mlp *m, double *maps_fp64, double *max_error, int32_t timeout_ms);

/* ------------------------------------------------------------------------
 * The array's own network.  A handle with per-camera gains, one block and
 * RT_FLAG_THUMBNAILS owns one surrogate network, created by the first
 * rt_surrogate_train or rt_surrogate_load; its surrogate mode
 * (rt_array_params.surrogate_mode) uses it.  These calls return when done
 * and must not overlap a capture; they leave the array's frame-set sequence
 * untouched (their frames go through the array's kernels in the handle's
 * own scratch buffers).
 * ------------------------------------------------------------------------ */

/* Train the handle's network for one pass over n_samples samples (batch
 * rows a step, Adam learning rate lr; n_samples / batch steps).  The samples
 * are synthetic frame sets of the array's own cameras, generated on the
 * device from seed -- one sample per camera: a random scene (sky, horizon,
 * ground, gradients), an illuminant common to the array drawn per channel
 * from U[0.8, 1.25] and per-camera per-channel gains from U[0.6, 1.5] times
 * it (clipped to [0.45, 1.9]), noise sigma 4, NV12 (12-bit mono for infrared
 * cameras); features = the thumbnail features (rt_get_thumb_features),
 * label = the log-gains of the array's per-camera gain fit of that frame set
 * (first of a sequence: no smoothing).  The first call draws the initial
 * weights from seed (He-style normal, zero biases).  Calling again continues
 * training with the optimiser state; the samples of the same (n_samples,
 * seed) are kept between calls and visited in another order each call.
 * batch 1..256, batch <= n_samples <= 2^26, 0 < lr < 1. */
rt_status rt_surrogate_train(rt_handle *h, int64_t n_samples, int32_t batch, double lr, uint64_t seed);

/* The batch losses of the last rt_surrogate_train, one per step: *n = the
 * number of steps, min(cap, *n) copied to losses (host; may be NULL). */
rt_status rt_surrogate_losses(rt_handle *h, float *losses, int64_t cap, int64_t *n);

/* Held-out error of the handle's network on ceil(n_samples / K) fresh
 * synthetic frame sets from seed (generated as for training): per camera,
 * max over channels of |exp(p - x) - 1|, p the prediction re-gauged per
 * seam chain (the chain's mean log-gain subtracted, the fit's gauge) and x
 * the fit's log-gain.  errors (host, may be NULL) receives min(cap, *n_out)
 * values, frame set by frame set, camera by camera; errors_identity (may be
 * NULL) the same error of leaving the camera uncorrected (p = 0). */
rt_status rt_surrogate_evaluate(rt_handle *h, int64_t n_samples, uint64_t seed, double *errors,
                                double *errors_identity, int64_t cap, int64_t *n_out);

/* Checkpoint of the handle's network: the FP32 master weights, both Adam
 * moments, the Adam step count and the training-call count, in one file
 * (binary, "RTSG" version 1).  rt_surrogate_load restores all of it into
 * the handle (creating its network if needed): training continued after a
 * load gives bit-identical weights to training that never stopped.
 * RT_ERR_INVALID for a file that is not such a checkpoint. */
rt_status rt_surrogate_save(rt_handle *h, const char *path);
rt_status rt_surrogate_load(rt_handle *h, const char *path);

/* The handle's network parameters (n = RT_MLP_PARAMS FP32, layout above). */
rt_status rt_surrogate_get_params(rt_handle *h, float *params, size_t n);

/* Change the surrogate mode's fallback tolerance (>= 0) for the frame sets
 * enqueued after this call (captured sequences included: the judge reads it
 * on the device). */
rt_status rt_surrogate_set_tolerance(rt_handle *h, double tol);

/* What the surrogate mode did, over the frame sets since the handle's first
 * surrogate-mode submit (waits, bounded, for pending work). */
typedef struct {
    int64_t frame_sets;      /* frame sets corrected in surrogate mode */
    int64_t predicted;       /* ... with the surrogate's gains */
    int64_t plain;           /* ... with the plain fit (first of a sequence, fallback) */
    int64_t judged;          /* predictions judged by the plain fit */
    int64_t judged_failed;   /* judgements above the tolerance */
    int32_t fallback;        /* 1 while the plain fit is applied */
    double last_error;       /* max |g_pred / g_fit - 1| of the last judgement */
    double max_error;        /* ... of all judgements */
    double tolerance;        /* the tolerance in force */
} rt_surrogate_report;
rt_status rt_surrogate_get_report(rt_handle *h, rt_surrogate_report *out, int32_t timeout_ms);

/* Text of the network's last error. */
const char *rt_mlp_last_error(rt_mlp *m);

void rt_mlp_destroy(rt_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* RT_SURROGATE_H */
