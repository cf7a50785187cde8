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
 * thumbnail features of every camera go through the network m; the
 * predicted log-gains are re-gauged per seam chain (the chain's mean
 * log-gain per channel subtracted, as the fit's gauge does) and turned into
 * gains clamped like the fit's.  Writes maps_fp64 (may be NULL; layout of
 * rt_get_gains, (g, 0) on both sides) and *max_error (may be NULL): the
 * largest |g_pred / g_fit - 1| over cameras and channels against the
 * per-camera gain fit of the same frame set (before smoothing).  A caller
 * uses the prediction while *max_error stays below its tolerance and the
 * plain fit otherwise. */
rt_status rt_surrogate_predict(rt_handle *h, rt_mlp *m, double *maps_fp64, double *max_error, int32_t timeout_ms);

/* Text of the network's last error. */
const char *rt_mlp_last_error(rt_mlp *m);

void rt_mlp_destroy(rt_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* RT_SURROGATE_H */
