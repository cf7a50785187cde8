/*
 * rt_check.h -- self-checks of librt.so's device arithmetic, for tests.
 *
 * No counterpart in the paper.  The per-camera gain fit (rt.h,
 * RT_FIT_GLOBAL; Sec. "White balance and exposure correction": log-gains
 * from the ratio of band means, gains as their exponentials) evaluates its
 * logarithm and exponential with table-driven methods (Tang, ACM TOMS 16(4)
 * 1990 and 15(2) 1989) instead of the CUDA math library: on GB300 each
 * FP64 instruction of a library call is a long serial step.  This entry
 * point runs those two device routines on given inputs so that tests can
 * hold them to their error bounds.
 */
#ifndef RT_CHECK_H
#define RT_CHECK_H

#include <stdint.h>

#include "rt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For i < n: log_ratio[i] = ln(a[i] / b[i]) for positive integers a[i], b[i]
 * (the solve's logarithm of a ratio of band sums), and exp_x[i] = e^x[i] for
 * x[i] in [-700, 700] (the solve's exponential).  All pointers are host
 * memory (n elements each; either pair may be NULL to skip it); the call
 * allocates device scratch, runs one kernel on the current device and
 * returns when done.  RT_ERR_INVALID for n < 0, a zero a[i] or b[i] or an x
 * outside the range; RT_ERR_CUDA if a CUDA call fails. */
rt_status rt_check_solve_math(int32_t n, const uint64_t *a, const uint64_t *b, double *log_ratio, const double *x,
                              double *exp_x);

/* Intermediate values of the learned surrogate's last rt_mlp_gradients call
 * (rt_surrogate.h), so that tests can run the FP64 oracle's layer steps on the
 * GPU's own operands (identical BF16 activations and ReLU masks) layer by
 * layer.  Host buffers (any may be NULL), for the call's n batch rows:
 *   h1, h2   BF16 bits [n][256]: relu(x W1^T + b1) and relu(h1 W2^T + b2);
 *   dz2      BF16 bits [n][256]: (dL/dy W3) masked by h2 > 0;
 *   dz1t     BF16 bits [256][256]: (dz2 W2) masked by h1 > 0, TRANSPOSED
 *            (column b = batch row b; columns >= n are zero);
 *   y        FP32 [n][3]: the network's outputs.
 * Waits for the network's stream.  RT_ERR_INVALID for n outside 1..256. */
typedef struct rt_mlp rt_mlp;
rt_status rt_mlp_check_activations(rt_mlp *m, int32_t n, uint16_t *h1, uint16_t *h2, uint16_t *dz2,
                                   uint16_t *dz1t, float *y);

#ifdef __cplusplus
}
#endif

#endif /* RT_CHECK_H */
