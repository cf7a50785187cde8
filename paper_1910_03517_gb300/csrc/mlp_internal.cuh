// Stream-ordered operations of the learned gain surrogate's network (k_mlp.cu)
// for the host runtime: no host synchronisation, so that they can be
// enqueued back to back (training) or captured in a CUDA graph (inference
// inside the frame-set pipeline).
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/rt.h"

typedef struct rt_mlp rt_mlp;

namespace rt {

constexpr int kMlpIn = 3 * RT_THUMB_H * RT_THUMB_W;   // 6912 thumbnail features
constexpr int kMlpOut = 3;                             // log-gains
constexpr int kMlpMaxRows = 256;                       // rows of one forward / training batch

// The network's input rows X [256][6912] (BF16, row-major): the forward
// reads rows 0 .. n-1, later rows are ignored.
__nv_bfloat16 *mlp_input(rt_mlp *m);
// Outputs of the last forward, FP32 [256][3].
const float *mlp_output(const rt_mlp *m);

// Y = network(X rows 0 .. n-1) on stream s (1 <= n <= 256).
cudaError_t mlp_forward_async(rt_mlp *m, int n, cudaStream_t s);

// One Adam step (learning rate lr) on the batch of rows idx[0 .. n-1] of a
// training set (features data_x [.][6912] BF16, targets data_t [.][3] FP32,
// both device memory): gathers the batch, runs the forward and backward
// passes and the update, and writes the batch loss (before the step) to the
// device float *loss_out.  Deterministic: the same parameters, batch and
// step count give bit-identical results.
cudaError_t mlp_train_batch_async(rt_mlp *m, const __nv_bfloat16 *data_x, const float *data_t, const int32_t *idx,
                                  int n, double lr, float *loss_out, cudaStream_t s);

// Adam steps taken so far.
int64_t mlp_steps(const rt_mlp *m);

// Waits for stream s and reports a GEMM that gave up waiting (RT_ERR_TIMEOUT).
rt_status mlp_check(rt_mlp *m, cudaStream_t s, std::string *msg);

// The FP32 master parameters, both Adam moments and the step count as one
// byte blob, and back (waits for stream s).
rt_status mlp_serialize(rt_mlp *m, cudaStream_t s, std::vector<uint8_t> *out);
rt_status mlp_deserialize(rt_mlp *m, cudaStream_t s, const uint8_t *p, size_t n);

}  // namespace rt
