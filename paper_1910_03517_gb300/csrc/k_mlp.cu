// Learned gain surrogate (no counterpart in the paper): a camera's 3x36x64
// thumbnail -> Linear(6912, 256) -> ReLU -> Linear(256, 256) -> ReLU ->
// Linear(256, 3) -> the camera's three log-gains.  BF16 operands, FP32
// accumulation on the tcgen05 tensor cores (tc_gemm.cuh), FP32 master
// weights and Adam moments.  Trained with the mean squared error against the
// log-gains of the per-camera gain fit.
//
// A training step for a batch of 256 thumbnails (M = 256):
//   fwd1  H1 = relu(X W1^T + b1)        GEMM 256x256x6912 split over K in 27
//                                       pieces of 256 (108 CTAs), partial sums
//                                       reduced in a fixed order with the bias
//                                       and ReLU, writing H1 and H1^T
//   fwd2  H2 = relu(H1 W2^T + b2)       GEMM 256x256x256
//   head  y = H2 W3^T + b3, e = y - t, dZ2 = (dy W3) * [H2 > 0]  (CUDA cores)
//         loss, dW3, db3: sums over the batch in a fixed order
//   dW2 = dZ2^T H1                      GEMM 256x256x256  (A = dZ2^T, B = H1^T)
//   dZ1 = (dZ2 W2) * [H1 > 0]           GEMM 256x256x256  (A = dZ2,  B = W2^T)
//   dW1 = dZ1^T X                       GEMM 256x6912x256 (A = dZ1^T, B = X^T)
//   db1, db2 (batch sums), Adam over all parameters, BF16 copies of W1, W2, W2^T.
// No floating-point atomics anywhere: a step is bit-for-bit reproducible.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rt_internal.cuh"
#include "mlp_internal.cuh"
#include "tc_gemm.cuh"
#include "../../include/rt_surrogate.h"
#include "../../include/rt_check.h"

using namespace rt;

namespace {

constexpr int D_IN = 3 * RT_THUMB_H * RT_THUMB_W;   // 6912
constexpr int D_H = 256;
constexpr int D_OUT = 3;
constexpr int MAXB = 256;
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (size_t)D_H * D_IN, OFF_W2 = OFF_B1 + D_H,
                 OFF_B2 = OFF_W2 + (size_t)D_H * D_H, OFF_W3 = OFF_B2 + D_H, OFF_B3 = OFF_W3 + (size_t)D_OUT * D_H,
                 N_PARAMS = OFF_B3 + D_OUT;
constexpr int kBN = 128;
constexpr int kSplit1 = 27;        // K pieces of the first layer's forward GEMM (6912 = 27 x 256)
static_assert(D_IN % (kSplit1 * tc::kBK) == 0, "split of the first layer");

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// GEMM kernels with fused epilogues
// ---------------------------------------------------------------------------

struct EpiReluBias {            // out = bf16(relu(v + bias[col])), row-major and (optionally) transposed
    const float *bias;
    bf16 *out; int ld;          // [M][N]
    bf16 *outT; int ldT;        // [N][M] or nullptr
    __device__ void operator()(int row, int col0, const float *v) const
    {
        bf16 h[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) h[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[col0 + i], 0.0f));
        uint4 *d = reinterpret_cast<uint4 *>(out + (size_t)row * ld + col0);
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = reinterpret_cast<const uint4 *>(h)[i];
        if (outT) {
#pragma unroll
            for (int i = 0; i < 32; ++i) outT[(size_t)(col0 + i) * ldT + row] = h[i];
        }
    }
};

struct EpiMaskT {               // outT[col][row] = bf16(v * [H[row][col] > 0])
    const bf16 *H; int ldH;
    bf16 *outT; int ldT;
    __device__ void operator()(int row, int col0, const float *v) const
    {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float hv = __bfloat162float(H[(size_t)row * ldH + col0 + i]);
            outT[(size_t)(col0 + i) * ldT + row] = __float2bfloat16_rn(hv > 0.0f ? v[i] : 0.0f);
        }
    }
};

struct EpiStore {               // out[row][col] = v (FP32)
    float *out; int ld;
    __device__ void operator()(int row, int col0, const float *v) const
    {
        float4 *d = reinterpret_cast<float4 *>(out + (size_t)row * ld + col0);
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
};

struct EpiPartial {             // part[z][row][col] = v (FP32), z = the K piece (blockIdx.z)
    float *part; int M;
    __device__ void operator()(int row, int col0, const float *v) const
    {
        float4 *d = reinterpret_cast<float4 *>(part + ((size_t)blockIdx.z * M + row) * D_H + col0);
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
};

// One 128 x kBN tile of D = A B^T over the K piece blockIdx.z of K / gridDim.z.
template <class Epi>
__global__ void __launch_bounds__(128, 1) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int K, Epi epi,
                                                      int *err)
{
    const int kz = K / (int)gridDim.z;
    tc::gemm_tile<kBN>(&tmA, &tmB, (int)blockIdx.z * kz, kz, epi, err);
}

// ---------------------------------------------------------------------------
// CUDA-core kernels
// ---------------------------------------------------------------------------

// Sum of the first layer's K pieces in a fixed order, + bias, ReLU, BF16:
// H [M][256] row-major and (optionally) HT [256][ldT] transposed.  One
// thread per row and 4 consecutive columns.
__global__ void __launch_bounds__(256) split_relu_kernel(const float *__restrict__ part, int M,
                                                         const float *__restrict__ bias, bf16 *__restrict__ H,
                                                         bf16 *__restrict__ HT, int ldT)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * (D_H / 4)) return;
    const int row = t / (D_H / 4), c0 = (t % (D_H / 4)) * 4;
    const size_t zs = (size_t)M * D_H / 4;
    const float4 *p = reinterpret_cast<const float4 *>(part + (size_t)row * D_H + c0);
    float4 acc = p[0];
#pragma unroll
    for (int z = 1; z < kSplit1; ++z) {
        const float4 v = p[z * zs];
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    const float a[4] = {acc.x, acc.y, acc.z, acc.w};
    bf16 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __float2bfloat16_rn(fmaxf(a[i] + bias[c0 + i], 0.0f));
    *reinterpret_cast<uint2 *>(H + (size_t)row * D_H + c0) = *reinterpret_cast<const uint2 *>(h);
    if (HT) {
#pragma unroll
        for (int i = 0; i < 4; ++i) HT[(size_t)(c0 + i) * ldT + row] = h[i];
    }
}

// Output layer and the start of its backward for one batch row per CTA (256
// threads): y = H2 W3^T + b3; with gradients, e = y - t for the n_valid real
// rows (0 for padding rows) and dZ2 = ((2 e / (3 n)) W3) * [H2 > 0].
__global__ void __launch_bounds__(256) head_kernel(const bf16 *__restrict__ H2, const float *__restrict__ P,
                                                   const float *__restrict__ T, int n_valid, float *__restrict__ Y,
                                                   float *__restrict__ Eo, bf16 *__restrict__ dZ2,
                                                   bf16 *__restrict__ dZ2T, int Mb, int want_grad)
{
    const int b = blockIdx.x, i = threadIdx.x;
    __shared__ float red[D_OUT][8];
    __shared__ float dy[D_OUT];
    const float h = __bfloat162float(H2[(size_t)b * D_H + i]);
    float w[D_OUT];
#pragma unroll
    for (int o = 0; o < D_OUT; ++o) w[o] = __bfloat162float(__float2bfloat16_rn(P[OFF_W3 + o * D_H + i]));
#pragma unroll
    for (int o = 0; o < D_OUT; ++o) {
        float s = h * w[o];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((i & 31) == 0) red[o][i >> 5] = s;
    }
    __syncthreads();
    if (i < D_OUT) {
        float s = 0;
        for (int q = 0; q < 8; ++q) s += red[i][q];
        const float y = s + P[OFF_B3 + i];
        Y[b * D_OUT + i] = y;
        float d = 0.0f;
        if (want_grad) {
            const float e = b < n_valid ? y - T[b * D_OUT + i] : 0.0f;
            Eo[b * D_OUT + i] = e;
            d = 2.0f * e / (float)(n_valid * D_OUT);
        }
        dy[i] = d;
    }
    __syncthreads();
    if (!want_grad) return;
    float g = 0.0f;
#pragma unroll
    for (int o = 0; o < D_OUT; ++o) g += dy[o] * w[o];
    const bf16 z = __float2bfloat16_rn(h > 0.0f ? g : 0.0f);
    dZ2[(size_t)b * D_H + i] = z;
    dZ2T[(size_t)i * Mb + b] = z;
}

// Batch sums of the output layer, each in a fixed order (no atomics), with
// dy = 2 e / (3 n) rounded as in the head: dW3[o][i] = sum_b dy[b][o] H2[b][i]
// (thread i), db3[o] = sum_b dy[b][o] and (CTA 0) loss = sum_b,o e^2 / (3 n),
// both by a fixed tree over the threads.  Grid of 3 CTAs (o) x 256 threads.
__global__ void __launch_bounds__(256) head_sums_kernel(const bf16 *__restrict__ H2, const float *__restrict__ Eo,
                                                        int n_valid, float *__restrict__ G, float *__restrict__ loss)
{
    __shared__ float s_db[256], s_l[256];
    const int o = blockIdx.x, i = threadIdx.x;
    const float den = (float)(n_valid * D_OUT);
    float acc = 0.0f;
#pragma unroll 8
    for (int b = 0; b < n_valid; ++b) acc += (2.0f * Eo[b * D_OUT + o] / den) * __bfloat162float(H2[(size_t)b * D_H + i]);
    G[OFF_W3 + o * D_H + i] = acc;
    float l = 0.0f;
    if (i < n_valid) {
#pragma unroll
        for (int q = 0; q < D_OUT; ++q) {
            const float e = Eo[i * D_OUT + q];
            l += e * e;
        }
    }
    s_db[i] = i < n_valid ? 2.0f * Eo[i * D_OUT + o] / den : 0.0f;
    s_l[i] = l;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (i < w) {
            s_db[i] += s_db[i + w];
            s_l[i] += s_l[i + w];
        }
        __syncthreads();
    }
    if (i == 0) {
        G[OFF_B3 + o] = s_db[0];
        if (o == 0 && loss) *loss = s_l[0] / den;
    }
}

// A training batch gathered from a training set: X[b] = data_x[idx[b]],
// X^T, T[b] = data_t[idx[b]] for b < n; rows n .. 255 are zero.  Tiles of
// 32 rows x 32 features through shared memory (coalesced X^T stores).
__global__ void gather_kernel(const bf16 *__restrict__ data_x, const float *__restrict__ data_t,
                              const int32_t *__restrict__ idx, int n, bf16 *__restrict__ X, bf16 *__restrict__ XT,
                              float *__restrict__ T)
{
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        const bf16 v = r < n ? data_x[(size_t)idx[r] * D_IN + c] : __float2bfloat16_rn(0.0f);
        t[i][threadIdx.x] = v;
        X[(size_t)r * D_IN + c] = v;
    }
    if (blockIdx.x == 0 && threadIdx.y == 0) {
        const int r = r0 + threadIdx.x;
        for (int q = 0; q < D_OUT; ++q) T[r * D_OUT + q] = r < n ? data_t[(size_t)idx[r] * D_OUT + q] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) XT[(size_t)(c0 + i) * MAXB + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// bias gradient: db[j] = sum over the batch of dZ^T[j][b]  (one warp per j)
__global__ void bias_grad_kernel(const bf16 *__restrict__ dZT, int Mb, int n_valid, float *__restrict__ db, int n)
{
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= n) return;
    float s = 0.0f;
    for (int b = lane; b < n_valid; b += 32) s += __bfloat162float(dZT[(size_t)j * Mb + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) db[j] = s;
}

// XT[c][b] = X[b][c]
__global__ void transpose_kernel(const bf16 *__restrict__ X, int rows, int cols, bf16 *__restrict__ XT)
{
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? X[(size_t)r * cols + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) XT[(size_t)c * rows + r] = t[threadIdx.x][i];
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters; refreshes BF16 copies.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ Mm,
                            float *__restrict__ Vv, float lr, float b1, float b2, float eps, float c1, float c2,
                            bf16 *__restrict__ W1b, bf16 *__restrict__ W2b, bf16 *__restrict__ W2bT)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N_PARAMS; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * Mm[i] + (1.0f - b1) * g;
        const float v = b2 * Vv[i] + (1.0f - b2) * g * g;
        Mm[i] = m;
        Vv[i] = v;
        const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        P[i] = p;
        const bf16 pb = __float2bfloat16_rn(p);
        if (i < OFF_B1) {
            W1b[i] = pb;
        } else if (i >= OFF_W2 && i < OFF_B2) {
            const size_t q = i - OFF_W2, r = q / D_H, c = q % D_H;
            W2b[q] = pb;
            W2bT[c * D_H + r] = pb;
        }
    }
}

__global__ void refresh_bf16_kernel(const float *__restrict__ P, bf16 *__restrict__ W1b, bf16 *__restrict__ W2b,
                                    bf16 *__restrict__ W2bT)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < OFF_B2; i += (size_t)gridDim.x * blockDim.x) {
        const bf16 pb = __float2bfloat16_rn(P[i]);
        if (i < OFF_B1) {
            W1b[i] = pb;
        } else if (i >= OFF_W2) {
            const size_t q = i - OFF_W2, r = q / D_H, c = q % D_H;
            W2b[q] = pb;
            W2bT[c * D_H + r] = pb;
        }
    }
}

// Predicted log-gains y[K][3] -> re-gauged, clamped gains per chain and the
// judge's error against the fitted gains (maps_fit [K][2][1][3][2]).  One
// thread per (chain, channel); single CTA.
__global__ void surrogate_gains_kernel(const float *__restrict__ y, const int32_t *__restrict__ group_start,
                                       const int32_t *__restrict__ group_members, int n_groups,
                                       const double *__restrict__ maps_fit, double gmin, double gmax,
                                       double *__restrict__ maps_out, double *__restrict__ err_out)
{
    __shared__ double worst[96];
    const int t = threadIdx.x;
    double e = 0.0;
    if (t < n_groups * 3) {
        const int grp = t / 3, c = t % 3;
        const int g0 = group_start[grp], n = group_start[grp + 1] - g0;
        double mean = 0.0;
        for (int i = 0; i < n; ++i) mean += (double)y[group_members[g0 + i] * 3 + c];
        mean /= n;
        for (int i = 0; i < n; ++i) {
            const int cam = group_members[g0 + i];
            const double g = fmin(fmax(exp((double)y[cam * 3 + c] - mean), gmin), gmax);
            for (int side = 0; side < 2; ++side) {
                maps_out[((cam * 2 + side) * 3 + c) * 2] = g;
                maps_out[((cam * 2 + side) * 3 + c) * 2 + 1] = 0.0;
            }
            e = fmax(e, fabs(g / maps_fit[((cam * 2) * 3 + c) * 2] - 1.0));
        }
    }
    if (t < 96) worst[t] = e;
    __syncthreads();
    if (t == 0) {
        double m = 0.0;
        for (int i = 0; i < 96 && i < n_groups * 3; ++i) m = fmax(m, worst[i]);
        *err_out = m;
    }
}

// ---------------------------------------------------------------------------
// tensor maps
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// K-major BF16 matrix [rows][cols] (cols = K contiguous), box 64 x box_rows, 128-byte swizzle
bool make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows)
{
    EncodeTiled enc = get_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct rt_mlp {
    cudaStream_t s = nullptr;
    float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr, *W2bT = nullptr;
    bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ2T = nullptr,
         *dZ1T = nullptr;
    float *T = nullptr, *Y = nullptr, *Eo = nullptr, *loss = nullptr, *part = nullptr;
    int *err = nullptr;
    int64_t steps = 0;
    // tensor maps (fixed buffers)
    CUtensorMap mX, mW1, mH1, mW2, mdZ2T, mH1T, mdZ2, mW2T, mdZ1T, mXT;
    std::string msg;
};

namespace {

rt_status mfail(rt_mlp *m, rt_status s, const std::string &msg)
{
    if (m) m->msg = msg;
    return s;
}

#define MC(m, call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return mfail(m, e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA,               \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

#define CE(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return e_;                                                             \
    } while (0)

// The GEMM kernels' dynamic shared memory limit is set once, in rt_mlp_create.
template <class Epi>
cudaError_t gemm_attr()
{
    return cudaFuncSetAttribute(gemm_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc::Smem<kBN>::kBytes);
}

template <class Epi>
cudaError_t run_gemm(rt_mlp *m, const CUtensorMap &A, const CUtensorMap &B, int M, int N, int K, int splits,
                     const Epi &epi, cudaStream_t st)
{
    dim3 grid(N / kBN, M / tc::kBM, splits);
    gemm_kernel<Epi><<<grid, 128, tc::Smem<kBN>::kBytes, st>>>(A, B, K, epi, m->err);
    return cudaGetLastError();
}

// Forward of Mb rows of m->X (n_valid real ones) and, with grad, the backward
// into m->G and the batch loss into *loss_out (device; may be null).
cudaError_t fwd_bwd(rt_mlp *m, int Mb, int n_valid, bool grad, float *loss_out, cudaStream_t st)
{
    EpiPartial ep{m->part, Mb};
    CE(run_gemm(m, m->mX, m->mW1, Mb, D_H, D_IN, kSplit1, ep, st));
    {
        const int threads = Mb * (D_H / 4);
        split_relu_kernel<<<(threads + 255) / 256, 256, 0, st>>>(m->part, Mb, m->P + OFF_B1, m->H1,
                                                                 grad ? m->H1T : nullptr, MAXB);
        CE(cudaGetLastError());
    }
    EpiReluBias e2{m->P + OFF_B2, m->H2, D_H, nullptr, 0};
    CE(run_gemm(m, m->mH1, m->mW2, Mb, D_H, D_H, 1, e2, st));
    head_kernel<<<grad ? MAXB : Mb, D_H, 0, st>>>(m->H2, m->P, m->T, n_valid, m->Y, m->Eo, m->dZ2, m->dZ2T, MAXB,
                                                  grad ? 1 : 0);
    CE(cudaGetLastError());
    if (!grad) return cudaSuccess;
    head_sums_kernel<<<D_OUT, D_H, 0, st>>>(m->H2, m->Eo, n_valid, m->G, loss_out);
    CE(cudaGetLastError());
    EpiStore s2{m->G + OFF_W2, D_H};
    CE(run_gemm(m, m->mdZ2T, m->mH1T, D_H, D_H, MAXB, 1, s2, st));
    EpiMaskT mk{m->H1, D_H, m->dZ1T, MAXB};
    CE(run_gemm(m, m->mdZ2, m->mW2T, MAXB, D_H, D_H, 1, mk, st));
    EpiStore s1{m->G + OFF_W1, D_IN};
    CE(run_gemm(m, m->mdZ1T, m->mXT, D_H, D_IN, MAXB, 1, s1, st));
    bias_grad_kernel<<<D_H / 8, 256, 0, st>>>(m->dZ1T, MAXB, n_valid, m->G + OFF_B1, D_H);
    bias_grad_kernel<<<D_H / 8, 256, 0, st>>>(m->dZ2T, MAXB, n_valid, m->G + OFF_B2, D_H);
    return cudaGetLastError();
}

cudaError_t adam(rt_mlp *m, double lr, cudaStream_t st)
{
    m->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m->steps)), c2 = (float)(1.0 - std::pow(0.999, (double)m->steps));
    adam_kernel<<<1024, 256, 0, st>>>(m->P, m->G, m->Mm, m->Vv, (float)lr, b1, b2, 1e-8f, c1, c2, m->W1b, m->W2b,
                                      m->W2bT);
    return cudaGetLastError();
}

// A caller's batch (host or device memory) into X (and X^T, T for training);
// padding rows are zero.
rt_status load_batch(rt_mlp *m, const void *x, const float *t, int n)
{
    MC(m, cudaMemsetAsync(m->X, 0, (size_t)MAXB * D_IN * 2, m->s));
    MC(m, cudaMemcpyAsync(m->X, x, (size_t)n * D_IN * 2, cudaMemcpyDefault, m->s));
    if (t) {
        MC(m, cudaMemsetAsync(m->T, 0, (size_t)MAXB * D_OUT * 4, m->s));
        MC(m, cudaMemcpyAsync(m->T, t, (size_t)n * D_OUT * 4, cudaMemcpyDefault, m->s));
        dim3 g(D_IN / 32, MAXB / 32), b(32, 8);
        transpose_kernel<<<g, b, 0, m->s>>>(m->X, MAXB, D_IN, m->XT);
        MC(m, cudaGetLastError());
    }
    return RT_OK;
}

rt_status check_err(rt_mlp *m)
{
    std::string msg;
    rt_status s = rt::mlp_check(m, m->s, &msg);
    if (s != RT_OK) m->msg = msg;
    return s;
}

}  // namespace

namespace rt {

__nv_bfloat16 *mlp_input(rt_mlp *m) { return m->X; }
const float *mlp_output(const rt_mlp *m) { return m->Y; }
int64_t mlp_steps(const rt_mlp *m) { return m->steps; }

cudaError_t mlp_forward_async(rt_mlp *m, int n, cudaStream_t s)
{
    if (n < 1 || n > MAXB) return cudaErrorInvalidValue;
    return fwd_bwd(m, n <= tc::kBM ? tc::kBM : MAXB, n, false, nullptr, s);
}

cudaError_t mlp_train_batch_async(rt_mlp *m, const __nv_bfloat16 *data_x, const float *data_t, const int32_t *idx,
                                  int n, double lr, float *loss_out, cudaStream_t s)
{
    if (n < 1 || n > MAXB) return cudaErrorInvalidValue;
    dim3 g(D_IN / 32, MAXB / 32), b(32, 8);
    gather_kernel<<<g, b, 0, s>>>(data_x, data_t, idx, n, m->X, m->XT, m->T);
    CE(cudaGetLastError());
    CE(fwd_bwd(m, MAXB, n, true, loss_out, s));
    return adam(m, lr, s);
}

rt_status mlp_check(rt_mlp *m, cudaStream_t s, std::string *msg)
{
    int e = 0;
    cudaError_t r = cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (r == cudaSuccess) r = cudaStreamSynchronize(s);
    if (r != cudaSuccess) {
        if (msg) *msg = std::string("surrogate network: ") + cudaGetErrorString(r);
        return RT_ERR_CUDA;
    }
    if (e) {
        if (msg) *msg = "a tensor-core GEMM gave up waiting (code " + std::to_string(e) + ")";
        return RT_ERR_TIMEOUT;
    }
    return RT_OK;
}

// Blob: magic, version, parameter count, step count, then P, Adam m, Adam v.
constexpr uint32_t kNetMagic = 0x534E5452u;   // "RTNS"
constexpr uint32_t kNetVersion = 1;

rt_status mlp_serialize(rt_mlp *m, cudaStream_t s, std::vector<uint8_t> *out)
{
    const size_t head = 4 + 4 + 8 + 8, body = (size_t)N_PARAMS * 4;
    out->assign(head + 3 * body, 0);
    uint8_t *p = out->data();
    const uint64_t np = N_PARAMS;
    const int64_t st = m->steps;
    memcpy(p, &kNetMagic, 4);
    memcpy(p + 4, &kNetVersion, 4);
    memcpy(p + 8, &np, 8);
    memcpy(p + 16, &st, 8);
    if (cudaMemcpyAsync(p + head, m->P, body, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(p + head + body, m->Mm, body, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(p + head + 2 * body, m->Vv, body, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return RT_ERR_CUDA;
    return RT_OK;
}

rt_status mlp_deserialize(rt_mlp *m, cudaStream_t s, const uint8_t *p, size_t n)
{
    const size_t head = 4 + 4 + 8 + 8, body = (size_t)N_PARAMS * 4;
    if (n != head + 3 * body) return RT_ERR_INVALID;
    uint32_t magic = 0, ver = 0;
    uint64_t np = 0;
    int64_t st = 0;
    memcpy(&magic, p, 4);
    memcpy(&ver, p + 4, 4);
    memcpy(&np, p + 8, 8);
    memcpy(&st, p + 16, 8);
    if (magic != kNetMagic || ver != kNetVersion || np != N_PARAMS || st < 0) return RT_ERR_INVALID;
    if (cudaMemcpyAsync(m->P, p + head, body, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(m->Mm, p + head + body, body, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(m->Vv, p + head + 2 * body, body, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return RT_ERR_CUDA;
    refresh_bf16_kernel<<<512, 256, 0, s>>>(m->P, m->W1b, m->W2b, m->W2bT);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return RT_ERR_CUDA;
    m->steps = st;
    return RT_OK;
}

}  // namespace rt

extern "C" {

rt_status rt_mlp_create(rt_mlp **out, void *cuda_stream)
{
    if (!out) return RT_ERR_INVALID;
    *out = nullptr;
    rt_mlp *m = new rt_mlp();
    m->s = static_cast<cudaStream_t>(cuda_stream);
    auto A = [&](auto **p, size_t n) {
        cudaError_t e = cudaMalloc((void **)p, n);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, n);
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = A(&m->P, N_PARAMS * 4);
    if (e == cudaSuccess) e = A(&m->G, N_PARAMS * 4);
    if (e == cudaSuccess) e = A(&m->Mm, N_PARAMS * 4);
    if (e == cudaSuccess) e = A(&m->Vv, N_PARAMS * 4);
    if (e == cudaSuccess) e = A(&m->W1b, (size_t)D_H * D_IN * 2);
    if (e == cudaSuccess) e = A(&m->W2b, (size_t)D_H * D_H * 2);
    if (e == cudaSuccess) e = A(&m->W2bT, (size_t)D_H * D_H * 2);
    if (e == cudaSuccess) e = A(&m->X, (size_t)MAXB * D_IN * 2);
    if (e == cudaSuccess) e = A(&m->XT, (size_t)MAXB * D_IN * 2);
    if (e == cudaSuccess) e = A(&m->H1, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->H1T, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->H2, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->dZ2, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->dZ2T, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->dZ1T, (size_t)MAXB * D_H * 2);
    if (e == cudaSuccess) e = A(&m->T, (size_t)MAXB * D_OUT * 4);
    if (e == cudaSuccess) e = A(&m->Y, (size_t)MAXB * D_OUT * 4);
    if (e == cudaSuccess) e = A(&m->Eo, (size_t)MAXB * D_OUT * 4);
    if (e == cudaSuccess) e = A(&m->part, (size_t)kSplit1 * MAXB * D_H * 4);
    if (e == cudaSuccess) e = A(&m->loss, 4);
    if (e == cudaSuccess) e = A(&m->err, 4);
    if (e == cudaSuccess) e = gemm_attr<EpiReluBias>();
    if (e == cudaSuccess) e = gemm_attr<EpiMaskT>();
    if (e == cudaSuccess) e = gemm_attr<EpiStore>();
    if (e == cudaSuccess) e = gemm_attr<EpiPartial>();
    if (e != cudaSuccess) {
        rt_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
    }
    bool ok = make_map(&m->mX, m->X, MAXB, D_IN, tc::kBM) && make_map(&m->mW1, m->W1b, D_H, D_IN, kBN) &&
              make_map(&m->mH1, m->H1, MAXB, D_H, tc::kBM) && make_map(&m->mW2, m->W2b, D_H, D_H, kBN) &&
              make_map(&m->mdZ2T, m->dZ2T, D_H, MAXB, tc::kBM) && make_map(&m->mH1T, m->H1T, D_H, MAXB, kBN) &&
              make_map(&m->mdZ2, m->dZ2, MAXB, D_H, tc::kBM) && make_map(&m->mW2T, m->W2bT, D_H, D_H, kBN) &&
              make_map(&m->mdZ1T, m->dZ1T, D_H, MAXB, tc::kBM) && make_map(&m->mXT, m->XT, D_IN, MAXB, kBN);
    if (!ok) {
        rt_mlp_destroy(m);
        return RT_ERR_CUDA;
    }
    *out = m;
    return RT_OK;
}

rt_status rt_mlp_set_params(rt_mlp *m, const float *params, size_t n)
{
    if (!m || !params) return RT_ERR_INVALID;
    if (n != N_PARAMS) return mfail(m, RT_ERR_INVALID, "expected 1836291 parameters");
    MC(m, cudaMemcpyAsync(m->P, params, N_PARAMS * 4, cudaMemcpyDefault, m->s));
    MC(m, cudaMemsetAsync(m->Mm, 0, N_PARAMS * 4, m->s));
    MC(m, cudaMemsetAsync(m->Vv, 0, N_PARAMS * 4, m->s));
    refresh_bf16_kernel<<<512, 256, 0, m->s>>>(m->P, m->W1b, m->W2b, m->W2bT);
    MC(m, cudaGetLastError());
    m->steps = 0;
    MC(m, cudaStreamSynchronize(m->s));
    return RT_OK;
}

rt_status rt_mlp_get_params(rt_mlp *m, float *params, size_t n)
{
    if (!m || !params) return RT_ERR_INVALID;
    if (n != N_PARAMS) return mfail(m, RT_ERR_INVALID, "expected 1836291 parameters");
    MC(m, cudaMemcpyAsync(params, m->P, N_PARAMS * 4, cudaMemcpyDefault, m->s));
    MC(m, cudaStreamSynchronize(m->s));
    return RT_OK;
}

rt_status rt_mlp_forward(rt_mlp *m, const void *x_bf16, int32_t n, float *y)
{
    if (!m || !x_bf16 || !y) return RT_ERR_INVALID;
    if (n < 1 || n > MAXB) return mfail(m, RT_ERR_INVALID, "n must be in 1..256");
    rt_status s = load_batch(m, x_bf16, nullptr, n);
    if (s != RT_OK) return s;
    MC(m, rt::mlp_forward_async(m, n, m->s));
    MC(m, cudaMemcpyAsync(y, m->Y, (size_t)n * D_OUT * 4, cudaMemcpyDefault, m->s));
    return check_err(m);
}

rt_status rt_mlp_gradients(rt_mlp *m, const void *x_bf16, const float *t, int32_t n, float *grads, float *loss)
{
    if (!m || !x_bf16 || !t) return RT_ERR_INVALID;
    if (n < 1 || n > MAXB) return mfail(m, RT_ERR_INVALID, "n must be in 1..256");
    rt_status s = load_batch(m, x_bf16, t, n);
    if (s != RT_OK) return s;
    MC(m, fwd_bwd(m, MAXB, n, true, m->loss, m->s));
    if (grads) MC(m, cudaMemcpyAsync(grads, m->G, N_PARAMS * 4, cudaMemcpyDefault, m->s));
    if (loss) MC(m, cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDefault, m->s));
    return check_err(m);
}

rt_status rt_mlp_train_step(rt_mlp *m, const void *x_bf16, const float *t, int32_t n, double lr, float *loss)
{
    if (!m || !x_bf16 || !t) return RT_ERR_INVALID;
    if (n < 1 || n > MAXB) return mfail(m, RT_ERR_INVALID, "n must be in 1..256");
    rt_status s = load_batch(m, x_bf16, t, n);
    if (s != RT_OK) return s;
    MC(m, fwd_bwd(m, MAXB, n, true, m->loss, m->s));
    MC(m, adam(m, lr, m->s));
    if (loss) MC(m, cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDefault, m->s));
    return check_err(m);
}

const char *rt_mlp_last_error(rt_mlp *m) { return m ? m->msg.c_str() : ""; }

rt_status rt_mlp_check_activations(rt_mlp *m, int32_t n, uint16_t *h1, uint16_t *h2, uint16_t *dz2,
                                   uint16_t *dz1t, float *y)
{
    if (!m) return RT_ERR_INVALID;
    if (n < 1 || n > MAXB) return mfail(m, RT_ERR_INVALID, "n must be in 1..256");
    const size_t row = (size_t)D_H * 2;
    if (h1) MC(m, cudaMemcpyAsync(h1, m->H1, (size_t)n * row, cudaMemcpyDeviceToHost, m->s));
    if (h2) MC(m, cudaMemcpyAsync(h2, m->H2, (size_t)n * row, cudaMemcpyDeviceToHost, m->s));
    if (dz2) MC(m, cudaMemcpyAsync(dz2, m->dZ2, (size_t)n * row, cudaMemcpyDeviceToHost, m->s));
    if (dz1t) MC(m, cudaMemcpyAsync(dz1t, m->dZ1T, (size_t)D_H * MAXB * 2, cudaMemcpyDeviceToHost, m->s));
    if (y) MC(m, cudaMemcpyAsync(y, m->Y, (size_t)n * D_OUT * 4, cudaMemcpyDeviceToHost, m->s));
    MC(m, cudaStreamSynchronize(m->s));
    return RT_OK;
}

}  // extern "C"

namespace rt {
cudaError_t launch_surrogate_gains(const float *y, const int32_t *group_start, const int32_t *group_members,
                                   int n_groups, const double *maps_fit, double gmin, double gmax, double *maps_out,
                                   double *err_out, cudaStream_t s)
{
    if (n_groups * 3 > 96) return cudaErrorInvalidValue;
    surrogate_gains_kernel<<<1, 96, 0, s>>>(y, group_start, group_members, n_groups, maps_fit, gmin, gmax, maps_out,
                                            err_out);
    return cudaGetLastError();
}
}  // namespace rt

extern "C" {

void rt_mlp_destroy(rt_mlp *m)
{
    if (!m) return;
    if (m->s) cudaStreamSynchronize(m->s);
    void *ps[] = {m->P, m->G, m->Mm, m->Vv, m->W1b, m->W2b, m->W2bT, m->X, m->XT, m->H1, m->H1T, m->H2,
                  m->dZ2, m->dZ2T, m->dZ1T, m->T, m->Y, m->Eo, m->part, m->loss, m->err};
    for (void *p : ps)
        if (p) cudaFree(p);
    delete m;
}

}  // extern "C"
