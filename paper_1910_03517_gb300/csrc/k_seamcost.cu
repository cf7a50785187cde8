// Seam quality telemetry: the gradient-continuity cost of Sec.
// "Quantitative", Eq. (gradientcost), on the corrected output of a frame
// set.  Per seam (left camera's right edge, right camera's left edge) both
// images are box-averaged over 8 x 8 pixels; only the last two averaged
// columns of the left image and the first two of the right are needed.  On
// averaged row i:
//   d+_i = |(R1 - R0) - (R0 - L0)|,  d-_i = |(L-1 - L0) - (L0 - R0)|,
// |.| the Euclidean norm over R, G, B, and the cost is the mean over the
// rows both images have of (d+_i + d-_i) / 2.
//
// One CTA per seam, one thread per averaged row; block sums are exact
// integers, the means and norms FP64 (a few operations per averaged row).
#include "rt_internal.cuh"

namespace rt {

namespace {

constexpr int kCostThreads = 128;

__global__ void __launch_bounds__(kCostThreads) seam_cost_kernel(const ArrayGeom g, const int2 *__restrict__ seams,
                                                                 double *__restrict__ cost)
{
    __shared__ double part[kCostThreads / 32];
    const int2 sm = seams[blockIdx.x];
    const CamGeom &L = g.cam[sm.x], &R = g.cam[sm.y];
    const int n = min(L.H / 8, R.H / 8);
    const int xl = (L.W / 8 - 2) * 8;     // first pixel column of the left image's column L-1
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        uint32_t sl[2][3] = {{0, 0, 0}, {0, 0, 0}}, sr[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int r = 0; r < 8; ++r) {
            const uint8_t *pl = L.rgb + (size_t)(8 * i + r) * L.rgb_pitch + 3 * xl;
            const uint8_t *pr = R.rgb + (size_t)(8 * i + r) * R.rgb_pitch;
#pragma unroll
            for (int col = 0; col < 16; ++col)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sl[col >> 3][c] += pl[3 * col + c];
                    sr[col >> 3][c] += pr[3 * col + c];
                }
        }
        double dp2 = 0.0, dm2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double lm1 = sl[0][c] / 64.0, l0 = sl[1][c] / 64.0, r0 = sr[0][c] / 64.0, r1 = sr[1][c] / 64.0;
            const double a = (r1 - r0) - (r0 - l0), b = (lm1 - l0) - (l0 - r0);
            dp2 += a * a;
            dm2 += b * b;
        }
        acc += 0.5 * (sqrt(dp2) + sqrt(dm2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        cost[blockIdx.x] = n > 0 ? s / n : 0.0;
    }
}

}  // namespace

cudaError_t launch_seam_cost(const ArrayGeom &g, const int2 *seams, int n_seams, double *cost, cudaStream_t s)
{
    if (n_seams <= 0) return cudaSuccess;
    seam_cost_kernel<<<n_seams, kCostThreads, 0, s>>>(g, seams, cost);
    return cudaGetLastError();
}

}  // namespace rt
