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
// seam_rows_kernel: one warp per (seam, averaged row); lane = (pixel row r,
// side s, 8-column half q) loads its 8 pixels (24 bytes, three aligned
// 8-byte loads) and the warp adds the 8 rows with shuffles -- exact integer
// block sums; lane 0 forms d+_i, d-_i in FP64 and stores their mean.
// seam_sum_kernel: one warp per seam adds its rows in a fixed order, so the
// cost does not depend on scheduling.
#include "rt_internal.cuh"

namespace rt {

namespace {

constexpr int kRowWarps = 4;

__global__ void __launch_bounds__(32 * kRowWarps) seam_rows_kernel(const ArrayGeom g, const int2 *__restrict__ seams,
                                                                  int max_rows, double *__restrict__ rows)
{
    const int seam = blockIdx.y;
    const int i = blockIdx.x * kRowWarps + (threadIdx.x >> 5);   // averaged row
    const int lane = threadIdx.x & 31;
    const int2 sm = seams[seam];
    const CamGeom &L = g.cam[sm.x], &R = g.cam[sm.y];
    const int n = min(L.H / 8, R.H / 8);
    if (i >= n) return;                                          // whole warps leave together
    const int r = lane >> 2, side = (lane >> 1) & 1, q = lane & 1;
    const CamGeom &cg = side ? R : L;
    const int x0 = (side ? 0 : (L.W / 8 - 2) * 8) + 8 * q;      // first of the lane's 8 pixels
    const uint8_t *p = cg.rgb + (size_t)(8 * i + r) * cg.rgb_pitch + 3 * x0;   // 8-byte aligned
    const uint2 a = *reinterpret_cast<const uint2 *>(p), b = *reinterpret_cast<const uint2 *>(p + 8),
                c = *reinterpret_cast<const uint2 *>(p + 16);
    const uint32_t w[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
    uint32_t s[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 24; ++j) s[j % 3] += (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
    // add the 8 pixel rows: lanes with equal (side, half) differ in bits 2..4
#pragma unroll
    for (int o = 4; o < 32; o <<= 1)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) s[ch] += __shfl_xor_sync(0xffffffffu, s[ch], o);
    // lanes 0..3 now hold (left, half 0) = L-1, (left, 1) = L0, (right, 0) = R0, (right, 1) = R1
    double m[4][3];
#pragma unroll
    for (int src = 0; src < 4; ++src)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) m[src][ch] = __shfl_sync(0xffffffffu, s[ch], src) / 64.0;
    if (lane == 0) {
        double dp2 = 0.0, dm2 = 0.0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const double lm1 = m[0][ch], l0 = m[1][ch], r0 = m[2][ch], r1 = m[3][ch];
            const double u = (r1 - r0) - (r0 - l0), v = (lm1 - l0) - (l0 - r0);
            dp2 += u * u;
            dm2 += v * v;
        }
        rows[(size_t)seam * max_rows + i] = 0.5 * (sqrt(dp2) + sqrt(dm2));
    }
}

__global__ void __launch_bounds__(32) seam_sum_kernel(const ArrayGeom g, const int2 *__restrict__ seams, int max_rows,
                                                     const double *__restrict__ rows, double *__restrict__ cost)
{
    const int seam = blockIdx.x, lane = threadIdx.x;
    const int2 sm = seams[seam];
    const int n = min(g.cam[sm.x].H / 8, g.cam[sm.y].H / 8);
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc += rows[(size_t)seam * max_rows + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) cost[seam] = n > 0 ? acc / n : 0.0;
}

}  // namespace

cudaError_t launch_seam_cost(const ArrayGeom &g, const int2 *seams, int n_seams, int max_rows, double *rows,
                             double *cost, cudaStream_t s)
{
    if (n_seams <= 0) return cudaSuccess;
    if (max_rows > 0) {
        dim3 grid((max_rows + kRowWarps - 1) / kRowWarps, n_seams);
        seam_rows_kernel<<<grid, 32 * kRowWarps, 0, s>>>(g, seams, max_rows, rows);
    }
    seam_sum_kernel<<<n_seams, 32, 0, s>>>(g, seams, max_rows, rows, cost);
    return cudaGetLastError();
}

}  // namespace rt
