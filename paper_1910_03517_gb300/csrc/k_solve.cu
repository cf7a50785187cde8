// The small per-frame FP64 solve (S3), exponential smoothing and Q16
// quantisation (S4) -- Sec. "White balance and exposure correction" and the
// Eq. of the exponential smoothing (alpha = 0.05).
//
// Per-camera gains: for each seam chain, channel and block one system
//   (L_w + lambda I + 1 1^T / K_g) x = B^T W r,
// x_k = log g_k, r = log mu^L(right camera) - log mu^R(left camera) over the
// valid seams, w = valid fraction of the band; solved by one warp with a
// right-looking Cholesky factorisation in FP64; g = clamp(exp(x)).
// Seam affine maps: one thread per (camera, side, block, channel) matches
// its band's mean and variance to the equal-weight mixture of the two bands
// of its seam: a = sd_s / sd_side, b = mu_s - a mu_side.
// Both: E = first ? E_new : (1 - alpha) E + alpha E_new; q = llround(65536 E).
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kMaxChain = 32;

__device__ __forceinline__ void smooth_store(const SolveArgs &a, size_t idx, double va, double vb)
{
    a.maps_new[idx] = va;
    a.maps_new[idx + 1] = vb;
    double ea = va, eb = vb;
    if (!a.first) {
        ea = (1.0 - a.alpha) * a.E[idx] + a.alpha * va;
        eb = (1.0 - a.alpha) * a.E[idx + 1] + a.alpha * vb;
    }
    a.E[idx] = ea;
    a.E[idx + 1] = eb;
    a.q16[idx] = (int32_t)llround(65536.0 * ea);
    a.q16[idx + 1] = (int32_t)llround(65536.0 * eb);
}

__device__ __forceinline__ int block_rows(int j, int H, int B) { return (int)(((long long)(j + 1) * H) / B - ((long long)j * H) / B); }

__device__ void clear_next(const SolveArgs &a)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nt = (size_t)gridDim.x * blockDim.x;
    for (size_t i = tid; i < a.clear_u32_n; i += nt) a.clear_u32[i] = 0u;
    for (size_t i = tid; i < a.clear_u64_n; i += nt) a.clear_u64[i] = 0ull;
    for (size_t i = tid; i < a.clear2_u32_n; i += nt) a.clear2_u32[i] = 0u;
}

__global__ void __launch_bounds__(32 * kWarpsPerCta) solve_global_kernel(const SolveArgs a)
{
    __shared__ double M[kWarpsPerCta][kMaxChain][kMaxChain + 1];
    __shared__ double rhs[kWarpsPerCta][kMaxChain];
    __shared__ double sw[kWarpsPerCta][kMaxChain], sr[kWarpsPerCta][kMaxChain];
    __shared__ int sb[kWarpsPerCta][kMaxChain];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_sys = a.n_groups * a.B * 3;
    for (int sys = blockIdx.x * kWarpsPerCta + warp; sys < n_sys; sys += gridDim.x * kWarpsPerCta) {
        const int c = sys % 3, j = (sys / 3) % a.B, grp = sys / (3 * a.B);
        const int g0 = a.group_start[grp];
        const int n = a.group_start[grp + 1] - g0;
        double (*m)[kMaxChain + 1] = M[warp];
        // M = lambda I + 1 1^T / n, rhs = 0
        if (lane < n) {
            for (int q = 0; q < n; ++q) m[lane][q] = 1.0 / n + (q == lane ? a.lambda : 0.0);
            rhs[warp][lane] = 0.0;
        }
        // the seam whose left camera is member `lane`
        sw[warp][lane] = 0.0;
        sb[warp][lane] = -1;
        if (lane < n) {
            const int kl = a.group_members[g0 + lane];
            const int kr = a.right_nbr[kl];
            if (kr >= 0 && kr != kl) {
                int bpos = -1;
                for (int q = 0; q < n; ++q)
                    if (a.group_members[g0 + q] == kr) bpos = q;
                const size_t iR = ((size_t)(kl * 2 + 1) * a.B + j) * 3 + c;
                const size_t iL = ((size_t)(kr * 2 + 0) * a.B + j) * 3 + c;
                const double nR = (double)a.n[iR], nL = (double)a.n[iL];
                if (bpos >= 0 && nR >= a.min_valid && nL >= a.min_valid) {
                    const double muR = fmax((double)a.sum[iR] / nR, 1.0);
                    const double muL = fmax((double)a.sum[iL] / nL, 1.0);
                    const int rows = min(block_rows(j, a.cam_H[kl], a.B), block_rows(j, a.cam_H[kr], a.B));
                    sw[warp][lane] = fmin(nR, nL) / ((double)a.S * rows);
                    sr[warp][lane] = log(muL) - log(muR);
                    sb[warp][lane] = bpos;
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            for (int e = 0; e < n; ++e) {
                const int b = sb[warp][e];
                if (b < 0) continue;
                const double w = sw[warp][e], r = sr[warp][e];
                m[e][e] += w;
                m[b][b] += w;
                m[e][b] -= w;
                m[b][e] -= w;
                rhs[warp][e] += w * r;
                rhs[warp][b] -= w * r;
            }
        }
        __syncwarp();
        // Cholesky M = L L^T, lower triangle in place
        for (int kk = 0; kk < n; ++kk) {
            if (lane == 0) m[kk][kk] = sqrt(m[kk][kk]);
            __syncwarp();
            const double d = m[kk][kk];
            if (lane > kk && lane < n) m[lane][kk] /= d;
            __syncwarp();
            if (lane > kk && lane < n)
                for (int q = kk + 1; q <= lane; ++q) m[lane][q] -= m[lane][kk] * m[q][kk];
            __syncwarp();
        }
        // L y = rhs
        for (int kk = 0; kk < n; ++kk) {
            if (lane == 0) rhs[warp][kk] /= m[kk][kk];
            __syncwarp();
            if (lane > kk && lane < n) rhs[warp][lane] -= m[lane][kk] * rhs[warp][kk];
            __syncwarp();
        }
        // L^T x = y
        for (int kk = n - 1; kk >= 0; --kk) {
            if (lane == 0) rhs[warp][kk] /= m[kk][kk];
            __syncwarp();
            if (lane < kk) rhs[warp][lane] -= m[kk][lane] * rhs[warp][kk];
            __syncwarp();
        }
        if (lane < n) {
            const int cam = a.group_members[g0 + lane];
            const double g = fmin(fmax(exp(rhs[warp][lane]), a.gmin), a.gmax);
            for (int side = 0; side < 2; ++side)
                smooth_store(a, (((size_t)(cam * 2 + side) * a.B + j) * 3 + c) * 2, g, 0.0);
        }
        __syncwarp();
    }
    clear_next(a);
}

__global__ void __launch_bounds__(128) solve_affine_kernel(const SolveArgs a)
{
    const int n_ent = a.K * 2 * a.B * 3;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_ent; e += gridDim.x * blockDim.x) {
        const int c = e % 3, j = (e / 3) % a.B, side = (e / (3 * a.B)) % 2, cam = e / (6 * a.B);
        // the seam on this side: (left camera's right band, right camera's left band)
        const int nb = side == 1 ? a.right_nbr[cam] : a.left_nbr[cam];
        double va = 1.0, vb = 0.0;
        if (nb >= 0 && nb != cam) {
            const int kl = side == 1 ? cam : nb, kr = side == 1 ? nb : cam;
            const size_t iR = ((size_t)(kl * 2 + 1) * a.B + j) * 3 + c;
            const size_t iL = ((size_t)(kr * 2 + 0) * a.B + j) * 3 + c;
            const double nR = (double)a.n[iR], nL = (double)a.n[iL];
            if (nR >= a.min_valid && nL >= a.min_valid) {
                const double muR = (double)a.sum[iR] / nR, muL = (double)a.sum[iL] / nL;
                const double vR = fmax((double)a.sumsq[iR] / nR - muR * muR, 0.0);
                const double vL = fmax((double)a.sumsq[iL] / nL - muL * muL, 0.0);
                const double mus = 0.5 * (muL + muR);
                const double dm = 0.5 * (muL - muR);
                const double vs = 0.5 * (vL + vR) + dm * dm;
                const double mu = side == 1 ? muR : muL;
                const double sd = sqrt(side == 1 ? vR : vL);
                double s = sd >= 0.5 ? sqrt(vs) / sd : 1.0;
                s = fmin(fmax(s, a.gmin), a.gmax);
                va = s;
                vb = mus - s * mu;
            }
        }
        smooth_store(a, (size_t)e * 2, va, vb);
    }
    clear_next(a);
}

}  // namespace

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s)
{
    size_t clear = a.clear_u32_n + a.clear_u64_n + a.clear2_u32_n;
    int grid_clear = (int)((clear + 128 * 16 - 1) / (128 * 16));
    if (a.fit_mode == RT_FIT_GLOBAL) {
        int n_sys = a.n_groups * a.B * 3;
        int grid = (n_sys + kWarpsPerCta - 1) / kWarpsPerCta;
        grid = grid < grid_clear ? grid_clear : grid;
        grid = grid > 1024 ? 1024 : (grid < 1 ? 1 : grid);
        solve_global_kernel<<<grid, 32 * kWarpsPerCta, 0, s>>>(a);
    } else {
        int n_ent = a.K * 2 * a.B * 3;
        int grid = (n_ent + 127) / 128;
        grid = grid < grid_clear ? grid_clear : grid;
        grid = grid > 1024 ? 1024 : (grid < 1 ? 1 : grid);
        solve_affine_kernel<<<grid, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace rt
