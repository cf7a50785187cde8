// The small per-frame FP64 solve (S3), exponential smoothing and Q16
// quantisation (S4) -- Sec. "White balance and exposure correction" and the
// Eq. of the exponential smoothing (alpha = 0.05).
//
// Per-camera gains: for each seam chain, channel and block one system
//   (L_w + lambda I + 1 1^T / K_g) x = B^T W r,
// x_k = log g_k, r = log mu^L(right camera) - log mu^R(left camera) over the
// valid seams, w = valid fraction of the band; solved in FP64 by one warp
// per system (tridiagonal factorisation plus a rank-two Woodbury correction,
// see solve_global_kernel); g = clamp(exp(x)).
// Seam affine maps: one thread per (camera, side, block, channel) matches
// its band's mean and variance to the equal-weight mixture of the two bands
// of its seam: a = sd_s / sd_side, b = mu_s - a mu_side.
// Both: E = first ? E_new : (1 - alpha) E + alpha E_new; q = llround(65536 E).
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

namespace {

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


// One system per CTA (one warp): the GPU's FP64 units are few, so systems
// are spread over SMs.  The chain's matrix is
//   M = T + u u^T + v v^T,   T = L_w(chain seams) + lambda I (tridiagonal),
//   u = 1/sqrt(K_g) (the gauge term), v = sqrt(w_c)(e_last - e_first) (the
// ring-closing seam, absent for a linear chain),
// so x = M^-1 rhs by the Woodbury identity from three tridiagonal solves
// with one factorisation (Thomas; T is symmetric, diagonally dominant).
__global__ void __launch_bounds__(32) solve_global_kernel(const SolveArgs a)
{
    __shared__ double sw[kMaxChain], sr[kMaxChain], cp[kMaxChain];
    __shared__ double zb[kMaxChain], zu[kMaxChain], zv[kMaxChain], x[kMaxChain];
    __shared__ int sb[kMaxChain];
    const int lane = threadIdx.x;
    const int sys = blockIdx.x;
    const int c = sys % 3, j = (sys / 3) % a.B, grp = sys / (3 * a.B);
    const int g0 = a.group_start[grp];
    const int n = a.group_start[grp + 1] - g0;
    // the seam whose left camera is member `lane`: weight and log-mean difference
    sw[lane] = 0.0;
    sr[lane] = 0.0;
    sb[lane] = -1;
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
                sw[lane] = fmin(nR, nL) / ((double)a.S * rows);
                sr[lane] = log(muL) - log(muR);
                sb[lane] = bpos;
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        // seams of a chain join members e and e+1; a ring's last seam joins n-1 and 0
        const bool ring = n >= 2 && sb[n - 1] == 0;
        const double wc = ring ? sw[n - 1] : 0.0;
        double rhs[kMaxChain];
        for (int e = 0; e < n; ++e) rhs[e] = 0.0;
        for (int e = 0; e < n; ++e) {
            const int b = sb[e];
            if (b < 0) continue;
            rhs[e] += sw[e] * sr[e];
            rhs[b] -= sw[e] * sr[e];
        }
        // Thomas factorisation of T: diag d_k = lambda + w_{k-1} + w_k, off -w_k
        const double su = 1.0 / sqrt((double)n);
        const double sv = sqrt(wc);
        double pb = 0.0, pu = 0.0, pv = 0.0;
        for (int k = 0; k < n; ++k) {
            const double wl = (k > 0 && sb[k - 1] == k) ? sw[k - 1] : 0.0;
            const double wr = (k + 1 < n && sb[k] == k + 1) ? sw[k] : 0.0;
            const double d = a.lambda + wl + wr;
            const double den = k == 0 ? d : d - wl * cp[k - 1];      // T_{k,k-1} = -wl
            const double id = 1.0 / den;
            cp[k] = -wr * id;                                        // T_{k,k+1} = -wr
            const double vk = ring ? (k == n - 1 ? sv : (k == 0 ? -sv : 0.0)) : 0.0;
            pb = (rhs[k] + wl * pb) * id;
            pu = (su + wl * pu) * id;
            pv = (vk + wl * pv) * id;
            zb[k] = pb;
            zu[k] = pu;
            zv[k] = pv;
        }
        for (int k = n - 2; k >= 0; --k) {
            zb[k] -= cp[k] * zb[k + 1];
            zu[k] -= cp[k] * zu[k + 1];
            zv[k] -= cp[k] * zv[k + 1];
        }
        // Woodbury: x = z_b - [z_u z_v] (I + U^T Z)^-1 U^T z_b
        double uzb = 0.0, uzu = 0.0, uzv = 0.0, vzb = 0.0, vzu = 0.0, vzv = 0.0;
        for (int k = 0; k < n; ++k) {
            const double vk = ring ? (k == n - 1 ? sv : (k == 0 ? -sv : 0.0)) : 0.0;
            uzb += su * zb[k]; uzu += su * zu[k]; uzv += su * zv[k];
            vzb += vk * zb[k]; vzu += vk * zu[k]; vzv += vk * zv[k];
        }
        double c00 = 1.0 + uzu, c01 = uzv, c10 = vzu, c11 = 1.0 + vzv;
        double alpha_u, alpha_v;
        if (ring) {
            const double det = c00 * c11 - c01 * c10;
            alpha_u = (c11 * uzb - c01 * vzb) / det;
            alpha_v = (c00 * vzb - c10 * uzb) / det;
        } else {
            alpha_u = uzb / c00;
            alpha_v = 0.0;
        }
        for (int k = 0; k < n; ++k) x[k] = zb[k] - zu[k] * alpha_u - zv[k] * alpha_v;
    }
    __syncwarp();
    if (lane < n) {
        const int cam = a.group_members[g0 + lane];
        const double g = fmin(fmax(exp(x[lane]), a.gmin), a.gmax);
        for (int side = 0; side < 2; ++side)
            smooth_store(a, (((size_t)(cam * 2 + side) * a.B + j) * 3 + c) * 2, g, 0.0);
    }
}

__global__ void __launch_bounds__(64) solve_affine_kernel(const SolveArgs a)
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
}

}  // namespace

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s)
{
    if (a.fit_mode == RT_FIT_GLOBAL) {
        const int n_sys = a.n_groups * a.B * 3;
        solve_global_kernel<<<n_sys, 32, 0, s>>>(a);
    } else {
        const int n_ent = a.K * 2 * a.B * 3;
        solve_affine_kernel<<<(n_ent + 63) / 64, 64, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace rt
