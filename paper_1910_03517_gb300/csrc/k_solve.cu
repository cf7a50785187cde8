// The small per-frame FP64 solve (S3), exponential smoothing and Q16
// quantisation (S4) -- Sec. "White balance and exposure correction" and the
// Eq. of the exponential smoothing (alpha = 0.05).
//
// Per-camera gains: for each seam chain, channel and block one system
//   (L_w + lambda I + 1 1^T / K_g) x = B^T W r,
// x_k = log g_k, r = log mu^L(right camera) - log mu^R(left camera) over the
// valid seams, w = valid fraction of the band; solved in FP64 by one warp
// per system (continuant elimination of the chain's tridiagonal matrix and a
// rank-one Woodbury correction for a ring, see solve_global_kernel);
// g = clamp(exp(x)).
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


// One system per CTA (one warp): the GPU's FP64 units are few and slow, so
// systems are spread over SMs and the sequential part is kept short.
//
// The right-hand side sums to zero (every seam adds w r to one camera and
// subtracts it from the other), so 1^T x = 0 and the gauge term 1 1^T / K_g
// leaves the solution unchanged: x solves (L_w + lambda I) x = rhs.  For a
// chain that matrix T is tridiagonal (diagonal d_k = lambda + w_{k-1} + w_k,
// off-diagonals -w); a ring adds its closing seam as a rank-one term
// v v^T, v = sqrt(w_c)(e_last - e_first), handled by the Woodbury identity.
// T is eliminated through its continuants
//   P_{-1} = 1, P_k = d_k P_{k-1} - w_{k-1}^2 P_{k-2},
//   s_k = rhs_k P_{k-1} + w_{k-1} s_{k-1}          (forward, one FMA per step)
//   x_k = s_k / P_k + (w_k P_{k-1} / P_k) x_{k+1}   (backward, one FMA per step)
// so the divisions run on all lanes at once and only FMAs stay sequential.
__global__ void __launch_bounds__(32) solve_global_kernel(const SolveArgs a)
{
    __shared__ double sw[kMaxChain], srw[kMaxChain], wp[kMaxChain], rh[kMaxChain], vv[kMaxChain];
    __shared__ double P[kMaxChain], Pp[kMaxChain], sB[kMaxChain], sV[kMaxChain];
    __shared__ double aB[kMaxChain], aV[kMaxChain], bt[kMaxChain], xb[kMaxChain], xv[kMaxChain];
    __shared__ int sb[kMaxChain];
    const int lane = threadIdx.x;
    const int sys = blockIdx.x;
    const int c = sys % 3, j = (sys / 3) % a.B, grp = sys / (3 * a.B);
    const int g0 = a.group_start[grp];
    const int n = a.group_start[grp + 1] - g0;
    // 1. the seam whose left camera is member `lane`: weight w and w * r,
    //    r = log mu^L - log mu^R (one logarithm of the ratio)
    double w = 0.0, wr = 0.0;
    int bpos = -1;
    if (lane < n) {
        const int kl = a.group_members[g0 + lane];
        const int kr = a.right_nbr[kl];
        if (kr >= 0 && kr != kl) {
            for (int q = 0; q < n; ++q)
                if (a.group_members[g0 + q] == kr) bpos = q;
            const size_t iR = ((size_t)(kl * 2 + 1) * a.B + j) * 3 + c;
            const size_t iL = ((size_t)(kr * 2 + 0) * a.B + j) * 3 + c;
            const uint32_t nR = a.n[iR], nL = a.n[iL];
            if (bpos >= 0 && nR >= (uint32_t)a.min_valid && nL >= (uint32_t)a.min_valid) {
                const unsigned long long sR = a.sum[iR], sL = a.sum[iL];
                double ratio;
                if (sR >= nR && sL >= nL)      // both means >= 1: exact integer products
                    ratio = (double)(sL * nR) / (double)(sR * nL);
                else
                    ratio = fmax((double)sL / (double)nL, 1.0) / fmax((double)sR / (double)nR, 1.0);
                const int rows = min(block_rows(j, a.cam_H[kl], a.B), block_rows(j, a.cam_H[kr], a.B));
                w = (double)min(nR, nL) / (double)(a.S * rows);
                wr = w * log(ratio);
            } else {
                bpos = -1;
            }
        }
    }
    sw[lane] = w;
    srw[lane] = wr;
    sb[lane] = bpos;
    __syncwarp();
    // right-hand side, the chain's path weights w_k (seam k, k+1) and the
    // ring's rank-one vector
    const bool ring = n >= 2 && sb[n - 1] == 0;
    const double sv = ring ? sqrt(sw[n - 1]) : 0.0;
    if (lane < n) {
        double r = sb[lane] >= 0 ? srw[lane] : 0.0;
        for (int e = 0; e < n; ++e)
            if (sb[e] == lane) r -= srw[e];
        rh[lane] = r;
        wp[lane] = (lane + 1 < n && sb[lane] == lane + 1) ? sw[lane] : 0.0;
        vv[lane] = ring ? (lane == n - 1 ? sv : (lane == 0 ? -sv : 0.0)) : 0.0;
    }
    __syncwarp();
    // 2. forward continuant recurrences (lane 0; one FMA per step each)
    if (lane == 0) {
        double Pm2 = 0.0, Pm1 = 1.0, sbm = 0.0, svm = 0.0;
        for (int k = 0; k < n; ++k) {
            const double wl = k > 0 ? wp[k - 1] : 0.0;
            const double d = a.lambda + wl + wp[k];
            const double pk = fma(d, Pm1, -(wl * wl) * Pm2);
            sbm = fma(wl, sbm, rh[k] * Pm1);
            svm = fma(wl, svm, vv[k] * Pm1);
            P[k] = pk;
            Pp[k] = Pm1;
            sB[k] = sbm;
            sV[k] = svm;
            Pm2 = Pm1;
            Pm1 = pk;
        }
    }
    __syncwarp();
    // 3. the divisions, all lanes at once
    if (lane < n) {
        const double ip = 1.0 / P[lane];
        aB[lane] = sB[lane] * ip;
        aV[lane] = sV[lane] * ip;
        bt[lane] = wp[lane] * Pp[lane] * ip;
    }
    __syncwarp();
    // 4. backward recurrences (lane 0)
    if (lane == 0) {
        double x1 = 0.0, x2 = 0.0;
        for (int k = n - 1; k >= 0; --k) {
            x1 = fma(bt[k], x1, aB[k]);
            x2 = fma(bt[k], x2, aV[k]);
            xb[k] = x1;
            xv[k] = x2;
        }
    }
    __syncwarp();
    // 5. ring: x = x_b - x_v (v^T x_b) / (1 + v^T x_v); gains, smoothing, Q16
    if (lane < n) {
        double x = xb[lane];
        if (ring) {
            const double vxb = sv * (xb[n - 1] - xb[0]), vxv = sv * (xv[n - 1] - xv[0]);
            x -= xv[lane] * vxb / (1.0 + vxv);
        }
        const int cam = a.group_members[g0 + lane];
        const double g = fmin(fmax(exp(x), a.gmin), a.gmax);
        const size_t i0 = (((size_t)(cam * 2 + 0) * a.B + j) * 3 + c) * 2;
        const size_t i1 = (((size_t)(cam * 2 + 1) * a.B + j) * 3 + c) * 2;
        // both sides carry the same gain: smooth and quantise once, store twice
        smooth_store(a, i0, g, 0.0);
        a.maps_new[i1] = a.maps_new[i0];
        a.maps_new[i1 + 1] = 0.0;
        a.E[i1] = a.E[i0];
        a.E[i1 + 1] = a.E[i0 + 1];
        a.q16[i1] = a.q16[i0];
        a.q16[i1 + 1] = a.q16[i0 + 1];
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
