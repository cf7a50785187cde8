// The small per-frame FP64 solve (S3), exponential smoothing and Q16
// quantisation (S4) -- Sec. "White balance and exposure correction" and the
// Eq. of the exponential smoothing (alpha = 0.05).
//
// Per-camera gains: for each seam chain, channel and block one system
//   (L_w + lambda I + 1 1^T / K_g) x = B^T W r,
// x_k = log g_k, r = log mu^L(right camera) - log mu^R(left camera) over the
// valid seams, w = valid fraction of the band; solved to FP64 accuracy by
// one warp per system (continuant elimination of the chain's tridiagonal
// matrix and a rank-one Sherman-Morrison correction for a ring, see
// solve_global_kernel); g = clamp(exp(x)).
// Seam affine maps: one thread per (camera, side, block, channel) matches
// its band's mean and variance to the equal-weight mixture of the two bands
// of its seam: a = sd_s / sd_side, b = mu_s - a mu_side.
// Both: E = first ? E_new : (1 - alpha) E + alpha E_new; q = 65536 E rounded
// half away from zero.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rt_internal.cuh"
#include "q16.cuh"
#include "../../include/rt_check.h"

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


// ---------------------------------------------------------------------------
// FP64 on GB300: one warp-wide FP64 instruction occupies a sub-partition's
// FP64 unit for ~64 cycles whatever the number of active lanes, and a library
// log / exp / division costs ~2100 / ~1300 / ~430 cycles.  The solve is a
// chain of such steps, so it is written to issue few FP64 instructions:
// logarithm and exponential are table-driven (FP64 only where the result's
// leading bits form, the small tails in FP32), the chain's unknowns stay on
// lanes, and the sequential recurrences cost one or two FP64 FMAs per camera.
// Results agree with plain FP64 arithmetic to ~1e-12 relative.
// ---------------------------------------------------------------------------

constexpr double kLn2 = 0.69314718055994530942;

// A = 2^e f with f in [1, 2); f = c_i (1 + u), |u| <= 1/256 (Tang's
// table-driven logarithm, ACM TOMS 16(4), 1990: ln A = e ln 2 + ln c_i +
// ln(1 + u)).  Requires A > 0; the leading 53 bits of A are used.
__device__ __forceinline__ void log_parts(unsigned long long A, const SolveTables &t, int &e, int &i, double &u)
{
    const int lz = __clzll((long long)A);
    const unsigned long long m = A << lz;             // leading one at bit 63
    e = 63 - lz;
    i = (int)((m >> 56) & 127);
    const double f = __longlong_as_double((long long)((1023ull << 52) | ((m << 1) >> 12)));
    u = fma(f, t.invc[i], -1.0);
}

// u - ln(1 + u) = u^2/2 - u^3/3 + u^4/4 - u^5/5 + ... for |u| <= 1/256: at
// most 7.7e-6, so FP32 leaves an absolute error near 1e-12; the first omitted
// term is below 3e-15.
__device__ __forceinline__ float log1p_tail(float u)
{
    return u * u * (0.5f - u * (0.333333343f - u * (0.25f - u * 0.2f)));
}

// ln(A / B) for positive integers A, B < 2^64.
__device__ __forceinline__ double log_ratio(unsigned long long A, unsigned long long B, const SolveTables &t)
{
    int eA, iA, eB, iB;
    double uA, uB;
    log_parts(A, t, eA, iA, uA);
    log_parts(B, t, eB, iB, uB);
    // no contraction into an FMA: equal arguments give exactly 0
    const float h = __fsub_rn(log1p_tail((float)uA), log1p_tail((float)uB));
    return fma((double)(eA - eB), kLn2, t.logc[iA] - t.logc[iB]) + ((uA - uB) - (double)h);
}

// e^x for x in [-700, 40] (Tang's table-driven exponential, ACM TOMS 15(2),
// 1989): x = (64 m + j) ln2/64 + r, |r| <= ln2/128 + tiny, e^x = 2^m 2^(j/64)
// (1 + r + q(r)), q = r^2/2 + r^3/6 + r^4/24 + r^5/120 below 1.5e-5 (FP32).
__device__ __forceinline__ double exp_table(double x, const SolveTables &t)
{
    const int k = __float2int_rn((float)x * 92.3324826168936579f);   // 64 / ln 2
    const double r = fma((double)(-k), kLn2 / 64.0, x);
    const float rf = (float)r;
    const float q = rf * rf * (0.5f + rf * (0.166666672f + rf * (0.0416666679f + rf * 0.00833333377f)));
    const double tj = t.exp2j[k & 63];
    const double y = fma(tj, r + (double)q, tj);
    return __hiloint2double(__double2hiint(y) + (k >> 6) * (1 << 20), __double2loint(y));
}

// One system (chain, block, channel) per CTA of one warp, one camera of the
// chain per lane; the systems of a frame set spread over SMs.
//
// The right-hand side sums to zero (every seam adds w r to one camera and
// subtracts it from the other), so 1^T x = 0 and the gauge term 1 1^T / K_g
// leaves the solution unchanged: x solves (L_w + lambda I) x = rhs.  For a
// chain that matrix T is tridiagonal (diagonal d_k = lambda + w_{k-1} + w_k,
// off-diagonals -w); a ring's closing seam adds w_c z z^T, z = e_last -
// e_first, handled by the Sherman-Morrison identity.  T is eliminated through
// its continuants
//   P_{-1} = 1, P_k = d_k P_{k-1} - w_{k-1}^2 P_{k-2}        (2 FP64 / step)
//   s_k = rhs_k P_{k-1} + w_{k-1} s_{k-1}                     (1 FP64 / step)
//   x_k = s_k / P_k + (w_k P_{k-1} / P_k) x_{k+1}             (1 FP64 / step)
// with the products and divisions done on all lanes at once.
__global__ void __launch_bounds__(32) solve_global_kernel(const SolveArgs a)
{
    __shared__ double s_in[kMaxChain], s_d[kMaxChain], s_q[kMaxChain], s_wp[kMaxChain], s_P[kMaxChain];
    __shared__ double s_t[kMaxChain], s_tz[kMaxChain], s_a[kMaxChain], s_az[kMaxChain], s_b[kMaxChain];
    __shared__ double s_x[kMaxChain], s_xz[kMaxChain];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    const int sys = blockIdx.x;
    if (a.gate && !a.gate[0]) return;                 // surrogate mode: no fit for this frame set
    const int c = sys % 3, j = (sys / 3) % a.B, grp = sys / (3 * a.B);
    const int g0 = a.topo.gstart[grp];
    const int n = a.topo.gstart[grp + 1] - g0;
    const bool act = lane < n;
    const int cam = act ? a.topo.member[g0 + lane] : 0;
    const int kr = act ? a.topo.right[cam] : -1;
    const int bpos = act ? a.topo.rpos[cam] : -1;     // position of kr in the chain
    const size_t i0 = (((size_t)(cam * 2 + 0) * a.B + j) * 3 + c) * 2;
    const size_t i1 = (((size_t)(cam * 2 + 1) * a.B + j) * 3 + c) * 2;
    // every load of the system in one round
    uint32_t nR = 0, nL = 0;
    unsigned long long sR = 0, sL = 0;
    if (bpos >= 0) {
        const size_t iR = ((size_t)(cam * 2 + 1) * a.B + j) * 3 + c;
        const size_t iL = ((size_t)(kr * 2 + 0) * a.B + j) * 3 + c;
        nR = a.n[iR]; nL = a.n[iL];
        sR = a.sum[iR]; sL = a.sum[iL];
    }
    double2 e_old = make_double2(0.0, 0.0);
    if (act && !a.first) e_old = *reinterpret_cast<const double2 *>(a.E + i0);
    // 1. the seam to the right of camera `lane`: weight w = valid fraction of
    //    the band, r = log max(mu^L, 1) - log max(mu^R, 1) as the log of an
    //    exact integer ratio
    const bool valid = bpos >= 0 && nR >= (uint32_t)a.min_valid && nL >= (uint32_t)a.min_valid;
    double w = 0.0, wr = 0.0;
    if (valid) {
        const bool lok = sL >= nL, rok = sR >= nR;    // means >= 1
        const unsigned long long A = (lok ? sL : 1ull) * (rok ? nR : 1ull);
        const unsigned long long Bq = (rok ? sR : 1ull) * (lok ? nL : 1ull);
        const double r = log_ratio(A, Bq, a.tab);
        const int rows = min(block_rows(j, a.topo.H[cam], a.B), block_rows(j, a.topo.H[kr], a.B));
        w = (double)min(nR, nL) / (double)(a.S * rows);
        wr = w * r;
    }
    // 2. right-hand side (own seam minus the incoming one), tridiagonal T
    s_in[lane] = 0.0;
    __syncwarp();
    if (valid) s_in[bpos] = wr;                       // each camera has one left neighbour
    __syncwarp();
    const double rh = wr - s_in[lane];
    const double wp = (valid && bpos == lane + 1) ? w : 0.0;   // path seam (lane, lane + 1)
    double wprev = __shfl_up_sync(full, wp, 1);
    if (lane == 0) wprev = 0.0;
    const bool ring = __ballot_sync(full, valid && bpos == 0 && lane == n - 1 && n >= 2) != 0;
    const double wc = __shfl_sync(full, w, n > 0 ? n - 1 : 0);
    if (act) {
        s_d[lane] = a.lambda + wprev + wp;
        s_q[lane] = wprev * wprev;
        s_wp[lane] = wp;
    }
    __syncwarp();
    // 3. continuants (lane 0)
    if (lane == 0) {
        double p2 = 0.0, p1 = 1.0;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            const double pk = fma(s_d[k], p1, -(s_q[k] * p2));
            s_P[k] = pk;
            p2 = p1;
            p1 = pk;
        }
    }
    __syncwarp();
    const double Pk = act ? s_P[lane] : 1.0;
    const double Pm = (act && lane > 0) ? s_P[lane - 1] : 1.0;
    const double ip = 1.0 / Pk;
    if (act) {
        s_t[lane] = rh * Pm;
        s_tz[lane] = lane == n - 1 ? Pm : (lane == 0 ? -Pm : 0.0);    // z = e_last - e_first
        s_b[lane] = wp * Pm * ip;
    }
    __syncwarp();
    // 4. forward sums (lane 0)
    if (lane == 0) {
        double sb = 0.0, sz = 0.0, wl = 0.0;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            sb = fma(wl, sb, s_t[k]);
            s_a[k] = sb;
            if (ring) {
                sz = fma(wl, sz, s_tz[k]);
                s_az[k] = sz;
            }
            wl = s_wp[k];
        }
    }
    __syncwarp();
    if (act) {
        s_a[lane] *= ip;
        if (ring) s_az[lane] *= ip;
    }
    __syncwarp();
    // 5. back substitution (lane 0)
    if (lane == 0) {
        double xb = 0.0, xz = 0.0;
#pragma unroll 4
        for (int k = n - 1; k >= 0; --k) {
            xb = fma(s_b[k], xb, s_a[k]);
            s_x[k] = xb;
            if (ring) {
                xz = fma(s_b[k], xz, s_az[k]);
                s_xz[k] = xz;
            }
        }
    }
    __syncwarp();
    if (!act) return;
    double x = s_x[lane];
    if (ring) {
        const double zx = s_x[n - 1] - s_x[0], zz = s_xz[n - 1] - s_xz[0];
        x -= s_xz[lane] * (wc * zx / fma(wc, zz, 1.0));
    }
    // 6. g = clamp(exp(x)); smoothing; Q16.  x is first kept inside a range
    //    whose exponentials lie beyond the clamp (same clamped result).
    const float xf = (float)x;
    if (!(xf >= a.xlo_f)) x = a.xlo;
    else if (xf > a.xhi_f) x = a.xhi;
    long long gb = __double_as_longlong(exp_table(x, a.tab));   // positive: bit order = value order
    gb = max(gb, __double_as_longlong(a.gmin));
    gb = min(gb, __double_as_longlong(a.gmax));
    const double g = __longlong_as_double(gb);
    const double2 m = make_double2(g, 0.0);
    // both sides carry the same gain
    *reinterpret_cast<double2 *>(a.maps_new + i0) = m;
    *reinterpret_cast<double2 *>(a.maps_new + i1) = m;
    if (a.fit_only) return;                           // smoothing and Q16 left to the caller
    double2 e;
    if (a.first) {
        e = make_double2(g, 0.0);
    } else {
        e.x = fma(a.one_m_alpha, e_old.x, a.alpha * g);
        e.y = a.one_m_alpha * e_old.y;
    }
    const int2 q = make_int2(q16_round(e.x), q16_round(e.y));
    *reinterpret_cast<double2 *>(a.E + i0) = e;
    *reinterpret_cast<double2 *>(a.E + i1) = e;
    *reinterpret_cast<int2 *>(a.q16 + i0) = q;
    *reinterpret_cast<int2 *>(a.q16 + i1) = q;
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

const SolveTables &solve_tables()
{
    static const SolveTables t = [] {
        SolveTables v;
        for (int i = 0; i < 128; ++i) {
            const double ci = 1.0 + (i + 0.5) / 128.0;   // exact
            v.invc[i] = 1.0 / ci;
            v.logc[i] = std::log(ci);
        }
        for (int i = 0; i < 64; ++i) v.exp2j[i] = std::exp2(i / 64.0);
        return v;
    }();
    return t;
}

// Quantile-LS affine maps: one warp per (camera, side, block, channel).
// Lane l holds bins 8l .. 8l+7 of both bands' histograms; a warp scan gives
// the cumulative counts c_R(v), c_L(v) in shared memory.  Lane i then finds,
// by binary search over v, its band's quantile x_i (the smallest v with
// 2 Q c_S(v) >= (2i + 1) n_S) and the mixture's y_i (the smallest v with
// Q (c_R(v) n_L + c_L(v) n_R) >= (2i + 1) n_R n_L), every comparison on exact
// integers; the line's integer sums come from a warp reduction, the slope is
// the ratio of two exact integer sums and b follows without FMA contraction
// -- the oracle's arithmetic, operation for operation.
constexpr int kQuantiles = 32;
// One map per CTA (2 KB of shared memory): beside the table variant of
// pass B, which leaves ~35 KB of shared memory per SM, CTAs of four maps
// (8 KB) found too few free slots and the solve took 64 us a frame set.
constexpr int kQuantWarps = 1;

__global__ void __launch_bounds__(32 * kQuantWarps) solve_quantile_kernel(const SolveArgs a)
{
    __shared__ uint32_t cum[kQuantWarps][2][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kQuantWarps + warp;
    if (e >= a.K * 2 * a.B * 3) return;   // whole warp
    const int c = e % 3, j = (e / 3) % a.B, side = (e / (3 * a.B)) % 2, cam = e / (6 * a.B);
    const int nb = side == 1 ? a.right_nbr[cam] : a.left_nbr[cam];
    double va = 1.0, vb = 0.0;
    if (nb >= 0 && nb != cam) {
        const int kl = side == 1 ? cam : nb, kr = side == 1 ? nb : cam;
        const size_t iR = ((size_t)(kl * 2 + 1) * a.B + j) * 3 + c;
        const size_t iL = ((size_t)(kr * 2 + 0) * a.B + j) * 3 + c;
        const long long nR = a.n[iR], nL = a.n[iL];
        if (nR >= a.min_valid && nL >= a.min_valid) {   // warp-uniform
            const uint4 *hR = reinterpret_cast<const uint4 *>(a.hist + iR * 256) + 2 * lane;
            const uint4 *hL = reinterpret_cast<const uint4 *>(a.hist + iL * 256) + 2 * lane;
            const uint4 r0 = hR[0], r1 = hR[1], l0 = hL[0], l1 = hL[1];
            uint32_t cr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            uint32_t cl[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                cr[q] += cr[q - 1];
                cl[q] += cl[q - 1];
            }
            // exclusive prefix of the lanes' totals
            uint32_t pr = cr[7], pl = cl[7];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t ur = __shfl_up_sync(0xffffffffu, pr, o), ul = __shfl_up_sync(0xffffffffu, pl, o);
                if (lane >= o) { pr += ur; pl += ul; }
            }
            pr -= cr[7];
            pl -= cl[7];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                cum[warp][0][8 * lane + q] = cr[q] + pr;
                cum[warp][1][8 * lane + q] = cl[q] + pl;
            }
            __syncwarp();
            const uint32_t *cR = cum[warp][0], *cL = cum[warp][1];
            const long long nS = side == 1 ? nR : nL;
            const uint32_t *cS = side == 1 ? cR : cL;
            const long long lev = 2LL * lane + 1;
            // smallest v in [0, 255] with the predicate true (true at 255)
            int lo = 0, hi = 255;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (2LL * kQuantiles * cS[mid] >= lev * nS) hi = mid; else lo = mid + 1;
            }
            const int x = lo;
            lo = 0; hi = 255;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)kQuantiles * ((long long)cR[mid] * nL + (long long)cL[mid] * nR) >= lev * nR * nL)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int y = lo;
            long long Sx = x, Sy = y, Sxx = x * x, Sxy = x * y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                Sx += __shfl_xor_sync(0xffffffffu, Sx, o);
                Sy += __shfl_xor_sync(0xffffffffu, Sy, o);
                Sxx += __shfl_xor_sync(0xffffffffu, Sxx, o);
                Sxy += __shfl_xor_sync(0xffffffffu, Sxy, o);
            }
            const long long den = kQuantiles * Sxx - Sx * Sx, num = kQuantiles * Sxy - Sx * Sy;
            double s = den != 0 ? (double)num / (double)den : 1.0;
            s = fmin(fmax(s, a.gmin), a.gmax);
            va = s;
            vb = __ddiv_rn(__dsub_rn((double)Sy, __dmul_rn(s, (double)Sx)), (double)kQuantiles);
        }
    }
    if (lane == 0) smooth_store(a, (size_t)e * 2, va, vb);
}

// Per-row maps by convex combination of adjacent blocks' maps: linear
// between the centres of consecutive blocks (doubled centres
// C_j = floor(j H / B) + floor((j + 1) H / B) - 1 keep it in integers), the
// edge blocks' maps beyond the first and last centre:
//   w = floor(65536 (2y - C_{j-1}) / (C_j - C_{j-1})),
//   m(y) = m_{j-1} + floor((m_j - m_{j-1}) w / 65536),
// for each of the nv values of a map (6: 3 x (a_q, b_q); 12: a 3 x 3
// matrix and its offsets).  One thread per (camera, side, row).
__global__ void __launch_bounds__(256) blend_rows_kernel(const ArrayGeom g, const int32_t *__restrict__ q16, int B,
                                                         int Hmax, int nv, int32_t *__restrict__ rows)
{
    const int total = g.K * 2 * Hmax;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int y = e % Hmax, side = (e / Hmax) % 2, cam = e / (2 * Hmax);
        const int H = g.cam[cam].H;
        if (y >= H) continue;
        const int Y = 2 * y;
        auto centre = [&](int j) {
            return (int)(((long long)j * H) / B + ((long long)(j + 1) * H) / B - 1);
        };
        const int32_t *src = q16 + (size_t)(cam * 2 + side) * B * nv;
        int32_t *dst = rows + ((size_t)(cam * 2 + side) * Hmax + y) * nv;
        if (Y <= centre(0)) {
            for (int i = 0; i < nv; ++i) dst[i] = src[i];
        } else if (Y >= centre(B - 1)) {
            for (int i = 0; i < nv; ++i) dst[i] = src[(B - 1) * nv + i];
        } else {
            int j = 1;
            while (Y >= centre(j)) ++j;
            const int c0 = centre(j - 1), c1 = centre(j);
            const long long w = (65536LL * (Y - c0)) / (c1 - c0);
            for (int i = 0; i < nv; ++i) {
                const long long m0 = src[(j - 1) * nv + i], m1 = src[j * nv + i];
                dst[i] = (int32_t)(m0 + (((m1 - m0) * w) >> 16));
            }
        }
    }
}

}  // namespace

cudaError_t launch_blend_rows(const ArrayGeom &g, const int32_t *q16, int B, int Hmax, int nv, int32_t *rows,
                              cudaStream_t s)
{
    const int total = g.K * 2 * Hmax;
    blend_rows_kernel<<<(total + 255) / 256, 256, 0, s>>>(g, q16, B, Hmax, nv, rows);
    return cudaGetLastError();
}

void fill_solve_topo(SolveTopo &t, int K, int n_groups, const int32_t *group_start, const int32_t *group_members,
                     const int32_t *right_nbr, const int32_t *cam_H)
{
    memset(&t, 0, sizeof t);
    for (int g = 0; g <= n_groups; ++g) t.gstart[g] = (int8_t)group_start[g];
    for (int i = 0; i < group_start[n_groups]; ++i) t.member[i] = (int8_t)group_members[i];
    for (int k = 0; k < K; ++k) {
        t.right[k] = (int8_t)right_nbr[k];
        t.rpos[k] = -1;
        t.H[k] = cam_H[k];
    }
    for (int g = 0; g < n_groups; ++g)
        for (int i = group_start[g]; i < group_start[g + 1]; ++i) {
            const int k = group_members[i], r = right_nbr[k];
            if (r < 0 || r == k) continue;
            for (int q = group_start[g]; q < group_start[g + 1]; ++q)
                if (group_members[q] == r) t.rpos[k] = (int8_t)(q - group_start[g]);
        }
}

cudaError_t launch_solve(const SolveArgs &args, cudaStream_t s)
{
    if (args.fit_mode == RT_FIT_GLOBAL) {
        SolveArgs a = args;
        a.tab = solve_tables();
        a.one_m_alpha = 1.0 - a.alpha;
        // beyond these the clamped gain is gmin / gmax whatever x is
        a.xlo = std::max(std::log(a.gmin) - 1.0, -700.0);
        a.xhi = std::log(a.gmax) + 1.0;
        a.xlo_f = (float)a.xlo;
        a.xhi_f = (float)a.xhi;
        const int n_sys = a.n_groups * a.B * 3;
        solve_global_kernel<<<n_sys, 32, 0, s>>>(a);
    } else if (args.fit_mode == RT_FIT_MATRIX) {
        return launch_solve_matrix(args, s);
    } else if (args.fit_mode == RT_FIT_QUANTILE_AFFINE) {
        const int n_ent = args.K * 2 * args.B * 3;
        solve_quantile_kernel<<<(n_ent + kQuantWarps - 1) / kQuantWarps, 32 * kQuantWarps, 0, s>>>(args);
    } else {
        const int n_ent = args.K * 2 * args.B * 3;
        solve_affine_kernel<<<(n_ent + 63) / 64, 64, 0, s>>>(args);
    }
    return cudaGetLastError();
}

}  // namespace rt

namespace {

__global__ void check_math_kernel(int n, const unsigned long long *a, const unsigned long long *b, double *lr,
                                  const double *x, double *ex, const rt::SolveTables tab)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (lr) lr[i] = rt::log_ratio(a[i], b[i], tab);
        if (ex) ex[i] = rt::exp_table(x[i], tab);
    }
}

}  // namespace

extern "C" rt_status rt_check_solve_math(int32_t n, const uint64_t *a, const uint64_t *b, double *log_ratio,
                                         const double *x, double *exp_x)
{
    if (n < 0) return RT_ERR_INVALID;
    if (n == 0) return RT_OK;
    const bool do_log = a && b && log_ratio, do_exp = x && exp_x;
    for (int i = 0; i < n; ++i) {
        if (do_log && (a[i] == 0 || b[i] == 0)) return RT_ERR_INVALID;
        if (do_exp && !(x[i] >= -700.0 && x[i] <= 700.0)) return RT_ERR_INVALID;
    }
    const size_t bytes = (size_t)n * 8;
    unsigned char *d = nullptr;
    if (cudaMalloc(&d, 5 * bytes) != cudaSuccess) return RT_ERR_CUDA;
    unsigned long long *da = reinterpret_cast<unsigned long long *>(d), *db = da + n;
    double *dl = reinterpret_cast<double *>(db + n), *dx = dl + n, *de = dx + n;
    cudaError_t e = cudaSuccess;
    if (do_log) {
        e = cudaMemcpy(da, a, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(db, b, bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && do_exp) e = cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        check_math_kernel<<<(n + 255) / 256, 256>>>(n, da, db, do_log ? dl : nullptr, dx, do_exp ? de : nullptr,
                                                    rt::solve_tables());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && do_log) e = cudaMemcpy(log_ratio, dl, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && do_exp) e = cudaMemcpy(exp_x, de, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}
