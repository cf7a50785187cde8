// 3 x 3 cross-channel maps (the conclusion's proposal of linear maps that
// mix the three colour channels), fitted like the paper's per-channel maps of
// Sec. "White balance and exposure correction": the shared spectrum of a seam
// is the equal-weight mixture of its two bands (mean mu_s = (mu_L + mu_R) / 2,
// covariance S_s = (S_L + S_R) / 2 + d d^T / 4, d = mu_L - mu_R), and each
// side's map out = M v + b matches its band's first two moments to it:
// M is the symmetric positive definite solution of M S M = S_s,
//   M = S^-1/2 (S^1/2 S_s S^1/2)^1/2 S^-1/2,
// its eigenvalues clamped to [gain_min, gain_max], b = mu_s - M mu.
// Covariances carry a ridge of 0.25 I.
//
// FP64 on this GPU costs ~64 cycles of a sub-partition per warp instruction
// whatever the active lanes, so a thread-serial FP64 eigen-solver would take
// tens of microseconds.  Instead, one warp per (camera, side, block):
//  1. lanes 0-8 / 16-24 form the two bands' moments in FP64 (one division a
//     lane), lanes 0-8 the mixture's (entry (i, j) in lane 3 i + j);
//  2. lane 0 builds an FP32 seed: S = F F^T (Cholesky), P = F^T S_s F =
//     U diag(l) U^T (cyclic Jacobi), M0 = W diag(sqrt l) W^T with W = F^-T U;
//  3. Newton on M S M = S_s with the seed's Jacobian: the FP64 residual
//     R = S_s - M S M (lane-parallel, 6 FMAs a lane), the correction from
//     the linearised equation in the seed's basis,
//       D^ = (H^T R H) ./ (sqrt l_i + sqrt l_j), H = F U,  D = W D^ W^T,
//     in FP32 and M += D in FP64, until |D| is below 1e-13 |M| or stops
//     shrinking (the FP64 residual's rounding floor); each step gains about
//     the seed's relative accuracy (1e-3 .. 1e-6 for band covariances);
//  4. eigenvalue clamp: FP32 Jacobi of M; only if an eigenvalue is not
//     inside the limits by a margin, FP64 Rayleigh quotients of its
//     eigenvectors give the eigenvalues and the clamp is applied as
//     f(M) = f[l1] I + f[l1,l2] (M - l1 I) + f[l1,l2,l3] (M - l1 I)(M - l2 I)
//     (Newton's divided differences over the sorted eigenvalues; stable for
//     a 1-Lipschitz f and needing no eigenvectors);
//  5. b, exponential smoothing and Q16 rounding of the 12 values, one lane
//     each.
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

namespace {

constexpr int kMatWarps = 1;       // problems per CTA
constexpr int kNewtonMax = 12;
constexpr double kRidge = 0.25;

struct MatShared {
    double x[2][9];      // per band: mu (3), then Q / n (6: 00 01 02 11 12 22)
    double Sb[2][9];     // per band: covariance + ridge, row-major
    double Ss[9];        // mixture covariance + ridge
    double mus[3];
    double M[9];
    double T[9];         // M S
    double lam[3];       // eigenvalues of M (clamp path)
    double dd[3];        // f[l1], f[l1,l2], f[l1,l2,l3]
    double l12[2];       // sorted l1, l2
    float Rf[9], X[9], D[9], Y[9];
    float H[9], W[9], inv[9];
    float V[9];          // eigenvectors of M (columns)
    int clamp;
};

__device__ __forceinline__ int sym6(int i, int j)
{
    const int u = i < j ? i : j, v = i < j ? j : i;
    return u == 0 ? v : (u == 1 ? 2 + v : 5);
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3 x 3 in FP32,
// A = V diag(A_ii) V^T on return.  Rotation from the symmetric 2 x 2 Schur
// decomposition: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c;
// A <- J^T A J, V <- V J.
__device__ void jacobi3f(float (&A)[3][3], float (&V)[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.f : 0.f;
    for (int sweep = 0; sweep < 10; ++sweep) {
        const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const float dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (!(off > 1e-15f * dia)) break;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
            const float apq = A[p][q];
            if (apq == 0.f) continue;
            const float tau = (A[q][q] - A[p][p]) / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            const float c = rsqrtf(1.f + t * t), s = t * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
}

// Step 2: the FP32 seed and the Newton basis (lane 0).
__device__ void seed(MatShared &sh)
{
    float S[3][3], Ss[3][3];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        S[i / 3][i % 3] = (float)sh.Sb[0][i];
        Ss[i / 3][i % 3] = (float)sh.Ss[i];
    }
    // S = F F^T, F lower triangular; G = F^-1
    const float tiny = 1e-30f;
    float F[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    F[0][0] = sqrtf(fmaxf(S[0][0], tiny));
    F[1][0] = S[1][0] / F[0][0];
    F[2][0] = S[2][0] / F[0][0];
    F[1][1] = sqrtf(fmaxf(S[1][1] - F[1][0] * F[1][0], tiny));
    F[2][1] = (S[2][1] - F[2][0] * F[1][0]) / F[1][1];
    F[2][2] = sqrtf(fmaxf(S[2][2] - F[2][0] * F[2][0] - F[2][1] * F[2][1], tiny));
    float G[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    G[0][0] = 1.f / F[0][0];
    G[1][1] = 1.f / F[1][1];
    G[2][2] = 1.f / F[2][2];
    G[1][0] = -F[1][0] * G[0][0] * G[1][1];
    G[2][1] = -F[2][1] * G[1][1] * G[2][2];
    G[2][0] = -(F[2][0] * G[0][0] + F[2][1] * G[1][0]) * G[2][2];
    // P = F^T S_s F (symmetrised)
    float K[3][3], P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) K[i][j] = Ss[i][0] * F[0][j] + Ss[i][1] * F[1][j] + Ss[i][2] * F[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = F[0][i] * K[0][j] + F[1][i] * K[1][j] + F[2][i] * K[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i + 1; j < 3; ++j) P[i][j] = P[j][i] = 0.5f * (P[i][j] + P[j][i]);
    float U[3][3];
    jacobi3f(P, U);
    float sq[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) sq[i] = sqrtf(fmaxf(P[i][i], tiny));
    // W = G^T U, H = F U
    float W[3][3], Hm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            W[i][j] = G[0][i] * U[0][j] + G[1][i] * U[1][j] + G[2][i] * U[2][j];
            Hm[i][j] = F[i][0] * U[0][j] + F[i][1] * U[1][j] + F[i][2] * U[2][j];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            sh.W[3 * i + j] = W[i][j];
            sh.H[3 * i + j] = Hm[i][j];
            sh.inv[3 * i + j] = 1.f / (sq[i] + sq[j]);
        }
    // M0 = W diag(sq) W^T, exactly symmetric
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const float m = W[i][0] * sq[0] * W[j][0] + W[i][1] * sq[1] * W[j][1] + W[i][2] * sq[2] * W[j][2];
            sh.M[3 * i + j] = sh.M[3 * j + i] = (double)m;
        }
}

// Step 4a (lane 0): does the clamp change M?  FP32 eigenvalues within
// the limits by a margin well above their error leave M as it is.
__device__ int clamp_needed(MatShared &sh, double gmin, double gmax)
{
    float A[3][3], V[3][3];
#pragma unroll
    for (int i = 0; i < 9; ++i) A[i / 3][i % 3] = (float)sh.M[i];
    jacobi3f(A, V);
    float big = fmaxf(fabsf(A[0][0]), fmaxf(fabsf(A[1][1]), fabsf(A[2][2])));
    const double margin = 1e-5 * (double)big + 1e-30;
    int need = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double l = (double)A[i][i];
        if (!(l >= gmin + margin && l <= gmax - margin)) need = 1;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) sh.V[i] = V[i / 3][i % 3];
    return need;
}

__device__ __forceinline__ double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// Step 4b (lane 0): sort the FP64 eigenvalues and form the divided
// differences of the clamp over them.
__device__ void clamp_differences(MatShared &sh, double lo, double hi)
{
    double l[3] = {sh.lam[0], sh.lam[1], sh.lam[2]};
    if (l[0] > l[1]) { const double t = l[0]; l[0] = l[1]; l[1] = t; }
    if (l[1] > l[2]) { const double t = l[1]; l[1] = l[2]; l[2] = t; }
    if (l[0] > l[1]) { const double t = l[0]; l[0] = l[1]; l[1] = t; }
    const double tol = 1e-13 * fmax(fabs(l[0]), fabs(l[2]));
    auto slope = [&](double a, double b) {
        // f[a, b] for a <= b; f' where the two coincide
        if (b - a > tol) return (clampd(b, lo, hi) - clampd(a, lo, hi)) / (b - a);
        return (a > lo && a < hi) ? 1.0 : 0.0;
    };
    const double f12 = slope(l[0], l[1]), f23 = slope(l[1], l[2]);
    sh.dd[0] = clampd(l[0], lo, hi);
    sh.dd[1] = f12;
    sh.dd[2] = l[2] - l[0] > tol ? (f23 - f12) / (l[2] - l[0]) : 0.0;
    sh.l12[0] = l[0];
    sh.l12[1] = l[1];
}

__device__ __forceinline__ void smooth_one(const SolveArgs &a, size_t idx, double v)
{
    a.maps_new[idx] = v;
    const double e = a.first ? v : (1.0 - a.alpha) * a.E[idx] + a.alpha * v;
    a.E[idx] = e;
    a.q16[idx] = (int32_t)llround(65536.0 * e);
}

__global__ void __launch_bounds__(32 * kMatWarps) solve_matrix_kernel(const SolveArgs a)
{
    __shared__ MatShared shm[kMatWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kMatWarps + warp;
    if (e >= a.K * 2 * a.B) return;   // whole warp
    MatShared &sh = shm[warp];
    const int j = e % a.B, side = (e / a.B) % 2, cam = e / (2 * a.B);
    // the seam on this side: this camera's band and the neighbour's facing band
    const int nb = side == 1 ? a.right_nbr[cam] : a.left_nbr[cam];
    const unsigned long long *q_own = a.joint + ((size_t)(cam * 2 + side) * a.B + j) * 10;
    const unsigned long long *q_oth = nullptr;
    bool valid = false;
    if (nb >= 0 && nb != cam) {
        q_oth = a.joint + ((size_t)(nb * 2 + (1 - side)) * a.B + j) * 10;
        valid = q_own[0] >= (unsigned long long)a.min_valid && q_oth[0] >= (unsigned long long)a.min_valid;
    }
    const int i3 = lane / 3, j3 = lane % 3;
    double out = (lane < 9 && i3 == j3) ? 1.0 : 0.0;   // identity
    if (valid) {
        // 1. moments: band 0 = this camera's, band 1 = the neighbour's
        const int hl = lane & 15, band = lane >> 4;
        if (hl < 9) {
            const unsigned long long *q = band == 0 ? q_own : q_oth;
            const unsigned long long num = hl < 3 ? q[1 + hl] : q[4 + (hl - 3)];
            sh.x[band][hl] = (double)num / (double)q[0];
        }
        __syncwarp();
        if (hl < 9) {
            const int i = hl / 3, jj = hl % 3;
            const double *x = sh.x[band];
            const double c = __dsub_rn(x[3 + sym6(i, jj)], __dmul_rn(x[i], x[jj]));
            sh.Sb[band][hl] = i == jj ? __dadd_rn(c, kRidge) : c;
        }
        __syncwarp();
        // the left camera's right band is "R", the right camera's left band "L"
        const double *muR = side == 1 ? sh.x[0] : sh.x[1], *muL = side == 1 ? sh.x[1] : sh.x[0];
        if (lane < 9) {
            const double di = __dsub_rn(muL[i3], muR[i3]), dj = __dsub_rn(muL[j3], muR[j3]);
            const double SL = side == 1 ? sh.Sb[1][lane] : sh.Sb[0][lane];
            const double SR = side == 1 ? sh.Sb[0][lane] : sh.Sb[1][lane];
            sh.Ss[lane] = __dadd_rn(__dmul_rn(0.5, __dadd_rn(SL, SR)), __dmul_rn(0.25, __dmul_rn(di, dj)));
            if (lane < 3) sh.mus[lane] = __dmul_rn(0.5, __dadd_rn(muL[lane], muR[lane]));
        }
        __syncwarp();
        // 2. FP32 seed
        if (lane == 0) seed(sh);
        __syncwarp();
        // 3. Newton steps
        const double *S = sh.Sb[0];
        float prev = INFINITY;
        for (int it = 0; it < kNewtonMax; ++it) {
            if (lane < 9) sh.T[lane] = fma(sh.M[3 * i3 + 2], S[6 + j3], fma(sh.M[3 * i3 + 1], S[3 + j3],
                                                                               sh.M[3 * i3] * S[j3]));
            __syncwarp();
            if (lane < 9) {
                double r = sh.Ss[lane];
                r = fma(-sh.T[3 * i3], sh.M[j3], r);
                r = fma(-sh.T[3 * i3 + 1], sh.M[3 + j3], r);
                r = fma(-sh.T[3 * i3 + 2], sh.M[6 + j3], r);
                sh.Rf[lane] = (float)r;
            }
            __syncwarp();
            if (lane < 9)
                sh.X[lane] = sh.Rf[3 * i3] * sh.H[j3] + sh.Rf[3 * i3 + 1] * sh.H[3 + j3] + sh.Rf[3 * i3 + 2] * sh.H[6 + j3];
            __syncwarp();
            if (lane < 9)
                sh.D[lane] = sh.inv[lane] *
                             (sh.H[i3] * sh.X[j3] + sh.H[3 + i3] * sh.X[3 + j3] + sh.H[6 + i3] * sh.X[6 + j3]);
            __syncwarp();
            if (lane < 9)
                sh.Y[lane] = sh.W[3 * i3] * sh.D[j3] + sh.W[3 * i3 + 1] * sh.D[3 + j3] + sh.W[3 * i3 + 2] * sh.D[6 + j3];
            __syncwarp();
            bool small = true;
            double mnew = 0.0;
            float ad = 0.f;
            if (lane < 9) {
                const int u = i3 < j3 ? i3 : j3, v = i3 < j3 ? j3 : i3;   // same value in (i, j) and (j, i)
                const float d = sh.Y[3 * u] * sh.W[3 * v] + sh.Y[3 * u + 1] * sh.W[3 * v + 1] +
                                sh.Y[3 * u + 2] * sh.W[3 * v + 2];
                mnew = sh.M[lane] + (double)d;
                small = fabs((double)d) <= 1e-13 * (fabs(sh.M[4 * i3]) + fabs(sh.M[4 * j3]));
                ad = fabsf(d);
            }
            // largest |D| of the step (non-negative floats order as their bits)
            const float amax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(ad)));
            __syncwarp();
            if (lane < 9) sh.M[lane] = mnew;
            __syncwarp();
            if (__all_sync(0xffffffffu, small) || amax > 0.25f * prev) break;
            prev = amax;
        }
        // 4. eigenvalue clamp
        if (lane == 0) sh.clamp = clamp_needed(sh, a.gmin, a.gmax);
        __syncwarp();
        if (sh.clamp) {
            if (lane < 3) {
                const double v0 = sh.V[lane], v1 = sh.V[3 + lane], v2 = sh.V[6 + lane];
                const double w0 = fma(sh.M[2], v2, fma(sh.M[1], v1, sh.M[0] * v0));
                const double w1 = fma(sh.M[5], v2, fma(sh.M[4], v1, sh.M[3] * v0));
                const double w2 = fma(sh.M[8], v2, fma(sh.M[7], v1, sh.M[6] * v0));
                const double num = fma(v2, w2, fma(v1, w1, v0 * w0));
                const double den = fma(v2, v2, fma(v1, v1, v0 * v0));
                sh.lam[lane] = num / den;
            }
            __syncwarp();
            if (lane == 0) clamp_differences(sh, a.gmin, a.gmax);
            __syncwarp();
            double mc = 0.0;
            if (lane < 9) {
                const int u = i3 < j3 ? i3 : j3, v = i3 < j3 ? j3 : i3;
                const double l1 = sh.l12[0], l2 = sh.l12[1];
                double z2 = 0.0;   // ((M - l1 I)(M - l2 I))_uv
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    z2 = fma(sh.M[3 * u + k] - (u == k ? l1 : 0.0), sh.M[3 * k + v] - (k == v ? l2 : 0.0), z2);
                const double z1 = sh.M[3 * u + v] - (u == v ? l1 : 0.0);
                mc = fma(sh.dd[2], z2, fma(sh.dd[1], z1, u == v ? sh.dd[0] : 0.0));
            }
            __syncwarp();
            if (lane < 9) sh.M[lane] = mc;
            __syncwarp();
        }
        // 5. b = mu_s - M mu, mu this camera's band
        if (lane < 9) {
            out = sh.M[lane];
        } else if (lane < 12) {
            const int c = lane - 9;
            const double *mu = sh.x[0];
            const double mm = fma(sh.M[3 * c + 2], mu[2], fma(sh.M[3 * c + 1], mu[1], sh.M[3 * c] * mu[0]));
            out = sh.mus[c] - mm;
        }
    }
    if (lane < 12) smooth_one(a, (size_t)e * 12 + lane, out);
}

}  // namespace

cudaError_t launch_solve_matrix(const SolveArgs &a, cudaStream_t s)
{
    const int n_ent = a.K * 2 * a.B;
    solve_matrix_kernel<<<(n_ent + kMatWarps - 1) / kMatWarps, 32 * kMatWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rt
