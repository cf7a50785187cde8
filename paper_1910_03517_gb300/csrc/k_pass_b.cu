// Pass B: NV12 / mono16 -> RGB24 conversion (S1), whole-frame histograms of
// the uncorrected RGB (S2 iii) and per-pixel Q16 application of the maps
// (S5, Sec. "White balance and exposure correction": the map f_c is applied
// from the image centre, identity, towards the border, full map, as a
// convex combination) -- one read of every input byte, one write of every
// output byte.
//
// Work decomposition: the array's pixels form one "unit" space (a unit is
// two rows x 16 columns of one camera: one 16-byte load per Y row, one per
// UV row, three 16-byte stores per RGB row).  Every CTA of a persistent grid
// takes an equal contiguous slice of that space across cameras of any size
// (load balance over uneven arrays); a slice that crosses a camera boundary
// is processed as one segment per camera, with the CTA's shared histogram
// flushed to the camera's global histogram between segments.
//
// Histograms: 3 channels x 256 bins x 32 lane-private copies of u32 in
// shared memory (96 KB); lane l only ever adds to copy l, so a warp's 32
// shared atomics always hit 32 distinct banks and 32 distinct words.
#include "rt_internal.cuh"
#include "pixel.cuh"

namespace rt {

namespace {

__device__ __forceinline__ uint4 ld_stream(const uint8_t *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void red_shared_inc(uint32_t addr)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}

// Apply constants of one row for the per-camera gain fit: t = a_q * vbits + cq
struct RowGain { uint32_t aq[3], cq[3]; };

__device__ __forceinline__ RowGain row_gain(const int32_t *__restrict__ q16, int cam, int j, int B)
{
    RowGain r;
    const int32_t *m = q16 + ((size_t)(cam * 2 + 0) * B + j) * 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r.aq[c] = (uint32_t)__ldg(m + 2 * c);
        r.cq[c] = 32768u - r.aq[c] * kMagicBits;          // modulo 2^32
    }
    return r;
}

// Seam-map application of channel c at column x (row block j):
//   A = 65536 + floor((a_q - 65536) w / 65536), Bq = floor(b_q w / 65536),
//   out = clamp(floor((A v + Bq + 32768) / 65536), 0, 255)
__device__ __forceinline__ uint32_t apply_seam(const CamGeom &cg, const int32_t *__restrict__ q16,
                                               int cam, int j, int B, int x, int c, uint32_t vb)
{
    const int side = x >= (cg.W >> 1) ? 1 : 0;
    const long long w = __ldg(cg.ramp + x);
    const int32_t *m = q16 + ((size_t)(cam * 2 + side) * B + j) * 6 + 2 * c;
    const int aq = __ldg(m), bq = __ldg(m + 1);
    const int A = 65536 + (int)(((long long)(aq - 65536) * w) >> 16);
    const int Bq = (int)(((long long)bq * w) >> 16);
    const uint32_t cst = (uint32_t)(Bq + 32768) - (uint32_t)A * kMagicBits;
    int t = (int)((uint32_t)A * vb + cst);
    t = t < 0 ? 0 : (t > 0xFFFFFF ? 0xFFFFFF : t);
    return (uint32_t)t;
}

template <int FIT, bool STATS, bool FULL>
__device__ __forceinline__ void unit_nv12(const CamGeom &cg, int cam, int rp, int ux, const ConvConsts &k,
                                          const int32_t *__restrict__ q16, int B, uint32_t hbase)
{
    const int x0 = ux * kUnitCols;
    const int y0 = rp * 2;
    const uint8_t *yp = cg.y + (size_t)y0 * cg.y_pitch + x0;
    const uint4 Y0 = ld_stream(yp);
    const uint4 Y1 = ld_stream(yp + cg.y_pitch);
    const uint4 UV = ld_stream(cg.uv + (size_t)rp * cg.uv_pitch + x0);
    const uint32_t yw[2][4] = {{Y0.x, Y0.y, Y0.z, Y0.w}, {Y1.x, Y1.y, Y1.z, Y1.w}};
    const uint32_t uvw[4] = {UV.x, UV.y, UV.z, UV.w};
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
    int jr[2];
    jr[0] = block_of_row(y0, cg.H, B);
    jr[1] = block_of_row(y0 + 1, cg.H, B);
    RowGain rg[2];
    if (FIT == RT_FIT_GLOBAL) {
        rg[0] = row_gain(q16, cam, jr[0], B);
        rg[1] = (jr[1] == jr[0]) ? rg[0] : row_gain(q16, cam, jr[1], B);
    }
    uint32_t ow[2][12];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) ow[r][i] = 0u;

#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const float Uf = byte_f(uvw[p >> 1], (p & 1) * 2);
        const float Vf = byte_f(uvw[p >> 1], (p & 1) * 2 + 1);
        const float cz[3] = {fmaf(Vf, k.krv, k.c_r0), fmaf(Uf, k.kgu, fmaf(Vf, k.kgv, k.c_g0)),
                             fmaf(Uf, k.kbu, k.c_b0)};
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = 2 * p + q;
                if (!FULL && i >= nvalid) continue;
                const float Yf = byte_f(yw[r][i >> 2], i & 3);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const uint32_t vb = zbits(Yf, k.ky, cz[c]);
                    if (STATS) red_shared_inc(hbase + vb * 128u + (uint32_t)c * 32768u);
                    uint32_t t;
                    if (FIT == RT_FIT_GLOBAL) {
                        t = rg[r].aq[c] * vb + rg[r].cq[c];
                        t = t > 0xFFFFFFu ? 0xFFFFFFu : t;
                    } else {
                        t = apply_seam(cg, q16, cam, jr[r], B, x0 + i, c, vb);
                    }
                    const int b = 3 * i + c;
                    ow[r][b >> 2] = put_byte2(ow[r][b >> 2], t, b & 3);
                }
            }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        uint8_t *dst = cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0;
        if (FULL) {
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            d4[0] = make_uint4(ow[r][0], ow[r][1], ow[r][2], ow[r][3]);
            d4[1] = make_uint4(ow[r][4], ow[r][5], ow[r][6], ow[r][7]);
            d4[2] = make_uint4(ow[r][8], ow[r][9], ow[r][10], ow[r][11]);
        } else {
            for (int b = 0; b < 3 * nvalid; ++b) dst[b] = (uint8_t)(ow[r][b >> 2] >> (8 * (b & 3)));
        }
    }
}

template <int FIT, bool STATS, bool FULL>
__device__ __forceinline__ void unit_mono(const CamGeom &cg, int cam, int rp, int ux,
                                          const int32_t *__restrict__ q16, int B, uint32_t hbase)
{
    const int x0 = ux * kUnitCols;
    const int y0 = rp * 2;
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
    uint32_t ow[2][12];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int i = 0; i < 12; ++i) ow[r][i] = 0u;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const uint8_t *yp = cg.y + (size_t)(y0 + r) * cg.y_pitch + 2 * x0;
        // a ragged tail of at most 8 samples reads only its first 16 bytes,
        // which the pitch (>= 2 W rounded up to 16) always covers
        const uint4 a = ld_stream(yp);
        const uint4 b = (FULL || nvalid > 8) ? ld_stream(yp + 16) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const int j = block_of_row(y0 + r, cg.H, B);
        RowGain rg;
        if (FIT == RT_FIT_GLOBAL) rg = row_gain(q16, cam, j, B);
#pragma unroll
        for (int i = 0; i < kUnitCols; ++i) {
            if (!FULL && i >= nvalid) continue;
            const uint32_t vb = mono_bits((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu, cg.shift);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (STATS) red_shared_inc(hbase + vb * 128u + (uint32_t)c * 32768u);
                uint32_t t;
                if (FIT == RT_FIT_GLOBAL) {
                    t = rg.aq[c] * vb + rg.cq[c];
                    t = t > 0xFFFFFFu ? 0xFFFFFFu : t;
                } else {
                    t = apply_seam(cg, q16, cam, j, B, x0 + i, c, vb);
                }
                const int bb = 3 * i + c;
                ow[r][bb >> 2] = put_byte2(ow[r][bb >> 2], t, bb & 3);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        uint8_t *dst = cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0;
        if (FULL) {
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            d4[0] = make_uint4(ow[r][0], ow[r][1], ow[r][2], ow[r][3]);
            d4[1] = make_uint4(ow[r][4], ow[r][5], ow[r][6], ow[r][7]);
            d4[2] = make_uint4(ow[r][8], ow[r][9], ow[r][10], ow[r][11]);
        } else {
            for (int b = 0; b < 3 * nvalid; ++b) dst[b] = (uint8_t)(ow[r][b >> 2] >> (8 * (b & 3)));
        }
    }
}

constexpr int kHistWords = 3 * 256 * kHistLanes;

template <int FIT, bool STATS>
__global__ void __launch_bounds__(512, 2) pass_b_kernel(const ArrayGeom g, const PassBArgs a)
{
    extern __shared__ uint32_t sh[];
    const int tid = threadIdx.x;
    const ConvConsts k = conv_consts(g.matrix);
    uint32_t ub = (uint32_t)(((unsigned long long)blockIdx.x * g.units_total) / gridDim.x);
    const uint32_t ue = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * g.units_total) / gridDim.x);
    int cam = 0;
    while (cam + 1 < g.K && g.cam[cam + 1].unit_base <= ub) ++cam;
    const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(sh) + (uint32_t)(tid & 31) * 4u -
                           kMagicBits * 128u;
    while (ub < ue) {
        const CamGeom &cg = g.cam[cam];
        const uint32_t cam_end = cam + 1 < g.K ? g.cam[cam + 1].unit_base : g.units_total;
        const uint32_t se = ue < cam_end ? ue : cam_end;
        if (STATS) {
            uint4 *s4 = reinterpret_cast<uint4 *>(sh);
            for (int i = tid; i < kHistWords / 4; i += blockDim.x) s4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
        }
        const uint32_t upr = cg.upr;
        const int full_units = cg.W / kUnitCols;
        for (uint32_t u = ub + tid; u < se; u += blockDim.x) {
            const uint32_t local = u - cg.unit_base;
            const int rp = (int)(local / upr);
            const int ux = (int)(local - (uint32_t)rp * upr);
            if (cg.fmt == RT_NV12) {
                if (ux < full_units) unit_nv12<FIT, STATS, true>(cg, cam, rp, ux, k, a.q16, g.B, hbase);
                else unit_nv12<FIT, STATS, false>(cg, cam, rp, ux, k, a.q16, g.B, hbase);
            } else {
                if (ux < full_units) unit_mono<FIT, STATS, true>(cg, cam, rp, ux, a.q16, g.B, hbase);
                else unit_mono<FIT, STATS, false>(cg, cam, rp, ux, a.q16, g.B, hbase);
            }
        }
        if (STATS) {
            __syncthreads();
            uint32_t *gh = a.frame_hist + (size_t)cam * 768;
            for (int b = tid; b < 768; b += blockDim.x) {
                uint32_t s = 0;
#pragma unroll 8
                for (int i = 0; i < kHistLanes; ++i) s += sh[b * kHistLanes + ((i + b) & 31)];
                if (s) atomicAdd(gh + b, s);
            }
            __syncthreads();
        }
        ub = se;
        ++cam;
    }
}

template <int FIT, bool STATS>
cudaError_t launch_one(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, size_t smem,
                       cudaStream_t s)
{
    pass_b_kernel<FIT, STATS><<<grid, threads, STATS ? smem : 0, s>>>(g, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t pass_b_prepare(int threads, size_t *smem_bytes)
{
    (void)threads;
    const size_t smem = (size_t)kHistWords * 4;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<RT_FIT_GLOBAL, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<RT_FIT_SEAM_AFFINE, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    *smem_bytes = smem;
    return cudaSuccess;
}

cudaError_t launch_pass_b(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, size_t smem,
                          cudaStream_t s)
{
    const bool stats = a.frame_hist != nullptr;
    if (g.fit_mode == RT_FIT_GLOBAL)
        return stats ? launch_one<RT_FIT_GLOBAL, true>(g, a, grid, threads, smem, s)
                     : launch_one<RT_FIT_GLOBAL, false>(g, a, grid, threads, smem, s);
    return stats ? launch_one<RT_FIT_SEAM_AFFINE, true>(g, a, grid, threads, smem, s)
                 : launch_one<RT_FIT_SEAM_AFFINE, false>(g, a, grid, threads, smem, s);
}

}  // namespace rt
