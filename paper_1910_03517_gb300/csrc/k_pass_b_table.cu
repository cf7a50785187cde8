// Pass B with the seam maps applied per block (Sec. "White balance and
// exposure correction": each seam side's map blended from the identity at
// the image centre to the full map at the border), reading every column's
// coefficients from a table instead of computing them per unit.
//
// The ramp gives every column its own coefficients A_c = delta 65536 +
// floor((m - delta 65536) w / 65536) and cst_c (k_pass_b.cu, col_coef).
// After each solve, seam_coef_kernel writes them for every (camera, block,
// column) with the same col_coef; pass B then loads them (6 words a column
// for the affine maps, 12 for the 3 x 3 maps) and applies them with the
// computing variant's arithmetic, so the outputs are the same bits.
//
// Work decomposition: a warp takes a tile of kTileRowPairs x kTileUnits = 4
// row pairs x 8 units (8 rows x 128 columns); lane l does unit (4 tr + l / 8,
// 8 tc + l % 8).  The 4 lanes of one unit column read the same coefficient
// words, so a warp's load of a word touches 8 consecutive 16-byte words (128
// bytes) where a warp along one row pair would touch 32; each input load
// reads 128 contiguous bytes of 4 rows, and each row pair of 8 units is 384
// contiguous output bytes.  (Of the tile shapes measured on tower12 with the
// affine maps, 4 x 8 ran fastest, then 2 x 16, one row pair of 32 units,
// 8 x 4 and 16 x 2.)  Per 4-column group of a unit the group's coefficient
// words are loaded once for both rows (again for the second row when the
// row pair straddles a block boundary).  Histograms and thumbnails as in
// k_pass_b.cu: one CTA per SM, a contiguous slice of the array's tiles, one
// segment per camera.
#include <algorithm>

#include "pass_b.cuh"

namespace rt {

namespace {

// Component q (0..3, known at compile time) of a 16-byte word.
__device__ __forceinline__ uint32_t word_q(const uint4 &v, int q)
{
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// First table word of unit ux of block j: the words of 4-column group g4 and
// value v follow at + (g4 nv + v) 32.
template <int NV>
__device__ __forceinline__ const uint4 *table_unit(const uint4 *__restrict__ coef, const CamGeom &cg, int j, int ux)
{
    const int nch = (int)((cg.upr + 31) >> 5);
    return coef + cg.coef_base + (size_t)(j * nch + (ux >> 5)) * (4 * NV * 32) + (ux & 31);
}

// Coefficient words stay in L1 (evict last); the output stores do not
// allocate there (st_v8, st_v4), so that streaming it does not evict them.
__device__ __forceinline__ uint4 ld_coef(const uint4 *p)
{
    uint4 v;
    asm("ld.global.nc.L1::evict_last.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// One full row of a unit (48 bytes at a), as store_unit stores each row.
__device__ __forceinline__ void store_row(const uint32_t (&w)[12], uint8_t *a)
{
    const bool odd = ((uintptr_t)a >> 4) & 1u;
    uint32_t w8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w8[i] = odd ? w[4 + i] : w[i];
    const uint4 w4 = odd ? make_uint4(w[0], w[1], w[2], w[3]) : make_uint4(w[8], w[9], w[10], w[11]);
    st_v8(a + (odd ? 16 : 0), w8);
    st_v4(a + (odd ? 0 : 32), w4);
}

// A row's 48 bytes: the full row through store_row, a ragged one (nvalid
// columns) through put_ragged.
template <bool FULL>
__device__ __forceinline__ void put_row(const uint32_t (&ow)[12], uint8_t *dst, int nvalid)
{
    if (FULL) store_row(ow, dst);
    else put_ragged(ow, dst, 3 * nvalid);
}

// t of the 4 columns' channel c (t[3 q + c]) of a 4-column group from the
// group's table words tg[32 v] (affine: A_c, cst_c; 3 x 3: A_cd row-major,
// cst_c), the channel's words loaded once -- the sums of col_apply.
template <int NV>
__device__ __forceinline__ void table_apply(const uint4 *__restrict__ tg, const uint32_t (&vbq)[4][3], uint32_t (&t)[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if constexpr (NV == 6) {
            const uint4 A = ld_coef(tg + 32 * c), C = ld_coef(tg + 32 * (3 + c));
#pragma unroll
            for (int q = 0; q < 4; ++q) t[3 * q + c] = word_q(A, q) * vbq[q][c] + word_q(C, q);
        } else {
            const uint4 A0 = ld_coef(tg + 32 * (3 * c)), A1 = ld_coef(tg + 32 * (3 * c + 1));
            const uint4 A2 = ld_coef(tg + 32 * (3 * c + 2)), C = ld_coef(tg + 32 * (9 + c));
#pragma unroll
            for (int q = 0; q < 4; ++q)
                t[3 * q + c] = word_q(A0, q) * vbq[q][0] + word_q(A1, q) * vbq[q][1] + word_q(A2, q) * vbq[q][2] +
                               word_q(C, q);
        }
    }
}

// An NV12 unit, both rows per 4-column group: the group's NV words are
// loaded once and serve both rows (reloaded for row 1 when the row pair
// straddles a block boundary), the chroma terms are converted once, and the
// unit's 2 x 12 output words go out through store_unit.
// TH: no thumbnails (0) or the camera's thumbnail width class (pass_b.cuh).
template <int NV, bool STATS, bool FULL, int TH>
__device__ __forceinline__ void unit_nv12_table2(const CamGeom &cg, int rp, int ux, const ConvConsts &k,
                                                 const uint4 *__restrict__ coef, uint32_t hbase, uint32_t *th,
                                                 const uint4 Y0, const uint4 Y1, const uint4 UV, uint32_t (&ow)[2][12])
{
    const int x0 = ux * kUnitCols, y0 = rp * 2;
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
    const uint32_t yw[2][4] = {{Y0.x, Y0.y, Y0.z, Y0.w}, {Y1.x, Y1.y, Y1.z, Y1.w}};
    const uint32_t uvw[4] = {UV.x, UV.y, UV.z, UV.w};
    const int j0 = block_of_row(y0, cg.H, cg.nblk), j1 = block_of_row(y0 + 1, cg.H, cg.nblk);
    const uint4 *tb[2] = {table_unit<NV>(coef, cg, j0, ux), table_unit<NV>(coef, cg, j1, ux)};
    constexpr bool THUMBS = TH != 0;
    [[maybe_unused]] ThumbAcc<2> ta;
    if constexpr (THUMBS) thumb_begin<TH>(ta, cg, y0, x0);
#pragma unroll
    for (int g4 = 0; g4 < 4; ++g4) {
        const F2 Uf = bytes_f2(uvw[g4], 0, 2), Vf = bytes_f2(uvw[g4], 1, 3);
        const F2 czR = fma2(Vf, k.krv, k.c_r0);
        const F2 czG = fma2(Uf, k.kgu, fma2(Vf, k.kgv, k.c_g0));
        const F2 czB = fma2(Uf, k.kbu, k.c_b0);
        uint4 cf[NV];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (r == 0 || j1 != j0) {
                const uint4 *tg = tb[r] + g4 * NV * 32;
#pragma unroll
                for (int v = 0; v < NV; ++v) cf[v] = ld_coef(tg + 32 * v);
            }
            uint32_t vbq[4][3];
            convert4(yw[r][g4], k, czR, czG, czB, vbq);
            uint32_t t[12];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * g4 + q;
                const bool live = FULL || i < nvalid;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if constexpr (THUMBS) {
                        if (live) thumb_add<TH>(ta, th, cg, r, x0, i, c, vbq[q][c]);
                    }
                    if (STATS && live) hist_inc(hbase + vbq[q][c] * 128u, c);
                    if constexpr (NV == 6)
                        t[3 * q + c] = word_q(cf[c], q) * vbq[q][c] + word_q(cf[3 + c], q);
                    else
                        t[3 * q + c] = word_q(cf[3 * c], q) * vbq[q][0] + word_q(cf[3 * c + 1], q) * vbq[q][1] +
                                       word_q(cf[3 * c + 2], q) * vbq[q][2] + word_q(cf[9 + c], q);
                }
            }
            ow[r][3 * g4 + 0] = even_bytes(clamp_hi2s(t[0], t[1]), clamp_hi2s(t[2], t[3]));
            ow[r][3 * g4 + 1] = even_bytes(clamp_hi2s(t[4], t[5]), clamp_hi2s(t[6], t[7]));
            ow[r][3 * g4 + 2] = even_bytes(clamp_hi2s(t[8], t[9]), clamp_hi2s(t[10], t[11]));
        }
    }
    if constexpr (THUMBS) {
        thumb_end<TH>(ta, th, nvalid);
    }
    if (!FULL) {
#pragma unroll
        for (int r = 0; r < 2; ++r) put_ragged(ow[r], cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0, 3 * nvalid);
    }
}

// A mono unit, row by row: the three channels of a pixel share its value.
template <int NV, bool STATS, bool FULL, int TH>
__device__ __forceinline__ void unit_mono_table(const CamGeom &cg, int rp, int ux, const uint4 *__restrict__ coef,
                                                uint32_t hbase, uint32_t *th)
{
    const int x0 = ux * kUnitCols, y0 = rp * 2;
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
        const uint8_t *yp = cg.y + (size_t)(y0 + r) * cg.y_pitch + 2 * x0;
        // a ragged tail of at most 8 samples reads only its first 16 bytes,
        // which the pitch (>= 2 W rounded up to 16) always covers
        const uint4 a = ld_stream(yp);
        const uint4 b = (FULL || nvalid > 8) ? ld_stream(yp + 16) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const uint4 *tb = table_unit<NV>(coef, cg, block_of_row(y0 + r, cg.H, cg.nblk), ux);
        uint32_t ow[12];
        [[maybe_unused]] ThumbAcc<1> ta;
        if constexpr (TH != 0) thumb_begin<TH>(ta, cg, y0 + r, x0);
#pragma unroll
        for (int g4 = 0; g4 < 4; ++g4) {
            const uint4 *tg = tb + g4 * NV * 32;
            uint32_t t[12];
            uint32_t vbq[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * g4 + q;
                const bool live = FULL || i < nvalid;
                const uint32_t v = mono_bits((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu, cg.shift);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    vbq[q][c] = v;
                    if constexpr (TH != 0) {
                        if (live) thumb_add<TH>(ta, th, cg, 0, x0, i, c, v);
                    }
                    if (STATS && live) hist_inc(hbase + v * 128u, c);
                }
            }
            table_apply<NV>(tg, vbq, t);
            ow[3 * g4 + 0] = even_bytes(clamp_hi2s(t[0], t[1]), clamp_hi2s(t[2], t[3]));
            ow[3 * g4 + 1] = even_bytes(clamp_hi2s(t[4], t[5]), clamp_hi2s(t[6], t[7]));
            ow[3 * g4 + 2] = even_bytes(clamp_hi2s(t[8], t[9]), clamp_hi2s(t[10], t[11]));
        }
        if constexpr (TH != 0) thumb_end<TH>(ta, th, nvalid);
        put_row<FULL>(ow, cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0, nvalid);
    }
}

// A unit with the camera's thumbnail width class (wide: TH = kThumbWide,
// else kThumbNarrow), or without thumbnails.
template <int NV, bool STATS, bool FULL, bool THUMBS, typename... A>
__device__ __forceinline__ void unit_nv12_table_th(bool wide, A &&...args)
{
    if constexpr (!THUMBS) unit_nv12_table2<NV, STATS, FULL, 0>(args...);
    else if (wide) unit_nv12_table2<NV, STATS, FULL, kThumbWide>(args...);
    else unit_nv12_table2<NV, STATS, FULL, kThumbNarrow>(args...);
}

template <int NV, bool STATS, bool FULL, bool THUMBS, typename... A>
__device__ __forceinline__ void unit_mono_table_th(bool wide, A &&...args)
{
    if constexpr (!THUMBS) unit_mono_table<NV, STATS, FULL, 0>(args...);
    else if (wide) unit_mono_table<NV, STATS, FULL, kThumbWide>(args...);
    else unit_mono_table<NV, STATS, FULL, kThumbNarrow>(args...);
}

// Both kernels hold a 4-column group's words for both rows of a unit: the
// affine maps' 6 (96 registers: compiled for 640 threads) and the 3 x 3
// maps' 12 (128 registers: compiled for 512).
template <int NV, bool THUMBS>
constexpr int kTableThreads = THUMBS ? 512 : (NV == 6 ? 640 : 512);

template <int NV, bool STATS, bool THUMBS>
__global__ void __launch_bounds__(kTableThreads<NV, THUMBS>, 1) pass_b_table_kernel(const ArrayGeom g, const PassBArgs a)
{
    extern __shared__ uint32_t sh[];
    uint32_t *th = sh + (STATS ? kHistWords : 0);   // [36][64][3] cell sums (THUMBS)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = (int)(blockDim.x >> 5);
    const ConvConsts &k = g.conv;
    allow_next_launch();
    // balanced contiguous slices of the tile space
    const uint32_t q = g.tiles_total / gridDim.x, r = g.tiles_total - q * gridDim.x;
    uint32_t tb = blockIdx.x * q + min(blockIdx.x, r);
    const uint32_t te = tb + q + (blockIdx.x < r ? 1u : 0u);
    int cam = 0;
    while (cam + 1 < g.K && g.cam[cam + 1].tile_base <= tb) ++cam;
    const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(sh) + (uint32_t)lane * 4u - kMagicBits * 128u;
    while (tb < te) {
        const CamGeom &cg = g.cam[cam];
        const uint32_t cam_end = cam + 1 < g.K ? g.cam[cam + 1].tile_base : g.tiles_total;
        const uint32_t se = te < cam_end ? te : cam_end;
        if (STATS || THUMBS) {
            uint4 *s4 = reinterpret_cast<uint4 *>(sh);
            const int words = (STATS ? kHistWords : 0) + (THUMBS ? kThumbWords : 0);
            for (int i = tid; i < words / 4; i += blockDim.x) s4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
        }
        const int nrp = cg.H >> 1, full_units = cg.W / kUnitCols;
        const bool twide = THUMBS && thumb_wide(cg);
        for (uint32_t t = tb + (uint32_t)warp; t < se; t += (uint32_t)nwarps) {
            const int local = (int)(t - cg.tile_base);
            const int tr = local / cg.ntc, tc = local - tr * cg.ntc;
            const int rp = tr * kTileRowPairs + lane / kTileUnits, ux = tc * kTileUnits + lane % kTileUnits;
            if (rp >= nrp || ux >= (int)cg.upr) continue;
            if (cg.fmt == RT_NV12) {
                const uint8_t *yp = cg.y + (size_t)(2 * rp) * cg.y_pitch + ux * kUnitCols;
                const uint4 Y0 = ld_stream(yp), Y1 = ld_stream(yp + cg.y_pitch);
                const uint4 UV = ld_stream(cg.uv + (size_t)rp * cg.uv_pitch + ux * kUnitCols);
                uint32_t ow[2][12];
                if (ux < full_units) {
                    unit_nv12_table_th<NV, STATS, true, THUMBS>(twide, cg, rp, ux, k, a.coef, hbase, th, Y0, Y1,
                                                                 UV, ow);
                    store_unit(ow, true, cg.rgb + (size_t)(2 * rp) * cg.rgb_pitch + 3 * kUnitCols * ux, cg.rgb_pitch);
                } else {
                    unit_nv12_table_th<NV, STATS, false, THUMBS>(twide, cg, rp, ux, k, a.coef, hbase, th, Y0, Y1,
                                                                 UV, ow);
                }
            } else {
                if (ux < full_units)
                    unit_mono_table_th<NV, STATS, true, THUMBS>(twide, cg, rp, ux, a.coef, hbase, th);
                else
                    unit_mono_table_th<NV, STATS, false, THUMBS>(twide, cg, rp, ux, a.coef, hbase, th);
            }
        }
        if (STATS || THUMBS) wait_prev_grid();   // the previous pass B cleared these accumulators
        if (THUMBS) {
            __syncthreads();
            // [36][64][3] shared -> [3][36][64] global
            uint32_t *gt = a.thumbs + (size_t)cam * kThumbWords;
            for (int i = tid; i < kThumbWords; i += blockDim.x) {
                const uint32_t v = th[i];
                if (v) {
                    const int c = i % 3, cell = i / 3;
                    atomicAdd(gt + c * (RT_THUMB_H * RT_THUMB_W) + cell, v);
                }
            }
            if (!STATS) __syncthreads();
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
        tb = se;
        ++cam;
    }
    // clear the accumulators the next frame set will use (other parity);
    // the previous pass B flushed its sums into them
    wait_prev_grid();
    for (uint32_t i = blockIdx.x * blockDim.x + tid; i < a.clear_a_n; i += gridDim.x * blockDim.x) a.clear_a[i] = 0u;
    for (uint32_t i = blockIdx.x * blockDim.x + tid; i < a.clear_b_n; i += gridDim.x * blockDim.x) a.clear_b[i] = 0u;
}

template <int NV, bool STATS, bool THUMBS>
cudaError_t launch_table(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, cudaStream_t s)
{
    if (threads > kTableThreads<NV, THUMBS>) threads = kTableThreads<NV, THUMBS>;
    const size_t smem = (size_t)((STATS ? kHistWords : 0) + (THUMBS ? kThumbWords : 0)) * 4;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pass_b_table_kernel<NV, STATS, THUMBS>, g, a);
}

template <int NV, bool THUMBS>
cudaError_t launch_table_nv(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, cudaStream_t s)
{
    return a.frame_hist ? launch_table<NV, true, THUMBS>(g, a, grid, threads, s)
                        : launch_table<NV, false, THUMBS>(g, a, grid, threads, s);
}

// Shared memory of the statistics and thumbnail variants; the carveout
// leaves the rest of the SM's 256 KB to L1, which holds the coefficient
// words of the blocks a CTA works on.
template <int NV>
cudaError_t prepare_nv()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pass_b_table_kernel<NV, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kHistWords * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_table_kernel<NV, true, false>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout, 50)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_table_kernel<NV, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (kHistWords + kThumbWords) * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_table_kernel<NV, true, true>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout, 60)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(pass_b_table_kernel<NV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kThumbWords * 4);
}

// The coefficient table: one thread per (block j, chunk of 32 units,
// 4-column group g4, unit) of camera blockIdx.y writes the NV words of
// columns 16 ux + 4 g4 + 0..3 with col_coef (columns past the row end and
// units past the last one of a chunk: weight 0).  Consecutive threads write
// consecutive words.
template <int NV>
__global__ void __launch_bounds__(256) seam_coef_kernel(const ArrayGeom g, const int32_t *__restrict__ q16,
                                                        uint4 *__restrict__ coef)
{
    const int cam = blockIdx.y;
    const CamGeom &cg = g.cam[cam];
    const uint32_t nch = (cg.upr + 31) >> 5;
    const uint32_t local = blockIdx.x * blockDim.x + threadIdx.x;   // ((j nch + chunk) 4 + g4) 32 + l
    if (local >= (uint32_t)cg.nblk * nch * 128u) return;
    const int l = (int)(local & 31u), g4 = (int)((local >> 5) & 3u);
    const uint32_t jc = local >> 7;                                  // j nch + chunk
    const int j = (int)(jc / nch), ux = (int)(jc % nch) * 32 + l;
    const int half = cg.W >> 1, xg = ux * kUnitCols + 4 * g4;
    // the ramp table covers the last unit of a row (64 bytes of tail)
    const int4 w4 = ramp4(cg.ramp, min(xg, (int)cg.upr * kUnitCols - 4));
    const int wq[4] = {w4.x, w4.y, w4.z, w4.w};
    uint32_t w[NV][4];
    int m[NV];
    load_map(q16, cam, xg >= half ? 1 : 0, j, g.B, m);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = xg + q;
        if (xg < half && x == half) load_map(q16, cam, 1, j, g.B, m);
        ColCoef<NV> cc;
        col_coef(m, (x < cg.W ? wq[q] : 0) << 14, cc);
#pragma unroll
        for (int v = 0; v < NV - 3; ++v) w[v][q] = cc.A[v];
#pragma unroll
        for (int c = 0; c < 3; ++c) w[NV - 3 + c][q] = cc.cst[c];
    }
    uint4 *dst = coef + cg.coef_base + (size_t)jc * (4 * NV * 32) + g4 * NV * 32 + l;
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[32 * v] = make_uint4(w[v][0], w[v][1], w[v][2], w[v][3]);
}

}  // namespace

cudaError_t launch_seam_coef(const ArrayGeom &g, const int32_t *q16, int nv, uint4 *coef, cudaStream_t s)
{
    uint32_t most = 0;   // threads of the largest camera
    for (int k = 0; k < g.K; ++k) most = std::max(most, (uint32_t)g.cam[k].nblk * ((g.cam[k].upr + 31) >> 5) * 128u);
    const dim3 grid((most + 255) / 256, g.K);
    if (nv == 12) seam_coef_kernel<12><<<grid, 256, 0, s>>>(g, q16, coef);
    else seam_coef_kernel<6><<<grid, 256, 0, s>>>(g, q16, coef);
    return cudaGetLastError();
}

cudaError_t pass_b_table_prepare()
{
    cudaError_t e;
    if ((e = prepare_nv<6>()) != cudaSuccess) return e;
    return prepare_nv<12>();
}

cudaError_t launch_pass_b_table(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, cudaStream_t s)
{
    const bool thumbs = a.thumbs != nullptr;
    if (g.fit_mode == RT_FIT_MATRIX)
        return thumbs ? launch_table_nv<12, true>(g, a, grid, threads, s)
                      : launch_table_nv<12, false>(g, a, grid, threads, s);
    return thumbs ? launch_table_nv<6, true>(g, a, grid, threads, s) : launch_table_nv<6, false>(g, a, grid, threads, s);
}

}  // namespace rt
