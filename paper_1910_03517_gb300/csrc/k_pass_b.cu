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
#include <algorithm>

#include <cuda_bf16.h>

#include "pass_b.cuh"

namespace rt {

namespace {

// TH: no thumbnails (0) or the camera's thumbnail width class (pass_b.cuh).
template <int FIT, bool STATS, bool FULL, int TH>
__device__ __forceinline__ void unit_nv12(const CamGeom &cg, int cam, int rp, int ux, const ConvConsts &k,
                                          const int32_t *__restrict__ q16, int B, uint32_t hbase, uint32_t *th,
                                          bool seg, uint32_t sa0, uint32_t sa1, uint32_t sa2,
                                          const uint4 Y0, const uint4 Y1, const uint4 UV, uint32_t (&ow)[2][12])
{
    const int x0 = ux * kUnitCols;
    const int y0 = rp * 2;
    const uint32_t yw[2][4] = {{Y0.x, Y0.y, Y0.z, Y0.w}, {Y1.x, Y1.y, Y1.z, Y1.w}};
    const uint32_t uvw[4] = {UV.x, UV.y, UV.z, UV.w};
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
    int jr[2] = {0, 0};
    RowGain rg[2];
    if (FIT == RT_FIT_GLOBAL) {
        if (seg) {
            // one block: the camera's gains, from the segment
            rg[0].aq[0] = sa0; rg[0].aq[1] = sa1; rg[0].aq[2] = sa2;
#pragma unroll
            for (int c = 0; c < 3; ++c) rg[0].cq[c] = 32768u - rg[0].aq[c] * kMagicBits;
            rg[1] = rg[0];
        } else {
            jr[0] = block_of_row(y0, cg.H, cg.nblk);
            jr[1] = block_of_row(y0 + 1, cg.H, cg.nblk);
            rg[0] = row_gain(q16, cam, jr[0], B);
            rg[1] = (jr[1] == jr[0]) ? rg[0] : row_gain(q16, cam, jr[1], B);
        }
    } else {
        jr[0] = block_of_row(y0, cg.H, cg.nblk);
        jr[1] = block_of_row(y0 + 1, cg.H, cg.nblk);
    }
    constexpr bool THUMBS = TH != 0;
    [[maybe_unused]] ThumbAcc<2> ta;
    if constexpr (THUMBS) thumb_begin<TH>(ta, cg, y0, x0);

#pragma unroll
    for (int g4 = 0; g4 < 4; ++g4) {                  // pixels 4 g4 .. 4 g4 + 3
        // chroma pairs 2 g4, 2 g4 + 1: (U, V) bytes 0, 1 and 2, 3 of the word,
        // both pairs' chroma terms at once in packed FP32x2
        const F2 Uf = bytes_f2(uvw[g4], 0, 2), Vf = bytes_f2(uvw[g4], 1, 3);
        const F2 czR = fma2(Vf, k.krv, k.c_r0);
        const F2 czG = fma2(Uf, k.kgu, fma2(Vf, k.kgv, k.c_g0));
        const F2 czB = fma2(Uf, k.kbu, k.c_b0);
        const float cz[2][3] = {{czR.x, czG.x, czB.x}, {czR.y, czG.y, czB.y}};
        if constexpr (FIT == RT_FIT_GLOBAL) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint32_t t[12];
                // conversion of the 4 pixels: luma pairs as packed floats,
                // 12 saturated z, rounded two at a time
                uint32_t vbq[4][3];
                convert4(yw[r][g4], k, czR, czG, czB, vbq);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * g4 + q;
                    const uint32_t *vb = vbq[q];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const bool live = FULL || i < nvalid;
                        if constexpr (THUMBS) {
                            if (live) thumb_add<TH>(ta, th, cg, r, x0, i, c, vb[c]);
                        }
                        if (STATS && live) hist_inc(hbase + vb[c] * 128u, c);
                        t[3 * q + c] = rg[r].aq[c] * vb[c] + rg[r].cq[c];   // 65536 out + low bits, unclamped
                    }
                }
                // clamp to 255 and pack: [R0 G0 B0 R1] [G1 B1 R2 G2] [B2 R3 G3 B3]
                ow[r][3 * g4 + 0] = even_bytes(clamp_hi2(t[0], t[1]), clamp_hi2(t[2], t[3]));
                ow[r][3 * g4 + 1] = even_bytes(clamp_hi2(t[4], t[5]), clamp_hi2(t[6], t[7]));
                ow[r][3 * g4 + 2] = even_bytes(clamp_hi2(t[8], t[9]), clamp_hi2(t[10], t[11]));
            }
        } else {
            // conversion of the 4 pixels of both rows: 12 saturated z per row,
            // rounded two at a time
            uint32_t vbq[2][4][3];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int h = 0; h < 2; ++h) {             // pixels 2h, 2h+1 share a chroma pair
                    const F2 Yf = bytes_f2(yw[r][g4], 2 * h, 2 * h + 1);
                    float z0[3], z1[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        z0[c] = __saturatef(fmaf(Yf.x, k.ky, cz[h][c]));
                        z1[c] = __saturatef(fmaf(Yf.y, k.ky, cz[h][c]));
                    }
                    magic2(z0[0], z0[1], vbq[r][2 * h][0], vbq[r][2 * h][1]);
                    magic2(z1[0], z1[1], vbq[r][2 * h + 1][0], vbq[r][2 * h + 1][1]);
                    magic2(z0[2], z1[2], vbq[r][2 * h][2], vbq[r][2 * h + 1][2]);
                }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * g4 + q;
                    const bool live = FULL || i < nvalid;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        if constexpr (THUMBS) {
                            if (live) thumb_add<TH>(ta, th, cg, r, x0, i, c, vbq[r][q][c]);
                        }
                        if (STATS && live) hist_inc(hbase + vbq[r][q][c] * 128u, c);
                    }
                }
            uint32_t t[2][12];
            // seam maps: the coefficients of a column serve both rows unless
            // the row pair straddles a block boundary; one map load per group
            // of 4 columns, another where the group crosses the image centre
            constexpr int NV = FIT == RT_FIT_MATRIX ? 12 : 6;
            const int half = cg.W >> 1, xg = x0 + 4 * g4;
            int m[NV];
            load_map(q16, cam, xg >= half ? 1 : 0, jr[0], B, m);
            const int4 w4 = ramp4(cg.ramp, xg);
            const int wq[4] = {w4.x << 14, w4.y << 14, w4.z << 14, w4.w << 14};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (xg < half && xg + q == half) load_map(q16, cam, 1, jr[0], B, m);
                ColCoef<NV> cc;
                col_coef(m, wq[q], cc);
                col_apply(cc, vbq[0][q], &t[0][3 * q]);
                if (jr[1] == jr[0]) {
                    col_apply(cc, vbq[1][q], &t[1][3 * q]);
                } else {
                    int m1[NV];
                    load_map(q16, cam, xg + q >= half ? 1 : 0, jr[1], B, m1);
                    ColCoef<NV> c1;
                    col_coef(m1, wq[q], c1);
                    col_apply(c1, vbq[1][q], &t[1][3 * q]);
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                ow[r][3 * g4 + 0] = even_bytes(clamp_hi2s(t[r][0], t[r][1]), clamp_hi2s(t[r][2], t[r][3]));
                ow[r][3 * g4 + 1] = even_bytes(clamp_hi2s(t[r][4], t[r][5]), clamp_hi2s(t[r][6], t[r][7]));
                ow[r][3 * g4 + 2] = even_bytes(clamp_hi2s(t[r][8], t[r][9]), clamp_hi2s(t[r][10], t[r][11]));
            }
        }
    }
    if constexpr (THUMBS) {
        thumb_end<TH>(ta, th, nvalid);
    }
    // a full unit's 48 bytes per row go out through store_unit; a ragged one
    // writes its bytes here
    if (!FULL) {
        if constexpr (FIT == RT_FIT_GLOBAL && STATS && TH == 0) {
            // this instance keeps its words in registers either way, and the
            // unrolled stores would cost it registers
            for (int r = 0; r < 2; ++r) {
                uint8_t *dst = cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0;
                for (int b = 0; b < 3 * nvalid; ++b) dst[b] = (uint8_t)(ow[r][b >> 2] >> (8 * (b & 3)));
            }
        } else {
#pragma unroll
            for (int r = 0; r < 2; ++r)
                put_ragged(ow[r], cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0, 3 * nvalid);
        }
    }
}

template <int FIT, bool STATS, bool FULL, int TH>
__device__ __forceinline__ void unit_mono(const CamGeom &cg, int cam, int rp, int ux,
                                          const int32_t *__restrict__ q16, int B, uint32_t hbase, uint32_t *th,
                                          uint32_t (&ow)[2][12])
{
    const int x0 = ux * kUnitCols;
    const int y0 = rp * 2;
    const int nvalid = FULL ? kUnitCols : (cg.W - x0);
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
        const int j = block_of_row(y0 + r, cg.H, cg.nblk);
        RowGain rg;
        if (FIT == RT_FIT_GLOBAL) rg = row_gain(q16, cam, j, B);
        constexpr int NV = FIT == RT_FIT_MATRIX ? 12 : 6;
        int mm[NV];
        int mside = -1;
        [[maybe_unused]] ThumbAcc<1> ta;
        if constexpr (TH != 0) thumb_begin<TH>(ta, cg, y0 + r, x0);
#pragma unroll
        for (int i = 0; i < kUnitCols; ++i) {
            if (!FULL && i >= nvalid) continue;
            const uint32_t vb = mono_bits((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu, cg.shift);
            if constexpr (TH != 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) thumb_add<TH>(ta, th, cg, 0, x0, i, c, vb);
            }
            if constexpr (FIT != RT_FIT_GLOBAL) {
                const int side = x0 + i >= (cg.W >> 1) ? 1 : 0;
                if (side != mside) {
                    load_map(q16, cam, side, j, B, mm);
                    mside = side;
                }
                ColCoef<NV> cc;
                col_coef(mm, __ldg(cg.ramp + x0 + i) << 14, cc);
                const uint32_t v3[3] = {vb, vb, vb};
                uint32_t t3[3];
                col_apply(cc, v3, t3);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (STATS) hist_inc(hbase + vb * 128u, c);
                    const int bb = 3 * i + c;
                    ow[r][bb >> 2] = put_byte2(ow[r][bb >> 2], clamp24(t3[c]), bb & 3);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (STATS) hist_inc(hbase + vb * 128u, c);
                    uint32_t t = rg.aq[c] * vb + rg.cq[c];
                    t = t > 0xFFFFFFu ? 0xFFFFFFu : t;
                    const int bb = 3 * i + c;
                    ow[r][bb >> 2] = put_byte2(ow[r][bb >> 2], t, bb & 3);
                }
            }
        }
        if constexpr (TH != 0) thumb_end<TH>(ta, th, nvalid);
    }
    // a full unit's 48 bytes per row go out through store_unit; a ragged one
    // writes its bytes here
    if (!FULL) {
        if constexpr (FIT == RT_FIT_GLOBAL && STATS && TH == 0) {
            // this instance keeps its words in registers either way, and the
            // unrolled stores would cost it registers
            for (int r = 0; r < 2; ++r) {
                uint8_t *dst = cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0;
                for (int b = 0; b < 3 * nvalid; ++b) dst[b] = (uint8_t)(ow[r][b >> 2] >> (8 * (b & 3)));
            }
        } else {
#pragma unroll
            for (int r = 0; r < 2; ++r)
                put_ragged(ow[r], cg.rgb + (size_t)(y0 + r) * cg.rgb_pitch + 3 * x0, 3 * nvalid);
        }
    }
}

// A unit with the camera's thumbnail width class (wide: TH = kThumbWide,
// else kThumbNarrow), or without thumbnails.
template <int FIT, bool STATS, bool FULL, bool THUMBS, typename... A>
__device__ __forceinline__ void unit_nv12_th(bool wide, A &&...args)
{
    if constexpr (!THUMBS) unit_nv12<FIT, STATS, FULL, 0>(args...);
    else if (wide) unit_nv12<FIT, STATS, FULL, kThumbWide>(args...);
    else unit_nv12<FIT, STATS, FULL, kThumbNarrow>(args...);
}

template <int FIT, bool STATS, bool FULL, bool THUMBS, typename... A>
__device__ __forceinline__ void unit_mono_th(bool wide, A &&...args)
{
    if constexpr (!THUMBS) unit_mono<FIT, STATS, FULL, 0>(args...);
    else if (wide) unit_mono<FIT, STATS, FULL, kThumbWide>(args...);
    else unit_mono<FIT, STATS, FULL, kThumbNarrow>(args...);
}

// The thumbnail variants get the registers of one CTA per SM, the seam maps
// those of RT_PASS_B_SEAM_CTAS_PER_SM.
template <int FIT, bool THUMBS>
constexpr int kMaxThreads = THUMBS ? 512 : (FIT == RT_FIT_GLOBAL ? RT_PASS_B_THREADS : RT_PASS_B_SEAM_THREADS);
template <int FIT, bool THUMBS>
constexpr int kMinCtas = THUMBS ? 1 : (FIT == RT_FIT_GLOBAL ? RT_PASS_B_CTAS_PER_SM : RT_PASS_B_SEAM_CTAS_PER_SM);

template <int FIT, bool STATS, bool THUMBS>
__global__ void __launch_bounds__(kMaxThreads<FIT, THUMBS>, kMinCtas<FIT, THUMBS>)
pass_b_kernel(const ArrayGeom g, const PassBArgs a)
{
    extern __shared__ uint32_t sh[];
    uint32_t *th = sh + (STATS ? kHistWords : 0);   // [36][64][3] cell sums (THUMBS)
    const int tid = threadIdx.x, lane = tid & 31;
    const ConvConsts &k = g.conv;
    allow_next_launch();
    // balanced contiguous slices: q units each, the first r slices one more
    const uint32_t q = g.units_total / gridDim.x, r = g.units_total - q * gridDim.x;
    uint32_t ub = blockIdx.x * q + min(blockIdx.x, r);
    const uint32_t ue = ub + q + (blockIdx.x < r ? 1u : 0u);
    int cam = 0;
    while (cam + 1 < g.K && g.cam[cam + 1].unit_base <= ub) ++cam;
    const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(sh) + (uint32_t)(tid & 31) * 4u -
                           kMagicBits * 128u;
    while (ub < ue) {
        const CamGeom &cg = g.cam[cam];
        const uint32_t cam_end = cam + 1 < g.K ? g.cam[cam + 1].unit_base : g.units_total;
        const uint32_t se = ue < cam_end ? ue : cam_end;
        if (STATS || THUMBS) {
            uint4 *s4 = reinterpret_cast<uint4 *>(sh);
            const int words = (STATS ? kHistWords : 0) + (THUMBS ? kThumbWords : 0);
            for (int i = tid; i < words / 4; i += blockDim.x) s4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
        }
        const int upr = (int)cg.upr;
        const int full_units = cg.W / kUnitCols;
        const bool twide = THUMBS && thumb_wide(cg);
        // per-camera gains hoisted out of the unit loop when there is one block
        const bool seg = FIT == RT_FIT_GLOBAL && g.B == 1;
        uint32_t sa0 = 0, sa1 = 0, sa2 = 0;
        if (seg) {
            const int32_t *m = a.q16 + (size_t)cam * 2 * 6;
            sa0 = (uint32_t)__ldg(m);
            sa1 = (uint32_t)__ldg(m + 2);
            sa2 = (uint32_t)__ldg(m + 4);
        }
        // (row pair, unit) of this thread's first unit, then stepped by blockDim
        const int first = (int)(ub - cg.unit_base) + tid;
        int rp = first / upr, ux = first - rp * upr;
        const int srp = (int)blockDim.x / upr, sux = (int)blockDim.x - srp * upr;
        const int nloc = (int)(se - cg.unit_base);
        // lane l of a warp handles unit base + l while that is below nloc
        uint32_t ow[2][12];
        if (cg.fmt == RT_NV12) {
            for (int base = first - lane; base < nloc; base += blockDim.x) {
                bool full = false;
                uint8_t *dst0 = nullptr;
                if (base + lane < nloc) {
                    const uint8_t *yp = cg.y + (size_t)(2 * rp) * cg.y_pitch + ux * kUnitCols;
                    const uint4 Y0 = ld_stream(yp), Y1 = ld_stream(yp + cg.y_pitch);
                    const uint4 UV = ld_stream(cg.uv + (size_t)rp * cg.uv_pitch + ux * kUnitCols);
                    if (ux < full_units) {
                        unit_nv12_th<FIT, STATS, true, THUMBS>(twide, cg, cam, rp, ux, k, a.q16, g.B, hbase, th, seg,
                                                                 sa0, sa1, sa2, Y0, Y1, UV, ow);
                        full = true;
                        dst0 = cg.rgb + (size_t)(2 * rp) * cg.rgb_pitch + 3 * kUnitCols * ux;
                    } else {
                        unit_nv12_th<FIT, STATS, false, THUMBS>(twide, cg, cam, rp, ux, k, a.q16, g.B, hbase, th, seg,
                                                                 sa0, sa1, sa2, Y0, Y1, UV, ow);
                    }
                }
                store_unit(ow, full, dst0, cg.rgb_pitch);
                ux += sux;
                rp += srp;
                if (ux >= upr) {
                    ux -= upr;
                    ++rp;
                }
            }
        } else {
            for (int base = first - lane; base < nloc; base += blockDim.x) {
                bool full = false;
                uint8_t *dst0 = nullptr;
                if (base + lane < nloc) {
                    if (ux < full_units) {
                        unit_mono_th<FIT, STATS, true, THUMBS>(twide, cg, cam, rp, ux, a.q16, g.B, hbase, th, ow);
                        full = true;
                        dst0 = cg.rgb + (size_t)(2 * rp) * cg.rgb_pitch + 3 * kUnitCols * ux;
                    } else {
                        unit_mono_th<FIT, STATS, false, THUMBS>(twide, cg, cam, rp, ux, a.q16, g.B, hbase, th, ow);
                    }
                }
                store_unit(ow, full, dst0, cg.rgb_pitch);
                ux += sux;
                rp += srp;
                if (ux >= upr) {
                    ux -= upr;
                    ++rp;
                }
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
        ub = se;
        ++cam;
    }
    // clear the accumulators the next frame set will use (other parity);
    // the previous pass B flushed its sums into them
    wait_prev_grid();
    for (uint32_t i = blockIdx.x * blockDim.x + tid; i < a.clear_a_n; i += gridDim.x * blockDim.x) a.clear_a[i] = 0u;
    for (uint32_t i = blockIdx.x * blockDim.x + tid; i < a.clear_b_n; i += gridDim.x * blockDim.x) a.clear_b[i] = 0u;
}

template <int FIT, bool STATS, bool THUMBS>
cudaError_t launch_one(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, cudaStream_t s)
{
    if (threads > kMaxThreads<FIT, THUMBS>) threads = kMaxThreads<FIT, THUMBS>;
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
    return cudaLaunchKernelEx(&cfg, pass_b_kernel<FIT, STATS, THUMBS>, g, a);
}

template <int FIT>
cudaError_t prepare_fit()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<FIT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kHistWords * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<FIT, true, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  100)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<FIT, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (kHistWords + kThumbWords) * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pass_b_kernel<FIT, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kThumbWords * 4)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

// Surrogate input features: x[k][c][j][i] = bf16(float(sum / area / 255 - 0.5))
// with the division done in double (cell area from the camera's size).
__global__ void thumb_features_kernel(const ArrayGeom g, const uint32_t *__restrict__ thumbs,
                                      __nv_bfloat16 *__restrict__ out)
{
    const int k = blockIdx.y;
    const CamGeom &cg = g.cam[k];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kThumbWords; e += gridDim.x * blockDim.x) {
        const int i = e % RT_THUMB_W, j = (e / RT_THUMB_W) % RT_THUMB_H;
        const long long cw = ((long long)(i + 1) * cg.W) / RT_THUMB_W - ((long long)i * cg.W) / RT_THUMB_W;
        const long long ch = ((long long)(j + 1) * cg.H) / RT_THUMB_H - ((long long)j * cg.H) / RT_THUMB_H;
        const double v = (double)thumbs[(size_t)k * kThumbWords + e] / (double)(cw * ch) / 255.0 - 0.5;
        out[(size_t)k * kThumbWords + e] = __float2bfloat16_rn((float)v);
    }
}

cudaError_t launch_thumb_features(const ArrayGeom &g, const uint32_t *thumbs, void *out, cudaStream_t s)
{
    dim3 grid(8, g.K);
    thumb_features_kernel<<<grid, 256, 0, s>>>(g, thumbs, static_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError();
}

cudaError_t pass_b_prepare(int threads, size_t *smem_bytes)
{
    (void)threads;
    cudaError_t e;
    if ((e = prepare_fit<RT_FIT_GLOBAL>()) != cudaSuccess) return e;
    if ((e = prepare_fit<RT_FIT_SEAM_AFFINE>()) != cudaSuccess) return e;
    if ((e = prepare_fit<RT_FIT_MATRIX>()) != cudaSuccess) return e;
    *smem_bytes = (size_t)kHistWords * 4;
    return cudaSuccess;
}

cudaError_t launch_pass_b(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, size_t smem,
                          cudaStream_t s)
{
    (void)smem;
    const bool stats = a.frame_hist != nullptr, thumbs = a.thumbs != nullptr;
    if (g.fit_mode == RT_FIT_GLOBAL) {
        if (thumbs) return stats ? launch_one<RT_FIT_GLOBAL, true, true>(g, a, grid, threads, s)
                                 : launch_one<RT_FIT_GLOBAL, false, true>(g, a, grid, threads, s);
        return stats ? launch_one<RT_FIT_GLOBAL, true, false>(g, a, grid, threads, s)
                     : launch_one<RT_FIT_GLOBAL, false, false>(g, a, grid, threads, s);
    }
    if (g.fit_mode == RT_FIT_MATRIX) {
        if (thumbs) return stats ? launch_one<RT_FIT_MATRIX, true, true>(g, a, grid, threads, s)
                                 : launch_one<RT_FIT_MATRIX, false, true>(g, a, grid, threads, s);
        return stats ? launch_one<RT_FIT_MATRIX, true, false>(g, a, grid, threads, s)
                     : launch_one<RT_FIT_MATRIX, false, false>(g, a, grid, threads, s);
    }
    if (thumbs) return stats ? launch_one<RT_FIT_SEAM_AFFINE, true, true>(g, a, grid, threads, s)
                             : launch_one<RT_FIT_SEAM_AFFINE, false, true>(g, a, grid, threads, s);
    return stats ? launch_one<RT_FIT_SEAM_AFFINE, true, false>(g, a, grid, threads, s)
                 : launch_one<RT_FIT_SEAM_AFFINE, false, false>(g, a, grid, threads, s);
}

}  // namespace rt
