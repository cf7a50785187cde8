// Device helpers shared by the pass B kernels (k_pass_b.cu: per-camera
// gains and the seam maps computed per unit; k_pass_b_table.cu: the seam maps
// read from a coefficient table): streaming loads, programmatic dependent
// launch, the lane-private histogram increments, the bit-exact conversion of
// 4 pixels, the Q16 application and packing, the seam maps' column
// coefficients along the ramp, thumbnail sums and the row stores.
#pragma once

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

// Programmatic dependent launch: the next pass B may be scheduled while this
// one runs (its CTAs take SMs as this grid's CTAs exit); it waits for this
// grid's completion, memory included, before touching the accumulators.
__device__ __forceinline__ void allow_next_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_prev_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void red_shared_inc(uint32_t addr)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}

// Histogram increment of channel C: the channel's 32 KB offset rides in the
// instruction's immediate address field.
template <int C>
__device__ __forceinline__ void red_shared_inc_c(uint32_t addr)
{
    asm volatile("red.shared.add.u32 [%0+%1], 1;" ::"r"(addr), "n"(C * 32768) : "memory");
}

__device__ __forceinline__ void hist_inc(uint32_t addr, int c)
{
    if (c == 0) red_shared_inc_c<0>(addr);
    else if (c == 1) red_shared_inc_c<1>(addr);
    else red_shared_inc_c<2>(addr);
}

// Apply constants of one row for the per-camera gain fit: t = a_q * vbits + cq
struct RowGain { uint32_t aq[3], cq[3]; };

// Two conversions' rounding step in one packed FP32x2 FMA:
// bits of (2^23 + 255 x) for x = z0, z1 (each already saturated to [0, 1]).
__device__ __forceinline__ void magic2(float z0, float z1, uint32_t &b0, uint32_t &b1)
{
    asm("{\n .reg .b64 a, k, m, r;\n"
        " mov.b64 a, {%2, %3};\n"
        " mov.b64 k, {%4, %4};\n"
        " mov.b64 m, {%5, %5};\n"
        " fma.rn.f32x2 r, a, k, m;\n"
        " mov.b64 {%0, %1}, r;\n}\n"
        : "=r"(b0), "=r"(b1) : "f"(z0), "f"(z1), "f"(255.0f), "f"(kMagic));
}

// Two values' float arithmetic in one packed FP32x2 instruction (the same
// round-to-nearest IEEE result per lane as the scalar instruction).
struct F2 { float x, y; };

__device__ __forceinline__ F2 fma2(F2 a, float k, F2 c)
{
    F2 d;
    asm("{\n .reg .b64 a, k, c, r;\n"
        " mov.b64 a, {%2, %3};\n"
        " mov.b64 k, {%4, %4};\n"
        " mov.b64 c, {%5, %6};\n"
        " fma.rn.f32x2 r, a, k, c;\n"
        " mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(k), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ F2 fma2(F2 a, float k, float c)
{
    F2 d;
    asm("{\n .reg .b64 a, k, c, r;\n"
        " mov.b64 a, {%2, %3};\n"
        " mov.b64 k, {%4, %4};\n"
        " mov.b64 c, {%5, %5};\n"
        " fma.rn.f32x2 r, a, k, c;\n"
        " mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(k), "f"(c));
    return d;
}

// Bytes i and j of w as floats (0..255): two PRMTs and one packed FADD that
// removes the 2^23 of the bit trick from both.
__device__ __forceinline__ F2 bytes_f2(uint32_t w, int i, int j)
{
    const uint32_t bi = __byte_perm(w, kMagicBits, 0x7440u | (uint32_t)i);
    const uint32_t bj = __byte_perm(w, kMagicBits, 0x7440u | (uint32_t)j);
    F2 d;
    asm("{\n .reg .b64 a, m, r;\n"
        " mov.b64 a, {%2, %3};\n"
        " mov.b64 m, {%4, %4};\n"
        " add.rn.f32x2 r, a, m;\n"
        " mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "r"(bi), "r"(bj), "f"(-kMagic));
    return d;
}

// Clamped output bytes of two applied values: t = 65536 v' + low bits, the
// result min(v', 255) (v' < 2^16).  Returns [min(t0>>16, 255), 0,
// min(t1>>16, 255), 0] -- one PRMT gathers the high halves, one packed
// 16-bit min clamps both.
__device__ __forceinline__ uint32_t clamp_hi2(uint32_t t0, uint32_t t1)
{
    const uint32_t hi = __byte_perm(t0, t1, 0x7632u);
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(hi), "r"(0x00FF00FFu));
    return r;
}

// The same for signed t (seam maps can give negative values): the high
// halves as signed 16-bit floor(t / 65536), clamped to [0, 255] by one packed
// min with ReLU.
__device__ __forceinline__ uint32_t clamp_hi2s(uint32_t t0, uint32_t t1)
{
    const uint32_t hi = __byte_perm(t0, t1, 0x7632u);
    uint32_t r;
    asm("min.relu.s16x2 %0, %1, %2;" : "=r"(r) : "r"(hi), "r"(0x00FF00FFu));
    return r;
}

// Bytes 0 and 2 of a and of b: [a.0, a.2, b.0, b.2].
__device__ __forceinline__ uint32_t even_bytes(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x6420u); }

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

// Seam maps along the ramp (Sec. "White balance and exposure correction":
// identity at the image centre, the full map at the border).  For column x
// with ramp weight w (Q16) and a map value m:
//   A = delta 65536 + floor((m - delta 65536) w / 65536),  Bq = floor(b_q w / 65536),
//   out = clamp(floor((sum A v + Bq + 32768) / 65536), 0, 255).
// floor(d w / 65536) is one 32-bit high multiply: mulhi(4 d, 16384 w) =
// floor(d w 2^16 / 2^32), exact while |4 d| < 2^31 and 16384 w <= 2^30 --
// |d| < 2^21 for slopes and matrix entries within the gain limits (<= 16)
// and |b_q| < 2^29 for offsets of 8-bit data; the map loads pre-shift d and b_q.
// Per column the coefficients fold the value bits' offset kMagicBits and the
// rounding term into one constant: t = sum_d A_d vbits_d + cst, output in
// byte 2 of t (t clamped to [0, 0xFFFFFF]).

// Affine map of one camera, side and row block, pre-shifted:
// m[2c] = 4 (a_q - 65536), m[2c+1] = 4 b_q (three 8-byte loads; a map starts on 24 bytes).
__device__ __forceinline__ void load_map6(const int32_t *__restrict__ q16, int cam, int side, int j, int B, int (&m)[6])
{
    const int2 *p = reinterpret_cast<const int2 *>(q16 + ((size_t)(cam * 2 + side) * B + j) * 6);
    const int2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    m[0] = (a.x - 65536) << 2; m[1] = a.y << 2;
    m[2] = (b.x - 65536) << 2; m[3] = b.y << 2;
    m[4] = (c.x - 65536) << 2; m[5] = c.y << 2;
}

// 3 x 3 map, pre-shifted: m[3c+d] = 4 (M_cd - delta_cd 65536), m[9+c] = 4 b_c
// (three 16-byte loads; a map starts on 48 bytes).
__device__ __forceinline__ void load_map12(const int32_t *__restrict__ q16, int cam, int side, int j, int B, int (&m)[12])
{
    const int4 *p = reinterpret_cast<const int4 *>(q16 + ((size_t)(cam * 2 + side) * B + j) * 12);
    const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    const int v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
    for (int i = 0; i < 12; ++i) m[i] = (v[i] - ((i == 0 || i == 4 || i == 8) ? 65536 : 0)) << 2;
}

// Ramp weights of 4 columns from x (a multiple of 4): one 16-byte load (each
// camera's ramp starts on 16 bytes and the table has 64 bytes of tail, enough
// for the last unit of a ragged row).
__device__ __forceinline__ int4 ramp4(const int32_t *__restrict__ ramp, int x)
{
    return __ldg(reinterpret_cast<const int4 *>(ramp + x));
}

__device__ __forceinline__ void load_map(const int32_t *__restrict__ q16, int cam, int side, int j, int B, int (&m)[6])
{
    load_map6(q16, cam, side, j, B, m);
}
__device__ __forceinline__ void load_map(const int32_t *__restrict__ q16, int cam, int side, int j, int B, int (&m)[12])
{
    load_map12(q16, cam, side, j, B, m);
}

// Column coefficients of a map: NV = 6 (affine: A_c, cst_c) or 12 (3 x 3:
// A_cd row-major, cst_c).  w14 = 16384 w.
template <int NV> struct ColCoef;
template <> struct ColCoef<6> { uint32_t A[3], cst[3]; };
template <> struct ColCoef<12> { uint32_t A[9], cst[3]; };

__device__ __forceinline__ void col_coef(const int (&m)[6], int w14, ColCoef<6> &o)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int A = 65536 + __mulhi(m[2 * c], w14);
        const int Bq = __mulhi(m[2 * c + 1], w14);
        o.A[c] = (uint32_t)A;
        o.cst[c] = (uint32_t)(Bq + 32768) - (uint32_t)A * kMagicBits;
    }
}

__device__ __forceinline__ void col_coef(const int (&m)[12], int w14, ColCoef<12> &o)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        uint32_t sumA = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int A = (c == d ? 65536 : 0) + __mulhi(m[3 * c + d], w14);
            o.A[3 * c + d] = (uint32_t)A;
            sumA += (uint32_t)A;
        }
        const int Bq = __mulhi(m[9 + c], w14);
        o.cst[c] = (uint32_t)(Bq + 32768) - sumA * kMagicBits;   // modulo 2^32
    }
}

// t = 65536 x (the unclamped result, as a signed 32-bit value) + low bits
// of one pixel's three value bits; clamp_hi2s turns pairs into bytes.
__device__ __forceinline__ void col_apply(const ColCoef<6> &k, const uint32_t (&vb)[3], uint32_t *t)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c] = k.A[c] * vb[c] + k.cst[c];
}

__device__ __forceinline__ void col_apply(const ColCoef<12> &k, const uint32_t (&vb)[3], uint32_t *t)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c] = k.A[3 * c] * vb[0] + k.A[3 * c + 1] * vb[1] + k.A[3 * c + 2] * vb[2] + k.cst[c];
}

// Output byte 2 of a seam-map value t, clamped (mono cameras, one value at a time).
__device__ __forceinline__ uint32_t clamp24(uint32_t t)
{
    const int v = (int)t;
    return (uint32_t)(v < 0 ? 0 : (v > 0xFFFFFF ? 0xFFFFFF : v));
}

// Thumbnail cell sums of a unit's R rows.  Cell (i, j) covers columns
// [floor(i W/64), floor((i+1) W/64)) and rows [floor(j H/36), floor((j+1)
// H/36)); th is the shared [36][64][3] u32 array.  The width class TH of the
// camera is fixed at compile time for the whole unit: on a camera at least
// 16 x 64 columns wide (TH = 1) a 16-column unit spans at most two cells --
// its columns before floor((c0 + 1) W/64), the first column of cell c0 + 1,
// lie in the cell c0 of its first column, the others in c0 + 1 -- so every
// row keeps, in registers, one sum per channel over its valid columns and
// one over those in c0, added to the cells at the end.  On a narrower camera
// (TH = 2) each value goes to its cell's shared word as it is converted.
// Sums of value bits wrap modulo 2^32; the n kMagicBits they carry are taken
// off at the end.
constexpr int kThumbWide = 1, kThumbNarrow = 2;

template <int R>
struct ThumbAcc {
    int c0, split;              // cell of the first column; columns of the unit in c0
    int off[R];                 // th offsets of the rows' cell rows
    uint32_t all[R][3], left[R][3];
};

// The width class of a camera's thumbnail sums (TH above).
__device__ __forceinline__ bool thumb_wide(const CamGeom &cg) { return cg.W >= kUnitCols * RT_THUMB_W; }

template <int TH, int R>
__device__ __forceinline__ void thumb_begin(ThumbAcc<R> &t, const CamGeom &cg, int y0, int x0)
{
#pragma unroll
    for (int r = 0; r < R; ++r) t.off[r] = block_of_row(y0 + r, cg.H, RT_THUMB_H) * RT_THUMB_W * 3;
    if constexpr (TH == kThumbWide) {
        t.c0 = (int)(((x0 + 1) * RT_THUMB_W - 1) / cg.W);
        t.split = (int)((t.c0 + 1) * cg.W / RT_THUMB_W) - x0;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) t.all[r][c] = t.left[r][c] = 0u;
    }
}

// Value bits vb of channel c of valid column x0 + i, row r of the unit.
template <int TH, int R>
__device__ __forceinline__ void thumb_add(ThumbAcc<R> &t, uint32_t *th, const CamGeom &cg, int r, int x0, int i,
                                          int c, uint32_t vb)
{
    if constexpr (TH == kThumbWide) {
        t.all[r][c] += vb;
        if (i < t.split) t.left[r][c] += vb;
    } else {
        const int cx = (int)(((x0 + i + 1) * RT_THUMB_W - 1) / cg.W);
        atomicAdd(th + t.off[r] + cx * 3 + c, vb - kMagicBits);
    }
}

// The rows' sums into their cells (nvalid valid columns).
template <int TH, int R>
__device__ __forceinline__ void thumb_end(const ThumbAcc<R> &t, uint32_t *th, int nvalid)
{
    if constexpr (TH == kThumbWide) {
        const int nl = min(t.split, nvalid), nr = nvalid - nl;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (nl > 0) atomicAdd(th + t.off[r] + t.c0 * 3 + c, t.left[r][c] - (uint32_t)nl * kMagicBits);
                if (nr > 0)
                    atomicAdd(th + t.off[r] + (t.c0 + 1) * 3 + c,
                              t.all[r][c] - t.left[r][c] - (uint32_t)nr * kMagicBits);
            }
    }
}

// Value bits of 4 pixels of one row (two chroma pairs, chroma terms czR,
// czG, czB of pairs 2 g4 and 2 g4 + 1): 12 saturated z rounded two at a time.
__device__ __forceinline__ void convert4(uint32_t yword, const ConvConsts &k, const F2 &czR, const F2 &czG,
                                         const F2 &czB, uint32_t (&vbq)[4][3])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {             // pixels 2h, 2h+1 share a chroma pair
        const F2 Yf = bytes_f2(yword, 2 * h, 2 * h + 1);
        const float czh[3] = {h ? czR.y : czR.x, h ? czG.y : czG.x, h ? czB.y : czB.x};
        float z0[3], z1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            z0[c] = __saturatef(fmaf(Yf.x, k.ky, czh[c]));
            z1[c] = __saturatef(fmaf(Yf.y, k.ky, czh[c]));
        }
        magic2(z0[0], z0[1], vbq[2 * h][0], vbq[2 * h][1]);
        magic2(z1[0], z1[1], vbq[2 * h + 1][0], vbq[2 * h + 1][1]);
        magic2(z0[2], z1[2], vbq[2 * h][2], vbq[2 * h + 1][2]);
    }
}

// Output stores: 256-bit (32-byte aligned p) and 128-bit, not allocating
// in L1 (the output is written once and never read back by the kernel;
// streaming it through L1 cost 5 % of pass B's time).
__device__ __forceinline__ void st_v8(uint8_t *p, const uint32_t (&w)[8])
{
    asm volatile("st.global.L1::no_allocate.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

__device__ __forceinline__ void st_v4(uint8_t *p, const uint4 &w)
{
    asm volatile("st.global.L1::no_allocate.v4.b32 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w) : "memory");
}

// The first nb bytes of a row's 12 output words, byte by byte (a ragged
// unit).  Every word is named by a compile-time index, so that the words stay
// in registers: a loop indexing them at run time puts the unit's output words
// in local memory, stored there for every unit.
__device__ __forceinline__ void put_ragged(const uint32_t (&w)[12], uint8_t *dst, int nb)
{
#pragma unroll
    for (int i = 0; i < 12; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * i + k < nb) dst[4 * i + k] = (uint8_t)(w[i] >> (8 * k));
}

// A full unit's two 48-byte rows, each as one 32-byte and one 16-byte store
// chosen by the row's alignment: at a 32-byte boundary bytes 0-31 then
// 32-47, 16 bytes past one bytes 16-47 then 0-15.  The 32-byte stores are
// whole sectors, and the 16-byte halves of two neighbouring units (the
// next lane's unit) share a sector and one store instruction, so the warp
// writes whole sectors (16 bytes every 48 would split every sector between
// two instructions).
__device__ __forceinline__ void store_unit(const uint32_t (&ow)[2][12], bool full, uint8_t *dst0, int pitch)
{
    if (!full) return;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        uint8_t *a = dst0 + (size_t)r * pitch;
        const bool odd = ((uintptr_t)a >> 4) & 1u;
        uint32_t w8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w8[i] = odd ? ow[r][4 + i] : ow[r][i];
        const uint4 w4 = odd ? make_uint4(ow[r][0], ow[r][1], ow[r][2], ow[r][3])
                             : make_uint4(ow[r][8], ow[r][9], ow[r][10], ow[r][11]);
        st_v8(a + (odd ? 16 : 0), w8);
        st_v4(a + (odd ? 0 : 32), w4);
    }
}

constexpr int kHistWords = 3 * 256 * kHistLanes;

constexpr int kThumbWords = RT_THUMB_H * RT_THUMB_W * 3;

}  // namespace

}  // namespace rt
