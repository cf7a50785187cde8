// Internal types shared by the kernels and the host runtime of librt.so.
// Everything a kernel needs per frame set travels by value in its parameter
// block (constant bank): camera geometry, this frame set's plane addresses,
// output addresses.  No per-frame host->device table copy is needed.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/rt.h"

namespace rt {

// Pass B (per-camera gains) is compiled for RT_PASS_B_CTAS_PER_SM CTAs of
// RT_PASS_B_THREADS threads per SM (64 registers a thread) and runs, by
// default, as a persistent grid of RT_PASS_B_RUN_CTAS CTAs per SM of
// RT_PASS_B_RUN_THREADS threads; each CTA holds its own 96 KB of histograms.
// The launch shape is a tuning parameter (rt_autotune).  With the output
// stores bypassing L1, one CTA of 512 threads per SM, next to 64-thread
// band-statistics CTAs, ran tower12 at 952k Mpix/s against 891k for two CTAs
// of 352 threads: the registers left per SM let the next frame set's
// statistics chain run beside pass B instead of waiting for its CTAs.
#ifndef RT_PASS_B_THREADS
#define RT_PASS_B_THREADS 512
#endif
#ifndef RT_PASS_B_CTAS_PER_SM
#define RT_PASS_B_CTAS_PER_SM 2
#endif
#ifndef RT_PASS_B_RUN_THREADS
#define RT_PASS_B_RUN_THREADS 512
#endif
#ifndef RT_PASS_B_RUN_CTAS
#define RT_PASS_B_RUN_CTAS 1
#endif
// Default threads of the pass B variants compiled for 128 registers (one CTA
// per SM): thumbnails, and the seam maps computed per unit.
#ifndef RT_PASS_B_WIDE_RUN_THREADS
#define RT_PASS_B_WIDE_RUN_THREADS 352
#endif

// The seam-map variants of pass B over units (blended per-row maps, or seam
// maps beside the thumbnails; per-column coefficients of both rows of a unit
// in registers) run RT_PASS_B_SEAM_CTAS_PER_SM CTAs of at most
// RT_PASS_B_SEAM_THREADS threads per SM.
#ifndef RT_PASS_B_SEAM_THREADS
#define RT_PASS_B_SEAM_THREADS 512
#endif
#ifndef RT_PASS_B_SEAM_CTAS_PER_SM
#define RT_PASS_B_SEAM_CTAS_PER_SM 1
#endif
// The table variant of pass B (seam maps per block) runs one CTA per SM:
// the affine maps' kernel (96 registers) with RT_PASS_B_TABLE6_RUN_THREADS
// threads, the 3 x 3 maps' (128 registers) with RT_PASS_B_TABLE12_RUN_THREADS;
// more threads speed pass B up but leave the next frame set's statistics
// chain no registers beside it.
#ifndef RT_PASS_B_TABLE12_RUN_THREADS
#define RT_PASS_B_TABLE12_RUN_THREADS 384
#endif
#ifndef RT_PASS_B_TABLE6_RUN_THREADS
#define RT_PASS_B_TABLE6_RUN_THREADS 512
#endif

constexpr int kUnitCols = 16;          // columns a thread converts per row
// Tile of a warp in the table variant of pass B: 4 row pairs x 8 units
// (8 rows x 128 columns); lane l takes row pair l / 8, unit l % 8.
constexpr int kTileRowPairs = 4, kTileUnits = 8;

// Values of one (camera, side, block) map: 3 channels x (a, b), or a 3 x 3
// cross-channel matrix (row-major) and its offset vector.
__host__ __device__ constexpr int map_vals(int fit_mode) { return fit_mode == RT_FIT_MATRIX ? 12 : 6; }
constexpr int kHistLanes = 32;         // lane-private copies of each histogram bin

struct CamGeom {
    const uint8_t *y;       // Y plane (NV12) or 16-bit mono plane, this frame set
    const uint8_t *uv;      // interleaved UV plane (NV12)
    uint8_t *rgb;           // corrected RGB24 output
    int32_t W, H, y_pitch, uv_pitch, rgb_pitch;
    int32_t fmt, shift;     // shift = bit_depth - 8 for mono
    int32_t nblk;           // blocks of this camera's rows in the applied map table
                            // (B; H when the table holds one map per row)
    uint32_t upr;           // units per row pair = ceil(W / 16)
    uint32_t unit_base;     // first unit of this camera in the array's unit space
    // table variant of pass B (seam maps per block): a warp takes a tile of
    // kTileRowPairs x kTileUnits units; ntr x ntc tiles per camera
    uint32_t tile_base;     // first tile of this camera in the array's tile space
    int32_t ntr, ntc;       // tiles per column (ceil(H / 2 / kTileRowPairs)), per row (ceil(upr / kTileUnits))
    uint32_t coef_base;     // first 16-byte word of this camera in a coefficient table
    const int32_t *ramp;    // Q16 ramp weight per column (seam maps)
};

// Colour-conversion constants (see pixel.cuh), computed on the host: the
// GB300's FP64 pipe is narrow, so device code never derives them itself.
struct ConvConsts {
    float ky;                    // 298 / 65280
    float krv, c_r0;             // z_R chroma part: V * krv + c_r0
    float kgu, kgv, c_g0;        // z_G chroma part: U * kgu + V * kgv + c_g0
    float kbu, c_b0;             // z_B chroma part: U * kbu + c_b0
};

struct ArrayGeom {
    CamGeom cam[RT_MAX_CAMERAS];
    ConvConsts conv;
    int32_t K, B, fit_mode, matrix;
    uint32_t units_total;   // sum over cameras of (H/2) * upr
    uint32_t tiles_total;   // table variant: sum over cameras of ntr * ntc
};

// Pass B: conversion + whole-frame statistics + Q16 application.
struct PassBArgs {
    const int32_t *q16;       // [K][2][B][3][2]
    const uint4 *coef;        // table variant: column coefficients of q16 (launch_seam_coef)
    uint32_t *frame_hist;     // [K][3][256] (nullptr: statistics off)
    uint32_t *thumbs;         // [K][3][36][64] (nullptr: off)
    // the next frame set's accumulators (the other parity), cleared here
    uint32_t *clear_a; uint32_t clear_a_n;
    uint32_t *clear_b; uint32_t clear_b_n;
};

// Pass A work item: one camera side, rows [row0, row1) all inside block j.
struct StripItem { int16_t cam, side, block, pad; int32_t row0, row1; };

struct PassAArgs {
    const StripItem *items;
    int32_t n_items, S, T, first;
    const uint8_t *prev_luma;   // [K][2][H][S] of the previous frame set
    uint8_t *cur_luma;          // [K][2][H][S] written for the next one
    int32_t luma_cam_stride;    // bytes per camera in the luma buffers (2 * Hmax * S)
    uint32_t *hist;             // [K][2][B][3][256]
    uint32_t *n;                // [K][2][B][3]
    unsigned long long *sum, *sumsq;
    unsigned long long *joint;  // [K][2][B][10] joint moments (3 x 3 maps), or nullptr
    // the other slot's statistics (read by the previous solve), cleared here
    // for the next frame set
    uint32_t *clear_u32; size_t clear_u32_n;
    unsigned long long *clear_u64; size_t clear_u64_n;
    // surrogate mode (nullptr otherwise): gate[0] = run the statistics,
    // gate[1] = the motion test may use prev_luma
    const int32_t *gate;
};

// Tables of the table-driven logarithm and exponential of the gain solve
// (filled on the host by launch_solve): c_i = 1 + (i + 1/2) / 128.
struct SolveTables {
    double invc[128];     // 1 / c_i
    double logc[128];     // ln c_i
    double exp2j[64];     // 2^(j / 64)
};

// The seam chains in a form the solve reads from its parameter block (no
// dependent loads): chain g holds member[gstart[g] .. gstart[g + 1]), by
// position; right[k] is the camera whose left band meets camera k's right
// band (-1 none) and rpos[k] its position in the chain.
struct SolveTopo {
    int8_t gstart[RT_MAX_CAMERAS + 1];
    int8_t member[RT_MAX_CAMERAS];
    int8_t right[RT_MAX_CAMERAS];
    int8_t rpos[RT_MAX_CAMERAS];
    int32_t H[RT_MAX_CAMERAS];
};

// Fills t from the chain arrays of the host (group_start[n_groups + 1],
// group_members, right_nbr[K], cam_H[K]).
void fill_solve_topo(SolveTopo &t, int K, int n_groups, const int32_t *group_start, const int32_t *group_members,
                     const int32_t *right_nbr, const int32_t *cam_H);

// Solve: fit + smoothing + quantisation.
struct SolveArgs {
    const uint32_t *hist;      // [K][2][B][3][256] band histograms (quantile fit)
    const uint32_t *n;
    const unsigned long long *sum, *sumsq;
    const unsigned long long *joint;   // [K][2][B][10] joint moments (3 x 3 maps)
    // [K][2][B][3][2] = (a, b) per channel, or [K][2][B][12] = (M row-major, b)
    // for the 3 x 3 maps
    double *maps_new;          // this frame set's estimate
    double *E;                 // smoothed estimate (state)
    int32_t *q16;
    int32_t K, B, S, fit_mode, min_valid, first;
    double alpha, lambda, gmin, gmax;
    // seam chains
    int32_t n_groups;
    const int32_t *group_start;   // [n_groups + 1] offsets into group_members
    const int32_t *group_members; // cameras of each chain, by position
    const int32_t *left_nbr;      // [K] camera whose right band meets my left band, -1 none
    const int32_t *right_nbr;     // [K]
    const int32_t *cam_H;         // [K]
    SolveTopo topo;               // the same chains, by value
    // surrogate mode: skip the fit unless gate[0] (nullptr: always fit); with
    // fit_only the per-camera gain fit writes maps_new only
    const int32_t *gate;
    int32_t fit_only;
    // filled by launch_solve
    SolveTables tab;
    double one_m_alpha;           // 1 - alpha
    double xlo, xhi;              // log-gain range kept before the exponential
    float xlo_f, xhi_f;
};

// Difference attention (k_attention.cu).
struct AttnArgs {
    const uint8_t *prev;                    // previous frame set's luma copies (nullptr: first frame set)
    uint8_t *cur;                           // this frame set's copies
    uint32_t *cells;                        // on-pixel counts per cell, camera k from cell_off[k]
    rt_crop *out;                           // proposals [max]
    int32_t *count;                         // number of proposals
    int32_t T, cell, min_on, max;
    uint32_t unit_base[RT_MAX_CAMERAS + 1]; // 16-byte row pieces: H * ceil(W / 16) per camera
    uint32_t cell_off[RT_MAX_CAMERAS + 1];
    uint32_t win_base[RT_MAX_CAMERAS + 1];  // windows max(ncx - 1, 1) * max(ncy - 1, 1) per camera
    int32_t ncx[RT_MAX_CAMERAS], ncy[RT_MAX_CAMERAS];
    size_t copy_off[RT_MAX_CAMERAS];
    int32_t copy_pitch[RT_MAX_CAMERAS];     // ceil(W / 16) * 16
};

struct CropArgs {
    const rt_crop *crops;     // device copy of this frame set's windows
    int32_t n, S;
    __half *out;              // [n][3][S][S]
    const int32_t *count;     // device count of valid windows (nullptr: all n)
};

// A synthetic frame set painted on the device (k_synth.cu): the learned
// surrogate's training and evaluation arrays.  Each camera sees its slice of
// a panorama (sky above a wavy horizon, smooth gradients, low-frequency
// sinusoids), scaled by its per-channel gain, with Gaussian noise, rounded to
// 8 bits and encoded as BT.709 limited-range NV12 (chroma the mean of each
// 2 x 2 block) or as 12-bit mono.
struct SynthArgs {
    uint8_t *y[RT_MAX_CAMERAS];         // Y plane (NV12) or 16-bit mono plane
    uint8_t *uv[RT_MAX_CAMERAS];        // UV plane (NV12)
    int32_t W[RT_MAX_CAMERAS], H[RT_MAX_CAMERAS], y_pitch[RT_MAX_CAMERAS], uv_pitch[RT_MAX_CAMERAS];
    int32_t fmt[RT_MAX_CAMERAS], bits[RT_MAX_CAMERAS];
    float x0[RT_MAX_CAMERAS];           // panorama column of the camera's first column
    float gain[RT_MAX_CAMERAS][3];
    float ph[16];                       // scene parameters in [0, 1)
    float noise;                        // noise standard deviation (8-bit levels)
    uint32_t key_lo, key_hi;            // noise counter key
    uint32_t block_base[RT_MAX_CAMERAS + 1];   // 2 x 2 blocks before camera k
    int32_t K;
};

// Launchers (each returns the launch's cudaError_t).
cudaError_t launch_synth(const SynthArgs &a, cudaStream_t s);
cudaError_t launch_pass_b(const ArrayGeom &g, const PassBArgs &a, int grid, int threads,
                          size_t smem, cudaStream_t s);
cudaError_t pass_b_prepare(int threads, size_t *smem_bytes);
// Column coefficients of the seam maps q16[K][2][B][nv] (nv = 6 or 12, B =
// every camera's nblk) for the table variant of pass B.  A camera's units
// are taken in chunks of 32 (nch = ceil(upr / 32) a row); for block j, unit
// ux = 32 chunk + l, group of 4 columns g4 and value v, the 16-byte word at
//   coef[cam.coef_base + ((j * nch + chunk) * 4 + g4) * nv * 32 + 32 v + l]
// holds value v (A_c then cst_c of the ramp blend, as the computing variant
// derives them) of columns 16 ux + 4 g4 + 0..3.  Words per camera:
// nblk * nch * 128 * nv.
cudaError_t launch_seam_coef(const ArrayGeom &g, const int32_t *q16, int nv, uint4 *coef, cudaStream_t s);
// Table variant of pass B (seam maps applied per block, a.coef set): grid
// CTAs of threads over the array's tiles.
cudaError_t launch_pass_b_table(const ArrayGeom &g, const PassBArgs &a, int grid, int threads, cudaStream_t s);
cudaError_t pass_b_table_prepare();
cudaError_t launch_pass_a(const ArrayGeom &g, const PassAArgs &a, int threads, cudaStream_t s);
cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_crops(const ArrayGeom &g, const CropArgs &a, int threads, int max_grid, cudaStream_t s);
cudaError_t launch_seam_cost(const ArrayGeom &g, const int2 *seams, int n_seams, int max_rows, double *rows,
                             double *cost, cudaStream_t s);
cudaError_t launch_attention(const ArrayGeom &g, const AttnArgs &a, int sm_count, cudaStream_t s);
// Per-row maps by convex blending of adjacent blocks: rows[K][2][Hmax][3][2]
// from q16[K][2][B][3][2].
cudaError_t launch_solve_matrix(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_blend_rows(const ArrayGeom &g, const int32_t *q16, int B, int Hmax, int nv, int32_t *rows,
                              cudaStream_t s);
cudaError_t launch_thumb_features(const ArrayGeom &g, const uint32_t *thumbs, void *out, cudaStream_t s);
cudaError_t launch_surrogate_gains(const float *y, const int32_t *group_start, const int32_t *group_members,
                                   int n_groups, const double *maps_fit, double gmin, double gmax, double *maps_out,
                                   double *err_out, cudaStream_t s);

}  // namespace rt
