/*
 * Plain, slow CPU oracle for the per-pixel steps of the remote-tower exposure
 * and white-balance correction (Sec. "White balance and exposure correction",
 * Eq. of the exponential smoothing; Sec. "Attention mechanisms" for the
 * detector-input crops).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this file's library.  It shares no code,
 * header, table or constant with the CUDA path, and it computes everything
 * from the definitions with one nested loop per pixel.
 *
 * Readings of what the paper leaves open (each one is listed, with its pin,
 * in the repository's design notes):
 *   - colour conversion: ITU-R BT.709 (or BT.601) limited range, integer
 *     coefficients round(256 * k * 255/219) and round(256 * k * 255/224)
 *     derived here from (Kr, Kb); chroma taken from the 2x2 block's sample;
 *   - narrow bands: the first and last S columns of each camera;
 *   - blocks of "identical size": rows [floor(j H / B), floor((j+1) H / B));
 *   - object removal: |Y_t - Y_{t-1}| > T on the band's luma excludes the
 *     pixel; saturated values 0 and 255 are excluded per channel;
 *   - the convex ramp from identity (image centre) to the map (border) is a
 *     Q16 weight linear in the column.
 * Integer right shifts of negative values are written as floor divisions.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* floor(a / b) for b > 0, independent of C's truncating division. */
static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int64_t clamp_i64(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Integer YCbCr -> RGB coefficients of the limited-range matrix.
 * out = {c_y, c_rv, c_gu, c_gv, c_bu}; matrix 0 = BT.709, 1 = BT.601.
 *   R' = Y' + 2(1-Kr) Cr',  G' = Y' - 2(1-Kb)Kb/Kg Cb' - 2(1-Kr)Kr/Kg Cr',
 *   B' = Y' + 2(1-Kb) Cb',  Y' = (Y-16)*255/219, C' = (C-128)*255/224.   */
void orc_color_coeffs(int matrix, int32_t out[5])
{
    double kr = matrix == 1 ? 0.299 : 0.2126;
    double kb = matrix == 1 ? 0.114 : 0.0722;
    double kg = 1.0 - kr - kb;
    double sy = 256.0 * 255.0 / 219.0, sc = 256.0 * 255.0 / 224.0;
    out[0] = (int32_t)lround(sy);
    out[1] = (int32_t)lround(sc * 2.0 * (1.0 - kr));
    out[2] = (int32_t)lround(sc * 2.0 * (1.0 - kb) * kb / kg);
    out[3] = (int32_t)lround(sc * 2.0 * (1.0 - kr) * kr / kg);
    out[4] = (int32_t)lround(sc * 2.0 * (1.0 - kb));
}

/* One pixel of the integer conversion. */
static void yuv_to_rgb(const int32_t k[5], int Y, int U, int V, uint8_t *rgb)
{
    int64_t C = Y - 16, D = U - 128, E = V - 128;
    rgb[0] = (uint8_t)clamp_i64(floor_div(k[0] * C + k[1] * E + 128, 256), 0, 255);
    rgb[1] = (uint8_t)clamp_i64(floor_div(k[0] * C - k[2] * D - k[3] * E + 128, 256), 0, 255);
    rgb[2] = (uint8_t)clamp_i64(floor_div(k[0] * C + k[4] * D + 128, 256), 0, 255);
}

/* NV12 (Y plane + interleaved U,V plane at half resolution) -> RGB24.
 * Pixel (x, y) takes the chroma sample of its 2x2 block: U at column
 * 2*(x/2), V at 2*(x/2)+1 of UV row y/2. */
void orc_convert_nv12(const uint8_t *yp, int64_t y_pitch, const uint8_t *uvp, int64_t uv_pitch,
                      int W, int H, int matrix, uint8_t *rgb, int64_t rgb_pitch)
{
    int32_t k[5];
    orc_color_coeffs(matrix, k);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int Y = yp[(int64_t)y * y_pitch + x];
            int U = uvp[(int64_t)(y / 2) * uv_pitch + 2 * (x / 2)];
            int V = uvp[(int64_t)(y / 2) * uv_pitch + 2 * (x / 2) + 1];
            yuv_to_rgb(k, Y, U, V, rgb + (int64_t)y * rgb_pitch + 3 * x);
        }
}

/* Mono (infrared) samples of bit_depth bits in 16-bit words -> gray RGB24:
 * v8 = min(255, v >> (bit_depth - 8)), R = G = B = v8. pitch in elements. */
void orc_convert_mono16(const uint16_t *p, int64_t pitch, int W, int H, int bit_depth,
                        uint8_t *rgb, int64_t rgb_pitch)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int v = p[(int64_t)y * pitch + x] >> (bit_depth - 8);
            uint8_t v8 = (uint8_t)(v > 255 ? 255 : v);
            uint8_t *o = rgb + (int64_t)y * rgb_pitch + 3 * x;
            o[0] = o[1] = o[2] = v8;
        }
}

/* Luma used by the motion test: the Y sample (NV12) or v8 (mono). */
void orc_luma_mono16(const uint16_t *p, int64_t pitch, int W, int H, int bit_depth,
                     uint8_t *out, int64_t out_pitch)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int v = p[(int64_t)y * pitch + x] >> (bit_depth - 8);
            out[(int64_t)y * out_pitch + x] = (uint8_t)(v > 255 ? 255 : v);
        }
}

/* First row of block j of B over H rows ("blocks of identical size" rounded
 * down to whole rows). */
static int block_row0(int j, int H, int B) { return (int)(((int64_t)j * H) / B); }

/* Narrow-band ("measured spectra") statistics of one camera.
 * Sides: 0 = left band, columns [0, S); 1 = right band, columns [W-S, W).
 * For each side s, block j, channel c, over the band's pixels that are not
 * moving (prev_luma == NULL, or |luma - prev_luma| <= T) and whose channel
 * value is neither 0 nor 255:  n += 1, sum += x, sumsq += x^2, hist[x] += 1.
 * Output layouts: n/sum/sumsq [2][B][3], hist [2][B][3][256]. */
void orc_strip_stats(const uint8_t *rgb, int64_t rgb_pitch,
                     const uint8_t *luma, int64_t luma_pitch,
                     const uint8_t *prev_luma, int64_t prev_pitch,
                     int W, int H, int S, int B, int T,
                     uint32_t *n, uint64_t *sum, uint64_t *sumsq, uint32_t *hist)
{
    memset(n, 0, sizeof(uint32_t) * 2 * B * 3);
    memset(sum, 0, sizeof(uint64_t) * 2 * B * 3);
    memset(sumsq, 0, sizeof(uint64_t) * 2 * B * 3);
    memset(hist, 0, sizeof(uint32_t) * 2 * B * 3 * 256);
    for (int s = 0; s < 2; ++s) {
        int x0 = s == 0 ? 0 : W - S;
        for (int j = 0; j < B; ++j)
            for (int y = block_row0(j, H, B); y < block_row0(j + 1, H, B); ++y)
                for (int x = x0; x < x0 + S; ++x) {
                    if (prev_luma) {
                        int d = (int)luma[(int64_t)y * luma_pitch + x] -
                                (int)prev_luma[(int64_t)y * prev_pitch + x];
                        if (d < 0) d = -d;
                        if (d > T) continue;
                    }
                    for (int c = 0; c < 3; ++c) {
                        int v = rgb[(int64_t)y * rgb_pitch + 3 * x + c];
                        if (v == 0 || v == 255) continue;
                        int64_t i = ((int64_t)s * B + j) * 3 + c;
                        n[i] += 1;
                        sum[i] += (uint64_t)v;
                        sumsq[i] += (uint64_t)v * (uint64_t)v;
                        hist[i * 256 + v] += 1;
                    }
                }
    }
}

/* Whole-frame statistics of the (uncorrected) RGB: per channel histogram,
 * sum and sum of squares over all pixels. hist [3][256], sum/sumsq [3]. */
void orc_frame_stats(const uint8_t *rgb, int64_t rgb_pitch, int W, int H,
                     uint32_t *hist, uint64_t *sum, uint64_t *sumsq)
{
    memset(hist, 0, sizeof(uint32_t) * 3 * 256);
    memset(sum, 0, sizeof(uint64_t) * 3);
    memset(sumsq, 0, sizeof(uint64_t) * 3);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < 3; ++c) {
                int v = rgb[(int64_t)y * rgb_pitch + 3 * x + c];
                hist[c * 256 + v] += 1;
                sum[c] += (uint64_t)v;
                sumsq[c] += (uint64_t)v * (uint64_t)v;
            }
}

/* Thumbnail cell sums of the uncorrected RGB on a TW x TH grid: cell (i, j)
 * covers columns [floor(i W/TW), floor((i+1) W/TW)) and rows
 * [floor(j H/TH), floor((j+1) H/TH)).  out [3][TH][TW]. */
void orc_thumbnail(const uint8_t *rgb, int64_t rgb_pitch, int W, int H, int TW, int TH,
                   uint32_t *out)
{
    memset(out, 0, sizeof(uint32_t) * 3 * TW * TH);
    for (int j = 0; j < TH; ++j)
        for (int i = 0; i < TW; ++i)
            for (int y = (int)((int64_t)j * H / TH); y < (int)((int64_t)(j + 1) * H / TH); ++y)
                for (int x = (int)((int64_t)i * W / TW); x < (int)((int64_t)(i + 1) * W / TW); ++x)
                    for (int c = 0; c < 3; ++c)
                        out[((int64_t)c * TH + j) * TW + i] += rgb[(int64_t)y * rgb_pitch + 3 * x + c];
}

/* Q16 weight of the map at column x: the convex combination runs from the
 * identity at the image centre to the full map at the border of the side
 * the column lies on (Fig. "exposure correction function ... applied to
 * half the image").  w = 65536 at columns 0 and W-1. */
int32_t orc_ramp_q16(int x, int W)
{
    int64_t h = W / 2;
    if (x < h) return (int32_t)(((h - x) * 65536) / h);
    return (int32_t)(((x - h + 1) * 65536) / h);
}

/* Per-pixel application of the Q16 maps f_c(x) = a_c x + b_c.
 * q16 layout [2 sides][B][3][2] = {a_q, b_q}.  fit_mode 0 (per-camera gains):
 * weight 65536 everywhere and the left-side table for every column; 1 (seam
 * maps): side = x < W/2 ? left : right, weight from orc_ramp_q16.
 *   A  = 65536 + floor((a_q - 65536) w / 65536),  Bq = floor(b_q w / 65536)
 *   out = clamp(floor((A v + Bq + 32768) / 65536), 0, 255). */
void orc_apply(const uint8_t *rgb, int64_t rgb_pitch, int W, int H, int B, int fit_mode,
               const int32_t *q16, uint8_t *out, int64_t out_pitch)
{
    for (int j = 0; j < B; ++j)
        for (int y = block_row0(j, H, B); y < block_row0(j + 1, H, B); ++y)
            for (int x = 0; x < W; ++x) {
                int side = (fit_mode == 1 && x >= W / 2) ? 1 : 0;
                int64_t w = fit_mode == 1 ? orc_ramp_q16(x, W) : 65536;
                for (int c = 0; c < 3; ++c) {
                    const int32_t *m = q16 + (((int64_t)side * B + j) * 3 + c) * 2;
                    int64_t A = 65536 + floor_div(((int64_t)m[0] - 65536) * w, 65536);
                    int64_t Bq = floor_div((int64_t)m[1] * w, 65536);
                    int64_t v = rgb[(int64_t)y * rgb_pitch + 3 * x + c];
                    out[(int64_t)y * out_pitch + 3 * x + c] =
                        (uint8_t)clamp_i64(floor_div(A * v + Bq + 32768, 65536), 0, 255);
                }
            }
}

/* Bilinear resample of the rectangle (x0, y0, w, h) of an RGB24 image to an
 * S x S square (the detector's fixed square input, Sec. "Detection"),
 * half-pixel centres, source coordinates clamped to the rectangle, values
 * scaled to [0, 1].  out [3][S][S] (planar, channel-major). */
void orc_crop(const uint8_t *rgb, int64_t rgb_pitch, int x0, int y0, int w, int h, int S,
              double *out)
{
    for (int oy = 0; oy < S; ++oy) {
        double sy = y0 + (oy + 0.5) * (double)h / S - 0.5;
        if (sy < y0) sy = y0;
        if (sy > y0 + h - 1) sy = y0 + h - 1;
        int ylo = (int)floor(sy);
        int yhi = ylo + 1 < y0 + h ? ylo + 1 : y0 + h - 1;
        double fy = sy - ylo;
        for (int ox = 0; ox < S; ++ox) {
            double sx = x0 + (ox + 0.5) * (double)w / S - 0.5;
            if (sx < x0) sx = x0;
            if (sx > x0 + w - 1) sx = x0 + w - 1;
            int xlo = (int)floor(sx);
            int xhi = xlo + 1 < x0 + w ? xlo + 1 : x0 + w - 1;
            double fx = sx - xlo;
            for (int c = 0; c < 3; ++c) {
                double p00 = rgb[(int64_t)ylo * rgb_pitch + 3 * xlo + c];
                double p01 = rgb[(int64_t)ylo * rgb_pitch + 3 * xhi + c];
                double p10 = rgb[(int64_t)yhi * rgb_pitch + 3 * xlo + c];
                double p11 = rgb[(int64_t)yhi * rgb_pitch + 3 * xhi + c];
                double v = (1.0 - fy) * ((1.0 - fx) * p00 + fx * p01) +
                           fy * ((1.0 - fx) * p10 + fx * p11);
                out[((int64_t)c * S + oy) * S + ox] = v / 255.0;
            }
        }
    }
}

/* Joint band statistics for 3 x 3 cross-channel maps: per band side and
 * block, over the pixels that are not moving and not saturated in any
 * channel (0 < v_c < 255 for all c): joint[s][j][10] =
 * {n, sum R, sum G, sum B, RR, RG, RB, GG, GB, BB}. */
void orc_strip_joint(const uint8_t *rgb, int64_t rgb_pitch,
                     const uint8_t *luma, int64_t luma_pitch,
                     const uint8_t *prev_luma, int64_t prev_pitch,
                     int W, int H, int S, int B, int T, uint64_t *joint)
{
    memset(joint, 0, sizeof(uint64_t) * 2 * B * 10);
    for (int s = 0; s < 2; ++s) {
        int x0 = s == 0 ? 0 : W - S;
        for (int j = 0; j < B; ++j)
            for (int y = block_row0(j, H, B); y < block_row0(j + 1, H, B); ++y)
                for (int x = x0; x < x0 + S; ++x) {
                    if (prev_luma) {
                        int d = (int)luma[(int64_t)y * luma_pitch + x] -
                                (int)prev_luma[(int64_t)y * prev_pitch + x];
                        if (d < 0) d = -d;
                        if (d > T) continue;
                    }
                    const uint8_t *p = rgb + (int64_t)y * rgb_pitch + 3 * x;
                    int ok = 1;
                    for (int c = 0; c < 3; ++c)
                        if (p[c] == 0 || p[c] == 255) ok = 0;
                    if (!ok) continue;
                    uint64_t *q = joint + ((int64_t)s * B + j) * 10;
                    uint64_t r = p[0], g = p[1], b = p[2];
                    q[0] += 1;
                    q[1] += r; q[2] += g; q[3] += b;
                    q[4] += r * r; q[5] += r * g; q[6] += r * b;
                    q[7] += g * g; q[8] += g * b; q[9] += b * b;
                }
    }
}

/* Apply 3 x 3 cross-channel maps along the ramp: q16 layout [2 sides][B][12]
 * = {M row-major (9), b (3)} in Q16.  For a pixel of side s, block j and
 * ramp weight w (orc_ramp_q16):
 *   A_cd = delta_cd 65536 + floor((m_cd - delta_cd 65536) w / 65536),
 *   B_c  = floor(b_c w / 65536),
 *   out_c = clamp(floor((sum_d A_cd v_d + B_c + 32768) / 65536), 0, 255). */
void orc_apply_matrix(const uint8_t *rgb, int64_t rgb_pitch, int W, int H, int B, const int32_t *q16,
                      uint8_t *out, int64_t out_pitch)
{
    for (int y = 0; y < H; ++y) {
        int j = 0;
        while (j + 1 < B && block_row0(j + 1, H, B) <= y) ++j;
        for (int x = 0; x < W; ++x) {
            int side = x >= W / 2 ? 1 : 0;
            int64_t w = orc_ramp_q16(x, W);
            const int32_t *m = q16 + ((int64_t)side * B + j) * 12;
            const uint8_t *p = rgb + (int64_t)y * rgb_pitch + 3 * x;
            for (int c = 0; c < 3; ++c) {
                int64_t acc = 32768;
                for (int d = 0; d < 3; ++d) {
                    int64_t delta = c == d ? 65536 : 0;
                    int64_t A = delta + floor_div((m[3 * c + d] - delta) * w, 65536);
                    acc += A * p[d];
                }
                acc += floor_div((int64_t)m[9 + c] * w, 65536);
                int64_t v = floor_div(acc, 65536);
                out[(int64_t)y * out_pitch + 3 * x + c] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
            }
        }
    }
}
