/*
 * rt.h -- C ABI of the GB300 camera-array correction library (librt.so).
 *
 * The library runs, per frame set of a multi-camera remote-tower array, the
 * pixel hot path of the automatic exposure and white-balance correction of
 * Sec. "White balance and exposure correction" and the detector-input crops
 * of Sec. "Detection" / "Attention mechanisms":
 *   S1  NV12 (or 12-bit mono infrared) -> RGB24 conversion of every camera;
 *   S2  integer statistics: histograms of the narrow bands on both sides of
 *       every seam, split into vertical blocks, with moving pixels removed
 *       (object removal, Fig. "thresholded difference"), and whole-frame
 *       histograms of every camera;
 *   S3  an FP64 fit: per-camera gains (least squares of log band means over
 *       the seams), or the paper's per-seam affine maps f_c(x) = a_c x + b_c
 *       matched to the shared spectrum of the seam;
 *   S4  exponential smoothing E <- (1 - alpha) E_prev + alpha E_new
 *       (alpha = 0.05) and Q16 quantisation;
 *   S5  per-pixel application of the maps along the convex ramp from the
 *       identity at the image centre to the map at the border;
 *   S6  bilinear resampling of attention windows into FP16 NCHW squares.
 *
 * Conventions for every call:
 *   - Every call returns an rt_status; nothing throws across the ABI.
 *   - Device pointers are CUDA device addresses of the current device; host
 *     pointers are ordinary process memory (pinned memory makes copies
 *     asynchronous and faster, but is not required).
 *   - Work is enqueued asynchronously.  The library orders its work after
 *     everything already queued on the caller's stream given to
 *     rt_array_config; results are waited for by the rt_get_* calls, which
 *     block for at most timeout_ms milliseconds (RT_ERR_TIMEOUT after that,
 *     never a hang).  timeout_ms < 0 waits without limit.
 *   - A handle must not be used from two threads at once.
 *   - Errors: RT_ERR_INVALID for arguments that break a stated rule (nothing
 *     is enqueued), RT_ERR_CUDA for a failed CUDA call (rt_last_error says
 *     which), RT_ERR_OOM when device memory runs out, RT_ERR_STATE when a
 *     call comes in the wrong order (e.g. a get before any submit).
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID = -1,
    RT_ERR_CUDA = -2,
    RT_ERR_OOM = -3,
    RT_ERR_NOT_READY = -4,
    RT_ERR_TIMEOUT = -5,
    RT_ERR_STATE = -6
} rt_status;

enum { RT_NV12 = 0, RT_MONO16 = 1 };                 /* camera pixel formats         */
enum { RT_LINEAR = 0, RT_RING = 1 };                 /* seam topology of every chain */
enum { RT_FIT_GLOBAL = 0, RT_FIT_SEAM_AFFINE = 1, RT_FIT_QUANTILE_AFFINE = 2, RT_FIT_MATRIX = 3 };  /* S3 fit */
enum { RT_SCHED_CURRENT = 0, RT_SCHED_LAGGED = 1 };  /* which statistics S5 applies  */
enum { RT_BT709 = 0, RT_BT601 = 1 };                 /* S1 colour matrix             */

#define RT_MAX_CAMERAS 32
#define RT_MAX_BLOCKS 64
#define RT_THUMB_W 64
#define RT_THUMB_H 36

/* One camera of the array.
 *   width, height  even, >= 2 * strip_width and >= 2 rows;
 *   format         RT_NV12 or RT_MONO16;
 *   bit_depth      significant bits of a mono sample (8..16), ignored for NV12;
 *   y_pitch        bytes per row of the Y plane (NV12) or of the 16-bit mono
 *                  plane; a multiple of 16 and >= width (2 * width for mono);
 *   uv_pitch       bytes per row of the interleaved U,V plane (NV12), a
 *                  multiple of 16 and >= width; ignored for mono;
 *   group          seam chain the camera belongs to (cameras of one chain are
 *                  side by side; chains are corrected independently);
 *   position       order of the camera inside its chain, left to right. */
typedef struct {
    int32_t width, height, format, bit_depth;
    int32_t y_pitch, uv_pitch, group, position;
} rt_camera_desc;

/* Array configuration (Sec. "White balance and exposure correction").
 *   num_cameras        1..RT_MAX_CAMERAS; cams points to that many entries;
 *   topology           RT_LINEAR (end cameras keep the identity on their
 *                      outer side) or RT_RING (last camera meets the first);
 *   strip_width        S: width in pixels of the narrow band at each seam,
 *                      a multiple of 16 (32 by default);
 *   num_blocks         B: vertical blocks of the band, 1..RT_MAX_BLOCKS
 *                      (the paper tests 16 and 64);
 *   fit_mode           RT_FIT_GLOBAL, RT_FIT_SEAM_AFFINE or RT_FIT_QUANTILE_AFFINE
 *                      (the affine map of each seam side as the least-squares
 *                      line through (band quantile, shared-spectrum quantile)
 *                      pairs at the levels (i + 1/2) / 32; the shared spectrum
 *                      is the equal-weight mixture of the two bands; applied
 *                      like RT_FIT_SEAM_AFFINE) or RT_FIT_MATRIX (3 x 3
 *                      cross-channel maps, the conclusion's proposal of linear
 *                      maps mixing the three channels: per seam side and block
 *                      the symmetric positive definite M with M S M^T = S_s,
 *                      S the band's RGB covariance, S_s that of the equal-weight
 *                      mixture of the two bands, both plus 0.25 I; M's
 *                      eigenvalues clamped to [gain_min, gain_max];
 *                      b = mu_s - M mu; moments over pixels neither moving nor
 *                      saturated in any channel; applied along the ramp);
 *   schedule           RT_SCHED_CURRENT: a frame set is corrected with the
 *                      estimate that includes its own statistics;
 *                      RT_SCHED_LAGGED: with the estimate of the previous
 *                      frame set (the first one with the identity);
 *   motion_threshold   T: a band pixel with |Y_t - Y_{t-1}| > T is moving;
 *   min_valid          a band side with fewer valid pixels is ignored;
 *   color_matrix       RT_BT709 or RT_BT601 (limited range);
 *   alpha              smoothing weight (0.05 in the paper), 0 < alpha <= 1;
 *   lambda             ridge term of the gain fit (> 0);
 *   gain_min/gain_max  clamp of gains and of affine slopes;
 *   max_crops          crops per frame set the library can hold (0 = none);
 *   crop_size          side of the square crops (>= 1 if max_crops > 0);
 *   flags              RT_FLAG_* below;
 *   attn_window        difference attention (RT_FLAG_ATTENTION): side of the
 *                      square windows, a multiple of 32 in 32..4096 (256);
 *                      windows step by attn_window / 2;
 *   attn_min_on        on-pixels (|Y_t - Y_{t-1}| > motion_threshold) a
 *                      window needs to be proposed, >= 1 (655, 1 % of 256^2);
 *   attn_max           proposals kept per frame set, 1..4096 (256);
 *   surrogate_mode     0: the gains are fitted every frame set (the paper's
 *                      method); 1: the learned surrogate (rt_surrogate.h)
 *                      predicts them from the previous frame set's
 *                      thumbnails and the fit runs only as its judge and
 *                      fallback; 2: the same from the thumbnails of the frame
 *                      set before the previous one, so that the prediction
 *                      runs beside the previous frame set's correction pass
 *                      instead of after it.  Modes 1 and 2 need RT_FIT_GLOBAL,
 *                      one block, RT_FLAG_THUMBNAILS, the current schedule and
 *                      a network (rt_surrogate_train or rt_surrogate_load)
 *                      before the first submit;
 *   judge_every        surrogate mode: the fit judges the prediction every
 *                      judge_every-th frame set of a sequence (>= 1; 8);
 *   fallback_tol       surrogate mode: a judged prediction whose largest
 *                      |g_pred / g_fit - 1| exceeds this (>= 0; 0.02) is
 *                      replaced by the fit, which stays applied (and judges
 *                      every frame set) until a judgement passes. */
typedef struct {
    int32_t num_cameras;
    const rt_camera_desc *cams;
    int32_t topology;
    int32_t strip_width, num_blocks, fit_mode, schedule;
    int32_t motion_threshold, min_valid, color_matrix;
    double alpha, lambda, gain_min, gain_max;
    int32_t max_crops, crop_size;
    int32_t flags;
    int32_t attn_window, attn_min_on, attn_max;
    int32_t surrogate_mode, judge_every;
    double fallback_tol;
} rt_array_params;

#define RT_FLAG_FRAME_STATS 1   /* whole-frame histograms of every camera (S2 iii) */
#define RT_FLAG_THUMBNAILS 2    /* 64x36 thumbnail cell sums of every camera (surrogate input);
                                   needs every camera at least 64 x 36 pixels */
#define RT_FLAG_SEAM_COST 4     /* gradient-continuity cost of every seam of the corrected
                                   output (rt_get_seam_costs); needs every camera >= 16 x 8 */
#define RT_FLAG_ATTENTION 8     /* difference attention: window proposals from the change of
                                   every camera's luma between frame sets (rt_get_proposals) */
#define RT_FLAG_BLEND_BLOCKS 16 /* with num_blocks > 1: apply per-row maps that blend adjacent
                                   blocks' maps convexly -- linear between the centres of two
                                   consecutive blocks (in Q16 integers), the edge blocks' maps
                                   beyond the first and last centre -- instead of switching
                                   maps at block borders */

/* n_crops value of rt_submit_frames / rt_capture_sequence: crop this frame
 * set's attention proposals (RT_FLAG_ATTENTION, max_crops > 0; at most
 * min(max_crops, attn_max) of them). */
#define RT_CROPS_FROM_PROPOSALS (-1)

/* An attention window: rectangle (x0, y0, w, h) of camera cam, inside it. */
typedef struct { int32_t cam, x0, y0, w, h; } rt_crop;

typedef struct rt_handle rt_handle;

/* Fill p with the defaults (S = 32, B = 1, per-camera gains, current
 * schedule, T = 24, min_valid = 64, BT.709, alpha = 0.05, lambda = 1e-6,
 * gains in [1/4, 4], no crops, frame statistics on, no surrogate mode,
 * judge_every = 8, fallback_tol = 0.02).  cams is left NULL. */
void rt_default_params(rt_array_params *p);

/* Validate the configuration, allocate every device buffer the array needs
 * (outputs, statistics, smoothing state, the previous frame's band luma)
 * and create the library's streams.  cuda_stream is the caller's stream
 * (cudaStream_t; NULL = legacy default stream) whose queued work every
 * submit waits for.  On success *out owns the handle (rt_destroy frees it). */
rt_status rt_array_config(const rt_array_params *params, void *cuda_stream, rt_handle **out);

/* Enqueue one frame set.  y_planes[k] / uv_planes[k] are device pointers to
 * camera k's Y and UV planes (NV12) or y_planes[k] to its 16-bit mono plane
 * (uv_planes may be NULL or hold NULL for mono cameras), 16-byte aligned,
 * laid out with the configured pitches.  They are read asynchronously and
 * must stay unchanged until this frame set's outputs have been waited for.
 * frame_index 0 restarts the sequence: no motion test (no previous frame)
 * and the smoothing starts from this frame set's estimate.  crops[0..n_crops)
 * are the attention windows of this frame set (n_crops <= max_crops).
 * Outputs live in library memory, double buffered: those of frame set t stay
 * valid until frame set t+2 is submitted. */
rt_status rt_submit_frames(rt_handle *h, const void *const *y_planes, const void *const *uv_planes,
                           int64_t frame_index, const rt_crop *crops, int32_t n_crops);

/* As rt_submit_frames, but the planes are in HOST memory (same pitches): the
 * library copies them into its own device staging buffers first, on a copy
 * stream that overlaps the previous frame set's processing.  If rgb_out is
 * not NULL, rgb_out[k] is a host buffer of height rows of rgb_out_pitch
 * bytes (>= 3 * width) that receives camera k's corrected RGB24 image,
 * copied back asynchronously as soon as the frame set is done.  Host
 * buffers (pinned memory makes the copies asynchronous) must stay unchanged
 * / untouched until rt_sync returns, or until a later rt_get_* of this frame
 * set returns. */
rt_status rt_submit_frames_host(rt_handle *h, const void *const *y_planes, const void *const *uv_planes,
                                int64_t frame_index, const rt_crop *crops, int32_t n_crops,
                                void *const *rgb_out, int64_t rgb_out_pitch);

/* Wait for the last submitted frame set and copy its smoothed maps.
 * maps_fp64 (may be NULL): doubles [K][2 sides][B][3 channels][2] = (a, b),
 * side 0 = left half, 1 = right half of the camera; with per-camera gains
 * both sides hold (g, 0).  maps_q16 (may be NULL): the same shape in int32,
 * round(65536 a), round(65536 b) -- the table the pixels were corrected
 * with.  With RT_FIT_MATRIX each (camera, side, block) holds 12 values
 * instead: M row-major (9) then b (3), out_c = sum_d M_cd v_d + b_c.
 * cap = elements each buffer holds (>= K*2*B*6, or K*2*B*12 for
 * RT_FIT_MATRIX). */
rt_status rt_get_gains(rt_handle *h, double *maps_fp64, int32_t *maps_q16, size_t cap, int32_t timeout_ms);

/* Wait for the last submitted frame set and return the device address of
 * camera cam's corrected RGB24 image (height rows of *pitch bytes, 3 bytes a
 * pixel, R G B).  The memory belongs to the library. */
rt_status rt_get_corrected(rt_handle *h, int32_t cam, const uint8_t **dev_rgb, int32_t *pitch, int32_t timeout_ms);

/* Wait, then copy camera cam's corrected RGB24 image into host (or device)
 * memory dst with row pitch dst_pitch bytes (>= 3 * width).  The copy runs on
 * the library's stream and is complete when the call returns. */
rt_status rt_copy_corrected(rt_handle *h, int32_t cam, void *dst, int64_t dst_pitch, int32_t timeout_ms);

/* Wait and return the device address of the last frame set's crops: FP16
 * [n][3][crop_size][crop_size] (planar R, G, B, values in [0, 1]). */
rt_status rt_get_crops(rt_handle *h, const void **dev_fp16_nchw, int32_t *n, int32_t timeout_ms);

/* Device addresses of the last frame set's statistics (library memory;
 * valid until the next submit).
 *   strip_hist   u32 [K][2][B][3][256]  band histograms (valid pixels)
 *   strip_n      u32 [K][2][B][3]       valid pixel counts
 *   strip_sum    u64 [K][2][B][3]       sums of valid values
 *   strip_sumsq  u64 [K][2][B][3]       sums of squares
 *   frame_hist   u32 [K][3][256]        whole-frame histograms (NULL if off)
 *   thumbs       u32 [K][3][36][64]     thumbnail cell sums (NULL if off)
 *   strip_joint  u64 [K][2][B][10]      RT_FIT_MATRIX only (else NULL): over
 *                the band pixels neither moving nor saturated in any channel,
 *                {n, sum R, sum G, sum B, RR, RG, RB, GG, GB, BB}
 *   uncorrected  optional: NULL (the library keeps no uncorrected RGB). */
typedef struct {
    const uint32_t *strip_hist, *strip_n;
    const uint64_t *strip_sum, *strip_sumsq;
    const uint32_t *frame_hist, *thumbs;
    int32_t num_cameras, num_blocks;
    const uint64_t *strip_joint;
} rt_stats_view;
rt_status rt_get_stats(rt_handle *h, rt_stats_view *out, int32_t timeout_ms);

/* Seam quality of the last frame set's corrected output (RT_FLAG_SEAM_COST),
 * the cost of Sec. "Quantitative", Eq. (gradientcost): both images of a seam
 * are box-averaged over 8 x 8 pixels (rows and columns beyond a multiple of
 * 8 dropped); on every averaged row i that both have, with columns L-1, L0
 * the last two of the left image and R0, R1 the first two of the right,
 *   d+_i = |(R1 - R0) - (R0 - L0)|,  d-_i = |(L-1 - L0) - (L0 - R0)|
 * (Euclidean norm over R, G, B), and cost = mean_i (d+_i + d-_i) / 2 --
 * whether the colour trend continues across the seam.  One entry per seam,
 * in chain order (groups ascending, cameras by position, a ring's closing
 * seam last in its group): left_cam[i], right_cam[i], cost[i] (FP64).  Any
 * output array may be NULL; cap = their capacity; *n = the number of seams
 * (RT_ERR_INVALID if it exceeds cap).  Waits at most timeout_ms. */
rt_status rt_get_seam_costs(rt_handle *h, int32_t *left_cam, int32_t *right_cam, double *cost, int32_t cap,
                            int32_t *n, int32_t timeout_ms);

/* Difference attention of the last frame set (RT_FLAG_ATTENTION; Sec.
 * "Attention mechanisms", the difference approach): the change map of a
 * camera holds the pixels whose luma (NV12 Y, or the 8-bit value of a mono
 * camera) differs from the previous frame set's by more than
 * motion_threshold; square windows of side attn_window slide over it at
 * stride attn_window / 2 (2 x 2 blocks of square cells of side
 * attn_window / 2, the last row and column of cells partial, windows clipped
 * to the frame), and every window with at least attn_min_on on-pixels is a
 * proposal, listed camera by camera, window row by window row, left to
 * right, at most attn_max.  The first frame set of a sequence, and the
 * first after rt_load_state or rt_autotune, proposes nothing.  out (may be NULL) receives min(cap, count) windows; *n the
 * count.  Waits at most timeout_ms. */
rt_status rt_get_proposals(rt_handle *h, rt_crop *out, int32_t cap, int32_t *n, int32_t timeout_ms);

/* Wait, then write the last frame set's thumbnail features into the DEVICE
 * buffer x_bf16: BF16 [K][3][36][64], cell mean / 255 - 0.5 (the learned
 * surrogate's input, rt_surrogate.h).  Needs RT_FLAG_THUMBNAILS. */
rt_status rt_get_thumb_features(rt_handle *h, void *x_bf16, int32_t timeout_ms);

/* Copy bytes from library memory (an address returned by rt_get_stats,
 * rt_get_crops or rt_get_corrected) to dst, host or device memory; complete
 * when the call returns (bounded by timeout_ms). */
rt_status rt_copy_out(rt_handle *h, void *dst, const void *src, size_t bytes, int32_t timeout_ms);

/* Make the CUDA stream `cuda_stream` (cudaStream_t) wait, on the device, for
 * all work enqueued so far by the handle, including pending device->host
 * copies.  Returns at once; lets a caller consume outputs stream-ordered. */
rt_status rt_stream_wait(rt_handle *h, void *cuda_stream);

/* Capture a CUDA graph that processes n_sets frame sets read from a fixed
 * ring of input buffers (a decoder's surface pool): set i uses
 * y_planes[i*K + k] / uv_planes[i*K + k] (device pointers, as for
 * rt_submit_frames) and crops[i*max_crops .. + n_crops[i]) (crops and
 * n_crops may be NULL for none).  n_sets >= 1.  The graph's buffer slots
 * repeat every 6 frame sets, so it can be launched whenever the frame sets
 * submitted since the capture are a multiple of 6: a graph of a multiple of 6
 * frame sets runs back to back; one of another length runs once, or again
 * after single submits restore the alignment.  At least one frame set must
 * have been submitted before (the graph continues a sequence; it never
 * restarts one).  The graph's parameters are fixed at capture; the buffers
 * must stay allocated while it exists.  A new capture replaces the previous
 * one. */
rt_status rt_capture_sequence(rt_handle *h, int32_t n_sets, const void *const *y_planes,
                              const void *const *uv_planes, const rt_crop *crops, const int32_t *n_crops);

/* Launch the captured graph once: n_sets more frame sets of the sequence,
 * one graph launch.  RT_ERR_STATE if nothing is captured or if the frame
 * sets submitted since the capture are not a multiple of 6. */
rt_status rt_launch_sequence(rt_handle *h);

/* Launch shapes of the per-frame-set kernels.  Throughput depends on them
 * (how many pass B threads per CTA, how many CTAs per SM, how the band
 * statistics and the crops are cut into CTAs) and on how they share the SMs
 * when they overlap, so rt_autotune measures them on the array itself. */
typedef struct {
    int32_t pass_b_threads;      /* threads per pass B CTA, 64..512, a multiple of 32 (the seam
                                    maps applied per block without thumbnails run a fixed shape:
                                    one CTA per SM of 512 threads, 384 for RT_FIT_MATRIX) */
    int32_t pass_b_ctas_per_sm;  /* 1 or 2 (the thumbnail variant always runs 1) */
    int32_t pass_a_rows;         /* rows per band-statistics work item, 8..1024 (a block's rows are
                                    split into round(rows / pass_a_rows) equal items, at least one) */
    int32_t pass_a_threads;      /* threads per band-statistics CTA: 64, 128 or 256 */
    int32_t crop_threads;        /* threads per crop CTA, 128 or 256 (crops over 2048 pixels a
                                    side; smaller ones run crop_size / 2 threads a CTA) */
    int32_t crop_grid;           /* at most this many CTAs per crop window, 1..4096 (row groups) */
    double step_us;              /* rt_autotune: measured time per frame set of this shape */
    int32_t from_cache;          /* rt_autotune: 1 if the shape came from the cache file */
    int32_t candidates;          /* rt_autotune: shapes timed (0 when cached) */
} rt_tuning;

/* Pick the launch shapes by timing candidates on n_sets frame sets of the
 * caller (n_sets a positive multiple of 6; planes and crops laid out as for
 * rt_capture_sequence): pass B's shape first, then the band statistics',
 * then the crops', each with the best of the earlier ones fixed; every
 * candidate is captured as a graph of the n_sets frame sets and timed over
 * three launches with CUDA events.  cache_path (may be NULL): a JSON file
 * mapping "device|SMs|array configuration" keys to shapes; a hit is applied
 * without timing, a miss is timed and written back (the file is created or
 * rewritten; other keys are kept).  The sequence state (smoothing state,
 * motion reference, restart flag) is restored afterwards; outputs of earlier
 * frame sets are overwritten and a captured sequence is dropped (capture
 * again).  out (may be NULL) receives the chosen shape.  Errors: as
 * rt_capture_sequence, RT_ERR_INVALID for a bad n_sets. */
rt_status rt_autotune(rt_handle *h, int32_t n_sets, const void *const *y_planes, const void *const *uv_planes,
                      const rt_crop *crops, const int32_t *n_crops, const char *cache_path, rt_tuning *out);

/* The launch shapes in use (step_us, from_cache, candidates as left by the
 * last rt_autotune, else 0). */
rt_status rt_get_tuning(rt_handle *h, rt_tuning *out);

/* Use the given launch shapes (validated as documented on rt_tuning; the
 * informational fields are ignored).  Drops a captured sequence. */
rt_status rt_set_tuning(rt_handle *h, const rt_tuning *t);

/* Per-pass device times, from CUDA events the library records around its
 * kernels when profiling is on.  rt_profile(h, RT_PROFILE_ALL) starts
 * collecting around every pass, rt_profile(h, RT_PROFILE_PASS_B) around the
 * correction pass only (the other totals stay 0; two events per frame set
 * instead of seven, so the timing disturbs a captured sequence less); both
 * clear what was collected.  rt_profile(h, 0) stops.  rt_get_profile waits
 * (bounded) and reports totals over the frame sets collected: for a captured
 * sequence, the frame sets of its last launch, with the mode in force at
 * capture. */
#define RT_PROFILE_ALL 1
#define RT_PROFILE_PASS_B 2
typedef struct {
    int32_t frame_sets;
    double pass_a_ms, solve_ms, pass_b_ms, crops_ms;   /* totals, milliseconds */
} rt_profile_report;
rt_status rt_profile(rt_handle *h, int32_t enable);
rt_status rt_get_profile(rt_handle *h, rt_profile_report *out, int32_t timeout_ms);

/* Block until all enqueued work of the handle has finished (bounded). */
rt_status rt_sync(rt_handle *h, int32_t timeout_ms);

/* Smoothing state (E, previous band luma, frame counter) as a byte blob.
 * rt_save_state: *len in = capacity of buf (buf NULL: only query), out =
 * bytes needed/written.  rt_load_state restores a blob saved by a handle of
 * the same configuration (RT_ERR_INVALID otherwise). */
rt_status rt_save_state(rt_handle *h, void *buf, size_t *len);
rt_status rt_load_state(rt_handle *h, const void *buf, size_t len);

/* Per-camera gains of ONE frame set without allocating anything.  No
 * counterpart in the paper: this is for callers that cannot call cudaMalloc
 * -- code that runs inside another framework's memory pool or allocator,
 * in a process whose device memory is reserved up front, or in a plug-in
 * that must not grow the device footprint -- and so cannot create a handle
 * (rt_array_config allocates its buffers).  It runs the band statistics and
 * the FP64 per-camera gain fit of the handle path's first frame set of a
 * sequence (no motion test, no smoothing history; defaults of
 * rt_default_params otherwise, BT.709, per-camera gains) and writes
 *   maps_dev  doubles [K][2][B][3][2] = (g, 0), as rt_get_gains;
 *   q16_dev   int32   [K][2][B][3][2] = round(65536 g), round(65536 * 0),
 * both DEVICE memory owned by the caller; the planes are device pointers
 * laid out as for rt_submit_frames.  All work is enqueued on cuda_stream
 * (cudaStream_t) and the call returns without waiting.
 * Limits (RT_ERR_INVALID beyond them): at most 16 cameras, 4 blocks, a band
 * width of 16 or 32, 2160 rows per camera.  Its working memory is one
 * 2.6 MB (2,632,704-byte) array inside librt.so that every GPU which loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address (make that first call before any
 * stream capture on the device).  Nothing is copied from host memory: the
 * work list and seam tables travel in a kernel's parameter block.
 * Every call uses the same array: calls whose work overlaps on the GPU race
 * with each other; the array keeps the last call's contents, and the
 * statistics part is cleared at the start of every call. */
rt_status rt_fit_gains_noalloc(const rt_camera_desc *cams, int32_t num_cameras,
                               const void *const *y_planes, const void *const *uv_planes,
                               int32_t strip_width, int32_t num_blocks, int32_t topology,
                               double *maps_dev, int32_t *q16_dev, void *cuda_stream);

/* Text of the last error on this handle (or of the last failed
 * rt_array_config when h is NULL).  Valid until the next call. */
const char *rt_last_error(rt_handle *h);

/* Wait (bounded) for pending work, free every resource of the handle. */
void rt_destroy(rt_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* RT_H */
