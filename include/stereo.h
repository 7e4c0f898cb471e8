/*
 * stereo.h -- C ABI of the B300 dense stereo-matching library (libstereo.so).
 *
 * The library implements the per-pixel stereo-matching path of Zhou &
 * Jagadeesan, "Real-time Dense Reconstruction of Tissue Surface from Stereo
 * Optical Video" (arXiv 2007.12623), Section II, as hand-written CUDA for
 * sm_103a:
 *
 *   gray conversion -> ZNCC cost over the disparity range (Sec. II-A)
 *   -> winner-take-all + parabola sub-pixel -> left-right check
 *   -> 3 x (radial outlier removal -> radial hole fill -> disc hole fill)
 *      (Sec. II-B)
 *   -> improved Laplacian refinement with the ZNCC o-update (Sec. II-C,
 *      Eqs. 1-4)
 *
 * plus a differentiable soft-argmin variant (forward and backward).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All image, map and cost pointers are DEVICE pointers owned by the
 *    caller, unless a comment says "host".  The library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work on that stream and returns; no
 *    call synchronises the device, so outputs are ready once the caller
 *    synchronises the stream.
 *  - Images are 8-bit, row-major, `pitch` bytes between rows (pitch >=
 *    width * channels).  channels = 1 (gray) or 3 (interleaved RGB, reduced
 *    to gray with (77 R + 150 G + 29 B + 128) >> 8).
 *  - Disparity d maps left pixel x to right pixel x - d.  Candidates are
 *    d_min .. d_min + num_disp - 1 (1 <= num_disp <= 256); a candidate is
 *    valid only when its whole (2r+1)^2 window lies inside both images.
 *  - Invalid / unknown disparities are STEREO_INVALID in int16 maps and NaN
 *    in float maps.
 *  - Errors are returned as stereo_status; arguments are checked on the host
 *    before anything is enqueued, so a call that fails with
 *    STEREO_ERR_INVALID_ARG or STEREO_ERR_UNSUPPORTED has enqueued nothing.
 *    No C++ exception crosses this boundary.  No kernel of this library waits
 *    on another, so no call returns STEREO_ERR_TIMEOUT (kept for callers'
 *    code).  The checked build of the library (libstereo_checked.so,
 *    compiled with -DSTEREO_CHECKED, for testing) checks the index ranges of
 *    its staged-row copies, cost stores, mask-word reads and writes,
 *    candidate loads, preparation writes and sub-pixel writes inside the
 *    kernels; a failed check records ST_DEVERR_BOUNDS (0x1000) | site in a
 *    device error word and skips the access (nothing traps), read and
 *    cleared with stereo_get_device_error().
 *  - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef STEREO_H
#define STEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STEREO_INVALID (-32768)
#define STEREO_MAX_DISP 256
#define STEREO_MAX_WIN_RADIUS 7

typedef enum {
    STEREO_OK = 0,
    STEREO_ERR_INVALID_ARG = 1,   /* NULL/misaligned pointer, bad size ...  */
    STEREO_ERR_CUDA = 2,          /* a CUDA runtime call failed             */
    STEREO_ERR_OOM = 3,           /* workspace allocation failed            */
    STEREO_ERR_UNSUPPORTED = 4,   /* valid request the library cannot serve */
    STEREO_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (unused) */
    STEREO_ERR_TOO_LARGE = 6      /* request exceeds the handle's capacity  */
} stereo_status;

typedef enum { STEREO_SAMPLE_FULL = 0, STEREO_SAMPLE_CHESSBOARD = 1 } stereo_sampling;

typedef enum {
    STEREO_COST_NONE = 0,   /* cost volume not kept (recomputed when needed) */
    STEREO_COST_F32 = 1,
    STEREO_COST_F16 = 2,
    STEREO_COST_BF16 = 3
} stereo_cost_dtype;

/* Method parameters.  Defaults (stereo_default_params) are the paper's
 * values: 11x11 window (Sec. II-A), outlier threshold 2.5 and 3 rounds with
 * radius 10, 20, 30 (Sec. II-B), hole-filling radii 50 and 20 (Sec. II-B),
 * smoothing radius 15, alpha 0.1, search +-5, eta 0.01 (Sec. II-C). */
typedef struct {
    int32_t max_width, max_height;  /* workspace sizing                        */
    int32_t d_min, num_disp;        /* candidate range                         */
    int32_t win_radius;             /* r: (2r+1)^2 window, 1..7                */
    int32_t sampling;               /* stereo_sampling                         */
    int32_t cost_dtype;             /* stereo_cost_dtype kept for refinement   */
    int32_t lr_thresh;              /* keep iff |dL - dR(x - dL)| <= thresh    */
    int32_t outlier_rounds, r0, dr; /* round t uses radius r0 + t*dr           */
    float outlier_thresh;           /* neighbouring disparities differ < this  */
    int32_t fill_radial_r;          /* radial search length                    */
    int32_t fill_radial_min_dirs;   /* directions needed to fill               */
    int32_t fill_disc_r;            /* disc radius                             */
    int32_t fill_disc_min_count;    /* valid pixels needed; -1 = 1/4 of disc   */
    int32_t smooth_radius;          /* box radius of Eqs. (1) and (3)          */
    int32_t smooth_iters;           /* K                                       */
    float alpha;                    /* Eq. (2)                                 */
    float eta;                      /* Eq. (4)                                 */
    int32_t refine_search;          /* o* in [d - S, d + S]                    */
    int32_t soft_argmin;            /* 1: also allocate the soft-argmin backward
                                       workspace (needs cost_dtype F32)       */
} stereo_params;

typedef struct stereo_handle stereo_handle;

/* One rectified stereo pair and its outputs.  Output pointers may be NULL
 * (not written).  disp_wta: winner-take-all disparity (int16); disp_sub:
 * disp_wta + parabola offset (float); disp_lr: after the left-right check
 * (int16); disp_post: after outlier removal / hole filling (int16); valid:
 * 1 where disp_post is valid (uint8); disp_final: refined disparity d^(K)
 * (float).  All maps are dense width*height, row stride = width. */
typedef struct {
    const uint8_t* left;
    const uint8_t* right;
    int32_t width, height, pitch, channels;
    int16_t* disp_wta;
    float* disp_sub;
    int16_t* disp_lr;
    int16_t* disp_post;
    uint8_t* valid;
    float* disp_final;
    /* Per-pair overrides used by stereo_match_batched (0 = handle's value;
     * d_min is used when num_disp != 0). */
    int32_t d_min, num_disp, win_radius;
} stereo_pair;

/* Fills *p with the paper's defaults (max_width/max_height 1920x1080,
 * d_min 0, num_disp 128, cost F32). */
void stereo_default_params(stereo_params* p);

/* Creates a handle and allocates its device workspace for up to `max_batch`
 * pairs of at most max_width x max_height with at most num_disp candidates.
 * The workspace belongs to the handle until stereo_destroy.  Returns
 * STEREO_ERR_OOM when the device allocation fails (*out untouched). */
stereo_status stereo_create(const stereo_params* p, int32_t max_batch, stereo_handle** out);

/* Frees the workspace and the handle.  Synchronises the handle's internal
 * work first.  NULL is accepted. */
stereo_status stereo_destroy(stereo_handle* h);

/* Whole path on one pair (Sec. II): gray -> ZNCC + WTA + sub-pixel ->
 * LR check -> outlier/hole loop -> Laplacian refinement.  Enqueued on
 * `stream`.  On a non-default stream the launch sequence is captured into a
 * CUDA graph on the first call with given pointers and sizes and replayed
 * on later calls with the same arguments; the handle keeps the graphs of the
 * 4 most recently used argument sets (e.g. the buffer sets of a
 * double-buffered loop).  When the caller's stream is itself being captured
 * the kernels are enqueued into the caller's capture.  Calls on one handle
 * share its workspace: they must be ordered (same stream, or synchronised). */
stereo_status stereo_match(stereo_handle* h, const stereo_pair* pair, void* stream);

/* The same path on n pairs of mixed sizes, disparity ranges (per-pair
 * d_min/num_disp) and windows (per-pair win_radius), n <= max_batch; pair i
 * uses workspace slot i.  The cost + winner-take-all stage of all pairs is
 * ONE persistent launch: resident warps take work units (pair, column run,
 * row band, disparity chunk) from a device counter.  The unit table is
 * rebuilt (and uploaded, outside any capture) when the pairs or the batch
 * configuration change.  When `use_graph` is non-zero and `stream` is not the
 * legacy default stream, the whole launch sequence is captured once into a
 * CUDA graph (keyed by the pairs' bytes) and replayed.  The per-pair stages
 * before and after the cost launch run on up to 8 streams owned by the
 * handle (parallel branches of the graph), forked from and joined back into
 * `stream`, so the call stays ordered on `stream`.  Returns
 * STEREO_ERR_UNSUPPORTED when called inside a caller's capture with pairs
 * that need new tables. */
stereo_status stereo_match_batched(stereo_handle* h, const stereo_pair* pairs, int32_t n,
                                   int32_t use_graph, void* stream);

/* Batch configuration: output rows per work unit (0 = default 16) and
 * disparities per lane K of the persistent cost launches (2 or 4 for every
 * pair; 0 = per pair, as the single-pair path splits its range: K = 2 for
 * D <= 64, K = 4 chunks of 128 disparities, and the rest of a range such as
 * D = 192 in K = 2 chunks of 64).  The K = 4 units and the K = 2 units run
 * as two persistent launches, one after the other. */
stereo_status stereo_set_batch_config(stereo_handle* h, int32_t rows, int32_t K);

/* How the per-pair stages of a batch (preparation, finalize, the outlier /
 * hole-filling rounds, the refinement iterations; Sec. II-B, II-C) run:
 * mode 0 (default) -- each pair's launches on up to 8 parallel streams
 * owned by the handle; mode 1 -- one launch per stage over all pairs of the
 * batch (a flat grid of every pair's blocks; each block finds its pair in a
 * table of cumulative block counts), with the per-pair launches as the
 * fallback when the post-processing or refinement parameters exceed the
 * tiled kernels' limits (outlier radius <= 64, radial fill radius <= 63,
 * disc radius <= 56, smoothing radius <= 32).  Both modes give the same
 * outputs bit for bit.  Returns STEREO_ERR_INVALID_ARG for another mode. */
stereo_status stereo_set_batch_stages(stereo_handle* h, int32_t mode);

/* The batch configuration in use: rows per unit, K (0 = per pair) and the
 * stage mode (any pointer may be NULL). */
stereo_status stereo_get_batch_config(const stereo_handle* h, int32_t* rows, int32_t* K, int32_t* stages);

/* Autotuner of the batched form: runs the batch once per candidate unit
 * configuration (K in {0 = per pair, 2, 4} x rows in {8, 12, 16, 24, 32,
 * 48}) and times the persistent cost stage with CUDA events; then times
 * whole passes in both stage modes with the fastest configuration, and keeps
 * the choices in the handle.  Synchronises `stream`; not allowed inside a
 * capture.  Writes the unit configuration and its cost-stage time (ms) when
 * the pointers are non-NULL (stereo_get_batch_config reads the stage mode). */
stereo_status stereo_autotune_batched(stereo_handle* h, const stereo_pair* pairs, int32_t n, void* stream,
                                      int32_t* best_rows, int32_t* best_K, float* best_ms);

/* Reads (and clears) the handle's device error word; synchronises `stream`
 * first.  *err = 0 when no device-side error was recorded.  In the checked
 * build it also reads and clears the words of the in-kernel index checks
 * (process-wide, one per translation unit of the library): the first failed
 * check's 0x1000 | site. */
stereo_status stereo_get_device_error(stereo_handle* h, int32_t* err, void* stream);

/* 1 in the checked build (in-kernel index checks), 0 otherwise. */
int32_t stereo_build_checked(void);

/* Checked build only: launches one check that cannot pass (an index one past
 * the end of a one-element buffer); its store is skipped and the error word
 * records 0x1000 | 0xfff.  STEREO_ERR_UNSUPPORTED in the normal build. */
stereo_status stereo_debug_check_selftest(void* stream);

/* Test hooks for allocation failures: after stereo_debug_fail_alloc(n) the
 * device allocation n + 1 calls later (counting every cudaMalloc that
 * stereo_create makes) fails as if the device had no memory left, without
 * calling cudaMalloc; n = -1 disarms.  stereo_create then returns
 * STEREO_ERR_OOM with everything it had allocated freed.
 * stereo_debug_live_allocations() counts the device allocations the
 * library's handles hold. */
stereo_status stereo_debug_fail_alloc(int32_t n);
int64_t stereo_debug_live_allocations(void);

const char* stereo_status_str(stereo_status s);

/* Tracing.  With stage timing on, stereo_match records CUDA events on its
 * stream around its stages: 0 input conversion, 1 window statistics, 2 cost
 * + winner-take-all kernel, 3 finalize (sub-pixel, LR check), 4 outlier /
 * hole-filling loop, 5 refinement.  stereo_match_batched does the same with
 * each stage covering all pairs of the batch (it then runs without a graph,
 * and one stage of every pair ends before the next stage starts).
 * The soft-argmin calls time their last pair: forward 0 statistics, 1 cost
 * kernel, 2 soft-argmin kernel (3..5 zero); backward 0 statistics, 1 cost
 * kernel, 2 dA kernel (A volume, per-pixel and diagonal sums), 3 window
 * sums of A with the T1 sums, 4 zero, 5 final gradient kernel.
 * stereo_get_stage_times waits for the last timed call of the handle and
 * writes min(n, STEREO_NUM_STAGES) durations in milliseconds. */
#define STEREO_NUM_STAGES 6
stereo_status stereo_set_stage_timing(stereo_handle* h, int32_t enable);
stereo_status stereo_get_stage_times(stereo_handle* h, float* ms, int32_t n);

/* Total number of CUDA kernels the library has enqueued since it was
 * loaded (all handles and streams). */
unsigned long long stereo_launch_count(void);

/* Process-wide tuning knobs.  "cost_rows": output rows per work unit of the
 * cost kernel (1..4096; 0 = automatic).  "soft_box_rows": output rows per
 * warp of the soft-argmin backward's window-sum kernel (1..4096; 0 =
 * automatic).  "graphs": 1 (default) replays
 * stereo_match / stereo_match_batched as captured CUDA graphs on non-default
 * streams, 0 launches kernels one by one.  Returns STEREO_ERR_INVALID_ARG
 * for an unknown name or value. */
stereo_status stereo_set_tuning(const char* name, int32_t value);

/* ------------------------------------------------------------------------
 * Stage entry points.  Each runs one step of the path on caller buffers, so
 * every step can be fed its input independently (stage-wise parity).
 * ---------------------------------------------------------------------- */

/* RGB (interleaved, `pitch` bytes per row) -> gray, (77R+150G+29B+128)>>8. */
stereo_status stereo_gray(const uint8_t* rgb, int32_t width, int32_t height, int32_t pitch,
                          uint8_t* gray, void* stream);

/* Sec. II-A: ZNCC of every valid candidate, winner-take-all for the left
 * view (ties -> smallest d) and for the right view (best left pixel u + d
 * for each right pixel u; used by the LR check), parabola sub-pixel offset
 * on c = 1 - ZNCC (its three costs read from an FP32 volume, else computed
 * in FP32 from the images: a parabola through FP16/BF16-rounded costs would
 * be off by up to ~0.03 px).  left/right: gray, row stride = width.  disp_left,
 * disp_right: int16 W*H; disp_sub: float W*H (NaN where invalid);
 * cost: optional [H][W][num_disp] volume of c = 1 - ZNCC in `cost_dtype`
 * (NaN for invalid candidates), NULL when cost_dtype is STEREO_COST_NONE.
 * Uses the handle's workspace; width/height/num_disp must fit the handle. */
stereo_status stereo_stage_match(stereo_handle* h, const uint8_t* left, const uint8_t* right,
                                 int32_t width, int32_t height, int32_t d_min, int32_t num_disp,
                                 int32_t win_radius, int32_t sampling, int32_t cost_dtype,
                                 int16_t* disp_left, int16_t* disp_right, float* disp_sub,
                                 void* cost, void* stream);

/* Left-right consistency check: out(x) = dL(x) when dL(x) is valid, x - dL(x)
 * is inside the image, dR(x - dL(x)) is valid and |dL - dR| <= thresh; else
 * STEREO_INVALID. */
stereo_status stereo_stage_lr(const int16_t* disp_left, const int16_t* disp_right, int32_t width,
                              int32_t height, int32_t thresh, int16_t* out, void* stream);

/* Sec. II-B radial outlier removal with the given radius (one pass).  Uses
 * the handle's workspace (line bitmasks); width/height must fit it. */
stereo_status stereo_stage_outlier(stereo_handle* h, const int16_t* in, int32_t width,
                                   int32_t height, int32_t radius, float thresh, int16_t* out,
                                   void* stream);

/* Sec. II-B first hole-filling method (8 radial directions).  Uses the
 * handle's workspace; width/height must fit it. */
stereo_status stereo_stage_fill_radial(stereo_handle* h, const int16_t* in, int32_t width,
                                       int32_t height, int32_t radius, int32_t min_dirs,
                                       int16_t* out, void* stream);

/* Sec. II-B second hole-filling method (disc), radius <= 56: a hole takes
 * the mean (rounded half up) of the valid pixels within Euclidean distance
 * `radius` when there are at least min_count of them.  min_count < 0 means a
 * quarter of the disc's pixel count, rounded up.  Uses no workspace memory
 * (width/height must still fit the handle). */
stereo_status stereo_stage_fill_disc(stereo_handle* h, const int16_t* in, int32_t width, int32_t height,
                                     int32_t radius, int32_t min_count, int16_t* out,
                                     void* stream);

/* Sec. II-B loop: `params->outlier_rounds` rounds of outlier removal (radius
 * r0 + t*dr) -> radial fill -> disc fill.  Uses the handle's workspace. */
stereo_status stereo_stage_postprocess(stereo_handle* h, const int16_t* in, int32_t width,
                                       int32_t height, int16_t* out, void* stream);

/* Sec. II-C refinement (Eqs. 1-4) for the handle's parameters.  o_in: int16
 * discrete disparities (STEREO_INVALID = none).  cost: [H][W][num_disp]
 * volume of 1 - ZNCC in cost_dtype (NaN = invalid candidate); when cost_dtype
 * is STEREO_COST_NONE the ZNCC is recomputed from left/right (gray).
 * d_out: float d^(K) (NaN where invalid); o_out: final int16 o (may be NULL). */
stereo_status stereo_stage_refine(stereo_handle* h, const int16_t* o_in, const void* cost,
                                  int32_t cost_dtype, const uint8_t* left, const uint8_t* right,
                                  int32_t width, int32_t height, int32_t d_min, int32_t num_disp,
                                  int32_t win_radius, float* d_out, int16_t* o_out, void* stream);

/* ------------------------------------------------------------------------
 * Differentiable soft-argmin variant (not in the paper): for every pixel,
 * p_d = softmax over the valid candidates of ZNCC(d) / tau and
 * d_soft = sum_d d p_d.  Images are float (batch x height x width,
 * contiguous, row stride = width); the handle must have been created with
 * soft_argmin = 1 (and cost_dtype F32) and sized for width, height,
 * num_disp.  Any tau > 0: below 0.025, where exp((ZNCC - 1) / tau) could
 * underflow for every candidate, the forward pass takes each pixel's
 * weights relative to its best candidate; win_radius <= 7.  Pixels without
 * a valid candidate get NaN.
 * ---------------------------------------------------------------------- */

/* Forward: d_soft and the log-sum-exp of the logits (both float B*H*W).
 * With num_disp <= 128 (one chunk of the cost kernel) the weights are summed
 * inside the cost kernel and no cost volume is written; larger num_disp
 * goes through the FP32 volume in the handle's workspace. */
stereo_status stereo_softargmin_fwd(stereo_handle* h, const float* left, const float* right,
                                    int32_t batch, int32_t width, int32_t height, int32_t d_min,
                                    int32_t num_disp, int32_t win_radius, float tau, float* d_soft,
                                    float* lse, void* stream);

/* Backward: given the forward outputs and grad_dsoft = dLoss/d d_soft
 * (float B*H*W), writes dLoss/dleft and dLoss/dright (float B*H*W).  Window
 * statistics and ZNCC are recomputed, not taken from the forward call (with
 * num_disp <= 128 inside the kernel that forms the backward terms; larger
 * num_disp through the FP32 volume).  A pixel whose d_soft is NaN (the
 * forward found no valid candidate) contributes nothing. */
stereo_status stereo_softargmin_bwd(stereo_handle* h, const float* left, const float* right,
                                    int32_t batch, int32_t width, int32_t height, int32_t d_min,
                                    int32_t num_disp, int32_t win_radius, float tau,
                                    const float* d_soft, const float* lse, const float* grad_dsoft,
                                    float* grad_left, float* grad_right, void* stream);

/* L1 loss of d_soft (n floats) against gt over the pixels where d_soft is
 * not NaN: *loss = mean |d_soft - gt| (device float), grad = sign(d_soft -
 * gt) / count, 0 elsewhere (device float n; may be NULL).  Needs a handle
 * created with soft_argmin = 1. */
stereo_status stereo_l1_loss(stereo_handle* h, const float* d_soft, const float* gt, int64_t n,
                             float* loss, float* grad, void* stream);

/* Calibration of a rectified pair: focal length f (pixels), principal point
 * (cx, cy) of the left camera (pixels), baseline (any length unit; points
 * come out in it), doffs = right principal point x minus left principal
 * point x (pixels). */
typedef struct {
    float f, cx, cy, baseline, doffs;
} stereo_camera;

/* Sec. II, depth from disparity (the reprojection of a rectified pair): for
 * every pixel (u, v) of the float disparity map `disp` (W*H, NaN = invalid,
 * e.g. disp_final) the point in the left camera frame
 *     Z = f baseline / (d + doffs), X = (u - cx) Z / f, Y = (v - cy) Z / f
 * (NaN where d is NaN or d + doffs <= 0), and its normal: the cross product
 * of the central differences (P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1)),
 * turned to face the camera and normalised (NaN on the image border, next
 * to a NaN point, or where the product vanishes).  xyz and normals are
 * float [H][W][3] device arrays; either may be NULL.  No handle needed. */
stereo_status stereo_depth_points(const float* disp, int32_t width, int32_t height, const stereo_camera* cam,
                                  float* xyz, float* normals, void* stream);

/* Histogram-voting preselection of feature-match inliers (Sec. II):
 * displacements (u2 - u1, v2 - v1) of n matches (uv1, uv2: float [n][2]
 * device arrays) are binned into an nb x nb histogram of bins of side `bin`
 * over [-range, range)^2, nb = stereo_vote_nbins(bin, range) (bin index
 * floor((d + range) / bin) in single precision; a displacement outside the
 * range votes for no bin); score[i] = the counts of the 3x3 bins around
 * match i's own (0 without a bin); order = the match indices by score,
 * higher first, ties by index.  hist (int32 nb*nb), score and order (int32
 * n) are caller-owned device arrays and all three are written.  n <= 16384
 * (STEREO_ERR_TOO_LARGE beyond), nb <= 4096. */
int32_t stereo_vote_nbins(float bin, float range);
stereo_status stereo_vote_matches(const float* uv1, const float* uv2, int32_t n, float bin, float range,
                                  int32_t* hist, int32_t* score, int32_t* order, void* stream);

/* Surface model of the point-based TSDF mosaicking (Sec. II, GPU-based TSDF
 * mosaicking): caller-owned device arrays of `capacity` points -- world
 * position (float [capacity][3]), RGB colour 0..255 (float [capacity][3]),
 * position weight and colour weight (float [capacity]) -- and two device
 * int32: count (points in use; read and updated) and dropped (written: new
 * points of the last call that did not fit). */
typedef struct {
    float* pos;
    float* rgb;
    float* wpos;
    float* wrgb;
    int32_t* count;
    int32_t* dropped;
    int32_t capacity;
} stereo_point_model;

/* Mosaics one key frame into the model: xyz = the frame's points in its
 * camera frame (float [H][W][3], NaN = no depth; e.g. stereo_depth_points of
 * disp_final), rgb = its colour image (u8 [H][W][3]), cam = its intrinsics
 * (f, cx, cy), R (9 floats, row-major) and t (3 floats) = the pose mapping
 * world to camera coordinates (host arrays).  Model points are projected
 * into the image (nearest point per pixel, in single precision: u =
 * floor(f X/Z + cx + 1/2)); a pixel with a point whose camera depth is
 * within `tau` of the projected model point's merges into it (position:
 * running mean, weight + 1; colour: mean weighted by the pixel's colour
 * weight, 1 inside the central disc of normalised radius r0 -- 1 at the
 * corners -- falling linearly to gmin at the corners); every other pixel
 * with a point is appended (row-major order) while capacity lasts.  Uses
 * the handle's workspace (width/height must fit the handle); ordered with
 * the handle's other calls. */
stereo_status stereo_mosaic_frame(stereo_handle* h, const stereo_point_model* model, const float* xyz,
                                  const uint8_t* rgb, int32_t width, int32_t height, const stereo_camera* cam,
                                  const float* R, const float* t, float tau, float r0, float gmin,
                                  void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant (no counterpart in the paper).
 *
 * For callers that must not allocate device memory at matching time -- e.g.
 * a real-time video pipeline that forbids allocation after start-up, or a
 * host that lends a plugin only its image and output buffers -- this runs
 * the same cost + winner-take-all stage as stereo_stage_match with
 * STEREO_COST_NONE (left and right WTA maps, sub-pixel from recomputed ZNCC)
 * without a handle: its scratch is a fixed 16 MiB device array inside the
 * library, which every GPU that loads the library keeps until process exit.
 * Limits: width <= 640, height <= 480, num_disp <= 128, |d_min| <= 64,
 * win_radius 1..7; larger requests return STEREO_ERR_TOO_LARGE and enqueue
 * nothing.  It calls no allocation routine.  The first call on each device
 * looks up the array's device address, so make it before any stream capture.
 * Every call reuses the same array: calls must not overlap on the GPU (use
 * one stream, or order them with events), or they race.  left/right: gray,
 * row stride = width; disp_left/disp_right: int16 W*H; disp_sub: float W*H
 * (may be NULL).
 * ---------------------------------------------------------------------- */
stereo_status stereo_match_wta_noalloc(const uint8_t* left, const uint8_t* right, int32_t width,
                                       int32_t height, int32_t d_min, int32_t num_disp,
                                       int32_t win_radius, int16_t* disp_left, int16_t* disp_right,
                                       float* disp_sub, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STEREO_H */
