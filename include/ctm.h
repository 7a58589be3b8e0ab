/*
 * ctm.h -- C ABI of the GB300 census template-matching library (libctm.so).
 *
 * Object-centric stereo ranging by Census template matching, arXiv 2604.07980,
 * Sec. 4.3 and Algorithm 2: for every detection box, census codes of the left
 * and right images (Sec. 4.3.1), an exhaustive Hamming-cost search per block
 * (Eq. census_cost) with first argmin and parabola refinement (Eq. subpixel),
 * a backward search and consistency test (Sec. 4.3.3), occlusion-aware point
 * sampling (Sec. 4.3.5), the far/close split and robust aggregation
 * (Sec. 4.3.4), and depth Z = f b / d (Eq. 1).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *    The caller owns every image, box and output buffer.  A context owns its
 *    workspace (census planes, plan, block results, counters).
 *  - Calls are asynchronous on `stream` unless stated otherwise; results are
 *    valid once that stream has synchronized.  A context is not thread-safe and
 *    must not run two calls concurrently on different streams.
 *  - Return value: CTM_OK (0) or a negative CTM_E* status.  Per-box outcomes
 *    are flags (CTM_BOX_*), never errors.  On error nothing has been enqueued
 *    unless the status is CTM_ECUDA; after CTM_ECUDA from a match call the
 *    context's device state is undefined and the context should be destroyed.
 *  - Disparities are in full-resolution pixels; the right-image match of a left
 *    pixel x is at x - d (d >= 0 for objects in front of the cameras).
 *  - No entry point falls back to a CPU implementation.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_ctx ctm_ctx;
/* A cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *ctm_stream;

/* Status codes. */
#define CTM_OK 0
#define CTM_EINVAL (-1)   /* bad argument: null pointer, size, window, range, pitch */
#define CTM_ENOMEM (-2)   /* workspace allocation failed or request exceeds capacity */
#define CTM_ECUDA (-3)    /* a CUDA call or launch failed */
#define CTM_ENODEV (-4)   /* no usable CUDA device */
#define CTM_ETOOBIG (-5)  /* beyond a fixed limit: ctm_match_boxes_noalloc's maxima, a server's frame size or arena */
#define CTM_EAGAIN (-6)   /* a server's admission queue is full; nothing was queued */
#define CTM_ETIMEOUT (-7) /* a bounded device-side wait expired: every box of the call that needed
                             a search has flags 0 and NaN outputs (returned by synchronous calls;
                             asynchronous ones set ctm_stats.error) */

/* Per-box flags (uint8), written by the match calls. */
#define CTM_BOX_VALID 0x01           /* disparity > 0 found; disp/depth finite         */
#define CTM_BOX_FB_REJECT 0x02       /* some block failed the forward-backward test     */
#define CTM_BOX_FEW_POINTS 0x04      /* some block had fewer than min_pts usable points */
#define CTM_BOX_NO_SEGMENT 0x08      /* CLOSE: no run of >= agg_nmin consistent blocks   */
#define CTM_BOX_NONPOS_DISP 0x10     /* the aggregated disparity was <= 0               */
#define CTM_BOX_EMPTY 0x20           /* box empty after clipping to the image           */
#define CTM_BOX_SUBPIX_CLAMPED 0x40  /* a valid block's argmin sat at a range end       */
#define CTM_BOX_FAR 0x80             /* classified FAR (matched at full resolution)     */
/* A box that needed a search carries flags 0 (neither VALID nor any reason bit)
 * and NaN disparity and depth when a bounded device wait of its call expired:
 * some of its blocks may not have been searched, so it is not aggregated. */

/* Per-block flags (ctm_block.flags). */
#define CTM_BLK_VALID 0x01
#define CTM_BLK_FB_REJECT 0x02
#define CTM_BLK_FEW_POINTS 0x04
#define CTM_BLK_SUBPIX_CLAMPED 0x08
#define CTM_BLK_PRESENT 0x10

/* Detection box: half-open rectangle [x0, x1) x [y0, y1) in full-resolution
 * pixels of its frame.  `frame` is informational; frame membership comes from
 * ctm_frame.box_begin / box_count. */
typedef struct {
    int32_t x0, y0, x1, y1, frame;
} ctm_box;

/* One stereo frame of a batch.  left/right: uint8 grayscale, `pitch` bytes per
 * row (pitch >= width).  Boxes [box_begin, box_begin + box_count) belong to it.
 * f_px * baseline_m is the Eq. 1 numerator. */
typedef struct {
    const uint8_t *left;
    const uint8_t *right;
    int32_t width, height, pitch;
    int32_t box_begin, box_count;
    float f_px, baseline_m;
} ctm_frame;

/* Matching parameters (Sec. 4.3).  Limits checked by ctm_create:
 * odd win_w, win_h <= 15 with win_w*win_h + sentinel <= 64; close_factor 1..8;
 * grid_g 1..8; pts_side 1..16; (dmax-dmin+1)*(dy_max-dy_min+1) <= 256 for both
 * ranges; min_pts >= 1; fb_tol >= 0; agg_nmin >= 1; 0 <= trim_frac < 0.5;
 * 0 <= max_occluders <= 32, 0 <= frontal_crop <= 1. */
typedef struct {
    int32_t win_w, win_h;     /* census window (Sec. 4.3.1: S_x = win_w/2, S_y = win_h/2) */
    int32_t sentinel;         /* 1: leading 1 bit above the comparison bits (Algorithm 1) */
    int32_t far_side_px;      /* tau_s: FAR iff max(clipped w, h) < tau_s; 0 = never FAR */
    int32_t close_factor;     /* k: CLOSE boxes match on the census of I(k x, k y)        */
    int32_t far_dmin, far_dmax;     /* FAR search range, full-res px                      */
    int32_t close_dmin, close_dmax; /* CLOSE search range, px of the decimated grid       */
    int32_t dy_min, dy_max;   /* vertical search range of both passes                    */
    int32_t grid_g;           /* CLOSE box -> grid_g x grid_g blocks                      */
    int32_t pts_side;         /* at most pts_side x pts_side points per block             */
    int32_t min_pts;          /* a block needs >= min_pts usable points                   */
    int32_t fb_tol;           /* accept iff |d_b - d_f| <= fb_tol (tau_v = fb_tol + 1)    */
    float agg_tau_d;          /* run: consecutive sorted differences < tau_d (full-res)   */
    int32_t agg_nmin;         /* run must hold >= agg_nmin blocks (N_min)                 */
    int32_t agg_mode;         /* 0: median of the run; 1: trimmed mean of the run         */
    float trim_frac;          /* trimmed mean drops floor(trim_frac * m) per end          */
    int32_t max_occluders;    /* at most this many occluders per box (Sec. 4.3.5)         */
    float frontal_crop;       /* ranking of occluders beyond the cap: 0 = nearest (largest
                                 bottom y) first; c in (0, 1] = those whose clipped box
                                 centre lies in the centred c W x c H crop first, each
                                 group nearest first (ties: lower index)                 */
} ctm_params;

/* Per-block diagnostic record (ctm_debug.blocks), slot = block index in
 * row-major grid order (FAR boxes use slot 0). */
typedef struct {
    int32_t n_pts, n_valid;
    int32_t d_f, dy_f, d_b, dy_b;
    int32_t s_m, s_0, s_p;    /* forward costs at d_f-1, d_f, d_f+1 (0 outside range) */
    float d_sub;              /* refined disparity on the matching grid                */
    float d_full;             /* d_sub * k                                             */
    int32_t flags;            /* CTM_BLK_*                                             */
} ctm_block;

/* Optional diagnostics for parity checks (all device pointers, may be NULL).
 * blocks: n_boxes * slots entries, slots = grid_g^2 (records only for blocks
 * that exist; the caller zero-fills).  cost_f / cost_b: n_boxes * slots * nc_stride
 * int32, nc_stride = max FAR/CLOSE candidate count, candidate c =
 * (dy - dy_min) * N_d + (d - dmin). */
typedef struct {
    ctm_block *blocks;
    int32_t *cost_f;
    int32_t *cost_b;
} ctm_debug;

/* Launch-shape tuning of a context (no effect on results).  Not described
 * by the paper: these are choices of this implementation's kernels. */
typedef struct {
    int32_t match_threads;  /* matching CTA size: 128 or 256 threads                    */
    int32_t strip_cols;     /* width, in codes, of the staged strip of one column chunk
                               of a block: a multiple of 8, at least the larger
                               disparity range + 2; larger values mean fewer chunks
                               and more shared memory per CTA                         */
    int32_t census_mode;    /* region-of-interest census (5x5, 7x7, 9x7 windows): 0 =
                               integer multiply-add compares, 4 CTAs per SM; 1 = the
                               same, 3 CTAs per SM; 2 = packed fp16 compares with
                               saturation, 4 CTAs per SM                              */
    int32_t queue_rounds;   /* fused matcher: 1 = the first blocks of a launch go out in
                               per-SM rounds (every SM one block of each round; the
                               queue runs from the largest blocks down), 0 = one
                               dynamic queue                                          */
    int32_t match_mode;     /* 0: fused matcher (one CTA runs both passes of a block);
                               1: two-pass pipelined matcher (a forward kernel, then a
                               backward kernel; each CTA loads its next block while it
                               scans the current one)                                 */
    int32_t split_ways;     /* fused matcher only: 0 = split every block's candidate range
                               into two (block, disparity-chunk) tiles when the queue
                               holds fewer than about 0.6 blocks per resident CTA and
                               the CLOSE range has at least 128 candidates; 1 = never
                               split; 2, 4 or 8 = always split into that many chunks.
                               Splitting needs one vertical offset (dy_min == dy_max) */
} ctm_tuning;

/* Counters of the last match call (ctm_get_stats). */
typedef struct {
    uint64_t cost_evals;   /* popcount(C_L xor C_R) evaluations, both passes */
    int32_t n_blocks;      /* blocks planned                                  */
    int32_t n_boxes;       /* boxes planned                                   */
    int32_t error;         /* nonzero: a bounded device wait expired and some
                              outputs of the call were not written            */
    int32_t census_tiles;  /* 32-pixel census row tiles computed (region of
                              interest of the batched and single-frame calls) */
    uint64_t host_bytes;   /* image bytes read from host memory by the device
                              (ctm_match_batch_mapped; 0 for other calls)      */
} ctm_stats;

/* Human-readable name of a status code (static string). */
const char *ctm_status_str(int status);

/* Fill *p with the library defaults (9x7 census with sentinel, tau_s 40, k 2,
 * FAR 0..31, CLOSE 0..127, dy 0, 4x4 blocks of <= 16x16 points, min_pts 16,
 * fb_tol 1, tau_d 1.0, N_min 6, median, 16 occluders). */
int ctm_default_params(ctm_params *p);

/* Create a context on the current CUDA device with capacity for max_frames
 * frames of at most max_width x max_height pixels and max_boxes boxes per call.
 * Allocates the device workspace (about 2.6 * 8 bytes per pixel per frame plus
 * per-box plans).  Errors: CTM_EINVAL (params or sizes), CTM_ENOMEM, CTM_ENODEV. */
int ctm_create(ctm_ctx **out, const ctm_params *p, int max_frames, int max_width,
               int max_height, int max_boxes);

/* Free the context and its workspace (synchronizes the device). NULL is a no-op. */
void ctm_destroy(ctm_ctx *ctx);

/* Census transform, Sec. 4.3.1 / Algorithm 1, of the decimated image
 * I_k(x, y) = I(k x, k y) (k = factor; k = 1 is the image itself).
 * img_dev: width x height uint8, `pitch` bytes per row.  codes_dev: uint64,
 * ceil(height/k) rows of codes_pitch elements (codes_pitch >= ceil(width/k)).
 * Bits are in raster window order, first neighbour highest; xi(a, b) = a > b;
 * with sentinel the bit win_w*win_h is set; pixels whose window leaves the
 * decimated image are 0.  No context needed.  Errors: CTM_EINVAL, CTM_ECUDA. */
int ctm_census_build(const uint8_t *img_dev, int width, int height, int pitch, int factor,
                     int win_w, int win_h, int sentinel, uint64_t *codes_dev,
                     int64_t codes_pitch, ctm_stream stream);

/* Algorithm 2 on one frame.  boxes_dev: n_boxes ctm_box (0 <= n_boxes <=
 * max_boxes).  Outputs (n_boxes each): disp_dev (float, full-res px, NaN unless
 * VALID), depth_dev (float, f_px*baseline_m/disp, NaN unless VALID), flags_dev
 * (uint8 CTM_BOX_*).  dbg may be NULL.  The launch sequence of the batch path on
 * one frame: device planning and point sampling, the census of the row tiles the
 * search reads (both images, both resolutions), one persistent matching kernel
 * and a per-box aggregation kernel.  Errors: CTM_EINVAL, CTM_ENOMEM (beyond
 * capacity), CTM_ECUDA. */
int ctm_match_boxes(ctm_ctx *ctx, const uint8_t *left_dev, const uint8_t *right_dev,
                    int width, int height, int pitch, const ctm_box *boxes_dev, int n_boxes,
                    float f_px, float baseline_m, float *disp_dev, float *depth_dev,
                    uint8_t *flags_dev, const ctm_debug *dbg, ctm_stream stream);

/* The plain per-box path: same inputs, outputs and results as ctm_match_boxes,
 * but one matching launch per box (no persistent queue, no graph). */
int ctm_match_boxes_plain(ctm_ctx *ctx, const uint8_t *left_dev, const uint8_t *right_dev,
                          int width, int height, int pitch, const ctm_box *boxes_dev,
                          int n_boxes, float f_px, float baseline_m, float *disp_dev,
                          float *depth_dev, uint8_t *flags_dev, ctm_stream stream);

/* Algorithm 2 on a batch of frames in one planned, persistent launch.
 * frames_dev: ctm_frame array in device memory; counts_dev: int32[2] in device
 * memory = {n_frames, n_boxes} (read on the device, so a captured graph replays
 * with new counts); boxes and outputs as in ctm_match_boxes, indexed over the
 * whole batch.  Counts beyond the context capacity are clamped on the device.
 * use_graph != 0 captures the launches into a CUDA graph on first use and
 * replays it while all pointers stay the same.  Errors: CTM_EINVAL, CTM_ECUDA. */
int ctm_match_batch(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                    const ctm_box *boxes_dev, float *disp_dev, float *depth_dev,
                    uint8_t *flags_dev, const ctm_debug *dbg, int use_graph, ctm_stream stream);

/* ctm_match_batch without a graph, recording eight caller-created CUDA events
 * (cudaEvent_t handles, created with timing enabled) on `stream` around its
 * launches: events[0] before planning, [1] before point sampling (which also
 * marks the census demand), [2] before the census (tile list and
 * region-of-interest kernel), [3] before matching, [4] before the per-box
 * aggregation, [5], [6] and [7] after it.  Used to time each
 * phase on the stream the kernels run on.  Errors as ctm_match_batch. */
int ctm_match_batch_profiled(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                             const ctm_box *boxes_dev, float *disp_dev, float *depth_dev,
                             uint8_t *flags_dev, void *const events[8], ctm_stream stream);

/* End-to-end batch from host memory: frames_host[i].left/right are HOST images
 * (page-locked for asynchronous copies), boxes_host and the outputs are host
 * arrays.  Copies the images and boxes in, runs the batched path, copies the
 * results out and synchronizes `stream` before returning.  When every frame's
 * boxes directly follow the previous frame's (box_begin of frame i + 1 = box_begin
 * + box_count of frame i), the frames go in up to 4 sub-batches: the copies of
 * sub-batch g + 1 (on a stream of the context) overlap the kernels of sub-batch
 * g (on `stream`), with results equal to one batch's; ctm_get_stats afterwards
 * sums the sub-batches.  Images packed at the staging pitch (pitch == width ==
 * max_width rounded up to 128) and, for runs of more than one, full height
 * (max_height) and laid out back to back in host memory as L0 R0 L1 R1 ... go
 * in one copy per sub-batch.  Errors as above, and CTM_ETIMEOUT when a bounded
 * device wait of the call expired (outputs incomplete; the context stays usable). */
int ctm_match_batch_host(ctm_ctx *ctx, const ctm_frame *frames_host, int n_frames,
                         const ctm_box *boxes_host, int n_boxes, float *disp_host,
                         float *depth_host, uint8_t *flags_host, ctm_stream stream);

/* End-to-end batch from host memory that moves only the image bytes the census
 * reads (no counterpart in the paper; same arguments, results and errors as
 * ctm_match_batch_host).  The planner marks, before any pixel moves, which
 * 32-pixel census tiles the search will read (Algorithm 2's blocks and their
 * disparity strips); a device kernel then reads, straight from the caller's
 * host images, the 64-byte segments of source rows those tiles' windows cover
 * and writes them into the context's staging images, and the batched path runs
 * on those.  A frame is read in place when the device can read its images at
 * their host address (page-locked memory, or any host memory where the device
 * reports pageable memory access, cudaDevAttrPageableMemoryAccess, e.g. GB300
 * with its host) and left, right, pitch and width are multiples of 16 bytes;
 * any other frame is copied whole first.  The host must not write the images
 * during the call.  One batch, no sub-batches; ctm_get_stats reports the bytes
 * read in place from host memory (host_bytes).  Synchronizes `stream` before
 * returning. */
int ctm_match_batch_mapped(ctm_ctx *ctx, const ctm_frame *frames_host, int n_frames,
                           const ctm_box *boxes_host, int n_boxes, float *disp_host,
                           float *depth_host, uint8_t *flags_host, ctm_stream stream);

/* Single-frame matching that allocates no device memory -- the paper has no
 * counterpart.  It is for callers that cannot call cudaMalloc while they run:
 * real-time control loops, where an allocation can synchronize the device and
 * take an unbounded time, and hosts that give this library a fixed memory budget
 * when it starts.  Same inputs, outputs and results as ctm_match_boxes without a
 * context: `p` is the parameter block, all other arguments as there.  Limits:
 * width <= 640, height <= 480, n_boxes <= 64; larger requests return
 * CTM_ETOOBIG.  The workspace is one 8 MiB array in static device memory that
 * every GPU loading the library holds until exit.  The first call on a device
 * does a one-time set-up with that device current (looks up the array's device
 * address, raises the matching kernel's shared-memory limit).  All calls share
 * the array and it keeps the previous call's contents (each call clears what
 * must start at zero); calls that overlap on the GPU race.  Not thread-safe.
 * Calls no cudaMalloc, cudaFree or allocating library routine.  A bounded-wait
 * expiry leaves the outputs as the CTM_ETIMEOUT rule says and the flag in
 * ctm_noalloc_get_stats.
 * Errors: CTM_EINVAL, CTM_ETOOBIG, CTM_ENODEV, CTM_ECUDA. */
int ctm_match_boxes_noalloc(const ctm_params *p, const uint8_t *left_dev, const uint8_t *right_dev,
                            int width, int height, int pitch, const ctm_box *boxes_dev, int n_boxes,
                            float f_px, float baseline_m, float *disp_dev, float *depth_dev,
                            uint8_t *flags_dev, ctm_stream stream);

/* Counters of the most recent match call on ctx.  Synchronizes `stream`. */
int ctm_get_stats(ctm_ctx *ctx, ctm_stats *out, ctm_stream stream);

/* Counters of the most recent ctm_match_boxes_noalloc call on the current
 * device (error != 0: a bounded device wait of that call expired), read from
 * the static array after synchronizing `stream`; allocates nothing.
 * Errors: CTM_EINVAL (null out, or no such call on this device yet),
 * CTM_ENODEV, CTM_ECUDA. */
int ctm_noalloc_get_stats(ctm_stats *out, ctm_stream stream);

/* Camera geometry of one frame for ctm_box_points (Sec. 4.3.6). */
typedef struct {
    float Q[16];          /* 4x4 row-major reprojection matrix: [X Y Z W]^T = Q [u v d 1]^T  */
    float T[12];          /* 3x4 row-major camera-to-vehicle transform [R | t]                */
    float disp_var;       /* sigma_d^2 (px^2): the configured disparity variance              */
    float f_px, baseline_m;
    int32_t width, height;    /* image size: boxes are clipped to it                          */
    int32_t reserved;
} ctm_geometry;

/* Sec. 4.3.6 disparity-to-depth conversion and the covariance estimation, per
 * box, after a match call: box i uses geo_dev[boxes_dev[i].frame].  For a box
 * whose flags have CTM_BOX_VALID: (u, v) = centre of the box clipped to the
 * image, in pixel coordinates (pixel c spans [c, c+1), so u = (x0 + x1 - 1) / 2),
 * d = disp_dev[i]; [X Y Z W] = Q [u v d 1]; p = (X, Y, Z) / W in the camera
 * frame; p_v = R p + t in the vehicle frame; sigma_Z^2 = Z^4 sigma_d^2 / (f b)^2
 * with Z = p.z.  out_dev (float, n_boxes x 8, row-major): p.x, p.y, p.z, p_v.x,
 * p_v.y, p_v.z, sigma_Z^2, W; all NaN for boxes that are not VALID, whose frame
 * index is outside [0, n_geo), or whose W is 0.  fp32 arithmetic in a fixed
 * order (no contraction).  out_dev must be 16-byte aligned.  Errors: CTM_EINVAL
 * (null pointer, n < 0, unaligned out_dev), CTM_ECUDA. */
int ctm_box_points(const ctm_box *boxes_dev, const float *disp_dev, const uint8_t *flags_dev,
                   int n_boxes, const ctm_geometry *geo_dev, int n_geo, float *out_dev,
                   ctm_stream stream);

/* Sec. 5.1 auto-rectification offset, with census matching in place of BM (no
 * counterpart in the paper's own design, which uses BM disparities).  For every
 * delta in [delta_min, delta_max] and every pixel (x, y) of the ROI
 * [rx0, rx1) x [ry0, ry1) (clipped to the image): the left pixel is read at
 * (x, y + delta); d_f = first argmin over d in [dmin, dmax] of
 * popcount(C_L(x, y + delta) ^ C_R(x - d, y)); d_b = first argmin over d' of
 * popcount(C_R(x - d_f, y) ^ C_L(x - d_f + d', y + delta)); the pixel counts when
 * its left census is defined (window inside the image), |d_b - d_f| <= fb_tol and
 * d_f > d_thresh.  Codes outside the image read as 0.  The census window is
 * p's (win_w, win_h, sentinel).  census_dev: caller-owned scratch of
 * 2 * width * height uint64 (overwritten); counts_dev: delta_max - delta_min + 1
 * counters (zeroed, then the counts); *delta_dev: the first delta with the
 * largest count (device int).  Asynchronous on `stream`.  Errors: CTM_EINVAL
 * (null pointer, bad sizes or window, more than 1024 disparities), CTM_ECUDA. */
int ctm_auto_rect(const ctm_params *p, const uint8_t *left_dev, const uint8_t *right_dev, int width,
                  int height, int pitch, int rx0, int ry0, int rx1, int ry1, int dmin, int dmax,
                  int delta_min, int delta_max, int d_thresh, int fb_tol, uint64_t *census_dev,
                  unsigned long long *counts_dev, int *delta_dev, ctm_stream stream);

/* Sec. 5.1 temporal filter (host): the median of the last n per-frame offsets
 * (even n: the lower of the middle two), with the change from prev clamped to
 * [-max_step, max_step].  Returns the filtered offset; prev for n < 1. */
int ctm_rect_filter(const int *estimates, int n, int prev, int max_step);

/* Current tuning of a context. */
int ctm_get_tuning(const ctm_ctx *ctx, ctm_tuning *out);

/* Set the tuning (CTM_EINVAL if a field is out of range or the strip does not
 * fit in shared memory; the context keeps its previous tuning then).  A
 * captured batch graph is dropped and recaptured by the next graph call.
 * Synchronous; do not call while a stream capture is active. */
int ctm_set_tuning(ctm_ctx *ctx, const ctm_tuning *t);

/* Autotuner: runs the batch of ctm_match_batch (same arguments, no debug
 * output) under candidate tunings -- every matching CTA size x strip width,
 * for each matcher, then each census variant, rounds on and off and automatic
 * or no disparity-chunk tiles around the best so far --
 * timing `reps` calls of each with CUDA events after one warm-up call, keeps
 * the fastest in the context and returns it in *best (and its time per call,
 * in ms, in *best_ms; either may be NULL).  The outputs are written by every
 * call and do not depend on the tuning.  Synchronizes `stream`; not
 * capturable.  On error the previous tuning is restored. */
int ctm_autotune(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                 const ctm_box *boxes_dev, float *disp_dev, float *depth_dev, uint8_t *flags_dev,
                 int reps, ctm_tuning *best, float *best_ms, ctm_stream stream);

/* Integer-pipe probe for roofline denominators (no counterpart in the paper):
 * runs `iters` iterations of independent chains of one instruction on every
 * SM -- kind 0: 32-bit popcount, 1: 3-input xor, 2: packed fp16 greater-than
 * mask, 3: 32-bit add, 4: 32-bit multiply-add, 5: packed fp16 fused
 * multiply-add with saturation -- and returns the operations (packed
 * instructions for kinds 2 and 5) per SM clock per SM.  Synchronizes the device.  Errors: CTM_EINVAL, CTM_ECUDA. */
int ctm_probe_int_rate(int kind, int iters, double *ops_per_clk_per_sm);

/* Fault injection for tests (no counterpart in the paper): arms ctx so that the
 * next match call on it that launches the fused persistent matcher directly
 * (ctm_match_boxes, ctm_match_batch with use_graph = 0, ctm_match_batch_host;
 * tuning match_mode 0; not a graph replay, not the plain per-box path) has its
 * CTA that takes the queue's first block (or first tile) announce a strip copy
 * on its mbarrier without issuing it.  That CTA's bounded wait then expires (about 1 s, then about 1 s more for the
 * copies in flight, of which there are none), it records the error and stops;
 * the other CTAs finish the queue.  The call's outputs follow the CTM_ETIMEOUT
 * rule above, and ctm_match_batch_host returns CTM_ETIMEOUT.  The arming is
 * consumed by that one call; the context stays usable.  No GPU fault is
 * involved.  Errors: CTM_EINVAL (null ctx). */
int ctm_inject_wait_expiry(ctm_ctx *ctx);

/* Fault injection for tests (no counterpart in the paper): of the device
 * allocations the library makes from now on (context workspaces, host-path
 * staging, server arenas and lane buffers), the first `skip` go through and the
 * next n fail on the host as a cudaMalloc on an exhausted device does, so the
 * call that makes them returns CTM_ENOMEM after releasing what it had
 * allocated.  n = 0 disarms.  Process-wide; nothing runs on a GPU.
 * Errors: CTM_EINVAL (skip < 0 or n < 0). */
int ctm_inject_alloc_failures(int skip, int n);

/* Bounded-wait probe (no counterpart in the paper): one CTA waits, with the
 * matching kernels' own bounded-wait routine, on an mbarrier phase that nothing
 * completes; the wait gives up after its time limit (about 1 s, then the same
 * again for copies in flight, of which there are none), records the expiry in a
 * device flag and the kernel returns.  *expired gets the flag (1), *waited_ms
 * the kernel's duration.  Shows on a GPU that an expired wait ends the kernel
 * with an error status and leaves the context usable.  Synchronous.
 * Errors: CTM_EINVAL (null pointer), CTM_ECUDA. */
int ctm_probe_bounded_wait(int *expired, float *waited_ms);

#ifdef __cplusplus
}
#endif
#endif /* CTM_H */
