// ctm_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctm.h"

namespace ctm {

constexpr int kMaxPtsSide = 16;
constexpr int kMaxPts = kMaxPtsSide * kMaxPtsSide;
constexpr int kMaxCand = 256;                    // candidates per pass (8 slices of 32)
constexpr int kMaxGrid = 8;
constexpr int kMaxSlots = kMaxGrid * kMaxGrid;
constexpr int kMaxOcc = 32;
constexpr int kMaxWin = 15;
constexpr int kPlanThreads = 256;

// The sampling kernel queues every searchable block twice.  The first queue
// keeps the blocks near their neighbours (sampling order: boxes of a frame
// together, so blocks whose strips overlap run close in time and share the L2):
// blocks with at least kBigWork usable points x candidates from the front, the
// others from the back.  The second is ordered by decreasing work without a
// sort: one of kQueueClasses classes of usable points x candidates per block
// (half-octave classes down from the largest possible block, kMaxPts x
// kMaxCand), each class a region of max_blocks entries, positions running
// through the classes in order.  The fused persistent matcher takes the second
// when the whole queue goes out in its first wave (see match.cu).
constexpr int kBigWork = 4096;
constexpr int kQueueClasses = 16;
// Per-SM rounds of the fused persistent matcher: arrival counters for SM ids below
// kSchedSMs, then one claim counter per round.
constexpr int kSchedSMs = 256;
constexpr int kMaxRounds = 8;
constexpr int kSchedInts = kSchedSMs + kMaxRounds;

// Device-side counters of one call.
struct Counts {
    int n_frames;    // clamped to capacity
    int n_boxes;     // clamped to capacity
    int n_blocks;    // total planned blocks
    int queue_head;  // next entry of the persistent work queue
    int error;       // nonzero: a bounded device wait expired (results incomplete)
    unsigned long long evals;
    int n_big;       // searchable blocks queued from the front (large work)
    int n_small;     // searchable blocks queued from the back (small work)
    int n_tiles;     // census tiles listed for the region-of-interest census
    int n_class[kQueueClasses];  // searchable blocks in each work class (ws.queue_w)
    unsigned long long host_bytes;  // image bytes the gather read from host memory (mapped calls)
};

// Planned box (device).
struct BoxPlan {
    int cx0, cy0, cx1, cy1;   // clipped full-res rectangle
    int sx0, sy0, sx1, sy1;   // the same box on the matching grid
    int frame, far, k, g;
    int nblk, nocc, dmin, dmax;
    int Ws, Hs;               // matching-grid size of the frame
    float fb;                 // f_px * baseline_m
};

// Sampled point grid of one block (Sec. 4.3.4) with its usable points
// (Sec. 4.3.5), computed once by the sampling kernel.
struct __align__(16) BlockGeom {
    int16_t X[kMaxPtsSide];           // sampled columns on the matching grid
    int16_t Y[kMaxPtsSide];           // sampled rows
    uint16_t colmask[kMaxPtsSide];    // bit m of colmask[j]: point (X_j, Y_m) usable
    uint16_t colprefix[kMaxPtsSide];  // usable points in columns < j
    int32_t n_valid;
    int32_t nx, ny;
    uint32_t cstart;                  // bit j: a strip column chunk starts at column j
    // the block's box plan, copied so that a matcher needs only this record
    int32_t box, slot, frame, k, far, dmin, dmax, Ws, Hs;
    // forward-pass result, written by the two-pass matcher's forward kernel
    int32_t d_f, dy_f;                // first argmin of the forward costs
    int32_t s_m, s_0, s_p;            // costs at d_f - 1, d_f, d_f + 1 (0 where outside)
    int32_t pad[2];
};
static_assert(sizeof(BlockGeom) % 16 == 0, "BlockGeom is moved by 16-byte copies");

// State of a block split into disparity-chunk tiles (match.cu): first-minimum
// keys (cost << 16 | candidate) merged by atomicMin, finished-tile tickets per
// pass, and the forward result published to the backward tiles.  Reset by the
// sampling kernel for every searchable block.
struct ChunkState {
    unsigned fkey, bkey;
    int fdone, bdone;
    int ready;
    int d_f, s_m, s_0, s_p;
    int pad[3];
};

// Result of one block kept for the aggregation (device).
struct BlockResult {
    float d_full;
    int flags;
};

// Device workspace of a context.
// One census plane of one frame (L1, R1, Lk, Rk), written by the planner so the
// census kernels need no per-tile divisions or address arithmetic.
struct PlaneDesc {
    const uint8_t *img;  // source image (full resolution)
    uint64_t *out;       // census plane
    int W, pitch, k;     // source width, row pitch (bytes), decimation
    int Ws, Hs;          // census grid
    int opitch;          // census row pitch (elements)
    int vec_load;        // word loads allowed (k in {1, 2}, aligned base and pitch)
    int pad;
};

struct Workspace {
    uint64_t *census;          // per frame: L1, R1, Lk, Rk planes
    long long frame_stride;    // elements per frame
    long long plane1_elems;    // elements of one full-res plane
    long long planek_elems;    // elements of one decimated plane
    long long pitch1, pitchk;  // row pitch in elements
    BoxPlan *plans;            // [max_boxes]
    int4 *occ;                 // [max_boxes * kMaxOcc]
    int *nblk;                 // [max_boxes]
    int *blk_base;             // [max_boxes]
    int2 *blocks;              // [max_blocks] (box, slot), flat in box order
    BlockGeom *geom;           // [max_blocks] indexed like blocks
    int *queue;                // [max_blocks] searchable blocks: large from the front, small from the back
    int *queue_w;              // [kQueueClasses * max_blocks] the same blocks by work class; null: none
    int *sched;                // [kSchedInts] rounds of the fused persistent matcher; null: none
    BlockResult *blkres;       // [max_blocks]
    const CUtensorMap *tmaps;  // [max_frames * 4 * kBoxClasses] census planes L1, R1, Lk, Rk as 2-D
                               // tensors, one map per box width of one row of 32 c codes (strip
                               // loads by tile::gather4); null: 1-D bulk copies, one per row
    ChunkState *chunk;         // [max_blocks]; null: no disparity-chunk tiles
    int32_t *chunk_cost;       // [max_blocks * nc_stride] forward cost rows of split blocks
    Counts *counts;            // counters of the call in progress (zero between calls)
    Counts *stats;             // the last finished call's counters
    ctm_frame *frames;         // staging for single-frame calls [max_frames]
    int *counts_in;            // staging {n_frames, n_boxes}
    // census demand bitmap: one bit per kCensusTilePx-pixel tile of a plane row, per frame
    // planes in the order L1, R1, Lk, Rk; words = 32 tiles
    uint32_t *bitmap;
    unsigned long long *tiles;  // [max_frames * bm_frame_words * 32] marked tiles, packed (census.cu)
    PlaneDesc *planes;          // [max_frames * 4]
    long long bm_frame_words;
    int bm_plane_off[5];       // word offset of each plane within a frame (+ end)
    int bm_row_words[4];       // words per row of each plane
};

struct Caps {
    int max_frames, max_width, max_height, max_boxes, max_blocks;
};

// Arguments of the planning and matching kernels (passed by value).
struct MatchArgs {
    Workspace ws;
    Caps caps;
    ctm_params p;
    const ctm_frame *frames;   // device
    const int *counts_in;      // device {n_frames, n_boxes}
    const ctm_box *boxes;      // device
    float *disp;
    float *depth;
    uint8_t *flags;
    ctm_debug dbg;
    int nc_stride;
    int strip_cols;            // columns of the shared-memory strip
    int queue_rounds;          // 1: when its whole queue fits its first wave, the fused persistent
                               // matcher hands the blocks out in per-SM rounds from the
                               // work-ordered queue (needs ws.queue_w, ws.sched); 0: never
    int sm_count;              // SMs of the device (rounds are sm_count positions wide)
    int match_mode;            // 0: fused single-kernel matcher, 1: two-pass pipelined matcher
    int split_ways;            // disparity-chunk tiles: 0 automatic, 1 never, 2/4/8 always
    int census_mode;           // region-of-interest census variant (census.cu)
    int strip_rows;            // rows of the shared-memory strip (pts_side * ndy, rounded up to 4)
    int stats_accumulate;      // 1: the aggregation adds the call's counters to the stats record
    const ctm_frame *gather_src;  // mapped calls: device copy of the caller's frame table (host
                                  // image pointers the device reads); the census then reads the
                                  // staging images of `frames`, filled by the gather.  Else null
    int inject_expiry;         // fault injection for tests: the CTA of the fused persistent matcher
                               // that takes queue position 0 withholds that block's first strip
                               // copy, so its bounded wait expires
};

__host__ __device__ inline int ceil_div_nn(int a, int b) { return (a + b - 1) / b; }

// Work class of a searchable block with `work` = usable points x candidates of
// one pass: 0 for the largest possible block, one class per half octave below.
__device__ __forceinline__ int queue_class(int work)
{
    if (work < 2) return kQueueClasses - 1;
    const int l = 31 - __clz(work);                   // floor(log2(work))
    const int s = 2 * l + ((work >> (l - 1)) & 1);    // + 1 from 1.5 * 2^l on
    constexpr int kTop = 2 * 16;                      // s of kMaxPts * kMaxCand = 2^16
    return min(max(kTop - s, 0), kQueueClasses - 1);
}

// Start of each class's positions in the work-ordered queue
// (start[kQueueClasses] = queue length), from the counters of the call.
__device__ __forceinline__ void queue_starts(const Counts *c, int *start)
{
    int n[kQueueClasses];
#pragma unroll
    for (int i = 0; i < kQueueClasses; ++i) n[i] = c->n_class[i];
    int acc = 0;
#pragma unroll
    for (int i = 0; i < kQueueClasses; ++i) {
        start[i] = acc;
        acc += n[i];
    }
    start[kQueueClasses] = acc;
}

// The work-ordered queue is written (by the sampling kernel) and read (by the
// fused persistent matcher) only when the call plans at most kMaxRounds blocks per
// SM: only then can the whole queue fit in the matcher's first wave, and larger
// calls skip its atomics.
__device__ __forceinline__ bool work_queue_on(const MatchArgs &a, int n_blocks)
{
    return a.ws.queue_w != nullptr && a.sm_count > 0 && n_blocks <= kMaxRounds * a.sm_count;
}

// Block at position p of the work-ordered queue (0 <= p < start[kQueueClasses]).
__device__ __forceinline__ int queue_w_at(const MatchArgs &a, const int *start, int p)
{
    int c = 0;
    while (c < kQueueClasses - 1 && p >= start[c + 1]) ++c;
    return a.ws.queue_w[(long long)c * a.caps.max_blocks + (p - start[c])];
}

// Block at position p of the first queue (n_big blocks from the front).
__device__ __forceinline__ int queue_at(const MatchArgs &a, int n_big, int p)
{
    return p < n_big ? a.ws.queue[p] : a.ws.queue[a.caps.max_blocks - 1 - (p - n_big)];
}

// Sampled coordinate j of n on [b0, b1): the centre of the j-th of n equal cells
// (Sec. 4.3.4's regular point grid).
__device__ __forceinline__ int point_coord(int b0, int b1, int n, int j)
{
    return b0 + ((2 * j + 1) * (b1 - b0)) / (2 * n);
}

// Rectangle of block `slot` (row-major in a g x g grid) of a planned box, on its
// matching grid, and its point counts per side.
struct BlockRect {
    int bx0, by0, bx1, by1, nx, ny;
};

__device__ __forceinline__ BlockRect block_rect(const BoxPlan &P, int slot, int pts_side)
{
    BlockRect r;
    const int ga = slot % P.g, gb = slot / P.g;
    const int bw = P.sx1 - P.sx0, bh = P.sy1 - P.sy0;
    r.bx0 = P.sx0 + (ga * bw) / P.g;
    r.bx1 = P.sx0 + ((ga + 1) * bw) / P.g;
    r.by0 = P.sy0 + (gb * bh) / P.g;
    r.by1 = P.sy0 + ((gb + 1) * bh) / P.g;
    r.nx = min(r.bx1 - r.bx0, pts_side);
    r.ny = min(r.by1 - r.by0, pts_side);
    return r;
}

// Census launches (census.cu)
constexpr int kCensusTilePx = 32;   // pixels per bitmap bit (a census tile: 8 lanes x 4 pixels)
// Grid columns a census tile x0 .. x0 + 31 reads: [x0 - L, x0 + R).  The fixed
// windows (5x5, 7x7, 9x7; census_roi4_kernel) load twelve pixels x - 4 .. x + 7
// per lane of four pixels; the other windows (census_roi_kernel) load 21 words
// of four pixels from x0 - 8.  Rows: the window's rows around the tile's row.
__host__ __device__ inline bool census_fixed_window(int win_w, int win_h)
{
    return (win_w == 9 && win_h == 7) || (win_w == 7 && win_h == 7) || (win_w == 5 && win_h == 5);
}
__host__ __device__ inline int census_reach_left(int win_w, int win_h) { return census_fixed_window(win_w, win_h) ? 4 : 8; }
__host__ __device__ inline int census_reach_right(int win_w, int win_h) { return census_fixed_window(win_w, win_h) ? 36 : 76; }

// Mapped calls (gather.cu): after the sampling kernel has marked the census
// tiles, copy from the caller's host images into the staging images the source
// bytes those tiles' census reads (64-byte segments of each source row).
cudaError_t launch_gather(const MatchArgs &a, int sm_count, cudaStream_t s);
constexpr int kGatherSegBytes = 64;
cudaError_t launch_census_single(const uint8_t *img, int W, int H, int pitch, int k, int win_w,
                                 int win_h, int sentinel, uint64_t *out, long long out_pitch,
                                 cudaStream_t s);
// Region-of-interest census over the marked tiles, `ctas_per_sm` resident CTAs
// per SM (census_roi_ctas_per_sm; the first call queries the occupancy, so make
// it before any stream capture).
int census_roi_ctas_per_sm(int win_w, int win_h, int mode);
cudaError_t launch_census_roi(const MatchArgs &a, int sm_count, cudaStream_t s);
size_t census_smem_bytes(int win_h);

// Planning (plan.cu)
cudaError_t launch_stage_frame(const MatchArgs &a, ctm_frame f, int n_boxes, cudaStream_t s);
cudaError_t launch_plan(const MatchArgs &a, cudaStream_t s);
cudaError_t launch_aggregate(const MatchArgs &a, cudaStream_t s);
cudaError_t launch_sample(const MatchArgs &a, cudaStream_t s);

// Matching (match.cu)
// threads per matching CTA: 128 or 256
size_t match_smem_bytes(const MatchArgs &a);
cudaError_t match_configure(const MatchArgs &a, int threads, int *ctas_per_sm);
// Like match_configure, but only ever raises the kernel's shared-memory limit.
cudaError_t match_configure_raise(const MatchArgs &a, int threads, int *ctas_per_sm);
cudaError_t launch_match_persistent(const MatchArgs &a, int threads, int grid, cudaStream_t s);
cudaError_t launch_match_box(const MatchArgs &a, int threads, int box, cudaStream_t s);

// Two-pass pipelined matcher (match_pipe.cu): forward kernel then backward
// kernel over the same queue, `grid` persistent CTAs each.
size_t match_pipe_smem_bytes(const MatchArgs &a);
cudaError_t match_pipe_configure(const MatchArgs &a, int threads, int *ctas_per_sm);
cudaError_t launch_match_pipe(const MatchArgs &a, int threads, int grid, cudaStream_t s);

// Probes (probe.cu)
cudaError_t run_int_probe(int kind, int iters, double *ops_per_clk_per_sm);
cudaError_t run_wait_probe(int *expired, float *waited_ms);

// Tensor-map box widths of the strip loads: 32, 64, ..., 256 codes (a box row is at
// most 256 elements).  A strip chunk stored SWa codes wide loads by tile::gather4
// with the narrowest box that holds it, its rows then kBox apart in shared memory
// (a multiple of 32 codes, so every four-row group starts 128-byte aligned).
constexpr int kBoxClasses = 8;
constexpr int kMaxMapFrames = 256;  // contexts with more frame slots use 1-D copies only
__host__ __device__ inline int box_width(int SWa) { return (SWa + 31) & ~31; }

// Build the census planes' tensor maps of a workspace (api.cu): host-encoded and
// copied to ws.tmaps; false if the driver's encoder is unavailable.
bool encode_plane_maps(const Workspace &ws, const Caps &caps, int close_factor, CUtensorMap *dev_maps);

// Parameter checks of ctm_create (limits in include/ctm.h and the matcher's
// strip budget) and the default strip width for a disparity range (api.cu).
bool params_valid(const ctm_params &p);
int default_strip_cols(int nd_max);

// ctm_match_batch with an optional gather (gather_src_dev: a device copy of a
// frame table holding each frame's host images, read by the gather of
// ctm_match_batch_mapped into the images of frames_dev; a frame with height 0
// there is not gathered).  Used by the serving loop.
int match_batch_dev(ctm_ctx *ctx, const ctm_frame *frames_dev, const ctm_frame *gather_src_dev,
                    const int32_t *counts_dev, const ctm_box *boxes_dev, float *disp_dev, float *depth_dev,
                    uint8_t *flags_dev, const ctm_debug *dbg, int use_graph, ctm_stream stream);

// Device address of the error flag of a context's last finished call
// (ctm_stats.error), for callers that read it back on their own stream.
const int32_t *context_error_flag(const ctm_ctx *ctx);

// Device allocation used for every workspace, staging buffer and arena of the
// library: cudaMalloc, unless ctm_inject_alloc_failures armed a failure, which
// this allocation then consumes (returning cudaErrorMemoryAllocation, as
// cudaMalloc does when the device is out of memory).
cudaError_t dev_alloc(void **ptr, size_t bytes);

// Bytes of device workspace a context holds (its one allocation at creation).
size_t context_device_bytes(const ctm_ctx *ctx);

}  // namespace ctm
