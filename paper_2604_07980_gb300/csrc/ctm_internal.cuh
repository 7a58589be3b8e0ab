// ctm_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctm.h"

namespace ctm {

constexpr int kMatchThreads = 256;               // one CTA matches one block
constexpr int kMatchWarps = kMatchThreads / 32;
constexpr int kMaxPtsSide = 16;
constexpr int kMaxPts = kMaxPtsSide * kMaxPtsSide;
constexpr int kMaxCand = 256;                    // candidates per pass (8 slices of 32)
constexpr int kMaxGrid = 8;
constexpr int kMaxSlots = kMaxGrid * kMaxGrid;
constexpr int kMaxOcc = 32;
constexpr int kMaxWin = 15;
constexpr int kCensusTileW = 32;
constexpr int kCensusTileH = 16;
constexpr int kPlanThreads = 128;
constexpr int kScanThreads = 1024;

// Device-side counters of one call.
struct Counts {
    int n_frames;    // clamped to capacity
    int n_boxes;     // clamped to capacity
    int n_blocks;    // total planned blocks
    int queue_head;  // next block index of the persistent queue
    unsigned long long evals;
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

// Result of one block kept for the aggregation (device).
struct BlockResult {
    float d_full;
    int flags;
};

// Device workspace of a context.
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
    int2 *blocks;              // [max_blocks] (box, slot)
    BlockResult *blkres;       // [max_blocks]
    int *box_done;             // [max_boxes]
    Counts *counts;
    ctm_frame *frames;         // staging for single-frame calls [max_frames]
    int *counts_in;            // staging {n_frames, n_boxes}
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
    int strip_rows;            // rows of the shared-memory strip (pts_side * ndy)
};

__host__ __device__ inline int ceil_div_nn(int a, int b) { return (a + b - 1) / b; }

// Census launches (census.cu)
cudaError_t launch_census_single(const uint8_t *img, int W, int H, int pitch, int k, int win_w,
                                 int win_h, int sentinel, uint64_t *out, long long out_pitch,
                                 cudaStream_t s);
cudaError_t launch_census_batch(const MatchArgs &a, cudaStream_t s);

// Planning (plan.cu)
cudaError_t launch_stage_frame(const MatchArgs &a, ctm_frame f, int n_boxes, cudaStream_t s);
cudaError_t launch_plan(const MatchArgs &a, cudaStream_t s);

// Matching (match.cu)
size_t match_smem_bytes(const MatchArgs &a);
cudaError_t match_configure(const MatchArgs &a, int *ctas_per_sm);
cudaError_t launch_match_persistent(const MatchArgs &a, int grid, cudaStream_t s);
cudaError_t launch_match_box(const MatchArgs &a, int box, cudaStream_t s);

// Probe (probe.cu)
cudaError_t run_int_probe(int kind, int iters, double *ops_per_clk_per_sm);

}  // namespace ctm
