// plan.cu -- device-side planning of Algorithm 2's per-box steps.
//
// plan_kernel (several CTAs per frame, each a slice of the frame's boxes,
// a warp per box): clip each box to its frame, classify it FAR
// or CLOSE by its larger side against tau_s (Sec. 4.3.4), map it to its matching
// grid (full resolution for FAR, the decimated grid for CLOSE), count its
// blocks, and select its occluders -- overlapping boxes of the same frame with a
// larger bottom y (Sec. 4.3.5), nearest (largest bottom y) first, at most
// max_occluders.  Boxes that are empty after clipping get their outputs here.
// Each slice's blocks get a contiguous range of the flat (box, slot) block list.
//
// sample_kernel (one warp per block): the block's point grid and its usable
// points; blocks with fewer than min_pts usable points are finished here, the
// others go to the work queue (large work first) and mark the census tiles
// their search can read.  All counts come from device memory so a captured
// graph replays with new inputs.
#include <math.h>

#include <algorithm>

#include "aggregate.cuh"
#include "ctm_internal.cuh"

namespace ctm {
namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int4 clip_box(const ctm_box &b, int W, int H)
{
    int4 r;
    r.x = b.x0 < 0 ? 0 : b.x0;
    r.y = b.y0 < 0 ? 0 : b.y0;
    r.z = b.x1 > W ? W : b.x1;
    r.w = b.y1 > H ? H : b.y1;
    if (r.z <= r.x || r.w <= r.y) r = make_int4(0, 0, 0, 0);
    return r;
}

// Priority rule of Sec. 4.3.5: an occluder is frontal if its clipped box
// centre lies in the centred crop [W (1 - c) / 2, W (1 + c) / 2) x [H (1 - c) / 2,
// H (1 + c) / 2), compared on doubled coordinates in fp32.
__device__ __forceinline__ bool frontal(int4 q, int W, int H, float c)
{
    if (!(c > 0.0f)) return false;
    const float sx = (float)(q.x + q.z), sy = (float)(q.y + q.w);
    const float om = __fsub_rn(1.0f, c), op = __fadd_rn(1.0f, c);
    return sx >= __fmul_rn((float)W, om) && sx < __fmul_rn((float)W, op) && sy >= __fmul_rn((float)H, om) &&
           sy < __fmul_rn((float)H, op);
}

__device__ __forceinline__ bool overlaps(int4 a, int4 b)
{
    const int ix0 = max(a.x, b.x), ix1 = min(a.z, b.z);
    const int iy0 = max(a.y, b.y), iy1 = min(a.w, b.w);
    return ix1 > ix0 && iy1 > iy0;
}

__global__ void stage_frame_kernel(ctm_frame *frames, int *counts_in, ctm_frame f, int n_boxes)
{
    frames[0] = f;
    counts_in[0] = 1;
    counts_in[1] = n_boxes;
}

constexpr int kStageBoxes = 1024;  // boxes of one frame staged in shared memory
constexpr int kKeyCache = 8;       // occluder keys per lane held in registers

// S CTAs per frame, each a slice of the frame's boxes: clip, classify,
// map to the matching grid and select the occluders of every box of the slice
// (the frame's clipped boxes are staged in shared memory for the pairwise
// test), then the slice's block counts are scanned and one atomic reserves the
// slice's range of the flat block list.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(MatchArgs a, int S)
{
    __shared__ int4 sbox[kStageBoxes];
    __shared__ int warp_tot[kPlanThreads / 32];
    __shared__ int s_run, s_base;
    const int f = blockIdx.x / S, slice = blockIdx.x % S;
    const int nf = clampi(a.counts_in[0], 0, a.caps.max_frames);
    const int nb_total = clampi(a.counts_in[1], 0, a.caps.max_boxes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) {
        a.ws.counts->n_frames = nf;
        a.ws.counts->n_boxes = nb_total;
        a.ws.counts->error = 0;  // the previous call's flag stays until here (see aggregate_kernel)
    }
    if (f >= nf) return;
    const ctm_frame fr = a.frames[f];
    const bool bad_frame = fr.width < 1 || fr.height < 1 || fr.width > a.caps.max_width ||
                           fr.height > a.caps.max_height || fr.pitch < fr.width ||
                           fr.left == nullptr || fr.right == nullptr;
    if (slice == 0 && tid < 4) {  // census plane descriptors of this frame: L1, R1, Lk, Rk
        PlaneDesc d;
        const int q = tid;
        d.img = (q & 1) ? fr.right : fr.left;
        d.W = fr.width;
        d.pitch = fr.pitch;
        d.k = q < 2 ? 1 : a.p.close_factor;
        d.Ws = ceil_div_nn(fr.width, d.k);
        d.Hs = ceil_div_nn(fr.height, d.k);
        uint64_t *cb = a.ws.census + (long long)f * a.ws.frame_stride;
        d.out = q < 2 ? cb + q * a.ws.plane1_elems : cb + 2 * a.ws.plane1_elems + (q - 2) * a.ws.planek_elems;
        d.opitch = (int)(q < 2 ? a.ws.pitch1 : a.ws.pitchk);
        d.vec_load = (d.k == 1 || d.k == 2) && (fr.pitch % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(d.img) & 7u) == 0);
        d.pad = 0;
        a.ws.planes[f * 4 + q] = d;
    }
    const int begin = clampi(fr.box_begin, 0, nb_total);
    const int end = clampi(fr.box_begin + fr.box_count, begin, nb_total);
    const int nloc = end - begin;
    const bool staged = nloc <= kStageBoxes;
    if (staged)
        for (int t = tid; t < nloc; t += blockDim.x) sbox[t] = clip_box(a.boxes[begin + t], fr.width, fr.height);
    __syncthreads();
    const ctm_params &p = a.p;
    const int K = p.max_occluders < kMaxOcc ? p.max_occluders : kMaxOcc;
    // this CTA's slice of the frame's boxes
    const int per = (nloc + S - 1) / S;
    const int sb = begin + min(slice * per, nloc), se = begin + min((slice + 1) * per, nloc);

    // a warp per box
    for (int i = sb + warp; i < se; i += kPlanThreads / 32) {
        const int4 r = staged ? sbox[i - begin] : clip_box(a.boxes[i], fr.width, fr.height);
        const int w = r.z - r.x, h = r.w - r.y;
        const int side = w > h ? w : h;
        const int far = side < p.far_side_px ? 1 : 0;
        const int k = far ? 1 : p.close_factor;
        BoxPlan P;
        P.cx0 = r.x; P.cy0 = r.y; P.cx1 = r.z; P.cy1 = r.w;
        // decimated pixel x belongs to the box iff its source pixel k x does
        P.sx0 = ceil_div_nn(r.x, k); P.sx1 = ceil_div_nn(r.z, k);
        P.sy0 = ceil_div_nn(r.y, k); P.sy1 = ceil_div_nn(r.w, k);
        P.frame = f;
        P.far = far;
        P.k = k;
        P.g = far ? 1 : p.grid_g;
        P.dmin = far ? p.far_dmin : p.close_dmin;
        P.dmax = far ? p.far_dmax : p.close_dmax;
        P.Ws = ceil_div_nn(fr.width, k);
        P.Hs = ceil_div_nn(fr.height, k);
        P.fb = __fmul_rn(fr.f_px, fr.baseline_m);
        const bool empty = bad_frame || w <= 0 || h <= 0 || P.sx1 <= P.sx0 || P.sy1 <= P.sy0;
        P.nblk = empty ? 0 : P.g * P.g;

        // occluders: overlap with positive area and strictly larger bottom y; keep
        // K of them: frontal ones first (frontal_crop > 0), then by largest bottom
        // y, ties to the lower index.  Key (frontal, bottom y, -index) is unique
        // per box, so round t takes the largest key below round t-1's: each lane
        // scans its share of the frame's boxes.
        // key of box j as an occluder of box i (0: it is not one)
        auto occ_key = [&](int j) -> unsigned long long {
            if (j >= end || j == i) return 0ull;
            const int4 q = staged ? sbox[j - begin] : clip_box(a.boxes[j], fr.width, fr.height);
            if (!(q.w > r.w) || !overlaps(r, q)) return 0ull;
            const unsigned front = frontal(q, fr.width, fr.height, p.frontal_crop) ? 0x80000000u : 0u;
            return ((unsigned long long)(front | (unsigned)q.w) << 32) | (unsigned)(0x7fffffff - (j - begin));
        };
        int nocc = 0;
        if (!empty && K > 0) {
            // frames of up to 32 * kKeyCache boxes keep every lane's keys in registers,
            // so a round is a register scan and two warp reductions
            const bool cached = nloc <= 32 * kKeyCache;
            unsigned long long kc[kKeyCache];
#pragma unroll
            for (int u = 0; u < kKeyCache; ++u) kc[u] = cached ? occ_key(begin + lane + 32 * u) : 0ull;
            unsigned long long prev = ~0ull;
            for (; nocc < K; ++nocc) {
                unsigned long long best = 0ull;
                if (cached) {
#pragma unroll
                    for (int u = 0; u < kKeyCache; ++u)
                        if (kc[u] < prev && kc[u] > best) best = kc[u];
                } else {
                    for (int j = begin + lane; j < end; j += 32) {
                        const unsigned long long key = occ_key(j);
                        if (key < prev && key > best) best = key;
                    }
                }
                // warp maximum of the 64-bit keys (two 32-bit reductions)
                const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(best >> 32));
                const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(best >> 32) == hi ? (unsigned)best : 0u);
                best = ((unsigned long long)hi << 32) | lo;
                if (best == 0ull) break;
                prev = best;
                if (lane == 0) {
                    const int j = begin + (0x7fffffff - (int)lo);
                    a.ws.occ[(long long)i * kMaxOcc + nocc] =
                        staged ? sbox[j - begin] : clip_box(a.boxes[j], fr.width, fr.height);
                }
            }
        }
        P.nocc = nocc;
        if (lane == 0) {
            a.ws.plans[i] = P;
            a.ws.nblk[i] = P.nblk;
            if (P.nblk == 0) {
                a.disp[i] = __int_as_float(0x7fc00000);
                a.depth[i] = __int_as_float(0x7fc00000);
                a.flags[i] = (uint8_t)((far ? CTM_BOX_FAR : 0) | CTM_BOX_EMPTY);
            }
        }
    }
    __syncthreads();

    // frame-local exclusive scan of the block counts, one reservation per frame
    if (tid == 0) s_run = 0;
    __syncthreads();
    for (int c0 = sb; c0 < se; c0 += blockDim.x) {
        const int i = c0 + tid;
        const int v = i < se ? a.ws.nblk[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        int wpre = 0, tot = 0;
        for (int wi = 0; wi < kPlanThreads / 32; ++wi) {
            if (wi < warp) wpre += warp_tot[wi];
            tot += warp_tot[wi];
        }
        if (i < se) a.ws.blk_base[i] = s_run + wpre + x - v;  // slice-local for now
        __syncthreads();
        if (tid == 0) s_run += tot;
        __syncthreads();
    }
    if (tid == 0) s_base = atomicAdd(&a.ws.counts->n_blocks, s_run);
    __syncthreads();
    const int base = s_base;
    // a warp per box writes the box's entries of the flat block list
    for (int i = sb + warp; i < se; i += kPlanThreads / 32) {
        const int bb = base + a.ws.blk_base[i];
        const int v = a.ws.nblk[i];
        __syncwarp();
        if (lane == 0) a.ws.blk_base[i] = bb;
        for (int s2 = lane; s2 < v; s2 += 32) a.ws.blocks[bb + s2] = make_int2(i, s2);
    }
}

// Mark, for one block, the census row tiles its two passes can read: the left
// plane at the sampled rows (plus the vertical spread of the backward pass) over
// [X_0 - (dmax - dmin), X_last + (dmax - dmin)], which holds the points and every
// backward strip; the right plane at rows Y_m + dy over [X_0 - dmax, X_last - dmin],
// which holds every forward strip and the backward queries.
__device__ __forceinline__ void mark_range(const MatchArgs &a, int f, int q, int y, int c0, int c1,
                                           int Ws, int Hs)
{
    if (y < 0 || y >= Hs) return;
    c0 = max(c0, 0);
    c1 = min(c1, Ws - 1);
    if (c1 < c0) return;
    const int t0 = c0 / kCensusTilePx, t1 = c1 / kCensusTilePx;
    uint32_t *row = a.ws.bitmap + (long long)f * a.ws.bm_frame_words + a.ws.bm_plane_off[q] +
                    (long long)y * a.ws.bm_row_words[q];
    for (int wi = t0 >> 5; wi <= (t1 >> 5); ++wi) {
        const int lo = max(t0 - wi * 32, 0), hi = min(t1 - wi * 32, 31);
        const uint32_t upto = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
        atomicOr(row + wi, upto & ~((1u << lo) - 1u));
    }
}

__global__ void __launch_bounds__(256) sample_kernel(MatchArgs a)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * 8 + warp;
    if (b >= a.ws.counts->n_blocks) return;
    const int2 bs = a.ws.blocks[b];
    const int box = bs.x, slot = bs.y;
    const BoxPlan P = a.ws.plans[box];
    const BlockRect r = block_rect(P, slot, a.p.pts_side);
    const int nx = r.nx, ny = r.ny;
    const int Xl = lane < nx ? point_coord(r.bx0, r.bx1, nx, lane) : 0;
    const int Yl = lane < ny ? point_coord(r.by0, r.by1, ny, lane) : 0;
    int4 occ = make_int4(0, 0, 0, 0);
    if (lane < P.nocc) occ = a.ws.occ[(long long)box * kMaxOcc + lane];
    // usable: left census defined (window inside the grid) and full-res position
    // k (x, y) in no kept occluder
    const int sxw = a.p.win_w >> 1, syw = a.p.win_h >> 1;
    const bool col_ok = lane < nx && Xl - sxw >= 0 && Xl + sxw < P.Ws;
    // Each occluder covers a column range x a row range of the point grid: lane q
    // forms the row mask of occluder q, then every column lane removes the rows
    // of the occluders whose x range holds it.
    const unsigned rowok = __ballot_sync(full, lane < ny && Yl - syw >= 0 && Yl + syw < P.Hs);
    unsigned occrows = 0u;
    if (P.nocc > 0) {
        for (int m = 0; m < ny; ++m) {
            const int fy = P.k * __shfl_sync(full, Yl, m);
            if (lane < P.nocc && fy >= occ.y && fy < occ.w) occrows |= 1u << m;
        }
    }
    unsigned colmask = col_ok ? rowok : 0u;
    const int fx = P.k * Xl;
    for (int q = 0; q < P.nocc; ++q) {
        const int ox0 = __shfl_sync(full, occ.x, q), ox1 = __shfl_sync(full, occ.z, q);
        const unsigned rows = __shfl_sync(full, occrows, q);
        if (fx >= ox0 && fx < ox1) colmask &= ~rows;
    }
    const int cnt = __popc(colmask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    const int n_valid = __shfl_sync(full, incl, 31);
    // column chunks whose strip (plus alignment) fits the shared-memory strip
    const int nd = P.dmax - P.dmin + 1;
    unsigned cstart = 1u;
    {
        int x0 = __shfl_sync(full, Xl, 0);
        for (int j = 1; j < nx; ++j) {
            const int xj = __shfl_sync(full, Xl, j);
            if (xj - x0 + nd + 2 > a.strip_cols) {
                cstart |= 1u << j;
                x0 = xj;
            }
        }
    }
    BlockGeom *g = a.ws.geom + b;
    if (lane < kMaxPtsSide) {
        g->X[lane] = (int16_t)Xl;
        g->Y[lane] = (int16_t)Yl;
        g->colmask[lane] = (uint16_t)colmask;
        g->colprefix[lane] = (uint16_t)(incl - cnt);
    }
    if (lane == 0) {
        g->n_valid = n_valid;
        g->nx = nx;
        g->ny = ny;
        g->cstart = cstart;
        g->box = box;
        g->slot = slot;
        g->frame = P.frame;
        g->k = P.k;
        g->far = P.far;
        g->dmin = P.dmin;
        g->dmax = P.dmax;
        g->Ws = P.Ws;
        g->Hs = P.Hs;
    }
    const int ndy = a.p.dy_max - a.p.dy_min + 1;
    if (n_valid < a.p.min_pts) {
        if (lane == 0) {
            ctm_block rec;
            rec.n_pts = nx * ny;
            rec.n_valid = n_valid;
            rec.d_f = rec.dy_f = rec.d_b = rec.dy_b = 0;
            rec.s_m = rec.s_0 = rec.s_p = 0;
            rec.d_sub = 0.0f;
            rec.d_full = 0.0f;
            rec.flags = CTM_BLK_PRESENT | CTM_BLK_FEW_POINTS;
            write_block(a, box, slot, rec);
        }
    } else {
        if (lane == 0) {
            if (a.ws.chunk) {  // state for disparity-chunk tiles (used only when the queue is short)
                ChunkState cs{};
                cs.fkey = cs.bkey = 0xffffffffu;
                a.ws.chunk[b] = cs;
            }
            const int work = n_valid * nd * ndy;
            if (work >= kBigWork) {
                const int q = atomicAdd(&a.ws.counts->n_big, 1);
                a.ws.queue[q] = b;
            } else {
                const int q = atomicAdd(&a.ws.counts->n_small, 1);
                a.ws.queue[a.caps.max_blocks - 1 - q] = b;
            }
            if (work_queue_on(a, a.ws.counts->n_blocks)) {
                const int c = queue_class(work);
                const int q = atomicAdd(&a.ws.counts->n_class[c], 1);
                a.ws.queue_w[(long long)c * a.caps.max_blocks + q] = b;
            }
        }
        // census demand of the searchable block (see mark_range)
        const int x_first = __shfl_sync(full, Xl, 0), x_last = __shfl_sync(full, Xl, nx - 1);
        const int qL = (P.far || a.p.close_factor == 1) ? 0 : 2;
        const int span = P.dmax - P.dmin;
        const int dyr = a.p.dy_max - a.p.dy_min;
        const int nl = 2 * dyr + 1, nr = dyr + 1;
        const int items = ny * (nl + nr);
        for (int it0 = 0; it0 < items; it0 += 32) {  // uniform trip count: the shuffle needs every lane
            const int it = it0 + lane;
            const int m = (it < items ? it : 0) / (nl + nr);
            const int e = it - m * (nl + nr);
            const int y = __shfl_sync(full, Yl, m);
            if (it >= items) continue;
            if (e < nl)
                mark_range(a, P.frame, qL, y + e - dyr, x_first - span, x_last + span, P.Ws, P.Hs);
            else
                mark_range(a, P.frame, qL + 1, y + a.p.dy_min + (e - nl), x_first - P.dmax, x_last - P.dmin,
                           P.Ws, P.Hs);
        }
    }
}

}  // namespace

cudaError_t launch_sample(const MatchArgs &a, cudaStream_t s)
{
    const int grid = ceil_div_nn(a.caps.max_blocks, 8);
    sample_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}


// One warp per planned box with blocks: Sec. 4.3.4 over its block records and
// Eq. 1 (boxes without blocks got their outputs from the planner).
//
// When a bounded wait of the matching kernel expired (counts->error), some
// blocks were never searched and their records are stale, so no box with
// blocks is aggregated: each gets NaN disparity and depth and flags 0 (neither
// VALID nor any reason bit), and the call's status says why.
//
// It is the last kernel of a call, so it also leaves the workspace ready for
// the next one: block 0 moves the counters to the stats record and zeroes
// them -- all but the error flag, which every CTA reads here and the next
// call's plan_kernel clears -- and the matcher's round counters, and every
// box's block count goes back to zero (no memset nodes at the start of a call).
__global__ void __launch_bounds__(256) aggregate_kernel(MatchArgs a)
{
    __shared__ float scratch[8][2 * kMaxSlots];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int failed = *reinterpret_cast<volatile int *>(&a.ws.counts->error);
    if (blockIdx.x == 0 && a.ws.sched)
        for (int i = threadIdx.x; i < kSchedInts; i += blockDim.x) a.ws.sched[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const Counts c = *a.ws.counts;
        if (a.stats_accumulate) {  // a later sub-batch of one call
            Counts t = *a.ws.stats;
            t.n_frames += c.n_frames;
            t.n_boxes += c.n_boxes;
            t.n_blocks += c.n_blocks;
            t.queue_head += c.queue_head;
            t.error |= c.error;
            t.evals += c.evals;
            t.n_big += c.n_big;
            t.n_small += c.n_small;
            t.n_tiles += c.n_tiles;
            t.host_bytes += c.host_bytes;
            for (int i = 0; i < kQueueClasses; ++i) t.n_class[i] += c.n_class[i];
            *a.ws.stats = t;
        } else {
            *a.ws.stats = c;
        }
        Counts z{};
        z.error = c.error;  // unchanged: other CTAs read it
        *a.ws.counts = z;
    }
    const int box = blockIdx.x * 8 + warp;
    if (box >= clampi(a.counts_in[1], 0, a.caps.max_boxes)) return;
    if (a.ws.nblk[box] == 0) return;
    if (failed) {
        if (lane == 0) {
            a.disp[box] = __int_as_float(0x7fc00000);
            a.depth[box] = __int_as_float(0x7fc00000);
            a.flags[box] = 0;
        }
    } else {
        aggregate_box(a, box, scratch[warp], lane);
    }
    __syncwarp();
    if (lane == 0) a.ws.nblk[box] = 0;
}

cudaError_t launch_aggregate(const MatchArgs &a, cudaStream_t s)
{
    aggregate_kernel<<<ceil_div_nn(a.caps.max_boxes, 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stage_frame(const MatchArgs &a, ctm_frame f, int n_boxes, cudaStream_t s)
{
    stage_frame_kernel<<<1, 1, 0, s>>>(a.ws.frames, a.ws.counts_in, f, n_boxes);
    return cudaGetLastError();
}

// The counters and block counts start at zero: the workspace is created zeroed
// and every call's aggregate_kernel zeroes them again.  A frame's boxes are
// planned a warp per box, so a frame with many boxes gets more CTAs when the
// call has few frames: about two CTAs per SM over the call's frame capacity,
// at least 4 and at most 32 per frame.
cudaError_t launch_plan(const MatchArgs &a, cudaStream_t s)
{
    const int nf = a.caps.max_frames > 0 ? a.caps.max_frames : 1;
    const int slices = std::min(std::max(ceil_div_nn(2 * a.sm_count, nf), 4), 32);
    plan_kernel<<<a.caps.max_frames * slices, kPlanThreads, 0, s>>>(a, slices);
    return cudaGetLastError();
}

}  // namespace ctm
