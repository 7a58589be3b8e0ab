// match.cu -- the Hamming-cost search of Algorithm 2, one CTA per block end to
// end (the fused kernel; match_pipe.cu has the two-pass pipelined variant):
//   1. the block's sampling record (point grid, usable-point masks from the
//      occlusion test of Sec. 4.3.5) is in shared memory; copy the left census
//      at every usable point (compacted column-major) and the first forward
//      strip chunk into shared memory with asynchronous copies issued together;
//   2. forward pass over the right-image strip the block can reach (sampled rows
//      x [x - dmax, x - dmin]): Eq. census_cost,
//      S(dy, d) = sum_p popc(C_L(p) ^ C_R(p.x - d, p.y + dy)), for every
//      candidate; lanes own consecutive candidates (conflict-free strip reads),
//      warps own point subsets, each thread keeps up to 8 candidate sums in
//      registers, and the warps' sums are combined in two shared rows by ordered
//      stores and adds (no atomics);
//   3. first argmin over (dy, d): after the last combining barrier every warp
//      reduces the rows to the minimum (cost << 16 | index) key itself, so the
//      result needs no broadcast; Eq. subpixel in fp32 with IEEE division;
//   4. backward pass (Sec. 4.3.3): the left strip [q.x + dmin, q.x + dmax] (bulk
//      copies, issued first) and the right codes at the matched positions (plain
//      loads) arrive in one round trip;
//   5. consistency |d_b - d_f| <= fb_tol and the block record; boxes are
//      aggregated afterwards (aggregate_kernel).
// Blocks wider than the strip are split into column chunks; chunk sums add up
// because Eq. census_cost is a sum over points.
#include <math.h>

#include "aggregate.cuh"
#include "ctm_internal.cuh"
#include "match_common.cuh"

namespace ctm {
namespace {

template <int NW>
struct Shared {
    BlockGeom geom[2];      // sampled grids: the current block's and the prefetched next one's
    uint64_t mbar;          // completion of the strip bulk copies
    uint64_t mbar_g;        // completion of the geometry prefetch
    int X[kMaxPtsSide];
    int Y[kMaxPtsSide];
    int colstart[kMaxPtsSide + 1];
    int next;               // queue position of the next block
    int next_b;             // its block
    int qstart[kQueueClasses + 1];  // position of each work class's first block (work-ordered queue)
    int gpend;              // a geometry copy is in flight on mbar_g
    int spend;              // a strip copy is in flight on mbar
    unsigned cstart;        // bit j set: a strip column chunk starts at point column j
    int nq;                 // rounds mode: queue length, -1 without a work-ordered queue
};

struct BlockCtx {
    int box, slot, b;
    int k, far;
    int dmin, dmax, nd, ndy, nc;
    int nx, ny, Ws, Hs;
    int tm_l, tm_r;           // tensor maps of the left and right planes (tile::gather4 loads)
    long long pitch;
    const uint64_t *CL;
    const uint64_t *CR;
};

// Geometry of a strip chunk whose columns start at colbase, SWc wide: rows load by
// tile::gather4 with the narrowest box that holds them when it fits the strip's
// shared-memory width, else by 1-D copies at the chunk's own width.
__device__ __forceinline__ ChunkGeom strip_geom(const MatchArgs &a, int colbase, int SWc)
{
    return chunk_geom(colbase, SWc, a.ws.tmaps != nullptr ? min(a.strip_cols, 32 * kBoxClasses) : 0);
}

// Row r = (m, e) of a strip chunk: the right plane at Y_m + dy_min + e (forward)
// or the left plane at Y_m + dy_f - (dy_min + e) (backward).
__device__ __forceinline__ int chunk_row_y(const MatchArgs &a, const BlockCtx &bc, const int *Y, bool fwd,
                                           int dy_f, int r)
{
    const int m = bc.ndy == 1 ? r : r / bc.ndy;
    const int e = r - m * bc.ndy;
    return fwd ? Y[m] + a.p.dy_min + e : Y[m] + dy_f - (a.p.dy_min + e);
}

// Warp 0: issue the bulk copies of one strip chunk (completion on sh.mbar).
// withhold (fault injection for tests only): announce bytes on the mbarrier but
// issue no copy, so the phase never completes and the bounded wait expires.
template <int NT>
__device__ __forceinline__ void issue_chunk(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                                            Shared<NT / 32> &sh, bool fwd, int dy_f, const ChunkGeom &g,
                                            bool withhold = false)
{
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid >= 32) return;
    const int rows = bc.ny * bc.ndy;
    if (g.box > 0) {
        // tile::gather4: four rows per copy, each the map's box of g.box codes from
        // colbase_a (columns outside the plane's allocation read as zero); rows outside
        // the grid are fetched as row 0 and zeroed by land_chunk, like the other columns
        // outside [0, Ws)
        const CUtensorMap *tm = a.ws.tmaps + (fwd ? bc.tm_r : bc.tm_l) * kBoxClasses + (g.box / 32 - 1);
        const int groups = (rows + 3) >> 2;
        const unsigned total = (unsigned)groups * 4u * (unsigned)g.box * 8u;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (lane == 0) {
            mbar_arrive_expect_tx(&sh.mbar, withhold ? total + 16u : total);
            sh.spend = 1;
        }
        __syncwarp();
        if (!withhold) {
            for (int q = lane; q < groups; q += 32) {
                int y[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = min(4 * q + i, rows - 1);
                    const int yy = chunk_row_y(a, bc, sh.Y, fwd, dy_f, r);
                    y[i] = (yy >= 0 && yy < bc.Hs) ? yy : 0;
                }
                gather4_g2s(sm.strip + 4 * q * g.stride, tm, g.colbase_a, y[0], y[1], y[2], y[3], &sh.mbar);
            }
        }
        return;
    }
    const uint64_t *plane = fwd ? bc.CR : bc.CL;
    const int Ws_even = (bc.Ws + 1) & ~1;   // the padding column after an odd width is readable
    const int x_lo = max(g.colbase_a, 0);
    const int x_hi = min(g.colbase_a + g.SWa, Ws_even);
    const unsigned row_bytes = x_hi > x_lo ? 8u * (unsigned)(x_hi - x_lo) : 0u;
    unsigned total = 0;
    for (int r = lane; r < rows; r += 32) {
        const int y = chunk_row_y(a, bc, sh.Y, fwd, dy_f, r);
        if (y >= 0 && y < bc.Hs) total += row_bytes;
    }
    total = __reduce_add_sync(0xffffffffu, total);
    // order earlier generic-proxy accesses of the strip before the bulk writes
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane == 0) {
        mbar_arrive_expect_tx(&sh.mbar, withhold ? total + 16u : total);
        sh.spend = 1;
    }
    __syncwarp();
    if (row_bytes > 0 && !withhold) {
        for (int r = lane; r < rows; r += 32) {
            const int y = chunk_row_y(a, bc, sh.Y, fwd, dy_f, r);
            if (y >= 0 && y < bc.Hs)
                bulk_g2s(sm.strip + r * g.stride + (x_lo - g.colbase_a), plane + (long long)y * bc.pitch + x_lo,
                         row_bytes, &sh.mbar);
        }
    }
}

// All threads: wait for the chunk issued last, then zero what lies outside the
// plane (rows outside it; columns < 0 or >= Ws), a warp per row (only edge
// chunks have any).  Returns false if the bounded wait expired.  The phase is
// only consumed when the wait succeeded, so a drain after a failure waits for
// the same copies.
template <int NT>
__device__ __forceinline__ bool land_chunk(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                                           Shared<NT / 32> &sh, unsigned &phase, bool fwd, int dy_f,
                                           const ChunkGeom &g)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const bool ok = mbar_wait_bounded(&sh.mbar, phase, &a.ws.counts->error);
    if (ok) phase ^= 1u;
    if (ok && tid == 0) sh.spend = 0;
    const int rows = bc.ny * bc.ndy;
    const bool edge = g.colbase_a < 0 || g.colbase_a + g.SWa > bc.Ws ||
                      sh.Y[0] + (fwd ? a.p.dy_min : dy_f - a.p.dy_max) < 0 ||
                      sh.Y[bc.ny - 1] + (fwd ? a.p.dy_max : dy_f - a.p.dy_min) >= bc.Hs;
    if (edge) {
        const int warp = tid >> 5;
        const int c_lo = min(max(-g.colbase_a, 0), g.SWa);             // [0, c_lo): x < 0
        const int c_hi = max(min(bc.Ws - g.colbase_a, g.SWa), c_lo);   // [c_hi, SWa): x >= Ws
        for (int r = warp; r < rows; r += NT / 32) {
            const int y = chunk_row_y(a, bc, sh.Y, fwd, dy_f, r);
            uint64_t *row = sm.strip + r * g.stride;
            if (y < 0 || y >= bc.Hs) {
                for (int c = lane; c < g.SWa; c += 32) row[c] = 0ull;
            } else {
                for (int c = lane; c < c_lo; c += 32) row[c] = 0ull;
                for (int c = c_hi + lane; c < g.SWa; c += 32) row[c] = 0ull;
            }
        }
    }
    return ok;
}

// Load one strip chunk: rows (m, e) of the right plane at Y_m + dy_min + e
// (forward) or of the left plane at Y_m + dy_f - (dy_min + e) (backward);
// issue, wait, zero-fill.
template <int NT>
__device__ __forceinline__ bool load_chunk(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                                           Shared<NT / 32> &sh, unsigned &phase, bool fwd, int dy_f,
                                           const ChunkGeom &g)
{
    issue_chunk<NT>(a, bc, sm, sh, fwd, dy_f, g);
    return land_chunk<NT>(a, bc, sm, sh, phase, fwd, dy_f, g);
}

// The scans of one search pass after its first strip chunk has landed and the
// point bases of the first chunk are set: every chunk (later ones loaded into
// the strip after the previous chunk's scan), sums kept in registers.  Returns
// false if a bounded wait expired.
template <int NT>
__device__ bool scan_chunks(const MatchArgs &a, const BlockCtx &bc, const Smem &sm, Shared<NT / 32> &sh,
                            unsigned &phase, bool fwd, ChunkGeom g, int (&acc)[8], int d_f, int dy_f)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int T = (bc.nc + 31) >> 5;
    const bool fast = bc.ndy == 1 && (bc.nd & 31) == 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0;
    const unsigned cs = sh.cstart;
    int j0 = 0;
    bool ok = true;
    while (j0 < bc.nx) {
        const unsigned later = cs & ~((2u << j0) - 1u);
        const int j1 = later ? __ffs(later) - 1 : bc.nx;
        const int xj0 = sh.X[j0];
        const int p0 = sh.colstart[j0], p1 = sh.colstart[j1];
        if (j0 > 0) {  // later chunks: load now (the first chunk was prefetched)
            const int SWc = sh.X[j1 - 1] - xj0 + bc.nd;
            g = strip_geom(a, fwd ? xj0 - bc.dmax : xj0 - d_f + bc.dmin, SWc);
            ok = load_chunk<NT>(a, bc, sm, sh, phase, fwd, dy_f, g) && ok;
            set_bases<NT>(sm, sh.X, p0, p1, bc.ndy, g.stride, xj0, g.delta);
            __syncthreads();
        }
        if (fast) {
            if (fwd)
                scan_dispatch_fast<NW, -1>(T, sm, p0, p1, bc.nd - 1 - lane, acc);
            else
                scan_dispatch_fast<NW, 1>(T, sm, p0, p1, lane, acc);
        } else {
            int coff[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int c = t * 32 + lane;
                int o = 0;
                if (c < bc.nc) {
                    int e = 0;
                    while (c >= bc.nd) { c -= bc.nd; ++e; }
                    o = e * g.stride + (fwd ? (bc.nd - 1 - c) : c);
                }
                coff[t] = o;
            }
            scan_dispatch<NW>(T, sm, p0, p1, coff, acc);
        }
        __syncthreads();
        j0 = j1;
    }
    return ok;
}

// The end of a pass: the warps' sums are combined in two rows, sm.cost and
// sm.cost_b, without atomics -- warps 0 and 1 store theirs, then each further pair
// of warps adds its sums to the rows in turn, a barrier between steps -- and
// every warp then reduces the whole row pair to the first argmin key
// (cost << 16 | c), so every thread holds it without a broadcast.  Warp 0 writes
// the debug costs.  The rows' previous readers (the other pass's argmin) are
// separated from the first store by a barrier of the caller.  False if a
// bounded wait expired anywhere.
template <int NT>
__device__ __forceinline__ bool combine_pass(const MatchArgs &a, const BlockCtx &bc, const Smem &sm, bool fwd,
                                             const int (&acc)[8], bool ok, unsigned &key, int coff = 0,
                                             int32_t *row_out = nullptr)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int T = (bc.nc + 31) >> 5;
    int *row = (warp & 1) ? sm.cost_b : sm.cost;
    if (warp < 2) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int c = t * 32 + lane;
            if (t < T && c < bc.nc) row[c] = acc[t];
        }
    }
    if (!__syncthreads_and(ok)) return false;
#pragma unroll
    for (int step = 1; step < NW / 2; ++step) {
        if ((warp >> 1) == step) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int c = t * 32 + lane;
                if (t < T && c < bc.nc) row[c] += acc[t];
            }
        }
        __syncthreads();
    }
    int32_t *dbgc = warp == 0 ? (fwd ? a.dbg.cost_f : a.dbg.cost_b) : nullptr;
    if (warp != 0) row_out = nullptr;
    const int slots = a.p.grid_g * a.p.grid_g;
    unsigned k = 0xffffffffu;
    for (int c = lane; c < bc.nc; c += 32) {
        const int s = sm.cost[c] + sm.cost_b[c];
        k = min(k, ((unsigned)s << 16) | (unsigned)c);
        if (dbgc) dbgc[((long long)bc.box * slots + bc.slot) * a.nc_stride + coff + c] = s;
        if (row_out) row_out[c] = s;
    }
    key = __reduce_min_sync(0xffffffffu, k);
    return true;
}

// Work distribution of the fused persistent kernel.  With more queued blocks
// than CTAs, every CTA takes blocks from the first queue (sampling order, for
// L2 locality) as it frees up, and the load evens out over the many blocks.
// When the whole queue goes out in the first wave (a single frame, a small
// batch), the dynamic queue alone lets one SM's CTAs take several of the
// largest blocks while another SM gets small ones, and the kernel lasts as long
// as the most loaded SM.  Then the blocks come from the work-ordered queue (the
// largest first) in rounds of sm_count positions: the r-th CTA to start on an
// SM takes a position of round r, so every SM gets one block of each round, of
// similar work.  A position of a round that no CTA of that rank took (an SM that
// ran fewer CTAs) is swept up by the next CTA that asks for work, so every
// position is taken exactly once whichever SMs the CTAs land on.
constexpr unsigned kRoundPauseNs = 1500;

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Thread 0, rounds mode (every position belongs to a round): a round position
// that no CTA of that rank took; nq when every position is taken.
__device__ __forceinline__ int sweep_rounds(int *sched, int nq, int R, int n_sm)
{
    for (int r = 0; r < R; ++r) {
        const int lim = min(n_sm, nq - r * n_sm);
        if (*reinterpret_cast<volatile int *>(sched + kSchedSMs + r) < lim) {
            const int k = atomicAdd(sched + kSchedSMs + r, 1);
            if (k < lim) return r * n_sm + k;
        }
    }
    return nq;
}

// Thread 0: first queue position of this CTA -- the round position of its rank
// on its SM (the order in which the SM's CTAs started), if any; CTAs without one pause briefly (bounded by the timer and an
// iteration cap) so that they do not sweep up positions before the CTAs of
// lower ranks that are still starting take them.
__device__ __forceinline__ int take_first_round(int *sched, int rank, int nq, int R, int n_sm)
{
    if (rank < R) {
        const int lim = min(n_sm, nq - rank * n_sm);
        const int k = atomicAdd(sched + kSchedSMs + rank, 1);
        if (k < lim) return rank * n_sm + k;
    }
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < 64 && global_ns() - t0 < kRoundPauseNs; ++it) __nanosleep(128);
    return sweep_rounds(sched, nq, R, n_sm);
}


// Block context from the block's sampling record (which carries its box plan).
__device__ __forceinline__ BlockCtx make_ctx(const MatchArgs &a, const BlockGeom &g, int b)
{
    BlockCtx bc;
    bc.box = g.box;
    bc.slot = g.slot;
    bc.b = b;
    bc.k = g.k;
    bc.far = g.far;
    bc.dmin = g.dmin;
    bc.dmax = g.dmax;
    bc.nd = g.dmax - g.dmin + 1;
    bc.ndy = a.p.dy_max - a.p.dy_min + 1;
    bc.nc = bc.nd * bc.ndy;
    bc.Ws = g.Ws;
    bc.Hs = g.Hs;
    bc.nx = g.nx;
    bc.ny = g.ny;
    const bool full = g.far || a.p.close_factor == 1;
    bc.tm_l = 4 * g.frame + (full ? 0 : 2);
    bc.tm_r = bc.tm_l + 1;
    const uint64_t *base = a.ws.census + (long long)g.frame * a.ws.frame_stride;
    bc.CL = full ? base : base + 2 * a.ws.plane1_elems;
    bc.CR = full ? base + a.ws.plane1_elems : base + 2 * a.ws.plane1_elems + a.ws.planek_elems;
    bc.pitch = full ? a.ws.pitch1 : a.ws.pitchk;
    return bc;
}

// Point layout of a block whose sampling record is in g: the column-major
// compaction of its usable points (sm.pmj), its sampled columns and rows, and,
// with left_codes, the left codes at its points (cp.async) and their strip bases
// in its first forward strip chunk g0.  Ends with a barrier.
template <int NT>
__device__ __forceinline__ void layout_block(const BlockCtx &bc, const BlockGeom &g, const Smem &sm,
                                             Shared<NT / 32> &sh, bool left_codes, int j1_first,
                                             const ChunkGeom &g0)
{
    const int tid = threadIdx.x;
    const int x0 = g.X[0];
    for (int t = tid; t < kMaxPts; t += NT) {
        const int j = t >> 4, m = t & 15;
        if (j < bc.nx && ((g.colmask[j] >> m) & 1u)) {
            const int idx = g.colprefix[j] + __popc(g.colmask[j] & ((1u << m) - 1u));
            const int x = g.X[j], y = g.Y[m];
            if (left_codes) {
                cp_async8(&sm.pcode[idx], bc.CL + (long long)y * bc.pitch + x);
                if (j < j1_first) sm.pbase[idx] = 8 * (m * bc.ndy * g0.stride + x - x0 + g0.delta);
            }
            sm.pmj[idx] = (m << 8) | j;
        }
    }
    if (tid < kMaxPtsSide) {
        sh.X[tid] = g.X[tid];
        sh.Y[tid] = g.Y[tid];
    }
    if (tid <= kMaxPtsSide) sh.colstart[tid] = tid < bc.nx ? g.colprefix[tid] : g.n_valid;
    if (tid == 0) sh.cstart = g.cstart;
    __syncthreads();  // sh.Y is read by the issuing warp
}

// First column chunk of a block: its end column and its forward strip geometry.
__device__ __forceinline__ int first_chunk_end(const BlockGeom &g, int nx)
{
    const unsigned later0 = g.cstart & ~1u;
    return later0 ? __ffs(later0) - 1 : nx;
}

// Start a block (or a disparity chunk of one: bc's candidate range) whose
// sampling record is in g: its point layout, the left codes at its points and
// its first forward strip chunk (bulk copies on sh.mbar).  Nothing is waited for
// here; the strip, the point arrays and sh.X / sh.Y must be free (the previous
// block's scans done).  withhold: see issue_chunk.
template <int NT>
__device__ void begin_block_ctx(const MatchArgs &a, const BlockCtx &bc, const BlockGeom &g, const Smem &sm,
                                Shared<NT / 32> &sh, bool withhold = false)
{
    const int j1_first = first_chunk_end(g, bc.nx);
    const int x0 = g.X[0];
    const ChunkGeom g0 = strip_geom(a, x0 - bc.dmax, g.X[j1_first - 1] - x0 + bc.nd);
    layout_block<NT>(bc, g, sm, sh, true, j1_first, g0);
    issue_chunk<NT>(a, bc, sm, sh, true, 0, g0, withhold);
}

// begin_block_ctx over block b's whole candidate range, its record in sh.geom[gbuf].
template <int NT>
__device__ void begin_block(const MatchArgs &a, int b, const Smem &sm, Shared<NT / 32> &sh, int gbuf,
                            bool withhold = false)
{
    begin_block_ctx<NT>(a, make_ctx(a, sh.geom[gbuf], b), sh.geom[gbuf], sm, sh, withhold);
}

// Block record from the two passes' results (Eq. subpixel on the forward costs
// around d_f, consistency |d_b - d_f| <= fb_tol); boxes are aggregated by
// aggregate_kernel.  bc: the block's whole candidate range.
__device__ __forceinline__ void write_record(const MatchArgs &a, const BlockCtx &bc, int total, int d_f, int dy_f,
                                             int d_b, int dy_b, int s_m, int s_0, int s_p)
{
    ctm_block rec;
    rec.n_pts = bc.nx * bc.ny;
    rec.n_valid = total;
    rec.flags = CTM_BLK_PRESENT;
    rec.d_f = d_f;
    rec.dy_f = dy_f;
    rec.d_b = d_b;
    rec.dy_b = dy_b;
    rec.s_m = s_m;
    rec.s_0 = s_0;
    rec.s_p = s_p;
    if (rec.d_f == bc.dmin || rec.d_f == bc.dmax) {
        rec.d_sub = (float)rec.d_f;
        rec.flags |= CTM_BLK_SUBPIX_CLAMPED;
    } else {
        // Eq. subpixel
        const float num = (float)(rec.s_p - rec.s_m);
        const float den = __fmul_rn(2.0f, (float)(rec.s_p + rec.s_m - 2 * rec.s_0));
        rec.d_sub = den == 0.0f ? (float)rec.d_f : __fsub_rn((float)rec.d_f, __fdiv_rn(num, den));
    }
    rec.d_full = __fmul_rn(rec.d_sub, (float)bc.k);
    const int dxv = abs(rec.d_b - rec.d_f);
    rec.flags |= dxv <= a.p.fb_tol ? CTM_BLK_VALID : CTM_BLK_FB_REJECT;
    write_block(a, bc.box, bc.slot, rec);
}

// Prefetch state of the persistent kernel.  A single-block launch has none.
struct Prefetch {
    bool on;
    int n_big, nq;  // first queue: blocks from the front; queue length
    int R, rank;    // rounds mode: rounds; thread 0: this CTA's rank on its SM
    int buf;        // geometry buffer of the next block
};

// Rounds mode, warp 0 after a block's forward pass: a round position that no CTA
// of that rank took, from the round counters lane r read (into h) when the block
// started -- a counter seen full stays full, one seen with room is claimed by an
// atomic that may still lose -- so the sweep adds no round trip to a block unless
// it finds one.  Lane 0 gets the position (nq: none).
__device__ __forceinline__ int sweep_rounds_warp(int *sched, int nq, int R, int n_sm, int h)
{
    const int lane = threadIdx.x & 31;
    const int lim = lane < R ? min(n_sm, nq - lane * n_sm) : 0;
    unsigned room = __ballot_sync(0xffffffffu, lane < R && h < lim);
    int pos = nq;
    if (lane == 0) {
        while (room) {
            const int r = __ffs(room) - 1;
            const int k = atomicAdd(sched + kSchedSMs + r, 1);
            if (k < min(n_sm, nq - r * n_sm)) {
                pos = r * n_sm + k;
                break;
            }
            room &= room - 1u;
        }
    }
    return pos;
}

template <bool ROUNDS, int NW>
__device__ __forceinline__ int queue_block(const MatchArgs &a, const Shared<NW> &sh, const Prefetch &pf, int p)
{
    return ROUNDS ? queue_w_at(a, sh.qstart, p) : queue_at(a, pf.n_big, p);
}

// One block end to end, after begin_block.  With pf.on, thread 0 takes the next
// queue index at the start and issues the next block's record copy once the
// forward pass is done; when the backward scans are over, the CTA waits for
// that record and begins the next block (its codes and first strip in flight)
// before thread 0 writes this block's record, so the next block's first round
// trip overlaps this block's end.  Forward and backward costs have their own
// rows, so no barrier separates one pass's argmin from the next pass's
// zeroing.  Returns false if a bounded wait expired.  evals: thread 0 adds this
// block's evaluation count.
template <int NT, bool ROUNDS = false>
__device__ bool process_block(const MatchArgs &a, int b, const Smem &sm, Shared<NT / 32> &sh,
                              unsigned &phase, int gbuf, Prefetch &pf, unsigned &gphase,
                              unsigned long long &evals)
{
    const int tid = threadIdx.x;
    int next_i = 0, h = 0;
    if (ROUNDS) {  // the round counters, read now and used after the forward pass
        if (pf.on && tid < pf.R) h = *reinterpret_cast<volatile int *>(a.ws.sched + kSchedSMs + tid);
    } else if (pf.on && tid == 0) {
        next_i = atomicAdd(&a.ws.counts->queue_head, 1);
    }
    const BlockGeom &g = sh.geom[gbuf];
    const BlockCtx bc = make_ctx(a, g, b);
    const int total = g.n_valid;
    const unsigned later0 = g.cstart & ~1u;
    const int j1_first = later0 ? __ffs(later0) - 1 : bc.nx;
    const int x0 = g.X[0];
    const int SW0 = g.X[j1_first - 1] - x0 + bc.nd;
    const ChunkGeom g0 = strip_geom(a, x0 - bc.dmax, SW0);

    // 1. the left codes and the first forward strip chunk (issued by begin_block)
    bool ok = land_chunk<NT>(a, bc, sm, sh, phase, true, 0, g0);
    cp_async_wait_all();
    int next_b = 0;
    if (!ROUNDS && pf.on && tid == 0 && next_i < pf.nq) next_b = queue_block<false>(a, sh, pf, next_i);
    if (!__syncthreads_and(ok)) return false;

    // 2-3. forward pass, argmin (every thread), parabola inputs
    int acc[8];
    ok = scan_chunks<NT>(a, bc, sm, sh, phase, true, g0, acc, 0, 0);
    unsigned key;
    if (!combine_pass<NT>(a, bc, sm, true, acc, ok, key)) return false;
    const int cf = (int)(key & 0xffffu);
    const int ef = bc.ndy == 1 ? 0 : cf / bc.nd;
    const int dif = cf - ef * bc.nd;
    const int d_f = bc.dmin + dif, dy_f = a.p.dy_min + ef;
    if (ROUNDS && pf.on && tid < 32) {
        next_i = sweep_rounds_warp(a.ws.sched, pf.nq, pf.R, a.sm_count, h);
        if (tid == 0 && next_i < pf.nq) next_b = queue_block<true>(a, sh, pf, next_i);
    }
    int s_m = 0, s_p = 0;
    if (tid == 0) {
        s_m = dif > 0 ? sm.cost[cf - 1] + sm.cost_b[cf - 1] : 0;
        s_p = dif < bc.nd - 1 ? sm.cost[cf + 1] + sm.cost_b[cf + 1] : 0;
        if (pf.on) {
            sh.next = next_i;
            sh.next_b = next_b;
            if (next_i < pf.nq) {  // the next block's record, in flight during this backward pass
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_expect_tx(&sh.mbar_g, (unsigned)sizeof(BlockGeom));
                bulk_g2s(&sh.geom[pf.buf], a.ws.geom + next_b, (unsigned)sizeof(BlockGeom), &sh.mbar_g);
                sh.gpend = 1;
            }
        }
    }

    // 4. backward pass: the right codes at the matched positions and the first left
    //    strip (every warp's forward scans ended at combine_pass's barrier).  A block
    //    whose forward strip was one chunk still holds every matched position in it
    //    (X_j - d_f lies in [X_j - dmax, X_j - dmin], row Y_m + dy_f among its rows,
    //    zero where outside the plane as a global read gives), so its codes come from
    //    shared memory before the backward copies overwrite the strip; otherwise they
    //    are plain global loads that overlap the copies' round trip.
    const ChunkGeom gb = strip_geom(a, x0 - d_f + bc.dmin, SW0);
    {
        constexpr int kPer = kMaxPts / NT;
        uint64_t v[kPer];
        if (j1_first == bc.nx) {
            const int col0 = bc.dmax + g0.delta - x0 - d_f;  // strip column of X_j - d_f is X_j + col0
            const int row_e = dy_f - a.p.dy_min;
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int t = tid + i * NT;
                v[i] = 0ull;
                if (t < total) {
                    const int mj = sm.pmj[t];
                    const int r = (mj >> 8) * bc.ndy + row_e;
                    v[i] = sm.strip[r * g0.stride + sh.X[mj & 255] + col0];
                }
            }
            __syncthreads();  // the strip's reads are done before the backward copies
            issue_chunk<NT>(a, bc, sm, sh, false, dy_f, gb);
        } else {
            issue_chunk<NT>(a, bc, sm, sh, false, dy_f, gb);
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int t = tid + i * NT;
                v[i] = 0ull;
                if (t < total) {
                    const int mj = sm.pmj[t];
                    const int qx = sh.X[mj & 255] - d_f, qy = sh.Y[mj >> 8] + dy_f;
                    if (qx >= 0 && qx < bc.Ws && qy >= 0 && qy < bc.Hs)
                        v[i] = __ldg(bc.CR + (long long)qy * bc.pitch + qx);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (tid + i * NT < total) sm.pcode[tid + i * NT] = v[i];
    }
    ok = land_chunk<NT>(a, bc, sm, sh, phase, false, dy_f, gb);
    set_bases<NT>(sm, sh.X, 0, sh.colstart[j1_first], bc.ndy, gb.stride, x0, gb.delta);
    if (!__syncthreads_and(ok)) return false;
    ok = scan_chunks<NT>(a, bc, sm, sh, phase, false, gb, acc, d_f, dy_f);
    unsigned keyb;
    if (!combine_pass<NT>(a, bc, sm, false, acc, ok, keyb)) return false;

    // the next block starts now: its record (wait) and its first loads (issued)
    const bool has_next = pf.on && sh.gpend;
    if (has_next) {
        const bool landed = mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
        if (landed) gphase ^= 1u;
        if (!__syncthreads_and(landed)) return false;
        if (tid == 0) sh.gpend = 0;
        begin_block<NT>(a, sh.next_b, sm, sh, pf.buf);
    }

    if (tid == 0) {
        const int cb = (int)(keyb & 0xffffu);
        const int eb = bc.ndy == 1 ? 0 : cb / bc.nd;
        // 5. block record; boxes are aggregated by aggregate_kernel
        write_record(a, bc, total, d_f, dy_f, bc.dmin + (cb - eb * bc.nd), a.p.dy_min + eb, s_m,
                     (int)(key >> 16), s_p);
        evals += 2ull * (unsigned long long)total * (unsigned long long)bc.nc;
    }
    return true;
}

// Disparity-chunk tiles.  When the work queue holds few blocks for the resident
// CTAs (a single frame, a small batch), the persistent kernel splits every
// searchable block's candidate range into `ways` chunks of whole 32-candidate
// slices and takes (block, chunk) tiles: first the forward tiles of every block,
// then the backward tiles, in queue order.  A forward tile scans its candidates,
// stores its costs in the block's cost row and merges its first minimum into the
// block's key with atomicMin on (cost << 16 | candidate) -- the minimum of the
// keys is the first minimum of the whole row whatever order the tiles finish
// in; the tile that finishes last (a ticket counter) reads the merged key, the
// costs beside it (Eq. subpixel) and publishes d_f.  A backward tile waits for
// that (bounded: every forward tile of its block was taken earlier by a running
// CTA, none of which waits on anything), scans its share of the backward
// candidates around d_f and merges its minimum the same way; the last one writes
// the block record.  Results equal the unsplit block's bit for bit.

// Bounded wait, by thread 0, for a flag another CTA of this launch sets: about
// one second of the global timer (an iteration cap as a backstop); false, with
// the error recorded, on expiry.
__device__ __forceinline__ bool wait_flag(const int *flag, int *error_flag)
{
    const volatile int *f = flag;
    if (*f) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < kWaitIters; ++it) {
        __nanosleep(64);
        if (*f) return true;
        if ((it & 15u) == 0 && global_ns() - t0 > kWaitNs) break;
    }
    atomicOr(error_flag, 1);
    return false;
}

__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }

// Candidate range [c0, c1) of chunk c of `ways` over nd candidates: whole
// 32-candidate slices, the last chunk ragged, trailing chunks possibly empty.
__device__ __forceinline__ void chunk_range(int nd, int ways, int c, int &c0, int &c1)
{
    const int cw = (((nd + ways - 1) / ways) + 31) & ~31;
    c0 = min(c * cw, nd);
    c1 = min(c0 + cw, nd);
}

// One tile after its record has landed in sh.geom[0].  False if a bounded wait
// expired (nothing of this tile is merged then).
template <int NT>
__device__ bool process_tile(const MatchArgs &a, int b, int c, int ways, bool bwd, const Smem &sm,
                             Shared<NT / 32> &sh, unsigned &phase, unsigned long long &evals, bool withhold)
{
    const int tid = threadIdx.x;
    const BlockGeom &g = sh.geom[0];
    const BlockCtx full = make_ctx(a, g, b);
    ChunkState *st = a.ws.chunk + b;
    int c0, c1;
    chunk_range(full.nd, ways, c, c0, c1);
    BlockCtx bc = full;
    bc.dmin = full.dmin + c0;
    bc.dmax = full.dmin + c1 - 1;
    bc.nd = c1 - c0;
    bc.nc = bc.nd;  // one dy row (ways > 1 only then)
    int d_f = 0;
    if (bwd) {  // the block's forward merge
        bool ready = true;
        if (tid == 0) ready = wait_flag(&st->ready, &a.ws.counts->error);
        if (!__syncthreads_and(ready)) return false;
        __threadfence();
        d_f = ld_cg(&st->d_f);
    }
    unsigned key = 0xffffffffu;
    if (c0 < c1) {
        const int total = g.n_valid;
        const int j1_first = first_chunk_end(g, bc.nx);
        const int x0 = g.X[0];
        const int SW0 = g.X[j1_first - 1] - x0 + bc.nd;
        int acc[8];
        bool ok;
        if (!bwd) {
            begin_block_ctx<NT>(a, bc, g, sm, sh, withhold);
            ok = land_chunk<NT>(a, bc, sm, sh, phase, true, 0, strip_geom(a, x0 - bc.dmax, SW0));
            cp_async_wait_all();
            if (!__syncthreads_and(ok)) return false;
            ok = scan_chunks<NT>(a, bc, sm, sh, phase, true, strip_geom(a, x0 - bc.dmax, SW0), acc, 0, 0);
            if (!combine_pass<NT>(a, bc, sm, true, acc, ok, key, c0, a.ws.chunk_cost + (long long)b * a.nc_stride + c0))
                return false;
        } else {
            const int dy_f = a.p.dy_min;
            const ChunkGeom gb = strip_geom(a, x0 - d_f + bc.dmin, SW0);
            layout_block<NT>(bc, g, sm, sh, false, j1_first, gb);
            issue_chunk<NT>(a, bc, sm, sh, false, dy_f, gb);
            for (int t = tid; t < total; t += NT) {  // right codes at the matched positions
                const int mj = sm.pmj[t];
                const int qx = sh.X[mj & 255] - d_f, qy = sh.Y[mj >> 8] + dy_f;
                sm.pcode[t] = (qx >= 0 && qx < bc.Ws && qy >= 0 && qy < bc.Hs)
                                  ? __ldg(bc.CR + (long long)qy * bc.pitch + qx) : 0ull;
            }
            ok = land_chunk<NT>(a, bc, sm, sh, phase, false, dy_f, gb);
            set_bases<NT>(sm, sh.X, 0, sh.colstart[j1_first], bc.ndy, gb.stride, x0, gb.delta);
            if (!__syncthreads_and(ok)) return false;
            ok = scan_chunks<NT>(a, bc, sm, sh, phase, false, gb, acc, d_f, dy_f);
            if (!combine_pass<NT>(a, bc, sm, false, acc, ok, key, c0)) return false;
        }
        if (tid == 0) evals += (unsigned long long)total * (unsigned long long)bc.nd;
        key += (unsigned)c0;  // candidate index within the block
    }
    __threadfence();  // warp 0's cost-row stores, before the ticket below
    __syncthreads();
    if (tid == 0) {
        if (key != 0xffffffffu) atomicMin(bwd ? &st->bkey : &st->fkey, key);
        __threadfence();
        const int ticket = atomicAdd(bwd ? &st->bdone : &st->fdone, 1);
        if (ticket == ways - 1) {  // the last tile of this pass merges
            __threadfence();
            const int32_t *row = a.ws.chunk_cost + (long long)b * a.nc_stride;
            if (!bwd) {
                const unsigned k = (unsigned)atomicOr(&st->fkey, 0u);
                const int cf = (int)(k & 0xffffu);
                st->s_0 = (int)(k >> 16);
                st->s_m = cf > 0 ? ld_cg(row + cf - 1) : 0;
                st->s_p = cf < full.nd - 1 ? ld_cg(row + cf + 1) : 0;
                st->d_f = full.dmin + cf;
                __threadfence();
                atomicExch(&st->ready, 1);
            } else {
                const unsigned k = (unsigned)atomicOr(&st->bkey, 0u);
                write_record(a, full, g.n_valid, ld_cg(&st->d_f), a.p.dy_min, full.dmin + (int)(k & 0xffffu),
                             a.p.dy_min, ld_cg(&st->s_m), ld_cg(&st->s_0), ld_cg(&st->s_p));
            }
        }
    }
    return true;
}

__device__ __forceinline__ Smem carve(const MatchArgs &a, unsigned char *raw)
{
    Smem sm;
    size_t off = 0;
    sm.strip = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols;
    sm.pcode = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * kMaxPts;
    sm.cost = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxCand;
    sm.cost_b = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxCand;
    sm.pmj = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxPts;
    sm.pbase = reinterpret_cast<int *>(raw + off);
    return sm;
}

// After a failed bounded wait: let every copy still in flight land before the
// CTA leaves (its shared memory may go to another CTA).
template <int NT>
__device__ __forceinline__ void drain(const MatchArgs &a, Shared<NT / 32> &sh, unsigned phase, unsigned gphase)
{
    cp_async_wait_all();
    __syncthreads();
    if (sh.gpend) mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
    if (sh.spend) mbar_wait_bounded(&sh.mbar, phase, &a.ws.counts->error);
}

// The persistent kernel over disparity-chunk tiles (see process_tile): thread 0
// takes the next tile index and fetches its block's record; no look-ahead.
template <int NT>
__device__ void run_tiles(const MatchArgs &a, const Smem &sm, Shared<NT / 32> &sh, int n_big, int nq, int ways)
{
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        mbar_init(&sh.mbar_g, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        sh.gpend = 0;
        sh.spend = 0;
    }
    __syncthreads();
    unsigned phase = 0, gphase = 0;
    unsigned long long evals = 0ull;
    const int n_fwd = nq * ways, n_tiles = 2 * n_fwd;
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = atomicAdd(&a.ws.counts->queue_head, 1);
            sh.next = i;
            if (i < n_tiles) {
                const int j = i < n_fwd ? i : i - n_fwd;
                sh.next_b = queue_at(a, n_big, j / ways);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_expect_tx(&sh.mbar_g, (unsigned)sizeof(BlockGeom));
                bulk_g2s(&sh.geom[0], a.ws.geom + sh.next_b, (unsigned)sizeof(BlockGeom), &sh.mbar_g);
                sh.gpend = 1;
            }
        }
        __syncthreads();
        const int i = sh.next;
        if (i >= n_tiles) break;
        const bool landed = mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
        if (landed) gphase ^= 1u;
        if (!__syncthreads_and(landed)) {
            drain<NT>(a, sh, phase, gphase);
            break;
        }
        if (threadIdx.x == 0) sh.gpend = 0;
        const bool bwd = i >= n_fwd;
        const int j = bwd ? i - n_fwd : i;
        const bool withhold = a.inject_expiry != 0 && i == 0;  // the first forward tile
        if (!process_tile<NT>(a, sh.next_b, j % ways, ways, bwd, sm, sh, phase, evals, withhold)) {
            drain<NT>(a, sh, phase, gphase);
            break;
        }
        __syncthreads();  // the tile's shared data is done with before the next record lands
    }
    if (threadIdx.x == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
}

// The persistent kernel's block loop: thread 0 takes the first queue position
// (ROUNDS: its SM rank's round) and fetches that block's record; then block after
// block, each taking and beginning the next one (process_block).
template <int NT, bool ROUNDS>
__device__ void run_blocks(const MatchArgs &a, const Smem &sm, Shared<NT / 32> &sh, Prefetch &pf)
{
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        mbar_init(&sh.mbar_g, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int i = ROUNDS ? take_first_round(a.ws.sched, pf.rank, pf.nq, pf.R, a.sm_count)
                             : atomicAdd(&a.ws.counts->queue_head, 1);
        sh.next = i;
        sh.gpend = 0;
        sh.spend = 0;
        if (i < pf.nq) {
            sh.next_b = queue_block<ROUNDS>(a, sh, pf, i);
            mbar_arrive_expect_tx(&sh.mbar_g, (unsigned)sizeof(BlockGeom));
            bulk_g2s(&sh.geom[0], a.ws.geom + sh.next_b, (unsigned)sizeof(BlockGeom), &sh.mbar_g);
            sh.gpend = 1;
        }
    }
    __syncthreads();
    unsigned phase = 0, gphase = 0;
    unsigned long long evals = 0ull;
    if (sh.gpend) {
        // the first block: wait for its record, begin it
        const bool landed = mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
        if (landed) gphase ^= 1u;
        if (__syncthreads_and(landed)) {
            if (threadIdx.x == 0) sh.gpend = 0;
            int b = sh.next_b;
            int buf = 0;
            begin_block<NT>(a, b, sm, sh, buf, a.inject_expiry != 0 && sh.next == 0);
            for (;;) {
                pf.buf = buf ^ 1;
                if (!process_block<NT, ROUNDS>(a, b, sm, sh, phase, buf, pf, gphase, evals)) {
                    drain<NT>(a, sh, phase, gphase);
                    break;
                }
                if (sh.next >= pf.nq) break;  // no block was begun
                b = sh.next_b;
                buf ^= 1;
            }
        } else {
            drain<NT>(a, sh, phase, gphase);
        }
    }
    if (threadIdx.x == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
}

// ROUNDS (chosen by the host, see rounds_kernel): the work-ordered queue in
// per-SM rounds; else the first queue, or disparity-chunk tiles.
template <int NT, bool ROUNDS>
__global__ void __launch_bounds__(NT, 1024 / NT)
    match_persistent_kernel(MatchArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Shared<NT / 32> sh;
    const Smem sm = carve(a, smem_raw);
    Prefetch pf;
    pf.on = true;
    pf.rank = 0;
    if (ROUNDS) {
        // thread 0: its rank on the SM and the class counts in one round trip
        if (threadIdx.x == 0) {
            const unsigned sid = sm_id();
            pf.rank = sid < (unsigned)kSchedSMs ? atomicAdd(a.ws.sched + sid, 1) : kMaxRounds;
            queue_starts(a.ws.counts, sh.qstart);
            sh.nq = work_queue_on(a, a.ws.counts->n_blocks) ? sh.qstart[kQueueClasses] : -1;
        }
        __syncthreads();
        pf.nq = sh.nq;
        pf.n_big = 0;
        if (pf.nq == 0) return;
        // the host's choice guarantees a written work-ordered queue of at most
        // kMaxRounds rounds; should it not hold, the call reports an error
        pf.R = ceil_div_nn(pf.nq, a.sm_count);
        if (pf.nq < 0 || pf.R > kMaxRounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ws.counts->error, 1);
            return;
        }
        run_blocks<NT, true>(a, sm, sh, pf);
        return;
    }
    const int n_big = a.ws.counts->n_big;
    pf.nq = n_big + a.ws.counts->n_small;
    pf.n_big = n_big;
    pf.R = 0;
    // fewer blocks than about 0.6 per resident CTA, and CLOSE blocks with at least 128
    // candidates: (block, disparity-chunk) tiles, two per block (measured: narrower
    // chunks and more of them only add per-tile cost); one vertical offset only, not
    // in the allocation-free path
    if (a.ws.chunk != nullptr && a.p.dy_min == a.p.dy_max && pf.nq > 0 && a.split_ways != 1) {
        const bool short_queue = 8 * pf.nq <= 5 * (int)gridDim.x && a.p.close_dmax - a.p.close_dmin + 1 >= 128;
        const int w = a.split_ways > 1 ? a.split_ways : (short_queue ? 2 : 1);
        const int ways = w >= 8 ? 8 : (w >= 4 ? 4 : (w >= 2 ? 2 : 1));
        if (ways > 1) {
            run_tiles<NT>(a, sm, sh, n_big, pf.nq, ways);
            return;
        }
    }
    run_blocks<NT, false>(a, sm, sh, pf);
}

template <int NT>
__global__ void __launch_bounds__(NT) match_box_kernel(MatchArgs a, int box)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Shared<NT / 32> sh;
    if ((int)blockIdx.x >= a.ws.nblk[box]) return;
    const int b = a.ws.blk_base[box] + blockIdx.x;
    if (a.ws.geom[b].n_valid < a.p.min_pts) return;  // finished by the sampling kernel
    const Smem sm = carve(a, smem_raw);
    if (threadIdx.x < (int)(sizeof(BlockGeom) / 16))
        cp_async16(reinterpret_cast<char *>(&sh.geom[0]) + 16 * threadIdx.x,
                   reinterpret_cast<const char *>(a.ws.geom + b) + 16 * threadIdx.x);
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        sh.gpend = 0;
        sh.spend = 0;
    }
    cp_async_wait_all();
    __syncthreads();
    unsigned phase = 0, gphase = 0;
    unsigned long long evals = 0ull;
    Prefetch pf;
    pf.on = false;
    pf.n_big = pf.nq = pf.R = pf.rank = 0;
    pf.buf = 1;
    begin_block<NT>(a, b, sm, sh, 0);
    if (!process_block<NT>(a, b, sm, sh, phase, 0, pf, gphase, evals)) drain<NT>(a, sh, phase, gphase);
    if (threadIdx.x == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
}

}  // namespace

size_t match_smem_bytes(const MatchArgs &a)
{
    return sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols + sizeof(uint64_t) * kMaxPts +
           2 * sizeof(int) * kMaxCand + 2 * sizeof(int) * kMaxPts;
}

// The dynamic shared-memory limit is a per-kernel, process-wide setting: it is
// only ever raised, so contexts with different strip sizes can coexist.
cudaError_t match_configure(const MatchArgs &a, int threads, int *ctas_per_sm)
{
    const int need = (int)match_smem_bytes(a);
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (threads == 128) {
        e = cudaFuncGetAttributes(&fa, match_box_kernel<128>);
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
            e = cudaFuncSetAttribute(match_box_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    } else {
        e = cudaFuncGetAttributes(&fa, match_box_kernel<256>);
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
            e = cudaFuncSetAttribute(match_box_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    }
    if (e != cudaSuccess) return e;
    return match_configure_raise(a, threads, ctas_per_sm);
}

namespace {

// Raise one persistent kernel's shared-memory limit to `need` and query its
// resident CTAs per SM.
template <int NT, bool ROUNDS>
cudaError_t raise_persistent(int need, int *ctas_per_sm)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, match_persistent_kernel<NT, ROUNDS>);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
        e = cudaFuncSetAttribute(match_persistent_kernel<NT, ROUNDS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 need);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,
                                                                           match_persistent_kernel<NT, ROUNDS>, NT, need);
    return e;
}

template <int NT>
cudaError_t raise_persistent_both(int need, int *ctas_per_sm)
{
    int c0 = 0, c1 = 0;
    cudaError_t e = raise_persistent<NT, false>(need, &c0);
    if (e == cudaSuccess) e = raise_persistent<NT, true>(need, &c1);
    *ctas_per_sm = c0 < c1 ? c0 : c1;
    return e;
}

// The rounds variant of the persistent kernel serves contexts whose whole
// capacity of blocks fits in kMaxRounds rounds (then the sampling kernel always
// writes the work-ordered queue, and every call's queue fits in them), unless
// rounds are tuned off or disparity-chunk tiles are forced.
bool rounds_kernel(const MatchArgs &a)
{
    return a.queue_rounds && a.ws.sched != nullptr && a.ws.queue_w != nullptr && a.split_ways <= 1 &&
           a.sm_count > 0 && a.caps.max_blocks <= kMaxRounds * a.sm_count;
}

}  // namespace

cudaError_t match_configure_raise(const MatchArgs &a, int threads, int *ctas_per_sm)
{
    const int need = (int)match_smem_bytes(a);
    return threads == 128 ? raise_persistent_both<128>(need, ctas_per_sm)
                          : raise_persistent_both<256>(need, ctas_per_sm);
}

cudaError_t launch_match_persistent(const MatchArgs &a, int threads, int grid, cudaStream_t s)
{
    const size_t smem = match_smem_bytes(a);
    const bool r = rounds_kernel(a);
    if (threads == 128) {
        if (r)
            match_persistent_kernel<128, true><<<grid, 128, smem, s>>>(a);
        else
            match_persistent_kernel<128, false><<<grid, 128, smem, s>>>(a);
    } else {
        if (r)
            match_persistent_kernel<256, true><<<grid, 256, smem, s>>>(a);
        else
            match_persistent_kernel<256, false><<<grid, 256, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_match_box(const MatchArgs &a, int threads, int box, cudaStream_t s)
{
    const int slots = a.p.grid_g * a.p.grid_g;
    if (threads == 128)
        match_box_kernel<128><<<slots, 128, match_smem_bytes(a), s>>>(a, box);
    else
        match_box_kernel<256><<<slots, 256, match_smem_bytes(a), s>>>(a, box);
    return cudaGetLastError();
}

}  // namespace ctm
