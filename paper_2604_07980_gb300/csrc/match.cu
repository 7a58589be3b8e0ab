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
//      registers, and warps combine them with shared-memory atomics;
//   3. first argmin over (dy, d) by warp min-reductions of (cost << 16 | index)
//      keys, then Eq. subpixel in fp32 with IEEE division;
//   4. backward pass (Sec. 4.3.3): the right codes at the matched positions and
//      the left strip [q.x + dmin, q.x + dmax] arrive in one round trip;
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
    unsigned warp_min[NW];
    int d_f, dy_f, s_m, s_0, s_p;
    int d_b, dy_b;
    int next;               // queue index of the next block
    int next_b;             // its block
    int gpend;              // a geometry copy is in flight on mbar_g
    unsigned cstart;        // bit j set: a strip column chunk starts at point column j
    int abort;              // a bounded wait expired: stop this CTA
};

struct BlockCtx {
    int box, slot, b;
    int k, far;
    int dmin, dmax, nd, ndy, nc;
    int nx, ny, Ws, Hs;
    long long pitch;
    const uint64_t *CL;
    const uint64_t *CR;
};

// Load one strip chunk: rows (m, e) of the right plane at Y_m + dy_min + e
// (forward) or of the left plane at Y_m + dy_f - (dy_min + e) (backward).
// Warp 0 issues one bulk copy per row for its in-plane part; lane 0 first
// registers the total byte count on the CTA's mbarrier.  After the copies land,
// positions outside the plane are zero-filled (only edge chunks have any).
// Returns false if the bounded wait expired.
template <int NT>
__device__ __forceinline__ bool load_chunk(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                                           Shared<NT / 32> &sh, unsigned &phase, bool fwd, int dy_f,
                                           const ChunkGeom &g)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int rows = bc.ny * bc.ndy;
    const uint64_t *plane = fwd ? bc.CR : bc.CL;
    const int Ws_even = (bc.Ws + 1) & ~1;   // the padding column after an odd width is readable
    const int x_lo = max(g.colbase_a, 0);
    const int x_hi = min(g.colbase_a + g.SWa, Ws_even);
    const unsigned row_bytes = x_hi > x_lo ? 8u * (unsigned)(x_hi - x_lo) : 0u;
    if (tid < 32) {
        unsigned total = 0;
        for (int r = lane; r < rows; r += 32) {
            const int m = bc.ndy == 1 ? r : r / bc.ndy;
            const int e = r - m * bc.ndy;
            const int y = fwd ? sh.Y[m] + a.p.dy_min + e : sh.Y[m] + dy_f - (a.p.dy_min + e);
            if (y >= 0 && y < bc.Hs) total += row_bytes;
        }
        total = __reduce_add_sync(0xffffffffu, total);
        // order earlier generic-proxy accesses of the strip before the bulk writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (lane == 0) mbar_arrive_expect_tx(&sh.mbar, total);
        __syncwarp();
        if (row_bytes > 0) {
            for (int r = lane; r < rows; r += 32) {
                const int m = bc.ndy == 1 ? r : r / bc.ndy;
                const int e = r - m * bc.ndy;
                const int y = fwd ? sh.Y[m] + a.p.dy_min + e : sh.Y[m] + dy_f - (a.p.dy_min + e);
                if (y >= 0 && y < bc.Hs)
                    bulk_g2s(sm.strip + r * g.SWa + (x_lo - g.colbase_a), plane + (long long)y * bc.pitch + x_lo,
                             row_bytes, &sh.mbar);
            }
        }
    }
    const bool ok = mbar_wait_bounded(&sh.mbar, phase, &a.ws.counts->error);
    phase ^= 1u;
    // zero-fill what lies outside the plane (rows outside it; columns < 0 or >= Ws)
    const bool edge = g.colbase_a < 0 || g.colbase_a + g.SWa > bc.Ws ||
                      sh.Y[0] + (fwd ? a.p.dy_min : dy_f - a.p.dy_max) < 0 ||
                      sh.Y[bc.ny - 1] + (fwd ? a.p.dy_max : dy_f - a.p.dy_min) >= bc.Hs;
    if (edge) {  // a warp per row: whole rows outside the plane, else the columns outside it
        const int warp = tid >> 5;
        const int c_lo = min(max(-g.colbase_a, 0), g.SWa);             // [0, c_lo): x < 0
        const int c_hi = max(min(bc.Ws - g.colbase_a, g.SWa), c_lo);   // [c_hi, SWa): x >= Ws
        for (int r = warp; r < rows; r += NT / 32) {
            const int m = bc.ndy == 1 ? r : r / bc.ndy;
            const int e = r - m * bc.ndy;
            const int y = fwd ? sh.Y[m] + a.p.dy_min + e : sh.Y[m] + dy_f - (a.p.dy_min + e);
            uint64_t *row = sm.strip + r * g.SWa;
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

// Warp and CTA minimum of the keys (cost << 16 | c) over the candidates; the
// result lands in sh.warp_min[0] and the costs stay in shared memory.
template <int NT>
__device__ __forceinline__ void argmin_pass(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                                            Shared<NT / 32> &sh, bool fwd)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned key = 0xffffffffu;
    int32_t *dbgc = fwd ? a.dbg.cost_f : a.dbg.cost_b;
    const int slots = a.p.grid_g * a.p.grid_g;
    for (int c = tid; c < bc.nc; c += NT) {
        const int s = sm.cost[c];
        key = min(key, ((unsigned)s << 16) | (unsigned)c);
        if (dbgc) dbgc[((long long)bc.box * slots + bc.slot) * a.nc_stride + c] = s;
    }
    key = __reduce_min_sync(0xffffffffu, key);
    if (lane == 0) sh.warp_min[warp] = key;
    __syncthreads();
    if (tid == 0) {
        unsigned m = sh.warp_min[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) m = min(m, sh.warp_min[w]);
        sh.warp_min[0] = m;
    }
    __syncthreads();
}

// One search pass after its first strip chunk has landed and the point bases of
// the first chunk are set.  Returns false if a bounded wait expired.
template <int NT>
__device__ bool search_pass(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                            Shared<NT / 32> &sh, unsigned &phase, bool fwd, ChunkGeom g)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int T = (bc.nc + 31) >> 5;
    const bool fast = bc.ndy == 1 && (bc.nd & 31) == 0;
    int acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0;
    const int d_f = sh.d_f, dy_f = sh.dy_f;
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
            g = chunk_geom(fwd ? xj0 - bc.dmax : xj0 - d_f + bc.dmin, SWc);
            ok = load_chunk<NT>(a, bc, sm, sh, phase, fwd, dy_f, g) && ok;
            set_bases<NT>(sm, sh.X, p0, p1, bc.ndy, g.SWa, xj0, g.delta);
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
                    o = e * g.SWa + (fwd ? (bc.nd - 1 - c) : c);
                }
                coff[t] = o;
            }
            scan_dispatch<NW>(T, sm, p0, p1, coff, acc);
        }
        __syncthreads();
        j0 = j1;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int c = t * 32 + lane;
        if (t < T && c < bc.nc) atomicAdd(&sm.cost[c], acc[t]);
    }
    __syncthreads();
    argmin_pass<NT>(a, bc, sm, sh, fwd);
    return ok;
}

// Queue entry i: large work from the front, small work from the back.
__device__ __forceinline__ int queue_block(const MatchArgs &a, int i, int n_big)
{
    return i < n_big ? a.ws.queue[i] : a.ws.queue[a.caps.max_blocks - 1 - (i - n_big)];
}

// Prefetch state of the persistent kernel: the queue index taken for the next
// block and the geometry buffer it goes to.  A single-block launch has none.
struct Prefetch {
    bool on;
    int n_big, nq;
    int buf;  // geometry buffer of the next block
};

// One block end to end.  Its geometry is in sh.geom[gbuf] (landed).  With
// pf.on, thread 0 takes the next queue index at the start, and once the
// forward pass is done issues the next block's geometry copy into the other
// buffer (completion on sh.mbar_g), so that round trip overlaps this block.
// Returns false if a bounded wait expired.  evals: thread 0 adds this block's
// evaluation count.
template <int NT>
__device__ bool process_block(const MatchArgs &a, int b, const Smem &sm, Shared<NT / 32> &sh,
                              unsigned &phase, int gbuf, const Prefetch &pf, unsigned long long &evals)
{
    int next_i = 0;
    if (pf.on && threadIdx.x == 0) next_i = atomicAdd(&a.ws.counts->queue_head, 1);
    const int tid = threadIdx.x;
    const int2 bs = a.ws.blocks[b];
    const BoxPlan P = a.ws.plans[bs.x];
    BlockCtx bc;
    bc.box = bs.x;
    bc.slot = bs.y;
    bc.b = b;
    bc.k = P.k;
    bc.far = P.far;
    bc.dmin = P.dmin;
    bc.dmax = P.dmax;
    bc.nd = P.dmax - P.dmin + 1;
    bc.ndy = a.p.dy_max - a.p.dy_min + 1;
    bc.nc = bc.nd * bc.ndy;
    bc.Ws = P.Ws;
    bc.Hs = P.Hs;
    {
        const bool full = P.far || a.p.close_factor == 1;
        const uint64_t *base = a.ws.census + (long long)P.frame * a.ws.frame_stride;
        bc.CL = full ? base : base + 2 * a.ws.plane1_elems;
        bc.CR = full ? base + a.ws.plane1_elems : base + 2 * a.ws.plane1_elems + a.ws.planek_elems;
        bc.pitch = full ? a.ws.pitch1 : a.ws.pitchk;
    }

    // 1a. the block's sampled grid and usable points (from the sampling kernel)
    for (int c = tid; c < bc.nc; c += NT) sm.cost[c] = 0;
    const BlockGeom &g = sh.geom[gbuf];
    bc.nx = g.nx;
    bc.ny = g.ny;
    const int total = g.n_valid;
    const unsigned later0 = g.cstart & ~1u;
    const int j1_first = later0 ? __ffs(later0) - 1 : bc.nx;
    const int x0 = g.X[0];
    const int SW0 = g.X[j1_first - 1] - x0 + bc.nd;
    const ChunkGeom g0 = chunk_geom(x0 - bc.dmax, SW0);

    // 1b. usable points at their compacted (column-major) index, left codes in flight
    for (int t = tid; t < kMaxPts; t += NT) {
        const int j = t >> 4, m = t & 15;
        if (j < bc.nx && ((g.colmask[j] >> m) & 1u)) {
            const int idx = g.colprefix[j] + __popc(g.colmask[j] & ((1u << m) - 1u));
            const int x = g.X[j], y = g.Y[m];
            cp_async8(&sm.pcode[idx], bc.CL + (long long)y * bc.pitch + x);
            sm.pmj[idx] = (m << 8) | j;
            if (j < j1_first) sm.pbase[idx] = 8 * (m * bc.ndy * g0.SWa + x - x0 + g0.delta);
        }
    }
    if (tid < kMaxPtsSide) {
        sh.X[tid] = g.X[tid];
        sh.Y[tid] = g.Y[tid];
    }
    if (tid <= kMaxPtsSide) sh.colstart[tid] = tid < bc.nx ? g.colprefix[tid] : total;
    if (tid == 0) sh.cstart = g.cstart;
    __syncthreads();
    // 1c. the first forward strip chunk
    bool ok = load_chunk<NT>(a, bc, sm, sh, phase, true, 0, g0);
    cp_async_wait_all();
    int next_b = 0;
    if (pf.on && tid == 0 && next_i < pf.nq) next_b = queue_block(a, next_i, pf.n_big);
    if (!__syncthreads_and(ok)) return false;

    ctm_block rec;
    rec.n_pts = bc.nx * bc.ny;
    rec.n_valid = total;
    rec.flags = CTM_BLK_PRESENT;

    // 2-3. forward pass, argmin, parabola
    ok = search_pass<NT>(a, bc, sm, sh, phase, true, g0);
    if (!__syncthreads_and(ok)) return false;
    if (tid == 0) {
        const unsigned key = sh.warp_min[0];
        const int c = (int)(key & 0xffffu);
        const int e = c / bc.nd, di = c - e * bc.nd;
        sh.d_f = bc.dmin + di;
        sh.dy_f = a.p.dy_min + e;
        sh.s_0 = (int)(key >> 16);
        sh.s_m = di > 0 ? sm.cost[c - 1] : 0;
        sh.s_p = di < bc.nd - 1 ? sm.cost[c + 1] : 0;
        if (pf.on) {
            sh.next = next_i;
            sh.next_b = next_b;
            if (next_i < pf.nq) {  // the next block's geometry, in flight during this backward pass
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_expect_tx(&sh.mbar_g, (unsigned)sizeof(BlockGeom));
                bulk_g2s(&sh.geom[pf.buf], a.ws.geom + next_b, (unsigned)sizeof(BlockGeom), &sh.mbar_g);
                sh.gpend = 1;
            }
        }
    }
    __syncthreads();
    // 4. backward pass: right codes at the matched positions + first left strip
    const int d_f = sh.d_f, dy_f = sh.dy_f;
    for (int t = tid; t < total; t += NT) {
        const int mj = sm.pmj[t];
        const int qx = sh.X[mj & 255] - d_f, qy = sh.Y[mj >> 8] + dy_f;
        if (qx >= 0 && qx < bc.Ws && qy >= 0 && qy < bc.Hs)
            cp_async8(&sm.pcode[t], bc.CR + (long long)qy * bc.pitch + qx);
        else
            sm.pcode[t] = 0ull;
    }
    for (int c = tid; c < bc.nc; c += NT) sm.cost[c] = 0;
    const ChunkGeom gb = chunk_geom(x0 - d_f + bc.dmin, SW0);
    ok = load_chunk<NT>(a, bc, sm, sh, phase, false, dy_f, gb);
    set_bases<NT>(sm, sh.X, 0, sh.colstart[j1_first], bc.ndy, gb.SWa, x0, gb.delta);
    cp_async_wait_all();
    if (!__syncthreads_and(ok)) return false;
    ok = search_pass<NT>(a, bc, sm, sh, phase, false, gb);
    if (!__syncthreads_and(ok)) return false;
    if (tid == 0) {
        const unsigned key = sh.warp_min[0];
        const int c = (int)(key & 0xffffu);
        const int e = c / bc.nd;
        sh.d_b = bc.dmin + (c - e * bc.nd);
        sh.dy_b = a.p.dy_min + e;
    }
    __syncthreads();

    // 5. block record (thread 0); boxes are aggregated by aggregate_kernel
    if (tid == 0) {
        rec.d_f = sh.d_f;
        rec.dy_f = sh.dy_f;
        rec.d_b = sh.d_b;
        rec.dy_b = sh.dy_b;
        rec.s_m = sh.s_m;
        rec.s_0 = sh.s_0;
        rec.s_p = sh.s_p;
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
        evals += 2ull * (unsigned long long)total * (unsigned long long)bc.nc;
    }
    __syncthreads();
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
    sm.pmj = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxPts;
    sm.pbase = reinterpret_cast<int *>(raw + off);
    return sm;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
    match_persistent_kernel(MatchArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Shared<NT / 32> sh;
    const Smem sm = carve(a, smem_raw);
    Prefetch pf;
    pf.on = true;
    pf.n_big = a.ws.counts->n_big;
    pf.nq = pf.n_big + a.ws.counts->n_small;
    if (threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        mbar_init(&sh.mbar_g, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int i = atomicAdd(&a.ws.counts->queue_head, 1);
        sh.next = i;
        sh.gpend = 0;
        if (i < pf.nq) {
            sh.next_b = queue_block(a, i, pf.n_big);
            mbar_arrive_expect_tx(&sh.mbar_g, (unsigned)sizeof(BlockGeom));
            bulk_g2s(&sh.geom[0], a.ws.geom + sh.next_b, (unsigned)sizeof(BlockGeom), &sh.mbar_g);
            sh.gpend = 1;
        }
    }
    __syncthreads();
    unsigned phase = 0, gphase = 0;
    unsigned long long evals = 0ull;
    int buf = 0;
    while (sh.gpend) {
        const int b = sh.next_b;
        const bool landed = mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
        gphase ^= 1u;
        if (!__syncthreads_and(landed)) break;  // (its copy landed or the wait gave up twice)
        if (threadIdx.x == 0) sh.gpend = 0;     // read by all threads before the barrier above
        pf.buf = buf ^ 1;
        if (!process_block<NT>(a, b, sm, sh, phase, buf, pf, evals)) {
            // a bounded wait expired: let a geometry copy in flight land before leaving
            __syncthreads();
            if (sh.gpend) mbar_wait_bounded(&sh.mbar_g, gphase, &a.ws.counts->error);
            break;
        }
        buf ^= 1;
    }
    if (threadIdx.x == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
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
    if (threadIdx.x == 0) mbar_init(&sh.mbar, 1);
    cp_async_wait_all();
    __syncthreads();
    unsigned phase = 0;
    unsigned long long evals = 0ull;
    Prefetch pf;
    pf.on = false;
    pf.n_big = pf.nq = 0;
    pf.buf = 1;
    process_block<NT>(a, b, sm, sh, phase, 0, pf, evals);
    if (threadIdx.x == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
}

}  // namespace

size_t match_smem_bytes(const MatchArgs &a)
{
    return sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols + sizeof(uint64_t) * kMaxPts +
           sizeof(int) * kMaxCand + 2 * sizeof(int) * kMaxPts;
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

cudaError_t match_configure_raise(const MatchArgs &a, int threads, int *ctas_per_sm)
{
    const int need = (int)match_smem_bytes(a);
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (threads == 128) {
        e = cudaFuncGetAttributes(&fa, match_persistent_kernel<128>);
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
            e = cudaFuncSetAttribute(match_persistent_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, match_persistent_kernel<128>, 128, need);
    } else {
        e = cudaFuncGetAttributes(&fa, match_persistent_kernel<256>);
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
            e = cudaFuncSetAttribute(match_persistent_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, match_persistent_kernel<256>, 256, need);
    }
    return e;
}

cudaError_t launch_match_persistent(const MatchArgs &a, int threads, int grid, cudaStream_t s)
{
    if (threads == 128)
        match_persistent_kernel<128><<<grid, 128, match_smem_bytes(a), s>>>(a);
    else
        match_persistent_kernel<256><<<grid, 256, match_smem_bytes(a), s>>>(a);
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
