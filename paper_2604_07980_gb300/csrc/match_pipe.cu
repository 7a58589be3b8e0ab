// match_pipe.cu -- the two-pass pipelined matcher.
//
// The fused kernel (match.cu) waits twice per block: for the point codes and
// forward strip, then -- after the forward argmin -- for the matched right
// codes and the backward strip.  Here the passes are split into two kernels
// over the same queue of searchable blocks:
//   match_fwd_kernel: Eq. census_cost for every candidate (forward), the first
//     argmin and the costs around it, stored in the block's sampling record;
//   match_bwd_kernel: the backward search of Sec. 4.3.3 from the stored d_f,
//     the consistency test and Eq. subpixel, then the block record.
// Within a pass the blocks of a CTA do not depend on one another, so each CTA
// keeps two data buffers: while it scans block k from one, the point codes and
// first strip chunk of block k+1 are already on their way into the other, and
// the sampling record of block k+2 into a third record buffer.  Blocks are
// assigned to CTAs round robin over the queue (large work first), so every CTA
// gets a similar mix.  Results equal the fused kernel's: the same sums in the
// same candidate order, the same argmin and the same fp32 parabola.
#include <math.h>

#include "aggregate.cuh"
#include "ctm_internal.cuh"
#include "match_common.cuh"

namespace ctm {
namespace {

constexpr int kGeomBufs = 3;

// The block held by one data buffer, as every thread of the CTA needs it.
struct Stage {
    const uint64_t *CL, *CR;
    long long pitch;
    int b, nd, ndy, nc, dmin, dmax, Ws, Hs;
    int nx, ny, total, j1_first, x0, SW0;
    int d_f, dy_f;   // backward pass: the forward result
    int gbuf;        // record buffer holding the block's sampling record
    ChunkGeom g0;    // first strip chunk of this pass
};

template <int NW>
struct PipeShared {
    BlockGeom geom[kGeomBufs];   // sampling records of blocks k, k+1, k+2
    uint64_t mbar_g[kGeomBufs];  // record copies
    uint64_t mbar_d[2];          // strip copies of the two data buffers
    Stage st[2];
    unsigned warp_min[NW];
    int pend_g[kGeomBufs];       // a record copy is in flight
    int pend_d[2];               // a strip copy is in flight
};

// Shared-memory views of the two data buffers (Smem of match_common.cuh).
__device__ __forceinline__ void carve_pipe(const MatchArgs &a, unsigned char *raw, Smem (&sm)[2])
{
    size_t off = 0;
    const size_t strip = sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols;
    int *cost = nullptr;
    for (int i = 0; i < 2; ++i) {
        sm[i].cost_b = nullptr;  // one cost row per pass kernel
        sm[i].strip = reinterpret_cast<uint64_t *>(raw + off);
        off += strip;
    }
    for (int i = 0; i < 2; ++i) {
        sm[i].pcode = reinterpret_cast<uint64_t *>(raw + off);
        off += sizeof(uint64_t) * kMaxPts;
    }
    cost = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxCand;
    for (int i = 0; i < 2; ++i) {
        sm[i].pmj = reinterpret_cast<int *>(raw + off);
        off += sizeof(int) * kMaxPts;
        sm[i].pbase = reinterpret_cast<int *>(raw + off);
        off += sizeof(int) * kMaxPts;
        sm[i].cost = cost;
    }
}

// Thread 0: start the copy of block b's sampling record into record buffer gb.
template <int NW>
__device__ __forceinline__ void issue_record(const MatchArgs &a, PipeShared<NW> &sh, int gb, int b)
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_arrive_expect_tx(&sh.mbar_g[gb], (unsigned)sizeof(BlockGeom));
    bulk_g2s(&sh.geom[gb], a.ws.geom + b, (unsigned)sizeof(BlockGeom), &sh.mbar_g[gb]);
    sh.pend_g[gb] = 1;
}

// Row (m, e) of a strip: the right plane at Y_m + dy_min + e (forward) or the
// left plane at Y_m + dy_f - (dy_min + e) (backward).
__device__ __forceinline__ int strip_row_y(const MatchArgs &a, const BlockGeom &g, const Stage &st, bool fwd,
                                           int r)
{
    const int m = st.ndy == 1 ? r : r / st.ndy;
    const int e = r - m * st.ndy;
    return fwd ? g.Y[m] + a.p.dy_min + e : g.Y[m] + st.dy_f - (a.p.dy_min + e);
}

// Warp 0: issue the bulk copies of one strip chunk into sm.strip (completion on
// mbar); the caller waits and zero-fills.
__device__ __forceinline__ void issue_strip(const MatchArgs &a, const BlockGeom &g, const Stage &st,
                                            const Smem &sm, uint64_t *mbar, bool fwd, const ChunkGeom &cg)
{
    const int lane = threadIdx.x & 31;
    const int rows = st.ny * st.ndy;
    const uint64_t *plane = fwd ? st.CR : st.CL;
    const int Ws_even = (st.Ws + 1) & ~1;  // the padding column after an odd width is readable
    const int x_lo = max(cg.colbase_a, 0);
    const int x_hi = min(cg.colbase_a + cg.SWa, Ws_even);
    const unsigned row_bytes = x_hi > x_lo ? 8u * (unsigned)(x_hi - x_lo) : 0u;
    unsigned total = 0;
    for (int r = lane; r < rows; r += 32) {
        const int y = strip_row_y(a, g, st, fwd, r);
        if (y >= 0 && y < st.Hs) total += row_bytes;
    }
    total = __reduce_add_sync(0xffffffffu, total);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(mbar, total);
    __syncwarp();
    if (row_bytes > 0) {
        for (int r = lane; r < rows; r += 32) {
            const int y = strip_row_y(a, g, st, fwd, r);
            if (y >= 0 && y < st.Hs)
                bulk_g2s(sm.strip + r * cg.SWa + (x_lo - cg.colbase_a), plane + (long long)y * st.pitch + x_lo,
                         row_bytes, mbar);
        }
    }
}

// After a strip chunk has landed: zero what lies outside the plane (whole rows
// outside it; columns < 0 or >= Ws), a warp per row.  Only edge chunks have any.
template <int NT>
__device__ __forceinline__ void zero_fill(const MatchArgs &a, const BlockGeom &g, const Stage &st,
                                          const Smem &sm, bool fwd, const ChunkGeom &cg)
{
    const int rows = st.ny * st.ndy;
    const bool edge = cg.colbase_a < 0 || cg.colbase_a + cg.SWa > st.Ws ||
                      g.Y[0] + (fwd ? a.p.dy_min : st.dy_f - a.p.dy_max) < 0 ||
                      g.Y[st.ny - 1] + (fwd ? a.p.dy_max : st.dy_f - a.p.dy_min) >= st.Hs;
    if (!edge) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c_lo = min(max(-cg.colbase_a, 0), cg.SWa);             // [0, c_lo): x < 0
    const int c_hi = max(min(st.Ws - cg.colbase_a, cg.SWa), c_lo);   // [c_hi, SWa): x >= Ws
    for (int r = warp; r < rows; r += NT / 32) {
        const int y = strip_row_y(a, g, st, fwd, r);
        uint64_t *row = sm.strip + r * cg.SWa;
        if (y < 0 || y >= st.Hs) {
            for (int c = lane; c < cg.SWa; c += 32) row[c] = 0ull;
        } else {
            for (int c = lane; c < c_lo; c += 32) row[c] = 0ull;
            for (int c = c_hi + lane; c < cg.SWa; c += 32) row[c] = 0ull;
        }
    }
}

// Everything about block b and this pass that follows from its sampling record.
__device__ __forceinline__ Stage make_stage(const MatchArgs &a, const BlockGeom &g, int b, int gbuf, bool fwd)
{
    Stage st;
    st.b = b;
    st.gbuf = gbuf;
    st.dmin = g.dmin;
    st.dmax = g.dmax;
    st.nd = g.dmax - g.dmin + 1;
    st.ndy = a.p.dy_max - a.p.dy_min + 1;
    st.nc = st.nd * st.ndy;
    st.Ws = g.Ws;
    st.Hs = g.Hs;
    st.nx = g.nx;
    st.ny = g.ny;
    st.total = g.n_valid;
    const bool full = g.far || a.p.close_factor == 1;
    const uint64_t *base = a.ws.census + (long long)g.frame * a.ws.frame_stride;
    st.CL = full ? base : base + 2 * a.ws.plane1_elems;
    st.CR = full ? base + a.ws.plane1_elems : base + 2 * a.ws.plane1_elems + a.ws.planek_elems;
    st.pitch = full ? a.ws.pitch1 : a.ws.pitchk;
    const unsigned later0 = g.cstart & ~1u;
    st.j1_first = later0 ? __ffs(later0) - 1 : st.nx;
    st.x0 = g.X[0];
    st.SW0 = g.X[st.j1_first - 1] - st.x0 + st.nd;
    st.d_f = fwd ? 0 : g.d_f;
    st.dy_f = fwd ? 0 : g.dy_f;
    st.g0 = chunk_geom(fwd ? st.x0 - st.dmax : st.x0 - st.d_f + st.dmin, st.SW0);
    return st;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// All threads: wait for block b's record in record buffer gb, then start its
// data into data buffer `buf`: the compacted point codes (left codes at the
// points forward; right codes at the matched positions backward) by cp.async,
// the point layout, and the first strip chunk by bulk copies (warp 0).
template <int NT, bool FWD>
__device__ __forceinline__ bool issue_block(const MatchArgs &a, PipeShared<NT / 32> &sh, const Smem &sm, int buf,
                                            int gb, int b, unsigned &par_g)
{
    const int tid = threadIdx.x;
    // (a phase is only counted as consumed when its wait succeeded, so that the
    // drain after a failed wait waits for that same phase)
    const bool ok = mbar_wait_bounded(&sh.mbar_g[gb], (par_g >> gb) & 1u, &a.ws.counts->error);
    if (ok) par_g ^= 1u << gb;
    const BlockGeom &g = sh.geom[gb];
    const Stage st = make_stage(a, g, b, gb, FWD);
    if (tid == 0) {
        sh.st[buf] = st;
        sh.pend_g[gb] = 0;
        sh.pend_d[buf] = 1;
    }
    for (int t = tid; t < kMaxPts; t += NT) {
        const int j = t >> 4, m = t & 15;
        if (j < st.nx && ((g.colmask[j] >> m) & 1u)) {
            const int idx = g.colprefix[j] + __popc(g.colmask[j] & ((1u << m) - 1u));
            const int x = g.X[j], y = g.Y[m];
            if (FWD) {
                cp_async8(&sm.pcode[idx], st.CL + (long long)y * st.pitch + x);
            } else {
                const int qx = x - st.d_f, qy = y + st.dy_f;
                if (qx >= 0 && qx < st.Ws && qy >= 0 && qy < st.Hs)
                    cp_async8(&sm.pcode[idx], st.CR + (long long)qy * st.pitch + qx);
                else
                    sm.pcode[idx] = 0ull;
            }
            sm.pmj[idx] = (m << 8) | j;
            if (j < st.j1_first) sm.pbase[idx] = 8 * (m * st.ndy * st.g0.SWa + x - st.x0 + st.g0.delta);
        }
    }
    if ((tid >> 5) == 0) issue_strip(a, g, st, sm, &sh.mbar_d[buf], FWD, st.g0);
    return ok;
}

// One pass of the block in data buffer `buf` after its first chunk has landed
// (and been zero-filled): all chunks, the cross-warp sums and the first argmin
// (key in sh.warp_min[0]; costs in sm.cost).  Later chunks are loaded into the
// same buffer.  Returns false if a bounded wait expired.
template <int NT, bool FWD>
__device__ bool scan_pass(const MatchArgs &a, PipeShared<NT / 32> &sh, const Smem &sm, const Stage &st,
                          const BlockGeom &g, int buf, unsigned &par_d)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = (st.nc + 31) >> 5;
    const bool fast = st.ndy == 1 && (st.nd & 31) == 0;
    int acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0;
    const unsigned cs = g.cstart;
    ChunkGeom cg = st.g0;
    bool ok = true;
    int j0 = 0;
    while (j0 < st.nx) {
        const unsigned later = cs & ~((2u << j0) - 1u);
        const int j1 = later ? __ffs(later) - 1 : st.nx;
        const int xj0 = g.X[j0];
        const int p0 = g.colprefix[j0];
        const int p1 = j1 < st.nx ? (int)g.colprefix[j1] : st.total;
        if (j0 > 0) {  // later chunks: into the same buffer, after the previous chunk's scan
            const int SWc = g.X[j1 - 1] - xj0 + st.nd;
            cg = chunk_geom(FWD ? xj0 - st.dmax : xj0 - st.d_f + st.dmin, SWc);
            if (warp == 0) issue_strip(a, g, st, sm, &sh.mbar_d[buf], FWD, cg);
            if (tid == 0) sh.pend_d[buf] = 1;
            for (int p = p0 + tid; p < p1; p += NT) {
                const int mj = sm.pmj[p];
                sm.pbase[p] = 8 * ((mj >> 8) * st.ndy * cg.SWa + g.X[mj & 255] - xj0 + cg.delta);
            }
            const bool landed = mbar_wait_bounded(&sh.mbar_d[buf], (par_d >> buf) & 1u, &a.ws.counts->error);
            if (landed) par_d ^= 1u << buf;
            ok = landed && ok;
            zero_fill<NT>(a, g, st, sm, FWD, cg);
            if (__syncthreads_and(landed) && tid == 0) sh.pend_d[buf] = 0;
        }
        if (fast) {
            if (FWD)
                scan_dispatch_fast<NW, -1>(T, sm, p0, p1, st.nd - 1 - lane, acc);
            else
                scan_dispatch_fast<NW, 1>(T, sm, p0, p1, lane, acc);
        } else {
            int coff[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int c = t * 32 + lane;
                int o = 0;
                if (c < st.nc) {
                    int e = 0;
                    while (c >= st.nd) { c -= st.nd; ++e; }
                    o = e * cg.SWa + (FWD ? (st.nd - 1 - c) : c);
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
        if (t < T && c < st.nc) atomicAdd(&sm.cost[c], acc[t]);
    }
    __syncthreads();
    // first argmin over (dy, d): keys (cost << 16 | c)
    unsigned key = 0xffffffffu;
    int32_t *dbgc = FWD ? a.dbg.cost_f : a.dbg.cost_b;
    const int slots = a.p.grid_g * a.p.grid_g;
    for (int c = tid; c < st.nc; c += NT) {
        const int s = sm.cost[c];
        key = min(key, ((unsigned)s << 16) | (unsigned)c);
        if (dbgc) dbgc[((long long)g.box * slots + g.slot) * a.nc_stride + c] = s;
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
    return ok;
}

// Thread 0, forward pass: the first argmin, the costs around it and the
// evaluation count; the result goes into the block's sampling record for the
// backward kernel.
__device__ __forceinline__ void forward_epilogue(const MatchArgs &a, const Smem &sm, const Stage &st,
                                                 unsigned key, unsigned long long &evals)
{
    const int c = (int)(key & 0xffffu);
    const int e = c / st.nd, di = c - e * st.nd;
    BlockGeom *g = a.ws.geom + st.b;
    g->d_f = st.dmin + di;
    g->dy_f = a.p.dy_min + e;
    g->s_0 = (int)(key >> 16);
    g->s_m = di > 0 ? sm.cost[c - 1] : 0;
    g->s_p = di < st.nd - 1 ? sm.cost[c + 1] : 0;
    evals += 2ull * (unsigned long long)st.total * (unsigned long long)st.nc;
}

// Thread 0, backward pass: d_b, the consistency test (Sec. 4.3.3), Eq. subpixel
// and the block record.
__device__ __forceinline__ void backward_epilogue(const MatchArgs &a, const BlockGeom &g, const Stage &st,
                                                  unsigned key)
{
    const int c = (int)(key & 0xffffu);
    const int e = c / st.nd;
    ctm_block rec;
    rec.n_pts = st.nx * st.ny;
    rec.n_valid = st.total;
    rec.flags = CTM_BLK_PRESENT;
    rec.d_f = g.d_f;
    rec.dy_f = g.dy_f;
    rec.d_b = st.dmin + (c - e * st.nd);
    rec.dy_b = a.p.dy_min + e;
    rec.s_m = g.s_m;
    rec.s_0 = g.s_0;
    rec.s_p = g.s_p;
    if (rec.d_f == st.dmin || rec.d_f == st.dmax) {
        rec.d_sub = (float)rec.d_f;
        rec.flags |= CTM_BLK_SUBPIX_CLAMPED;
    } else {
        // Eq. subpixel
        const float num = (float)(rec.s_p - rec.s_m);
        const float den = __fmul_rn(2.0f, (float)(rec.s_p + rec.s_m - 2 * rec.s_0));
        rec.d_sub = den == 0.0f ? (float)rec.d_f : __fsub_rn((float)rec.d_f, __fdiv_rn(num, den));
    }
    rec.d_full = __fmul_rn(rec.d_sub, (float)g.k);
    rec.flags |= abs(rec.d_b - rec.d_f) <= a.p.fb_tol ? CTM_BLK_VALID : CTM_BLK_FB_REJECT;
    write_block(a, g.box, g.slot, rec);
}

// One pass over this CTA's share of the queue (entries blockIdx.x + k * gridDim.x).
template <int NT, bool FWD>
__global__ void __launch_bounds__(NT, 512 / NT) match_pass_kernel(MatchArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ PipeShared<NT / 32> sh;
    Smem sm[2];
    carve_pipe(a, smem_raw, sm);
    const int tid = threadIdx.x;
    const int n_big = a.ws.counts->n_big;
    const int nq = n_big + a.ws.counts->n_small;
    const int G = gridDim.x;
    auto qblock = [&](int k) -> int {
        const long long i = (long long)blockIdx.x + (long long)k * G;
        return i < nq ? queue_at(a, n_big, (int)i) : -1;
    };
    const int b0 = qblock(0);
    if (b0 < 0) return;
    const int b1 = qblock(1);
    if (tid == 0) {
        for (int i = 0; i < kGeomBufs; ++i) {
            mbar_init(&sh.mbar_g[i], 1);
            sh.pend_g[i] = 0;
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sh.mbar_d[i], 1);
            sh.pend_d[i] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        issue_record(a, sh, 0, b0);
        if (b1 >= 0) issue_record(a, sh, 1, b1);
    }
    __syncthreads();
    unsigned par_g = 0u, par_d = 0u;
    unsigned long long evals = 0ull;
    bool ok = issue_block<NT, FWD>(a, sh, sm[0], 0, 0, b0, par_g);
    cp_async_commit();
    for (int k = 0;; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        const int b_next = k == 0 ? b1 : qblock(k + 1);
        const int b_next2 = qblock(k + 2);
        // the record of block k+2 (its buffer held block k-1's record)
        if (tid == 0 && b_next2 >= 0) issue_record(a, sh, (k + 2) % kGeomBufs, b_next2);
        // the data of block k+1 (its buffer held block k-1's data)
        if (b_next >= 0) ok = issue_block<NT, FWD>(a, sh, sm[nxt], nxt, (k + 1) % kGeomBufs, b_next, par_g) && ok;
        cp_async_commit();
        // block k: its codes (all but the newest cp.async group) and first strip chunk
        cp_async_wait_prev();
        const bool landed = mbar_wait_bounded(&sh.mbar_d[cur], (par_d >> cur) & 1u, &a.ws.counts->error);
        if (landed) par_d ^= 1u << cur;
        ok = landed && ok;
        if (!__syncthreads_and(ok)) break;  // also publishes sh.st[cur], written by thread 0
        const Stage st = sh.st[cur];
        if (tid == 0) sh.pend_d[cur] = 0;
        for (int c = tid; c < st.nc; c += NT) sm[cur].cost[c] = 0;
        const BlockGeom &g = sh.geom[st.gbuf];
        zero_fill<NT>(a, g, st, sm[cur], FWD, st.g0);
        __syncthreads();
        ok = scan_pass<NT, FWD>(a, sh, sm[cur], st, g, cur, par_d);
        if (!__syncthreads_and(ok)) break;
        if (tid == 0) {
            if (FWD)
                forward_epilogue(a, sm[cur], st, sh.warp_min[0], evals);
            else
                backward_epilogue(a, g, st, sh.warp_min[0]);
        }
        __syncthreads();
        if (b_next < 0) break;
    }
    if (!ok) {
        // a bounded wait expired: let every copy still in flight land before leaving
        cp_async_wait_all();
        __syncthreads();
        for (int i = 0; i < 2; ++i)
            if (sh.pend_d[i]) mbar_wait_bounded(&sh.mbar_d[i], (par_d >> i) & 1u, &a.ws.counts->error);
        for (int i = 0; i < kGeomBufs; ++i)
            if (sh.pend_g[i]) mbar_wait_bounded(&sh.mbar_g[i], (par_g >> i) & 1u, &a.ws.counts->error);
    }
    if (tid == 0 && evals) atomicAdd(&a.ws.counts->evals, evals);
}

}  // namespace

size_t match_pipe_smem_bytes(const MatchArgs &a)
{
    return 2 * sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols + 2 * sizeof(uint64_t) * kMaxPts +
           sizeof(int) * kMaxCand + 4 * sizeof(int) * kMaxPts;
}

template <int NT>
static cudaError_t configure_one(int need, int *ctas)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, match_pass_kernel<NT, true>);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
        e = cudaFuncSetAttribute(match_pass_kernel<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, match_pass_kernel<NT, false>);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < need)
        e = cudaFuncSetAttribute(match_pass_kernel<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    int c1 = 0, c2 = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c1, match_pass_kernel<NT, true>, NT, need);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c2, match_pass_kernel<NT, false>, NT, need);
    *ctas = c1 < c2 ? c1 : c2;
    return e;
}

// Raises (never lowers) the kernels' dynamic shared-memory limit, as
// match_configure does, and returns the resident CTAs per SM.
cudaError_t match_pipe_configure(const MatchArgs &a, int threads, int *ctas_per_sm)
{
    const int need = (int)match_pipe_smem_bytes(a);
    return threads == 128 ? configure_one<128>(need, ctas_per_sm) : configure_one<256>(need, ctas_per_sm);
}

cudaError_t launch_match_pipe(const MatchArgs &a, int threads, int grid, cudaStream_t s)
{
    const size_t smem = match_pipe_smem_bytes(a);
    if (threads == 128) {
        match_pass_kernel<128, true><<<grid, 128, smem, s>>>(a);
        match_pass_kernel<128, false><<<grid, 128, smem, s>>>(a);
    } else {
        match_pass_kernel<256, true><<<grid, 256, smem, s>>>(a);
        match_pass_kernel<256, false><<<grid, 256, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace ctm
