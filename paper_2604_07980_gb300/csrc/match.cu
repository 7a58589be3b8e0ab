// match.cu -- the Hamming-cost search of Algorithm 2 for every planned block.
//
// One CTA takes one block end to end:
//   1. sample the block's point grid (Sec. 4.3.4); copy the left census at every
//      grid point, the block's occluders and the first forward strip into shared
//      memory with asynchronous copies issued together (one memory round trip);
//      drop points whose left census is undefined or whose full-res position
//      lies in a kept occluder (Sec. 4.3.5) and compact the survivors
//      column-major;
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
//   5. consistency |d_b - d_f| <= fb_tol, block record; the last CTA to finish a
//      box (atomic counter after a fence) aggregates its blocks with one warp
//      (Sec. 4.3.4) and writes disparity, Eq. 1 depth and flags.
// Blocks wider than the strip are split into column chunks; chunk sums add up
// because Eq. census_cost is a sum over points.
#include <math.h>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

struct Smem {
    uint64_t *strip;   // strip_rows * strip_cols
    uint64_t *praw;    // kMaxPts: left code of grid point t = 16 j + m
    uint64_t *pcode;   // kMaxPts: compacted codes (left, then right queries)
    int *cost;         // kMaxCand
    int *pmj;          // kMaxPts: (m << 8) | j
    int *pbase;        // kMaxPts: byte offset of the point's strip row + column in the chunk
};

template <int NW>
struct Shared {
    int X[kMaxPtsSide];
    int Y[kMaxPtsSide];
    int colstart[kMaxPtsSide + 1];
    int4 occ[kMaxOcc];
    int warp_cnt[NW];
    unsigned warp_min[NW];
    float agg[kMaxSlots];
    float agg_sorted[kMaxSlots];
    int d_f, dy_f, s_m, s_0, s_p;
    int d_b, dy_b;
    int last;
    int next;
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

// Sum of popcounts over the points [p0, p1) of one chunk; T candidate slices,
// any (dy, d) layout: coff[t] is the element offset of this lane's candidate t.
template <int NW, int T>
__device__ __forceinline__ void scan_chunk(const Smem &sm, int p0, int p1, const int (&coff)[8],
                                           int (&acc)[8])
{
    const int warp = threadIdx.x >> 5;
    const char *strip = reinterpret_cast<const char *>(sm.strip);
    int p = p0 + warp;
    for (; p + NW < p1; p += 2 * NW) {
        const uint64_t c0 = sm.pcode[p], c1 = sm.pcode[p + NW];
        const char *b0 = strip + sm.pbase[p], *b1 = strip + sm.pbase[p + NW];
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
        const uint32_t l1 = (uint32_t)c1, h1 = (uint32_t)(c1 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = *reinterpret_cast<const uint64_t *>(b0 + 8 * coff[t]);
            const uint64_t r1 = *reinterpret_cast<const uint64_t *>(b1 + 8 * coff[t]);
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32)) +
                      __popc(l1 ^ (uint32_t)r1) + __popc(h1 ^ (uint32_t)(r1 >> 32));
        }
    }
    if (p < p1) {
        const uint64_t c0 = sm.pcode[p];
        const char *b0 = strip + sm.pbase[p];
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = *reinterpret_cast<const uint64_t *>(b0 + 8 * coff[t]);
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32));
        }
    }
}

// Fast path for one dy row and N_d a multiple of 32: this lane's candidate t
// sits at lane_off + DIR * 32 t elements from the point's base, so every strip
// load has an immediate offset and the inner loop is one load, two xors, two
// popcounts and one add per evaluation.
template <int NW, int T, int DIR>
__device__ __forceinline__ void scan_chunk_fast(const Smem &sm, int p0, int p1, int lane_off,
                                                int (&acc)[8])
{
    const int warp = threadIdx.x >> 5;
    const char *strip = reinterpret_cast<const char *>(sm.strip) + 8 * lane_off;
    int p = p0 + warp;
    for (; p + NW < p1; p += 2 * NW) {
        const uint64_t c0 = sm.pcode[p], c1 = sm.pcode[p + NW];
        const uint64_t *b0 = reinterpret_cast<const uint64_t *>(strip + sm.pbase[p]);
        const uint64_t *b1 = reinterpret_cast<const uint64_t *>(strip + sm.pbase[p + NW]);
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
        const uint32_t l1 = (uint32_t)c1, h1 = (uint32_t)(c1 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = b0[DIR * 32 * t];
            const uint64_t r1 = b1[DIR * 32 * t];
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32)) +
                      __popc(l1 ^ (uint32_t)r1) + __popc(h1 ^ (uint32_t)(r1 >> 32));
        }
    }
    if (p < p1) {
        const uint64_t c0 = sm.pcode[p];
        const uint64_t *b0 = reinterpret_cast<const uint64_t *>(strip + sm.pbase[p]);
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = b0[DIR * 32 * t];
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32));
        }
    }
}

template <int NW>
__device__ __forceinline__ void scan_dispatch(int T, const Smem &sm, int p0, int p1,
                                              const int (&coff)[8], int (&acc)[8])
{
    switch (T) {
    case 1: scan_chunk<NW, 1>(sm, p0, p1, coff, acc); break;
    case 2: scan_chunk<NW, 2>(sm, p0, p1, coff, acc); break;
    case 3: scan_chunk<NW, 3>(sm, p0, p1, coff, acc); break;
    case 4: scan_chunk<NW, 4>(sm, p0, p1, coff, acc); break;
    case 5: scan_chunk<NW, 5>(sm, p0, p1, coff, acc); break;
    case 6: scan_chunk<NW, 6>(sm, p0, p1, coff, acc); break;
    case 7: scan_chunk<NW, 7>(sm, p0, p1, coff, acc); break;
    default: scan_chunk<NW, 8>(sm, p0, p1, coff, acc); break;
    }
}

template <int NW, int DIR>
__device__ __forceinline__ void scan_dispatch_fast(int T, const Smem &sm, int p0, int p1, int lane_off,
                                                   int (&acc)[8])
{
    switch (T) {
    case 1: scan_chunk_fast<NW, 1, DIR>(sm, p0, p1, lane_off, acc); break;
    case 2: scan_chunk_fast<NW, 2, DIR>(sm, p0, p1, lane_off, acc); break;
    case 3: scan_chunk_fast<NW, 3, DIR>(sm, p0, p1, lane_off, acc); break;
    case 4: scan_chunk_fast<NW, 4, DIR>(sm, p0, p1, lane_off, acc); break;
    case 5: scan_chunk_fast<NW, 5, DIR>(sm, p0, p1, lane_off, acc); break;
    case 6: scan_chunk_fast<NW, 6, DIR>(sm, p0, p1, lane_off, acc); break;
    case 7: scan_chunk_fast<NW, 7, DIR>(sm, p0, p1, lane_off, acc); break;
    default: scan_chunk_fast<NW, 8, DIR>(sm, p0, p1, lane_off, acc); break;
    }
}

// Byte offsets of the compacted points [p0, p1) into a strip chunk of width SWc
// whose first column is point column xj0: row m * ndy, column X_j - xj0.
template <int NT>
__device__ __forceinline__ void set_bases(const Smem &sm, const int *X, int p0, int p1, int ndy,
                                          int SWc, int xj0)
{
    for (int p = p0 + (int)threadIdx.x; p < p1; p += NT) {
        const int mj = sm.pmj[p];
        sm.pbase[p] = 8 * ((mj >> 8) * ndy * SWc + X[mj & 255] - xj0);
    }
}

// Last point column of the chunk starting at j0 whose strip fits strip_cols.
__device__ __forceinline__ int chunk_end(const int *X, int j0, int nx, int nd, int strip_cols)
{
    int j1 = j0 + 1;
    while (j1 < nx && X[j1] - X[j0] + nd <= strip_cols) ++j1;
    return j1;
}

// Issue the asynchronous copies of one strip chunk: rows (m, e) of the right
// plane at Y_m + dy_min + e (forward) or of the left plane at
// Y_m + dy_f - (dy_min + e) (backward), columns [colbase, colbase + SWc).
// Positions outside the plane are written as 0.
template <int NT>
__device__ __forceinline__ void issue_strip(const BlockCtx &bc, const Smem &sm, const int *Y, bool fwd,
                                            int dy_min, int dy_f, int colbase, int SWc)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = bc.ny * bc.ndy;
    const uint64_t *plane = fwd ? bc.CR : bc.CL;
    for (int r = warp; r < rows; r += NT / 32) {
        const int m = bc.ndy == 1 ? r : r / bc.ndy;
        const int e = r - m * bc.ndy;
        const int y = fwd ? Y[m] + dy_min + e : Y[m] + dy_f - (dy_min + e);
        uint64_t *dst = sm.strip + r * SWc;
        const bool row_ok = y >= 0 && y < bc.Hs;
        const uint64_t *src = plane + (row_ok ? (long long)y * bc.pitch : 0);
        for (int c = lane; c < SWc; c += 32) {
            const int x = colbase + c;
            if (row_ok && x >= 0 && x < bc.Ws)
                cp_async8(dst + c, src + x);
            else
                dst[c] = 0ull;
        }
    }
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

// One search pass after its first strip chunk has been issued and landed and
// the point bases of the first chunk are set.
template <int NT>
__device__ void search_pass(const MatchArgs &a, const BlockCtx &bc, const Smem &sm,
                            Shared<NT / 32> &sh, bool fwd)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int T = (bc.nc + 31) >> 5;
    const bool fast = bc.ndy == 1 && (bc.nd & 31) == 0;
    int acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0;
    const int d_f = sh.d_f, dy_f = sh.dy_f;
    int j0 = 0;
    bool first = true;
    while (j0 < bc.nx) {
        const int j1 = chunk_end(sh.X, j0, bc.nx, bc.nd, a.strip_cols);
        const int xj0 = sh.X[j0];
        const int SWc = sh.X[j1 - 1] - xj0 + bc.nd;
        const int p0 = sh.colstart[j0], p1 = sh.colstart[j1];
        if (!first) {  // later chunks: load now (the first chunk was prefetched)
            const int colbase = fwd ? xj0 - bc.dmax : xj0 - d_f + bc.dmin;
            issue_strip<NT>(bc, sm, sh.Y, fwd, a.p.dy_min, dy_f, colbase, SWc);
            set_bases<NT>(sm, sh.X, p0, p1, bc.ndy, SWc, xj0);
            cp_async_wait_all();
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
                    o = e * SWc + (fwd ? (bc.nd - 1 - c) : c);
                }
                coff[t] = o;
            }
            scan_dispatch<NW>(T, sm, p0, p1, coff, acc);
        }
        __syncthreads();
        first = false;
        j0 = j1;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int c = t * 32 + lane;
        if (t < T && c < bc.nc) atomicAdd(&sm.cost[c], acc[t]);
    }
    __syncthreads();
    argmin_pass<NT>(a, bc, sm, sh, fwd);
}

// Sec. 4.3.4 on the block records of one box, by warp 0 of the CTA that
// finished the box last.
template <int NW>
__device__ void aggregate_box(const MatchArgs &a, int box, Shared<NW> &sh)
{
    const int lane = threadIdx.x & 31;
    const BoxPlan P = a.ws.plans[box];
    const int base = a.ws.blk_base[box];
    float d[2];
    int f[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        f[h] = 0;
        d[h] = 0.0f;
        if (s < P.nblk) {
            const int2 raw = __ldcg(reinterpret_cast<const int2 *>(a.ws.blkres + base + s));
            d[h] = __int_as_float(raw.x);
            f[h] = raw.y;
        }
    }
    const unsigned full = 0xffffffffu;
    const int fb_any = __any_sync(full, ((f[0] | f[1]) & CTM_BLK_FB_REJECT) != 0);
    const int few_any = __any_sync(full, ((f[0] | f[1]) & CTM_BLK_FEW_POINTS) != 0);
    const bool v0 = (f[0] & CTM_BLK_VALID) != 0, v1 = (f[1] & CTM_BLK_VALID) != 0;
    const int clamp_any = __any_sync(full, (v0 && (f[0] & CTM_BLK_SUBPIX_CLAMPED)) ||
                                               (v1 && (f[1] & CTM_BLK_SUBPIX_CLAMPED)));
    const unsigned b0 = __ballot_sync(full, v0), b1 = __ballot_sync(full, v1);
    const unsigned lt = (1u << lane) - 1u;
    const int nv = __popc(b0) + __popc(b1);
    if (v0) sh.agg[__popc(b0 & lt)] = d[0];
    if (v1) sh.agg[__popc(b0) + __popc(b1 & lt)] = d[1];
    __syncwarp();
    // rank sort (ties by position) into agg_sorted
    for (int e = lane; e < nv; e += 32) {
        const float x = sh.agg[e];
        int rank = 0;
        for (int q = 0; q < nv; ++q) {
            const float y = sh.agg[q];
            rank += (y < x) || (y == x && q < e);
        }
        sh.agg_sorted[rank] = x;
    }
    __syncwarp();
    if (lane != 0) return;
    int fl = P.far ? CTM_BOX_FAR : 0;
    if (fb_any) fl |= CTM_BOX_FB_REJECT;
    if (few_any) fl |= CTM_BOX_FEW_POINTS;
    if (clamp_any) fl |= CTM_BOX_SUBPIX_CLAMPED;
    bool have = false;
    float d_box = 0.0f;
    const float *v = sh.agg_sorted;
    if (P.far) {
        if (nv == 1) { have = true; d_box = v[0]; }
    } else if (nv > 0) {
        // longest run with consecutive differences < tau_d; first on ties
        int best_start = 0, best_len = 1, cur_start = 0, cur_len = 1;
        for (int i = 1; i < nv; ++i) {
            if (__fsub_rn(v[i], v[i - 1]) < a.p.agg_tau_d) {
                ++cur_len;
            } else {
                cur_start = i;
                cur_len = 1;
            }
            if (cur_len > best_len) { best_len = cur_len; best_start = cur_start; }
        }
        if (best_len >= a.p.agg_nmin) {
            have = true;
            const float *run = v + best_start;
            const int m = best_len;
            if (a.p.agg_mode == 0) {
                d_box = (m & 1) ? run[m / 2] : __fmul_rn(__fadd_rn(run[m / 2 - 1], run[m / 2]), 0.5f);
            } else {
                const int t = (int)floorf(__fmul_rn(a.p.trim_frac, (float)m));
                float s = 0.0f;
                for (int i = t; i < m - t; ++i) s = __fadd_rn(s, run[i]);
                d_box = __fdiv_rn(s, (float)(m - 2 * t));
            }
        }
    }
    if (!P.far && !have) fl |= CTM_BOX_NO_SEGMENT;
    float disp = __int_as_float(0x7fc00000), dep = __int_as_float(0x7fc00000);
    if (have) {
        if (d_box > 0.0f) {
            fl |= CTM_BOX_VALID;
            disp = d_box;
            dep = __fdiv_rn(P.fb, d_box);  // Eq. 1
        } else {
            fl |= CTM_BOX_NONPOS_DISP;
        }
    }
    a.disp[box] = disp;
    a.depth[box] = dep;
    a.flags[box] = (uint8_t)fl;
}

template <int NT>
__device__ void process_block(const MatchArgs &a, int b, const Smem &sm, Shared<NT / 32> &sh)
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    const BlockRect br = block_rect(P, bs.y, a.p.pts_side);
    bc.nx = br.nx;
    bc.ny = br.ny;
    const int np_nom = bc.nx * bc.ny;

    // 1a. geometry to shared memory, occluders in flight
    if (tid < bc.nx) sh.X[tid] = point_coord(br.bx0, br.bx1, bc.nx, tid);
    if (tid < bc.ny) sh.Y[tid] = point_coord(br.by0, br.by1, bc.ny, tid);
    if (tid < P.nocc) cp_async16(&sh.occ[tid], a.ws.occ + (long long)bc.box * kMaxOcc + tid);
    for (int c = tid; c < bc.nc; c += NT) sm.cost[c] = 0;
    __syncthreads();
    // 1b. grid-point codes (point t = 16 j + m) and the first forward strip chunk
    // join the same round trip
    for (int t = tid; t < kMaxPts; t += NT) {
        const int j = t >> 4, m = t & 15;
        if (j < bc.nx && m < bc.ny) {
            const int x = sh.X[j], y = sh.Y[m];
            if (x >= 0 && x < bc.Ws && y >= 0 && y < bc.Hs)
                cp_async8(&sm.praw[t], bc.CL + (long long)y * bc.pitch + x);
            else
                sm.praw[t] = 0ull;
        }
    }
    const int j1_first = bc.nx > 0 ? chunk_end(sh.X, 0, bc.nx, bc.nd, a.strip_cols) : 0;
    const int SW0 = bc.nx > 0 ? sh.X[j1_first - 1] - sh.X[0] + bc.nd : 0;
    if (bc.nx > 0 && bc.ny > 0)
        issue_strip<NT>(bc, sm, sh.Y, true, a.p.dy_min, 0, sh.X[0] - bc.dmax, SW0);
    cp_async_wait_all();
    __syncthreads();

    // 1c. usable points, compacted column-major, with their first-chunk bases
    const int sxw = a.p.win_w >> 1, syw = a.p.win_h >> 1;
    int total = 0;
    for (int t0 = 0; t0 < kMaxPts; t0 += NT) {
        const int t = t0 + tid;
        const int j = t >> 4, m = t & 15;
        const bool grid_pt = j < bc.nx && m < bc.ny;
        bool valid = false;
        if (grid_pt) {
            const int x = sh.X[j], y = sh.Y[m];
            valid = x - sxw >= 0 && x + sxw < bc.Ws && y - syw >= 0 && y + syw < bc.Hs;
            const int fx = P.k * x, fy = P.k * y;
            for (int q = 0; q < P.nocc && valid; ++q) {
                const int4 o = sh.occ[q];
                if (fx >= o.x && fx < o.z && fy >= o.y && fy < o.w) valid = false;
            }
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) sh.warp_cnt[warp] = __popc(ballot);
        __syncthreads();
        int wpre = 0, sum = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int c = sh.warp_cnt[w];
            if (w < warp) wpre += c;
            sum += c;
        }
        const int idx = total + wpre + __popc(ballot & ((1u << lane) - 1u));
        if (valid) {
            sm.pcode[idx] = sm.praw[t];
            sm.pmj[idx] = (m << 8) | j;
            if (j < j1_first) sm.pbase[idx] = 8 * (m * bc.ndy * SW0 + sh.X[j] - sh.X[0]);
        }
        if (grid_pt && m == 0) sh.colstart[j] = idx;
        total += sum;
        __syncthreads();
    }
    if (tid == 0) sh.colstart[bc.nx] = total;
    __syncthreads();

    const int slots = a.p.grid_g * a.p.grid_g;
    ctm_block rec;
    rec.n_pts = np_nom;
    rec.n_valid = total;
    rec.d_f = rec.dy_f = rec.d_b = rec.dy_b = 0;
    rec.s_m = rec.s_0 = rec.s_p = 0;
    rec.d_sub = 0.0f;
    rec.d_full = 0.0f;
    rec.flags = CTM_BLK_PRESENT;

    if (total < a.p.min_pts) {
        rec.flags |= CTM_BLK_FEW_POINTS;
    } else {
        // 2-3. forward pass, argmin, parabola
        search_pass<NT>(a, bc, sm, sh, true);
        if (tid == 0) {
            const unsigned key = sh.warp_min[0];
            const int c = (int)(key & 0xffffu);
            const int e = c / bc.nd, di = c - e * bc.nd;
            sh.d_f = bc.dmin + di;
            sh.dy_f = a.p.dy_min + e;
            sh.s_0 = (int)(key >> 16);
            sh.s_m = di > 0 ? sm.cost[c - 1] : 0;
            sh.s_p = di < bc.nd - 1 ? sm.cost[c + 1] : 0;
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
        // chunk 0's point bases are still those of 1c: later chunks own other points
        issue_strip<NT>(bc, sm, sh.Y, false, a.p.dy_min, dy_f, sh.X[0] - d_f + bc.dmin, SW0);
        cp_async_wait_all();
        __syncthreads();
        search_pass<NT>(a, bc, sm, sh, false);
        if (tid == 0) {
            const unsigned key = sh.warp_min[0];
            const int c = (int)(key & 0xffffu);
            const int e = c / bc.nd, di = c - e * bc.nd;
            sh.d_b = bc.dmin + di;
            sh.dy_b = a.p.dy_min + e;
        }
        __syncthreads();
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
    }

    // 5. block record, completion count, the last CTA of the box aggregates
    if (tid == 0) {
        BlockResult r;
        r.d_full = rec.d_full;
        r.flags = rec.flags;
        a.ws.blkres[a.ws.blk_base[bc.box] + bc.slot] = r;
        if (a.dbg.blocks) a.dbg.blocks[(long long)bc.box * slots + bc.slot] = rec;
        if (!(rec.flags & CTM_BLK_FEW_POINTS))
            atomicAdd(&a.ws.counts->evals, 2ull * (unsigned long long)total * (unsigned long long)bc.nc);
        __threadfence();
        const int prev = atomicAdd(&a.ws.box_done[bc.box], 1);
        sh.last = (prev == P.nblk - 1);
    }
    __syncthreads();
    if (sh.last && warp == 0) {
        __threadfence();
        aggregate_box<NW>(a, bc.box, sh);
    }
    __syncthreads();
}

__device__ __forceinline__ Smem carve(const MatchArgs &a, unsigned char *raw)
{
    Smem sm;
    size_t off = 0;
    sm.strip = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols;
    sm.praw = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * kMaxPts;
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
__global__ void __launch_bounds__(NT, 1536 / NT)
    match_persistent_kernel(MatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT / 32> sh;
    const Smem sm = carve(a, smem_raw);
    const int nblocks = a.ws.counts->n_blocks;
    for (;;) {
        if (threadIdx.x == 0) sh.next = atomicAdd(&a.ws.counts->queue_head, 1);
        __syncthreads();
        const int b = sh.next;
        __syncthreads();
        if (b >= nblocks) break;
        process_block<NT>(a, b, sm, sh);
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) match_box_kernel(MatchArgs a, int box)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<NT / 32> sh;
    if ((int)blockIdx.x >= a.ws.nblk[box]) return;
    const Smem sm = carve(a, smem_raw);
    process_block<NT>(a, a.ws.blk_base[box] + blockIdx.x, sm, sh);
}

}  // namespace

size_t match_smem_bytes(const MatchArgs &a)
{
    return sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols + 2 * sizeof(uint64_t) * kMaxPts +
           sizeof(int) * kMaxCand + 2 * sizeof(int) * kMaxPts;
}

cudaError_t match_configure(const MatchArgs &a, int threads, int *ctas_per_sm)
{
    const int smem = (int)match_smem_bytes(a);
    cudaError_t e = cudaSuccess;
    if (threads == 128) {
        e = cudaFuncSetAttribute(match_persistent_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(match_box_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, match_persistent_kernel<128>, 128, smem);
    } else {
        e = cudaFuncSetAttribute(match_persistent_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(match_box_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, match_persistent_kernel<256>, 256, smem);
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
