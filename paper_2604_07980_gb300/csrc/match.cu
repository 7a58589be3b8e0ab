// match.cu -- the Hamming-cost search of Algorithm 2 for every planned block.
//
// One CTA (256 threads) takes one block end to end:
//   1. sample the block's point grid (Sec. 4.3.4), drop points whose left census
//      is undefined or whose full-res position lies in a kept occluder
//      (Sec. 4.3.5), and compact the survivors column-major in shared memory;
//   2. forward pass: stage the right-image census strip the block can reach
//      (sampled rows x [x - dmax, x - dmin]) in shared memory and evaluate
//      Eq. census_cost, S(dy, d) = sum_p popc(C_L(p) ^ C_R(p.x - d, p.y + dy)),
//      for every candidate: lanes own consecutive candidates, warps own point
//      subsets, each thread keeps up to 8 candidate sums in registers;
//   3. first argmin over (dy, d) by warp min-reductions of (cost << 16 | index)
//      keys, then Eq. subpixel in fp32 with IEEE division;
//   4. backward pass (Sec. 4.3.3): queries are the right codes at the matched
//      positions, the strip is the left census at [q.x + dmin, q.x + dmax];
//   5. consistency |d_b - d_f| <= fb_tol, block record, and the last CTA to
//      finish a box (atomic counter after a fence) aggregates its blocks
//      (Sec. 4.3.4) and writes disparity, Eq. 1 depth and flags.
// Wide blocks are split into column chunks whose strip fits; chunk sums add up
// because Eq. census_cost is a sum over points.
#include <math.h>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

__device__ __forceinline__ int point_coord(int b0, int b1, int n, int j)
{
    return b0 + ((2 * j + 1) * (b1 - b0)) / (2 * n);
}

struct Smem {
    uint64_t *strip;   // strip_rows * strip_cols
    uint64_t *pcode;   // kMaxPts (left codes, later right query codes)
    int *partial;      // kMatchWarps * kMaxCand
    int *cost;         // kMaxCand
    int *pmj;          // kMaxPts: (m << 8) | j
};

struct BlockCtx {
    int box, slot, b;
    int g, k, far;
    int dmin, dmax, nd, ndy, nc;
    int nx, ny, Ws, Hs;
    long long pitch;
    const uint64_t *CL;
    const uint64_t *CR;
};

struct Shared {
    int X[kMaxPtsSide];
    int Y[kMaxPtsSide];
    int colstart[kMaxPtsSide + 1];
    int4 occ[kMaxOcc];
    int warp_cnt[kMatchWarps];
    unsigned warp_min[kMatchWarps];
    int n_valid;
    int d_f, dy_f, s_m, s_0, s_p;
    int d_b, dy_b;
    int last;
    int next;
};

// Sum of popcounts over the points of one chunk; T candidate slices per thread.
template <int T>
__device__ __forceinline__ void scan_chunk(const Smem &sm, const Shared &sh, int p0, int p1,
                                           int ndy, int SWc, int xj0, const int (&coff)[8],
                                           int (&acc)[8])
{
    const int warp = threadIdx.x >> 5;
    int p = p0 + warp;
    for (; p + kMatchWarps < p1; p += 2 * kMatchWarps) {
        const uint64_t c0 = sm.pcode[p], c1 = sm.pcode[p + kMatchWarps];
        const int mj0 = sm.pmj[p], mj1 = sm.pmj[p + kMatchWarps];
        const int base0 = (mj0 >> 8) * ndy * SWc + sh.X[mj0 & 255] - xj0;
        const int base1 = (mj1 >> 8) * ndy * SWc + sh.X[mj1 & 255] - xj0;
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
        const uint32_t l1 = (uint32_t)c1, h1 = (uint32_t)(c1 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = sm.strip[base0 + coff[t]];
            const uint64_t r1 = sm.strip[base1 + coff[t]];
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32)) +
                      __popc(l1 ^ (uint32_t)r1) + __popc(h1 ^ (uint32_t)(r1 >> 32));
        }
    }
    if (p < p1) {
        const uint64_t c0 = sm.pcode[p];
        const int mj0 = sm.pmj[p];
        const int base0 = (mj0 >> 8) * ndy * SWc + sh.X[mj0 & 255] - xj0;
        const uint32_t l0 = (uint32_t)c0, h0 = (uint32_t)(c0 >> 32);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint64_t r0 = sm.strip[base0 + coff[t]];
            acc[t] += __popc(l0 ^ (uint32_t)r0) + __popc(h0 ^ (uint32_t)(r0 >> 32));
        }
    }
}

__device__ __forceinline__ void scan_dispatch(int T, const Smem &sm, const Shared &sh, int p0,
                                              int p1, int ndy, int SWc, int xj0,
                                              const int (&coff)[8], int (&acc)[8])
{
    switch (T) {
    case 1: scan_chunk<1>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 2: scan_chunk<2>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 3: scan_chunk<3>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 4: scan_chunk<4>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 5: scan_chunk<5>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 6: scan_chunk<6>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    case 7: scan_chunk<7>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    default: scan_chunk<8>(sm, sh, p0, p1, ndy, SWc, xj0, coff, acc); break;
    }
}

// One search pass; fwd = true: right strip, candidates d in [dmin, dmax] at
// x - d, y + dy.  fwd = false: left strip around the forward match,
// candidates at q.x + d', q.y - dy'.  Leaves cost[c] in shared memory and
// returns the winning key (cost << 16 | c) in sh.warp_min[0].
__device__ void search_pass(const MatchArgs &a, const BlockCtx &bc, const Smem &sm, Shared &sh,
                            bool fwd)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = (bc.nc + 31) >> 5;
    int acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0;
    const uint64_t *plane = fwd ? bc.CR : bc.CL;
    const int d_f = sh.d_f, dy_f = sh.dy_f;
    const int dy_min = a.p.dy_min;

    int j0 = 0;
    while (j0 < bc.nx) {
        int j1 = j0 + 1;
        while (j1 < bc.nx && sh.X[j1] - sh.X[j0] + bc.nd <= a.strip_cols) ++j1;
        const int xj0 = sh.X[j0];
        const int SWc = sh.X[j1 - 1] - xj0 + bc.nd;
        const int rows = bc.ny * bc.ndy;
        const int colbase = fwd ? xj0 - bc.dmax : xj0 - d_f + bc.dmin;
        const int total = rows * SWc;
        for (int idx = tid; idx < total; idx += kMatchThreads) {
            const int r = idx / SWc;
            const int c = idx - r * SWc;
            const int m = r / bc.ndy;
            const int e = r - m * bc.ndy;
            const int y = fwd ? sh.Y[m] + dy_min + e : sh.Y[m] + dy_f - (dy_min + e);
            const int x = colbase + c;
            uint64_t v = 0;
            if (x >= 0 && x < bc.Ws && y >= 0 && y < bc.Hs) v = plane[(long long)y * bc.pitch + x];
            sm.strip[idx] = v;
        }
        __syncthreads();
        int coff[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int c = t * 32 + lane;
            int o = 0;
            if (c < bc.nc) {
                const int e = c / bc.nd;
                const int di = c - e * bc.nd;
                o = e * SWc + (fwd ? (bc.nd - 1 - di) : di);
            }
            coff[t] = o;
        }
        scan_dispatch(T, sm, sh, sh.colstart[j0], sh.colstart[j1], bc.ndy, SWc, xj0, coff, acc);
        __syncthreads();
        j0 = j1;
    }

#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int c = t * 32 + lane;
        if (t < T && c < bc.nc) sm.partial[warp * kMaxCand + c] = acc[t];
    }
    __syncthreads();
    unsigned key = 0xffffffffu;
    if (tid < bc.nc) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kMatchWarps; ++w) s += sm.partial[w * kMaxCand + tid];
        sm.cost[tid] = s;
        key = ((unsigned)s << 16) | (unsigned)tid;
        int32_t *dbgc = fwd ? a.dbg.cost_f : a.dbg.cost_b;
        if (dbgc) {
            const int slots = a.p.grid_g * a.p.grid_g;
            dbgc[((long long)bc.box * slots + bc.slot) * a.nc_stride + tid] = s;
        }
    }
    key = __reduce_min_sync(0xffffffffu, key);
    if (lane == 0) sh.warp_min[warp] = key;
    __syncthreads();
    if (tid == 0) {
        unsigned m = sh.warp_min[0];
#pragma unroll
        for (int w = 1; w < kMatchWarps; ++w) m = min(m, sh.warp_min[w]);
        sh.warp_min[0] = m;
    }
    __syncthreads();
}

__device__ void aggregate_box(const MatchArgs &a, int box)
{
    const BoxPlan P = a.ws.plans[box];
    const int base = a.ws.blk_base[box];
    float v[kMaxSlots];
    int nv = 0;
    int fb_any = 0, few_any = 0, clamp_any = 0;
    for (int s = 0; s < P.nblk; ++s) {
        const int2 raw = __ldcg(reinterpret_cast<const int2 *>(a.ws.blkres + base + s));
        const float d = __int_as_float(raw.x);
        const int f = raw.y;
        if (f & CTM_BLK_FB_REJECT) fb_any = 1;
        if (f & CTM_BLK_FEW_POINTS) few_any = 1;
        if (f & CTM_BLK_VALID) {
            if (f & CTM_BLK_SUBPIX_CLAMPED) clamp_any = 1;
            v[nv++] = d;
        }
    }
    int fl = P.far ? CTM_BOX_FAR : 0;
    if (fb_any) fl |= CTM_BOX_FB_REJECT;
    if (few_any) fl |= CTM_BOX_FEW_POINTS;
    if (clamp_any) fl |= CTM_BOX_SUBPIX_CLAMPED;
    bool have = false;
    float d_box = 0.0f;
    if (P.far) {
        if (nv == 1) { have = true; d_box = v[0]; }
    } else if (nv > 0) {
        // Sec. 4.3.4: sort, longest run with consecutive differences < tau_d
        for (int i = 1; i < nv; ++i) {
            const float t = v[i];
            int j = i - 1;
            while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
            v[j + 1] = t;
        }
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

__device__ void process_block(const MatchArgs &a, int b, const Smem &sm, Shared &sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int2 bs = a.ws.blocks[b];
    const BoxPlan P = a.ws.plans[bs.x];
    BlockCtx bc;
    bc.box = bs.x;
    bc.slot = bs.y;
    bc.b = b;
    bc.g = P.g;
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
    const int ga = bs.y % P.g, gb = bs.y / P.g;
    const int bw = P.sx1 - P.sx0, bh = P.sy1 - P.sy0;
    const int bx0 = P.sx0 + (ga * bw) / P.g, bx1 = P.sx0 + ((ga + 1) * bw) / P.g;
    const int by0 = P.sy0 + (gb * bh) / P.g, by1 = P.sy0 + ((gb + 1) * bh) / P.g;
    bc.nx = min(bx1 - bx0, a.p.pts_side);
    bc.ny = min(by1 - by0, a.p.pts_side);
    if (tid < bc.nx) sh.X[tid] = point_coord(bx0, bx1, bc.nx, tid);
    if (tid < bc.ny) sh.Y[tid] = point_coord(by0, by1, bc.ny, tid);
    if (tid < P.nocc) sh.occ[tid] = a.ws.occ[(long long)bc.box * kMaxOcc + tid];
    __syncthreads();

    // 1. usable points, compacted column-major (index = j * ny + m)
    const int np_nom = bc.nx * bc.ny;
    const int sxw = a.p.win_w >> 1, syw = a.p.win_h >> 1;
    bool valid = false;
    int m = 0, j = 0, x = 0, y = 0;
    if (tid < np_nom) {
        j = tid / bc.ny;
        m = tid - j * bc.ny;
        x = sh.X[j];
        y = sh.Y[m];
        valid = x - sxw >= 0 && x + sxw < bc.Ws && y - syw >= 0 && y + syw < bc.Hs;
        const int fx = P.k * x, fy = P.k * y;
        for (int t = 0; t < P.nocc && valid; ++t) {
            const int4 o = sh.occ[t];
            if (fx >= o.x && fx < o.z && fy >= o.y && fy < o.w) valid = false;
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) sh.warp_cnt[warp] = __popc(ballot);
    __syncthreads();
    int wpre = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kMatchWarps; ++w) {
        const int c = sh.warp_cnt[w];
        if (w < warp) wpre += c;
        total += c;
    }
    const int idx = wpre + __popc(ballot & ((1u << lane) - 1u));
    if (valid) {
        sm.pcode[idx] = bc.CL[(long long)y * bc.pitch + x];
        sm.pmj[idx] = (m << 8) | j;
    }
    if (tid < np_nom && m == 0) sh.colstart[j] = idx;
    if (tid == 0) {
        sh.colstart[bc.nx] = total;
        sh.n_valid = total;
    }
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
        search_pass(a, bc, sm, sh, true);
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
        // 4. backward pass: query codes are the right codes at the matched positions
        for (int t = tid; t < total; t += kMatchThreads) {
            const int mj = sm.pmj[t];
            const int qx = sh.X[mj & 255] - sh.d_f, qy = sh.Y[mj >> 8] + sh.dy_f;
            uint64_t v = 0;
            if (qx >= 0 && qx < bc.Ws && qy >= 0 && qy < bc.Hs) v = bc.CR[(long long)qy * bc.pitch + qx];
            sm.pcode[t] = v;
        }
        __syncthreads();
        search_pass(a, bc, sm, sh, false);
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

    // 5. block record, completion count, last CTA aggregates the box
    if (tid == 0) {
        BlockResult br;
        br.d_full = rec.d_full;
        br.flags = rec.flags;
        a.ws.blkres[b] = br;
        if (a.dbg.blocks) a.dbg.blocks[(long long)bc.box * slots + bc.slot] = rec;
        if (!(rec.flags & CTM_BLK_FEW_POINTS))
            atomicAdd(&a.ws.counts->evals, 2ull * (unsigned long long)total * (unsigned long long)bc.nc);
        __threadfence();
        const int prev = atomicAdd(&a.ws.box_done[bc.box], 1);
        sh.last = (prev == P.nblk - 1);
    }
    __syncthreads();
    if (sh.last && tid == 0) {
        __threadfence();
        aggregate_box(a, bc.box);
    }
    __syncthreads();
}

__device__ __forceinline__ Smem carve(const MatchArgs &a, unsigned char *raw)
{
    Smem sm;
    size_t off = 0;
    sm.strip = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols;
    sm.pcode = reinterpret_cast<uint64_t *>(raw + off);
    off += sizeof(uint64_t) * kMaxPts;
    sm.partial = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMatchWarps * kMaxCand;
    sm.cost = reinterpret_cast<int *>(raw + off);
    off += sizeof(int) * kMaxCand;
    sm.pmj = reinterpret_cast<int *>(raw + off);
    return sm;
}

__global__ void __launch_bounds__(kMatchThreads) match_persistent_kernel(MatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;
    const Smem sm = carve(a, smem_raw);
    const int nblocks = a.ws.counts->n_blocks;
    for (;;) {
        if (threadIdx.x == 0) sh.next = atomicAdd(&a.ws.counts->queue_head, 1);
        __syncthreads();
        const int b = sh.next;
        __syncthreads();
        if (b >= nblocks) break;
        process_block(a, b, sm, sh);
    }
}

__global__ void __launch_bounds__(kMatchThreads) match_box_kernel(MatchArgs a, int box)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared sh;
    if ((int)blockIdx.x >= a.ws.nblk[box]) return;
    const Smem sm = carve(a, smem_raw);
    process_block(a, a.ws.blk_base[box] + blockIdx.x, sm, sh);
}

}  // namespace

size_t match_smem_bytes(const MatchArgs &a)
{
    return sizeof(uint64_t) * (size_t)a.strip_rows * a.strip_cols + sizeof(uint64_t) * kMaxPts +
           sizeof(int) * kMatchWarps * kMaxCand + sizeof(int) * kMaxCand + sizeof(int) * kMaxPts;
}

cudaError_t match_configure(const MatchArgs &a, int *ctas_per_sm)
{
    const int smem = (int)match_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(match_persistent_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(match_box_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, match_persistent_kernel,
                                                         kMatchThreads, smem);
}

cudaError_t launch_match_persistent(const MatchArgs &a, int grid, cudaStream_t s)
{
    match_persistent_kernel<<<grid, kMatchThreads, match_smem_bytes(a), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_match_box(const MatchArgs &a, int box, cudaStream_t s)
{
    const int slots = a.p.grid_g * a.p.grid_g;
    match_box_kernel<<<slots, kMatchThreads, match_smem_bytes(a), s>>>(a, box);
    return cudaGetLastError();
}

}  // namespace ctm
