// match_common.cuh -- device pieces shared by the matching kernels (match.cu,
// match_pipe.cu): asynchronous-copy and mbarrier primitives with bounded waits,
// the shared-memory view of one block's data, the Hamming-sum scan loops and
// the strip chunk geometry.  Not part of the ABI.
#pragma once

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

// mbarrier + bulk copy (TMA, 1-D) primitives.
__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase `parity` of mbar: about one second of try_waits
// (global timer; an iteration cap as a backstop).  On expiry the CTA
// records an error, waits once more (bounded) for its copies in flight and
// reports false.
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr unsigned kWaitIters = 1u << 26;
__device__ __forceinline__ bool mbar_wait_for(uint64_t *mbar, unsigned parity)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < kWaitIters; ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((it & 15u) == 0 && global_ns() - t0 > kWaitNs) break;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, unsigned parity, int *error_flag)
{
    if (mbar_wait_for(mbar, parity)) return true;
    atomicOr(error_flag, 1);
    mbar_wait_for(mbar, parity);
    return false;
}

struct Smem {
    uint64_t *strip;   // strip_rows * strip_cols
    uint64_t *pcode;   // kMaxPts: compacted codes (left, then right queries)
    int *cost;         // kMaxCand
    int *cost_b;       // kMaxCand: backward costs (fused matcher; forward in cost)
    int *pmj;          // kMaxPts: (m << 8) | j
    int *pbase;        // kMaxPts: byte offset of the point's strip row + column in the chunk
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

// Byte offsets of the compacted points [p0, p1) into a strip chunk with row
// stride SWa whose element 0 is column xj0 - delta: row m * ndy, column
// X_j - xj0 + delta.
template <int NT>
__device__ __forceinline__ void set_bases(const Smem &sm, const int *X, int p0, int p1, int ndy,
                                          int SWa, int xj0, int delta)
{
    for (int p = p0 + (int)threadIdx.x; p < p1; p += NT) {
        const int mj = sm.pmj[p];
        sm.pbase[p] = 8 * ((mj >> 8) * ndy * SWa + X[mj & 255] - xj0 + delta);
    }
}

// Strip chunk geometry: columns [colbase, colbase + SWc) are stored from the even
// column colbase & ~1, so rows are 16-byte aligned for bulk copies.
struct ChunkGeom {
    int colbase_a;  // first stored column (even)
    int delta;      // colbase - colbase_a (0 or 1)
    int SWa;        // stored width in elements (even)
    int box;        // tensor-map box width when the rows load by tile::gather4, else 0
    int stride;     // row stride of the strip in shared memory, elements (box or SWa)
};

// gather_max: the widest box the caller's strip holds (0: 1-D copies only).
__device__ __forceinline__ ChunkGeom chunk_geom(int colbase, int SWc, int gather_max = 0)
{
    ChunkGeom g;
    g.colbase_a = colbase & ~1;
    g.delta = colbase - g.colbase_a;
    g.SWa = (SWc + g.delta + 1) & ~1;
    const int box = box_width(g.SWa);
    g.box = gather_max > 0 && box <= gather_max ? box : 0;
    g.stride = g.box > 0 ? g.box : g.SWa;
    return g;
}

// tile::gather4: rows y0..y3 of a 2-D tensor, one box of columns from x (the
// tensor map's one-row box), into four consecutive rows of shared memory at dst.
__device__ __forceinline__ void gather4_g2s(void *dst, const CUtensorMap *tm, int x, int y0, int y1, int y2,
                                           int y3, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n"
        ::"r"(smem_addr(dst)), "l"(tm), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_addr(mbar))
        : "memory");
}

}  // namespace
}  // namespace ctm
