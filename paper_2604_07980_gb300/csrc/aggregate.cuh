// aggregate.cuh -- block records and per-box aggregation (Sec. 4.3.4).  The
// sampling kernel (blocks with too few points) and the matching kernels
// (searched blocks) write block records; aggregate_kernel (plan.cu) then
// aggregates every box with one warp.
#pragma once

#include <math.h>

#include "ctm_internal.cuh"

namespace ctm {

// Sec. 4.3.4 on the block records of one box, by one full warp: FAR boxes take their single block; CLOSE boxes sort the
// valid block disparities, take the longest run whose consecutive differences
// are below tau_d (first run on ties), require N_min members and return its
// median (even length: mean of the middle two) or trimmed mean (floor(trim m)
// dropped per end, sum in ascending order); then Eq. 1.  `scratch` holds
// 2 * kMaxSlots floats of shared memory private to the warp.
__device__ __forceinline__ void aggregate_box(const MatchArgs &a, int box, float *scratch, int lane)
{
    const unsigned full = 0xffffffffu;
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
    const int fb_any = __any_sync(full, ((f[0] | f[1]) & CTM_BLK_FB_REJECT) != 0);
    const int few_any = __any_sync(full, ((f[0] | f[1]) & CTM_BLK_FEW_POINTS) != 0);
    const bool v0 = (f[0] & CTM_BLK_VALID) != 0, v1 = (f[1] & CTM_BLK_VALID) != 0;
    const int clamp_any = __any_sync(full, (v0 && (f[0] & CTM_BLK_SUBPIX_CLAMPED)) ||
                                               (v1 && (f[1] & CTM_BLK_SUBPIX_CLAMPED)));
    const unsigned b0 = __ballot_sync(full, v0), b1 = __ballot_sync(full, v1);
    const unsigned lt = (1u << lane) - 1u;
    const int nv = __popc(b0) + __popc(b1);
    float *vals = scratch, *sorted = scratch + kMaxSlots;
    if (v0) vals[__popc(b0 & lt)] = d[0];
    if (v1) vals[__popc(b0) + __popc(b1 & lt)] = d[1];
    __syncwarp();
    // rank sort (ties by position)
    for (int e = lane; e < nv; e += 32) {
        const float x = vals[e];
        int rank = 0;
        for (int q = 0; q < nv; ++q) {
            const float y = vals[q];
            rank += (y < x) || (y == x && q < e);
        }
        sorted[rank] = x;
    }
    __syncwarp();
    if (lane == 0) {
        int fl = P.far ? CTM_BOX_FAR : 0;
        if (fb_any) fl |= CTM_BOX_FB_REJECT;
        if (few_any) fl |= CTM_BOX_FEW_POINTS;
        if (clamp_any) fl |= CTM_BOX_SUBPIX_CLAMPED;
        bool have = false;
        float d_box = 0.0f;
        const float *v = sorted;
        if (P.far) {
            if (nv == 1) { have = true; d_box = v[0]; }
        } else if (nv > 0) {
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
    __syncwarp();
}

// Record a finished block: its aggregation record and the optional diagnostic
// record.  Boxes are aggregated after all blocks are written (aggregate_kernel).
__device__ __forceinline__ void write_block(const MatchArgs &a, int box, int slot, const ctm_block &rec)
{
    BlockResult r;
    r.d_full = rec.d_full;
    r.flags = rec.flags;
    a.ws.blkres[a.ws.blk_base[box] + slot] = r;
    if (a.dbg.blocks) a.dbg.blocks[(long long)box * (a.p.grid_g * a.p.grid_g) + slot] = rec;
}

}  // namespace ctm
