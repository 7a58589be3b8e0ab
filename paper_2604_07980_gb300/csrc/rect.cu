// rect.cu -- Sec. 5.1 auto-rectification offset, with census matching in place
// of block matching: for every vertical offset delta and every ROI pixel, the
// winner-take-all disparity of the left pixel read delta rows lower, checked by
// the backward search; the offset with the most consistent disparities above a
// threshold wins.  Not on the per-frame path; run now and then on a stream of
// its own.  Also the temporal filter of the per-frame estimates (host code).
#include <cuda_runtime.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

__device__ __forceinline__ uint64_t code_or_zero(const uint64_t *C, long long pitch, int W, int H, int x, int y)
{
    return (x >= 0 && x < W && y >= 0 && y < H) ? __ldg(C + (long long)y * pitch + x) : 0ull;
}

constexpr int kRectThreads = 128;

// Thread per ROI pixel of one row and one offset (grid: x tiles, rows, offsets).
// The CTA stages the two code rows its pixels search: the right row y over
// columns x0 - dmax .. x0 + 127 - dmin (forward candidates x - d) and the left
// row y + delta over x0 + dmin - dmax .. x0 + 127 + dmax - dmin (backward
// candidates x - d_f + d for any d_f), codes outside the image as 0.  Each scan
// keeps the first minimum as the least key (cost << 11 | candidate index).
__global__ void __launch_bounds__(kRectThreads) rect_kernel(const uint64_t *CL, const uint64_t *CR, long long pitch,
                                                            int W, int H, int sx, int sy, int rx0, int rx1, int ry0,
                                                            int dmin, int dmax, int delta_min, int d_thresh,
                                                            int fb_tol, unsigned long long *counts)
{
    extern __shared__ uint64_t rect_smem[];
    const int nd = dmax - dmin + 1;
    const int x0 = rx0 + blockIdx.x * kRectThreads;
    const int x = x0 + threadIdx.x;
    const int y = ry0 + blockIdx.y;
    const int delta = delta_min + blockIdx.z;
    const int yl = y + delta;
    uint64_t *rrow = rect_smem;                     // columns x0 - dmax + i
    uint64_t *lrow = rect_smem + kRectThreads + nd;  // columns x0 + dmin - dmax + i
    const int nr = kRectThreads + nd - 1, nl = kRectThreads + 2 * (nd - 1);
    for (int i = threadIdx.x; i < nr; i += kRectThreads) rrow[i] = code_or_zero(CR, pitch, W, H, x0 - dmax + i, y);
    for (int i = threadIdx.x; i < nl; i += kRectThreads)
        lrow[i] = code_or_zero(CL, pitch, W, H, x0 + dmin - dmax + i, yl);
    __syncthreads();
    bool hit = false;
    if (x < rx1 && x - sx >= 0 && x + sx < W && yl - sy >= 0 && yl + sy < H) {
        const int t = threadIdx.x;
        const uint64_t cl = lrow[t + dmax - dmin];  // column x
        unsigned kf = 0xffffffffu;
        for (int i = 0; i < nd; ++i)  // candidate d = dmin + i at column x - d: rrow[t + dmax - d]
            kf = min(kf, ((unsigned)__popcll(cl ^ rrow[t + nd - 1 - i]) << 11) | (unsigned)i);
        const int i_f = (int)(kf & 2047u);
        const uint64_t cq = rrow[t + nd - 1 - i_f];   // column x - d_f
        const int b0 = t + nd - 1 - i_f;              // lrow index of column x - d_f + dmin
        unsigned kb = 0xffffffffu;
        for (int i = 0; i < nd; ++i) kb = min(kb, ((unsigned)__popcll(cq ^ lrow[b0 + i]) << 11) | (unsigned)i);
        const int d_f = dmin + i_f, d_b = dmin + (int)(kb & 2047u);
        hit = abs(d_b - d_f) <= fb_tol && d_f > d_thresh;
    }
    const int n = __syncthreads_count(hit);
    if (threadIdx.x == 0 && n) atomicAdd(counts + blockIdx.z, (unsigned long long)n);
}

// First offset with the largest count.
__global__ void rect_argmax_kernel(const unsigned long long *counts, int n, int delta_min, int *delta_out)
{
    if (threadIdx.x != 0) return;
    int best = 0;
    for (int i = 1; i < n; ++i)
        if (counts[i] > counts[best]) best = i;
    *delta_out = delta_min + best;
}

}  // namespace
}  // namespace ctm

using namespace ctm;

extern "C" int ctm_auto_rect(const ctm_params *p, const uint8_t *left_dev, const uint8_t *right_dev, int width,
                             int height, int pitch, int rx0, int ry0, int rx1, int ry1, int dmin, int dmax,
                             int delta_min, int delta_max, int d_thresh, int fb_tol, uint64_t *census_dev,
                             unsigned long long *counts_dev, int *delta_dev, ctm_stream stream)
{
    if (!p || !left_dev || !right_dev || !census_dev || !counts_dev || !delta_dev) return CTM_EINVAL;
    if (width < 1 || height < 1 || pitch < width || dmin > dmax || dmax - dmin + 1 > 1024 ||
        delta_min > delta_max || delta_max - delta_min + 1 > 65535 || fb_tol < 0)
        return CTM_EINVAL;
    if (p->win_w < 1 || p->win_h < 1 || (p->win_w & 1) == 0 || (p->win_h & 1) == 0 || p->win_w > kMaxWin ||
        p->win_h > kMaxWin || p->win_w * p->win_h + (p->sentinel ? 1 : 0) > 64)
        return CTM_EINVAL;
    rx0 = std::max(rx0, 0);
    ry0 = std::max(ry0, 0);
    rx1 = std::min(rx1, width);
    ry1 = std::min(ry1, height);
    cudaStream_t s = (cudaStream_t)stream;
    const int nd = delta_max - delta_min + 1;
    const long long cpitch = width;  // census planes: width codes per row, left then right
    uint64_t *CL = census_dev, *CR = census_dev + (long long)width * height;
    cudaError_t e = cudaMemsetAsync(counts_dev, 0, sizeof(unsigned long long) * nd, s);
    if (e == cudaSuccess)
        e = launch_census_single(left_dev, width, height, pitch, 1, p->win_w, p->win_h, p->sentinel, CL, cpitch, s);
    if (e == cudaSuccess)
        e = launch_census_single(right_dev, width, height, pitch, 1, p->win_w, p->win_h, p->sentinel, CR, cpitch, s);
    if (e == cudaSuccess && rx1 > rx0 && ry1 > ry0) {
        const dim3 grid((rx1 - rx0 + kRectThreads - 1) / kRectThreads, ry1 - ry0, nd);
        const int ndisp = dmax - dmin + 1;
        const size_t smem = sizeof(uint64_t) * (size_t)(2 * kRectThreads + 3 * ndisp);
        e = cudaFuncSetAttribute(rect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            rect_kernel<<<grid, kRectThreads, smem, s>>>(CL, CR, cpitch, width, height, p->win_w / 2, p->win_h / 2,
                                                         rx0, rx1, ry0, dmin, dmax, delta_min, d_thresh, fb_tol,
                                                         counts_dev);
        e = e == cudaSuccess ? cudaGetLastError() : e;
    }
    if (e == cudaSuccess) {
        rect_argmax_kernel<<<1, 32, 0, s>>>(counts_dev, nd, delta_min, delta_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

extern "C" int ctm_rect_filter(const int *estimates, int n, int prev, int max_step)
{
    if (!estimates || n < 1) return prev;
    if (max_step < 0) max_step = 0;
    std::vector<int> v(estimates, estimates + n);
    std::sort(v.begin(), v.end());
    const int med = v[(n - 1) / 2];
    const int step = std::min(std::max(med - prev, -max_step), max_step);
    return prev + step;
}
