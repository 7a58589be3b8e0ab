// gather.cu -- the image bytes a call's census reads, copied by the device straight
// from the caller's host memory (ctm_match_batch_mapped).
//
// The planner knows before any pixel moves which census tiles the search will
// read: the sampling kernel marks them in the demand bitmap (one bit per
// 32-pixel tile of a plane row).  A tile's census reads a fixed window of its
// plane (grid columns [x0 - L, x0 + R) of the window's rows; see
// census_reach_left/right), which at decimation k is every k-th column and row
// of the source image.  Each warp of gather_kernel takes one source row of one
// image and 32 segments of kGatherSegBytes bytes of it: lane s decides from the
// bitmap whether any marked tile of a plane made from this image reads its
// segment, then the warp copies the needed segments from host memory into the
// staging image.  Bytes of the staging images that no marked tile reads are never
// written and never read.  The bitmap is read, not cleared (tile_list_kernel
// consumes it next).
#include <algorithm>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

constexpr int kSegsPerWarp = 32;
constexpr int kGatherThreads = 256;  // one persistent CTA per SM

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Does any marked tile of plane q (decimation k) read source bytes [x_lo, x_lo +
// kGatherSegBytes) of source row sy?  Tile t reads source bytes [k (32 t - L),
// k (32 t + R)) of its window's rows; the tiles that can reach the segment are
// consecutive bits t_lo .. t_hi (at most six, so at most two bitmap words), and
// the rows' words are OR-ed first (independent loads, one round trip).
__device__ __forceinline__ bool plane_needs(const MatchArgs &a, const uint32_t *fbm, int q, int k, int sy,
                                            int height, int width, int L, int R, int x_lo)
{
    if (sy % k) return false;
    const int gy = sy / k;  // grid row of this source row
    const int Hs = (height + k - 1) / k;
    const int ntiles = ((width + k - 1) / k + kCensusTilePx - 1) / kCensusTilePx;
    const int tp = kCensusTilePx * k;
    const int t_lo = max(floor_div(x_lo - k * R, tp) + 1, 0);
    const int t_hi = min(floor_div(x_lo + kGatherSegBytes + k * L - 1, tp), ntiles - 1);
    if (t_lo > t_hi) return false;
    const int wh = a.p.win_h, sy_w = wh / 2;
    // tile rows y whose window rows y - sy_w .. y - sy_w + wh - 1 hold gy
    const int y0 = max(gy + sy_w - wh + 1, 0), y1 = min(gy + sy_w, Hs - 1);
    const int w0 = t_lo >> 5, w1 = t_hi >> 5;
    const uint32_t *p = fbm + a.ws.bm_plane_off[q] + (long long)y0 * a.ws.bm_row_words[q];
    uint32_t lo = 0u, hi = 0u;
    for (int y = y0; y <= y1; ++y, p += a.ws.bm_row_words[q]) {
        lo |= p[w0];
        hi |= p[w1];
    }
    const unsigned long long m = ((unsigned long long)hi << 32) | lo;  // bits of tiles 32 w0 ..
    const int b0 = t_lo - 32 * w0, nb = t_hi - t_lo + 1;
    const unsigned long long range = ((nb >= 64 ? 0ull : (1ull << nb)) - 1ull) << b0;
    // with w1 == w0 the high word repeats the low one; only bits below 32 + b0 .. count then
    return (m & (w1 == w0 ? (range & 0xffffffffull) : range)) != 0ull;
}

// One (frame, image, source row, chunk of 32 segments) per warp: the needed
// segments (a ballot of the lanes' plane_needs), then their bytes, 16 per lane
// (kGatherSegBytes / 16 lanes per segment, 512 contiguous bytes per pass), all
// reads before the writes.  Returns the bytes this lane copied.
__device__ __forceinline__ unsigned long long gather_item(const MatchArgs &a, long long item, int chunks, int nf,
                                                          int lane)
{
    long long r = item;
    const int chunk = (int)(r % chunks);
    r /= chunks;
    const int sy = (int)(r % a.caps.max_height);
    r /= a.caps.max_height;
    const int img = (int)(r % 2);
    const int f = (int)(r / 2);
    if (f >= nf) return 0ull;
    const ctm_frame src = a.gather_src[f];
    const int W = src.width;
    if (sy >= src.height || chunk * kSegsPerWarp * kGatherSegBytes >= W) return 0ull;
    const int L = census_reach_left(a.p.win_w, a.p.win_h);
    const int R = census_reach_right(a.p.win_w, a.p.win_h);
    const int x_lo = (chunk * kSegsPerWarp + lane) * kGatherSegBytes;
    const uint32_t *fbm = a.ws.bitmap + (long long)f * a.ws.bm_frame_words;
    bool need = false;
    if (x_lo < W) {
        // planes made from this image: full resolution (plane img) and, at
        // decimation close_factor > 1, plane 2 + img
        need = plane_needs(a, fbm, img, 1, sy, src.height, W, L, R, x_lo);
        if (a.p.close_factor > 1)
            need = plane_needs(a, fbm, 2 + img, a.p.close_factor, sy, src.height, W, L, R, x_lo) || need;
    }
    const unsigned needm = __ballot_sync(0xffffffffu, need);
    if (!needm) return 0ull;
    const ctm_frame dst = a.frames[f];
    constexpr int kLanesPerSeg = kGatherSegBytes / 16, kSegsPerPass = 32 / kLanesPerSeg;
    constexpr int kPasses = kSegsPerWarp / kSegsPerPass;
    const int part = lane % kLanesPerSeg;
    const long long off = (long long)chunk * kSegsPerWarp * kGatherSegBytes + 16 * part;
    const uint8_t *srow = (img ? src.right : src.left) + (long long)sy * src.pitch + off;
    uint8_t *drow = const_cast<uint8_t *>(img ? dst.right : dst.left) + (long long)sy * dst.pitch + off;
    uint4 v[kPasses];
    bool on[kPasses];
#pragma unroll
    for (int pass = 0; pass < kPasses; ++pass) {
        const int sl = pass * kSegsPerPass + lane / kLanesPerSeg;  // segment within the chunk
        on[pass] = ((needm >> sl) & 1u) && off + sl * kGatherSegBytes < W;
        if (on[pass]) v[pass] = *reinterpret_cast<const uint4 *>(srow + sl * kGatherSegBytes);
    }
    unsigned long long bytes = 0ull;
#pragma unroll
    for (int pass = 0; pass < kPasses; ++pass) {
        if (on[pass]) {
            *reinterpret_cast<uint4 *>(drow + (pass * kSegsPerPass + lane / kLanesPerSeg) * kGatherSegBytes) = v[pass];
            bytes += 16;
        }
    }
    return bytes;
}

// One persistent CTA per SM walking the row chunks: the gather mostly waits on
// the host link, and a small footprint leaves the SM's other slots to the kernels
// of calls running beside it.
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(MatchArgs a, int chunks, long long items)
{
    __shared__ unsigned long long cta_bytes;
    if (threadIdx.x == 0) cta_bytes = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nf = min(max(a.counts_in[0], 0), a.caps.max_frames);
    const long long warps = (long long)gridDim.x * (kGatherThreads / 32);
    // items run frame-major: the call's frames are the first nf of the capacity's
    const long long lim = min(items, (long long)nf * 2 * a.caps.max_height * chunks);
    unsigned long long bytes = 0ull;
    for (long long it = (long long)blockIdx.x * (kGatherThreads / 32) + (threadIdx.x >> 5); it < lim; it += warps)
        bytes += gather_item(a, it, chunks, nf, lane);
    if (bytes) atomicAdd(&cta_bytes, bytes);
    __syncthreads();
    if (threadIdx.x == 0 && cta_bytes) atomicAdd(&a.ws.counts->host_bytes, cta_bytes);
}

}  // namespace

cudaError_t launch_gather(const MatchArgs &a, int sm_count, cudaStream_t s)
{
    const int chunks = ceil_div_nn(a.caps.max_width, kSegsPerWarp * kGatherSegBytes);
    const long long items = (long long)a.caps.max_frames * 2 * a.caps.max_height * chunks;
    const long long grid = std::min<long long>((items + kGatherThreads / 32 - 1) / (kGatherThreads / 32), sm_count);
    if (grid > 0) gather_kernel<<<(unsigned)grid, kGatherThreads, 0, s>>>(a, chunks, items);
    return cudaGetLastError();
}

}  // namespace ctm
