// census.cu -- census transform kernels (Sec. 4.3.1, Algorithm 1).
//
// Work unit: one warp computes a 64-pixel row tile of codes on the grid
// I_k(x, y) = I(k x, k y) (k = 1 is the image itself; k > 1 is the
// multi-resolution census of Sec. 4.3.1 taken by decimation).  The warp stages
// the tile's window rows in shared memory as fp16 bit patterns 0x6400 | v, which
// is exactly 1024 + v, so fp16 order equals pixel order with no conversion.  Each
// lane owns two adjacent pixels: one packed compare (__hgt2_mask) gives xi for
// both pixels at one window offset, and one LOP3 ORs it into the bit position of
// that offset in a 16-bit-per-pixel accumulator.  Bits follow the raster order of
// the window (row j outer, column i inner), first neighbour in the highest
// comparison bit, with the optional sentinel above them; pixels whose window
// leaves the grid get 0.
//
// Two drivers: the full-image kernel (ctm_census_build, one warp per tile) and
// the region-of-interest kernel of the matching path, which computes only the
// tiles the planner marked in a per-plane bitmap (one bit per 64-pixel tile of
// a row) and clears the marks it consumed.
#include <cuda_fp16.h>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

constexpr int kTile = kCensusTilePx;               // pixels per warp tile
constexpr int kColsMax = kTile + kMaxWin - 1;      // staged columns (78)
constexpr int kWordsMax = (kColsMax + 1) / 2 + 1;  // half2 words per staged row (40)
constexpr int kWarpsPerCta = 8;

// Per-warp staging buffers: `rows` window rows, each as half2 pairs (c, c+1)
// starting at even c (even) and at odd c (odd), kWordsMax words per row.
struct WarpStage {
    uint32_t *even;
    uint32_t *odd;
};

__device__ __forceinline__ WarpStage warp_stage(uint32_t *smem, int warp, int rows)
{
    WarpStage st;
    st.even = smem + (size_t)warp * 2 * rows * kWordsMax;
    st.odd = st.even + rows * kWordsMax;
    return st;
}

struct Plane {
    const uint8_t *img;   // source image (full resolution)
    int W, H, pitch, k;   // source size and decimation
    int Ws, Hs;           // census grid size
    uint64_t *out;
    long long opitch;
    int vec_ok;           // 16-byte stores allowed (even pitch, 16-byte aligned base)
};

__device__ __forceinline__ __half2 as_h2(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

// Stage the WH window rows of tile (x0, y): every load of the tile is issued
// before any is used, so a warp waits for one memory round trip per tile.
template <int WW, int WH>
__device__ __forceinline__ void stage_rows(const Plane &pl, int x0, int y, const WarpStage &st, int lane)
{
    constexpr int sx = WW / 2, sy = WH / 2, ncols = kTile + 2 * sx;
    constexpr int per_lane = (ncols + 31) / 32;
    uint16_t v[WH][per_lane];
#pragma unroll
    for (int r = 0; r < WH; ++r) {
        const uint8_t *src = pl.img + (long long)pl.k * (y - sy + r) * pl.pitch;
#pragma unroll
        for (int t = 0; t < per_lane; ++t) {
            const int c = lane + 32 * t;
            const int xs = x0 - sx + c;
            uint16_t val = 0x6400;
            if (c < ncols && xs >= 0 && xs < pl.Ws) val = (uint16_t)(0x6400 | src[(long long)pl.k * xs]);
            v[r][t] = val;
        }
    }
    uint16_t *ev = reinterpret_cast<uint16_t *>(st.even);
    uint16_t *od = reinterpret_cast<uint16_t *>(st.odd);
#pragma unroll
    for (int r = 0; r < WH; ++r) {
#pragma unroll
        for (int t = 0; t < per_lane; ++t) {
            const int c = lane + 32 * t;
            if (c < ncols) {
                ev[r * 2 * kWordsMax + c] = v[r][t];
                if (c > 0) od[r * 2 * kWordsMax + c - 1] = v[r][t];
            }
        }
    }
}

// Any window: staging with runtime sizes.
__device__ __forceinline__ void stage_rows_any(const Plane &pl, int x0, int y, int sx, int sy,
                                               const WarpStage &st, int lane)
{
    const int ncols = kTile + 2 * sx;
    uint16_t *ev = reinterpret_cast<uint16_t *>(st.even);
    for (int r = 0; r < 2 * sy + 1; ++r) {
        const uint8_t *src = pl.img + (long long)pl.k * (y - sy + r) * pl.pitch;
        for (int c = lane; c < ncols; c += 32) {
            const int xs = x0 - sx + c;
            uint16_t val = 0x6400;
            if (xs >= 0 && xs < pl.Ws) val = (uint16_t)(0x6400 | src[(long long)pl.k * xs]);
            ev[r * 2 * kWordsMax + c] = val;
        }
    }
}

// Codes of pixels (x0 + 2 lane, x0 + 2 lane + 1) from the staged rows.
template <int WW, int WH>
__device__ __forceinline__ void tile_codes(const WarpStage &st, int lane, int sentinel, uint64_t &c0,
                                           uint64_t &c1)
{
    constexpr int sx = WW / 2, sy = WH / 2;
    constexpr int n = WW * WH;
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    const uint32_t cw = (sx & 1) ? st.odd[sy * kWordsMax + lane + (sx - 1) / 2]
                                 : st.even[sy * kWordsMax + lane + sx / 2];
    const __half2 centre = as_h2(cw);
#pragma unroll
    for (int j = 0; j < WH; ++j) {
#pragma unroll
        for (int i = 0; i < WW; ++i) {
            // staged column of the neighbour, relative to the lane's pair base 2*lane
            const uint32_t nb = (i & 1) ? st.odd[j * kWordsMax + lane + (i - 1) / 2]
                                        : st.even[j * kWordsMax + lane + i / 2];
            const uint32_t m = __hgt2_mask(as_h2(nb), centre);
            const int k = j * WW + i;     // raster index of the window offset
            const int p = n - 1 - k;      // its code bit
            const uint32_t pos = (1u << (p & 15)) | (1u << (16 + (p & 15)));
            acc[p >> 4] |= m & pos;
        }
    }
    if (sentinel) {
        const uint32_t pos = (1u << (n & 15)) | (1u << (16 + (n & 15)));
        acc[n >> 4] |= pos;
    }
    const uint32_t lo0 = __byte_perm(acc[0], acc[1], 0x5410), hi0 = __byte_perm(acc[2], acc[3], 0x5410);
    const uint32_t lo1 = __byte_perm(acc[0], acc[1], 0x7632), hi1 = __byte_perm(acc[2], acc[3], 0x7632);
    c0 = ((uint64_t)hi0 << 32) | lo0;
    c1 = ((uint64_t)hi1 << 32) | lo1;
}

// Any window: plain per-pixel loop over the staged rows.
__device__ __forceinline__ uint64_t code_any(const WarpStage &st, int px, int win_w, int win_h,
                                             int sentinel)
{
    const uint16_t *ev = reinterpret_cast<const uint16_t *>(st.even);
    constexpr int rowh = 2 * kWordsMax;
    const int sx = win_w / 2, sy = win_h / 2;
    const uint16_t centre = ev[sy * rowh + px + sx];
    uint64_t c = sentinel ? 1ull : 0ull;
    for (int j = 0; j < win_h; ++j)
        for (int i = 0; i < win_w; ++i) c = (c << 1) | (uint64_t)(ev[j * rowh + px + i] > centre);
    return c;
}

__device__ __forceinline__ void store_pair(const Plane &pl, int x, int y, uint64_t c0, uint64_t c1)
{
    uint64_t *dst = pl.out + (long long)y * pl.opitch + x;
    if (x + 1 < pl.Ws) {
        if (pl.vec_ok) {
            *reinterpret_cast<ulonglong2 *>(dst) = make_ulonglong2(c0, c1);
        } else {
            dst[0] = c0;
            dst[1] = c1;
        }
    } else if (x < pl.Ws) {
        dst[0] = c0;
    }
}

// One 64-pixel tile of row y starting at x0 (x0 a multiple of 64).
template <int WW, int WH>
__device__ void census_tile(const Plane &pl, int x0, int y, int win_w, int win_h, int sentinel,
                            const WarpStage &st)
{
    const int lane = threadIdx.x & 31;
    const int sx = win_w / 2, sy = win_h / 2;
    const int x = x0 + 2 * lane;
    if (y - sy < 0 || y + sy >= pl.Hs) {  // whole row undefined
        store_pair(pl, x, y, 0ull, 0ull);
        return;
    }
    uint64_t c0, c1;
    if constexpr (WW > 0) {
        stage_rows<WW, WH>(pl, x0, y, st, lane);
        __syncwarp();
        tile_codes<WW, WH>(st, lane, sentinel, c0, c1);
    } else {
        stage_rows_any(pl, x0, y, sx, sy, st, lane);
        __syncwarp();
        c0 = code_any(st, 2 * lane, win_w, win_h, sentinel);
        c1 = code_any(st, 2 * lane + 1, win_w, win_h, sentinel);
    }
    if (x - sx < 0 || x + sx >= pl.Ws) c0 = 0ull;
    if (x + 1 - sx < 0 || x + 1 + sx >= pl.Ws) c1 = 0ull;
    store_pair(pl, x, y, c0, c1);
    __syncwarp();
}

__device__ __forceinline__ void census_tile_any(const Plane &pl, int x0, int y, int win_w, int win_h,
                                                int sentinel, const WarpStage &st)
{
    if (win_w == 9 && win_h == 7)
        census_tile<9, 7>(pl, x0, y, win_w, win_h, sentinel, st);
    else if (win_w == 7 && win_h == 7)
        census_tile<7, 7>(pl, x0, y, win_w, win_h, sentinel, st);
    else if (win_w == 5 && win_h == 5)
        census_tile<5, 5>(pl, x0, y, win_w, win_h, sentinel, st);
    else
        census_tile<0, 0>(pl, x0, y, win_w, win_h, sentinel, st);
}

// Full image: warp w of CTA (bx, by) takes tile bx of row by * 8 + w.
__global__ void __launch_bounds__(32 * kWarpsPerCta) census_full_kernel(Plane pl, int win_w, int win_h,
                                                                        int sentinel)
{
    extern __shared__ uint32_t stage_mem[];
    const int warp = threadIdx.x >> 5;
    const int y = blockIdx.y * kWarpsPerCta + warp;
    if (y >= pl.Hs) return;
    const WarpStage st = warp_stage(stage_mem, warp, win_h);
    census_tile_any(pl, blockIdx.x * kTile, y, win_w, win_h, sentinel, st);
}

// Region of interest: warps stride over the bitmap words of all frames' planes.
__global__ void __launch_bounds__(32 * kWarpsPerCta) census_roi_kernel(MatchArgs a)
{
    extern __shared__ uint32_t stage_mem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WarpStage st = warp_stage(stage_mem, warp, a.p.win_h);
    int nf = a.counts_in[0];
    nf = nf < 0 ? 0 : (nf > a.caps.max_frames ? a.caps.max_frames : nf);
    const long long total = (long long)nf * a.ws.bm_frame_words;
    const long long gwarp = (long long)blockIdx.x * kWarpsPerCta + warp;
    const long long nwarps = (long long)gridDim.x * kWarpsPerCta;
    for (long long w = gwarp; w < total; w += nwarps) {
        uint32_t bits = a.ws.bitmap[w];
        if (bits == 0u) continue;
        __syncwarp();
        if (lane == 0) a.ws.bitmap[w] = 0u;  // consumed: the bitmap is clear for the next call
        const int f = (int)(w / a.ws.bm_frame_words);
        int r = (int)(w - (long long)f * a.ws.bm_frame_words);
        int q = 0;
        while (q < 3 && r >= a.ws.bm_plane_off[q + 1]) ++q;
        r -= a.ws.bm_plane_off[q];
        const int y = r / a.ws.bm_row_words[q];
        const int wi = r - y * a.ws.bm_row_words[q];
        const ctm_frame fr = a.frames[f];
        Plane pl;
        pl.img = (q & 1) ? fr.right : fr.left;
        pl.W = fr.width;
        pl.H = fr.height;
        pl.pitch = fr.pitch;
        pl.k = q < 2 ? 1 : a.p.close_factor;
        pl.Ws = ceil_div_nn(fr.width, pl.k);
        pl.Hs = ceil_div_nn(fr.height, pl.k);
        uint64_t *base = a.ws.census + (long long)f * a.ws.frame_stride;
        pl.out = q < 2 ? base + q * a.ws.plane1_elems : base + 2 * a.ws.plane1_elems + (q - 2) * a.ws.planek_elems;
        pl.opitch = q < 2 ? a.ws.pitch1 : a.ws.pitchk;
        pl.vec_ok = 1;  // workspace planes: 256-byte aligned, pitch a multiple of 32
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int x0 = (wi * 32 + b) * kTile;
            if (x0 < pl.Ws && y < pl.Hs)
                census_tile_any(pl, x0, y, a.p.win_w, a.p.win_h, a.p.sentinel, st);
        }
    }
}

}  // namespace

size_t census_smem_bytes(int win_h)
{
    return sizeof(uint32_t) * (size_t)kWarpsPerCta * 2 * win_h * kWordsMax;
}

cudaError_t launch_census_single(const uint8_t *img, int W, int H, int pitch, int k, int win_w,
                                 int win_h, int sentinel, uint64_t *out, long long out_pitch,
                                 cudaStream_t s)
{
    Plane pl;
    pl.img = img;
    pl.W = W;
    pl.H = H;
    pl.pitch = pitch;
    pl.k = k;
    pl.Ws = ceil_div_nn(W, k);
    pl.Hs = ceil_div_nn(H, k);
    pl.out = out;
    pl.opitch = out_pitch;
    pl.vec_ok = (out_pitch % 2 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    dim3 grid(ceil_div_nn(pl.Ws, kTile), ceil_div_nn(pl.Hs, kWarpsPerCta));
    census_full_kernel<<<grid, 32 * kWarpsPerCta, census_smem_bytes(win_h), s>>>(pl, win_w, win_h, sentinel);
    return cudaGetLastError();
}

cudaError_t launch_census_roi(const MatchArgs &a, int grid, cudaStream_t s)
{
    census_roi_kernel<<<grid, 32 * kWarpsPerCta, census_smem_bytes(a.p.win_h), s>>>(a);
    return cudaGetLastError();
}

}  // namespace ctm
