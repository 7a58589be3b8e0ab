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
    int vec_load;         // word loads allowed: k in {1, 2}, 8-byte aligned base, pitch % 4 == 0
};

__device__ __forceinline__ __half2 as_h2(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

// Staged row layout: H[b] = 0x6400 | I_k(x0 - 8 + b, row) for b in [0, 80), kept
// twice as half2 words: even[t] = (H[2t], H[2t+1]) and odd[t] = (H[2t+1], H[2t+2]),
// so every pair of adjacent pixels is one aligned 32-bit word in one of the two.
// Lane l < 21 loads H[4l .. 4l+3] with one 32-bit load (k = 1) or one 64-bit
// load (k = 2) where the four pixels lie inside the image, else byte by byte.
__device__ __forceinline__ uint32_t load_quad(const Plane &pl, int x0, int ys, int lane)
{
    const uint8_t *row = pl.img + (long long)pl.k * ys * pl.pitch;
    uint32_t v = 0u;
    if (lane < 21) {
        const int xs = x0 - 8 + 4 * lane;
        if (pl.vec_load && pl.k == 1 && xs >= 0 && xs + 3 < pl.W) {
            v = __ldg(reinterpret_cast<const uint32_t *>(row + xs));
        } else if (pl.vec_load && pl.k == 2 && xs >= 0 && 2 * xs + 7 < pl.W) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(row + 2 * xs));
            v = __byte_perm(w.x, w.y, 0x6420);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int xq = xs + q;
                if (xq >= 0 && xq < pl.Ws) v |= (uint32_t)__ldg(row + (long long)pl.k * xq) << (8 * q);
            }
        }
    }
    return v;
}

// All WH window rows of tile (x0, y) for this lane, with one uniform decision per
// tile: interior tiles of a word-aligned image take straight-line word loads,
// edge tiles take the per-pixel path.  Rows must lie inside the grid.
template <int WH>
__device__ __forceinline__ void load_tile(const Plane &pl, int x0, int y, int lane, uint32_t (&v)[WH])
{
    constexpr int sy = WH / 2;
    const int xs = x0 - 8 + 4 * lane;
    const bool interior = pl.vec_load && x0 - 8 >= 0 &&
                          (pl.k == 1 ? x0 + 76 <= pl.W : 2 * (x0 + 76) <= pl.W);
    if (interior) {
        const long long step = (long long)pl.k * pl.pitch;
        const uint8_t *row = pl.img + (long long)pl.k * (y - sy) * pl.pitch + (long long)pl.k * xs;
        if (lane < 21) {
            if (pl.k == 1) {
#pragma unroll
                for (int r = 0; r < WH; ++r) v[r] = __ldg(reinterpret_cast<const uint32_t *>(row + r * step));
            } else {
#pragma unroll
                for (int r = 0; r < WH; ++r) {
                    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(row + r * step));
                    v[r] = __byte_perm(w.x, w.y, 0x6420);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < WH; ++r) v[r] = 0u;
        }
    } else {
#pragma unroll
        for (int r = 0; r < WH; ++r) v[r] = load_quad(pl, x0, y - sy + r, lane);
    }
}

// Convert one loaded row (4 pixels per lane) to the two half2 copies.
__device__ __forceinline__ void store_quad(uint32_t v, uint32_t *even, uint32_t *odd, int lane)
{
    const uint32_t nxt = __shfl_down_sync(0xffffffffu, v, 1);
    if (lane < 20) {
        const uint32_t C = 0x64646464u;
        uint2 e, o;
        e.x = __byte_perm(v, C, 0x4140);                            // H[4l],   H[4l+1]
        e.y = __byte_perm(v, C, 0x4342);                            // H[4l+2], H[4l+3]
        o.x = __byte_perm(v, C, 0x4241);                            // H[4l+1], H[4l+2]
        o.y = __byte_perm(__byte_perm(v, nxt, 0x0043), C, 0x4140);  // H[4l+3], H[4l+4]
        *reinterpret_cast<uint2 *>(even + 2 * lane) = e;
        *reinterpret_cast<uint2 *>(odd + 2 * lane) = o;
    }
}

// Stage the window rows y - sy .. y + sy of tile x0: all loads first (they are
// independent and in flight together), then the conversions.
template <int WH>
__device__ __forceinline__ void stage_rows(const Plane &pl, int x0, int y, const WarpStage &st, int lane)
{
    constexpr int sy = WH / 2;
    uint32_t v[WH];
#pragma unroll
    for (int r = 0; r < WH; ++r) v[r] = load_quad(pl, x0, y - sy + r, lane);
#pragma unroll
    for (int r = 0; r < WH; ++r) store_quad(v[r], st.even + r * kWordsMax, st.odd + r * kWordsMax, lane);
}

__device__ __forceinline__ void stage_rows_any(const Plane &pl, int x0, int y, int sy,
                                               const WarpStage &st, int lane)
{
    for (int r = 0; r < 2 * sy + 1; ++r)
        store_quad(load_quad(pl, x0, y - sy + r, lane), st.even + r * kWordsMax, st.odd + r * kWordsMax, lane);
}

// Codes of pixels (x0 + 2 lane, x0 + 2 lane + 1) from the staged rows.
template <int WW, int WH>
__device__ __forceinline__ void tile_codes(const WarpStage &st, int lane, int sentinel, uint64_t &c0,
                                           uint64_t &c1)
{
    constexpr int sx = WW / 2, sy = WH / 2;
    constexpr int n = WW * WH;
    constexpr int OFF = 8 - sx;  // H index of the window's left column, relative to 2*lane
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    const __half2 centre = as_h2(st.even[sy * kWordsMax + lane + 4]);  // H[2*lane + 8]
#pragma unroll
    for (int j = 0; j < WH; ++j) {
#pragma unroll
        for (int i = 0; i < WW; ++i) {
            const int b = i + OFF;  // H index of the neighbour pair, relative to 2*lane
            const uint32_t nb = (b & 1) ? st.odd[j * kWordsMax + lane + (b - 1) / 2]
                                        : st.even[j * kWordsMax + lane + b / 2];
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
    const int off = 8 - sx;
    const uint16_t centre = ev[sy * rowh + px + 8];
    uint64_t c = sentinel ? 1ull : 0ull;
    for (int j = 0; j < win_h; ++j)
        for (int i = 0; i < win_w; ++i) c = (c << 1) | (uint64_t)(ev[j * rowh + px + i + off] > centre);
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
        stage_rows<WH>(pl, x0, y, st, lane);
        __syncwarp();
        tile_codes<WW, WH>(st, lane, sentinel, c0, c1);
    } else {
        stage_rows_any(pl, x0, y, sy, st, lane);
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
    extern __shared__ __align__(16) uint32_t stage_mem[];
    const int warp = threadIdx.x >> 5;
    const int y = blockIdx.y * kWarpsPerCta + warp;
    if (y >= pl.Hs) return;
    const WarpStage st = warp_stage(stage_mem, warp, win_h);
    census_tile_any(pl, blockIdx.x * kTile, y, win_w, win_h, sentinel, st);
}

// Region of interest.  Each warp walks the set bits of its bitmap words
// (grid-stride over the words of all frames' planes) as one stream of tiles and
// clears every word it consumed.
struct TileCursor {
    long long w;       // current word index (grid-stride)
    uint32_t bits;     // tiles of the current word not yet taken
    Plane pl;          // plane of the current word
    int y, wi;         // row and word-in-row of the current word
};

__device__ __forceinline__ void decode_word(const MatchArgs &a, long long w, TileCursor &c)
{
    const int f = (int)(w / a.ws.bm_frame_words);
    int r = (int)(w - (long long)f * a.ws.bm_frame_words);
    int q = 0;
    while (q < 3 && r >= a.ws.bm_plane_off[q + 1]) ++q;
    r -= a.ws.bm_plane_off[q];
    c.y = r / a.ws.bm_row_words[q];
    c.wi = r - c.y * a.ws.bm_row_words[q];
    const ctm_frame fr = a.frames[f];
    Plane &pl = c.pl;
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
    pl.vec_load = (pl.k == 1 || pl.k == 2) && (fr.pitch % 4 == 0) &&
                  ((reinterpret_cast<uintptr_t>(pl.img) & 7u) == 0);
}

// Next tile of this warp's stream; false when its words are exhausted.
__device__ __forceinline__ bool next_tile(const MatchArgs &a, TileCursor &c, long long nwarps,
                                          long long total, int lane, int &x0, int &y)
{
    for (;;) {
        while (c.bits == 0u) {
            c.w += nwarps;
            if (c.w >= total) return false;
            const uint32_t bits = a.ws.bitmap[c.w];
            if (bits == 0u) continue;
            __syncwarp();
            if (lane == 0) a.ws.bitmap[c.w] = 0u;  // consumed: clear for the next call
            decode_word(a, c.w, c);
            c.bits = bits;
        }
        const int b = __ffs(c.bits) - 1;
        c.bits &= c.bits - 1u;
        x0 = (c.wi * 32 + b) * kTile;
        y = c.y;
        if (x0 < c.pl.Ws && y < c.pl.Hs) return true;
    }
}

// Fixed windows: the loads of the next tile are issued before the current
// tile is converted and computed, so memory latency overlaps compute.
template <int WW, int WH>
__device__ void roi_stream(const MatchArgs &a, const WarpStage &st, TileCursor &c, long long nwarps,
                           long long total, int lane)
{
    constexpr int sx = WW / 2, sy = WH / 2;
    int xA = 0, yA = 0;
    bool okA = next_tile(a, c, nwarps, total, lane, xA, yA);
    Plane plA = c.pl;
    uint32_t vA[WH];
#pragma unroll
    for (int r = 0; r < WH; ++r) vA[r] = 0u;
    if (okA && yA - sy >= 0 && yA + sy < plA.Hs) load_tile<WH>(plA, xA, yA, lane, vA);
    while (okA) {
        int xB = 0, yB = 0;
        const bool okB = next_tile(a, c, nwarps, total, lane, xB, yB);
        const Plane plB = c.pl;
        uint32_t vB[WH];
#pragma unroll
        for (int r = 0; r < WH; ++r) vB[r] = 0u;
        if (okB && yB - sy >= 0 && yB + sy < plB.Hs) load_tile<WH>(plB, xB, yB, lane, vB);
        // compute tile A
        const int x = xA + 2 * lane;
        uint64_t c0 = 0ull, c1 = 0ull;
        if (yA - sy >= 0 && yA + sy < plA.Hs) {
#pragma unroll
            for (int r = 0; r < WH; ++r) store_quad(vA[r], st.even + r * kWordsMax, st.odd + r * kWordsMax, lane);
            __syncwarp();
            tile_codes<WW, WH>(st, lane, a.p.sentinel, c0, c1);
            if (x - sx < 0 || x + sx >= plA.Ws) c0 = 0ull;
            if (x + 1 - sx < 0 || x + 1 + sx >= plA.Ws) c1 = 0ull;
            __syncwarp();
        }
        store_pair(plA, x, yA, c0, c1);
        plA = plB;
        xA = xB;
        yA = yB;
        okA = okB;
#pragma unroll
        for (int r = 0; r < WH; ++r) vA[r] = vB[r];
    }
}

__global__ void __launch_bounds__(32 * kWarpsPerCta, 4) census_roi_kernel(MatchArgs a)
{
    extern __shared__ __align__(16) uint32_t stage_mem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WarpStage st = warp_stage(stage_mem, warp, a.p.win_h);
    int nf = a.counts_in[0];
    nf = nf < 0 ? 0 : (nf > a.caps.max_frames ? a.caps.max_frames : nf);
    const long long total = (long long)nf * a.ws.bm_frame_words;
    const long long gwarp = (long long)blockIdx.x * kWarpsPerCta + warp;
    const long long nwarps = (long long)gridDim.x * kWarpsPerCta;
    TileCursor c;
    c.w = gwarp - nwarps;
    c.bits = 0u;
    const int ww = a.p.win_w, wh = a.p.win_h;
    if (ww == 9 && wh == 7) {
        roi_stream<9, 7>(a, st, c, nwarps, total, lane);
    } else if (ww == 7 && wh == 7) {
        roi_stream<7, 7>(a, st, c, nwarps, total, lane);
    } else if (ww == 5 && wh == 5) {
        roi_stream<5, 5>(a, st, c, nwarps, total, lane);
    } else {
        int x0, y;
        while (next_tile(a, c, nwarps, total, lane, x0, y))
            census_tile<0, 0>(c.pl, x0, y, ww, wh, a.p.sentinel, st);
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
    pl.vec_load = (k == 1 || k == 2) && (pitch % 4 == 0) && ((reinterpret_cast<uintptr_t>(img) & 7u) == 0);
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
