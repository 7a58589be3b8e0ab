// census.cu -- census transform kernels (Sec. 4.3.1, Algorithm 1).
//
// Codes on the grid I_k(x, y) = I(k x, k y) (k = 1 is the image itself; k > 1
// is the multi-resolution census of Sec. 4.3.1 taken by decimation).  Bits
// follow the raster order of the window (row j outer, column i inner), first
// neighbour in the highest comparison bit, with the optional sentinel above
// them; pixels whose window leaves the grid get 0.
//
// Fixed windows (5x5, 7x7, 9x7) use census4: four pixels per lane, compares on
// the integer multiply-add pipe, rows loaded straight into registers.  The
// full-image kernel (ctm_census_build) gives a half-warp a 64-pixel row tile;
// the region-of-interest kernel of the matching path gives eight lanes a
// 32-pixel tile from the list of tiles the planner marked.  Other windows use
// a warp per 64-pixel tile, staging the window rows in shared memory as fp16
// bit patterns 0x6400 | v (exactly 1024 + v, so fp16 order is pixel order) and
// comparing two pixels per __hgt2_mask.
#include <cuda_fp16.h>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

constexpr int kTile = 64;                          // pixels per warp tile of the full-image kernels
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


// ---------------------------------------------------------------------------
// Fixed windows (5x5, 7x7, 9x7): four pixels per lane.
//
// Lane l of a tile's lane group owns pixels x .. x+3 (x = x0 + 4 l).  It
// loads the twelve pixels I_k(x-4 .. x+7) of every window row straight into
// registers (three 32-bit loads at k = 1, three 64-bit loads compacted with
// PRMT at k = 2; adjacent lanes share bytes through L1) and forms the eleven
// words (b[t], b[t+1]) of pixel pairs in registers, so no shared
// memory is involved.  Pixel pairs (x, x+1) and (x+2, x+3) are compared two at
// a time in the 16-bit halves of a word (codes4).

// Pixels xs .. xs+3 of a row at k = 1 (one aligned word; xs is a multiple of 4):
// 0 where the word lies outside [0, W), bytes where it straddles W.
__device__ __forceinline__ uint32_t word_k1(const uint8_t *row, int xs, int W)
{
    if (xs >= 0 && xs + 4 <= W) return __ldg(reinterpret_cast<const uint32_t *>(row + xs));
    if (xs + 4 <= 0 || xs >= W) return 0u;
    uint32_t w = 0u;
    for (int t = 0; t < 4; ++t) {
        const int xt = xs + t;
        if (xt >= 0 && xt < W) w |= (uint32_t)__ldg(row + xt) << (8 * t);
    }
    return w;
}

// Decimated pixels xs .. xs+3 of a row at k = 2 (source bytes 2 xs .. 2 xs + 7,
// one aligned 8-byte word compacted with PRMT): 0 outside the grid [0, Ws),
// bytes where the word straddles the source row end W.
__device__ __forceinline__ uint32_t word_k2(const uint8_t *row, int xs, int W, int Ws)
{
    if (xs >= 0 && 2 * xs + 8 <= W) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(row + 2 * xs));
        return __byte_perm(u.x, u.y, 0x6420);
    }
    if (xs + 4 <= 0 || xs >= Ws) return 0u;
    uint32_t w = 0u;
    for (int t = 0; t < 4; ++t) {
        const int xt = xs + t;
        if (xt >= 0 && xt < Ws) w |= (uint32_t)__ldg(row + 2 * xt) << (8 * t);
    }
    return w;
}

// Twelve pixels I_k(x - 4 .. x + 7) of grid row `yr` for this lane, as three
// little-endian words; pixels outside the grid read as 0 (they only feed
// pixels whose codes are zeroed).  Lanes whose twelve pixels lie inside a
// word-aligned image take word loads, the others (image borders, other
// decimations or alignments) byte loads.
__device__ __forceinline__ void load_row12(const PlaneDesc &d, bool inside, int x, int yr, uint32_t (&v)[3])
{
    if (inside && d.k == 1) {
        const uint32_t *q = reinterpret_cast<const uint32_t *>(d.img + (long long)yr * d.pitch + (x - 4));
        v[0] = __ldg(q);
        v[1] = __ldg(q + 1);
        v[2] = __ldg(q + 2);
    } else if (inside) {  // k == 2: every other source byte
        const uint2 *q = reinterpret_cast<const uint2 *>(d.img + 2LL * yr * d.pitch + 2 * (x - 4));
        const uint2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
        v[0] = __byte_perm(a.x, a.y, 0x6420);
        v[1] = __byte_perm(b.x, b.y, 0x6420);
        v[2] = __byte_perm(c.x, c.y, 0x6420);
    } else {
        const uint8_t *row = d.img + (long long)d.k * yr * d.pitch;
        uint32_t w[3] = {0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 12; ++t) {
            const int xs = x - 4 + t;
            const uint32_t b = (xs >= 0 && xs < d.Ws) ? (uint32_t)__ldg(row + (long long)d.k * xs) : 0u;
            w[t >> 2] |= b << (8 * (t & 3));
        }
        v[0] = w[0];
        v[1] = w[1];
        v[2] = w[2];
    }
}

// Codes of the four pixels x .. x+3 of a lane (bit layout as tile_codes) from
// its window rows: row(j, v) gives the twelve pixels I_k(x - 4 .. x + 7) of
// window row j as three little-endian words (row(sy, v) first, for the centre
// pixels).
//
// The compares run on the integer multiply-add pipe: with both pixels of a
// pair in the two 16-bit halves of a word w (plain values, upper bytes zero),
// e = w * 2^s + K_s, K_s = (2^16 - 2^(8+s) - 1 - c 2^s) per half, is per half
// the complement of 2^(8+s) + (c - nb) 2^s, which lies in [1, 2^16) for
// s <= 7; so no carry crosses the halves and bit 8 + s of each half is
// [nb > c].  Code bit p = 8 a + s is taken from bit 8 + s (and 24 + s) of e
// into accumulator a with one LOP3; accumulator a ends up holding code byte a
// of the low pixel in its byte 1 and of the high pixel in its byte 3.
template <int WW, int WH, typename RowFn>
__device__ __forceinline__ void codes4(RowFn row, int sentinel, uint64_t (&c)[4])
{
    constexpr int sx = WW / 2, sy = WH / 2;
    constexpr int n = WW * WH;
    constexpr int OFF = 4 - sx;  // byte index of the window's left column for pixel x
    uint32_t vc[3];
    row(sy, vc);
    uint32_t accA[8], accB[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) accA[q] = accB[q] = 0u;
    if (sentinel) {
        accA[n >> 3] = (0x100u << (n & 7)) | (0x1000000u << (n & 7));
        accB[n >> 3] = accA[n >> 3];
    }
    const uint32_t cA = __byte_perm(vc[1], 0u, 0x4140);  // pixels x, x+1
    const uint32_t cB = __byte_perm(vc[1], 0u, 0x4342);  // pixels x+2, x+3
    uint32_t KA[8], KB[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t h = 0x10000u - (0x100u << q) - 1u;
        KA[q] = (h | (h << 16)) - (cA << q);
        KB[q] = (h | (h << 16)) - (cB << q);
    }
#pragma unroll
    for (int j = 0; j < WH; ++j) {
        uint32_t v[3];
        row(j, v);
        // w[t] = (b[t], b[t+1]) in the two halves, t = 0 .. 10
        uint32_t w[11];
        const uint32_t s1 = __funnelshift_r(v[0], v[1], 8);  // b1 .. b4
        const uint32_t s2 = __funnelshift_r(v[1], v[2], 8);  // b5 .. b8
        w[0] = __byte_perm(v[0], 0u, 0x4140);
        w[1] = __byte_perm(s1, 0u, 0x4140);
        w[2] = __byte_perm(v[0], 0u, 0x4342);
        w[3] = __byte_perm(s1, 0u, 0x4342);
        w[4] = __byte_perm(v[1], 0u, 0x4140);
        w[5] = __byte_perm(s2, 0u, 0x4140);
        w[6] = __byte_perm(v[1], 0u, 0x4342);
        w[7] = __byte_perm(s2, 0u, 0x4342);
        w[8] = __byte_perm(v[2], 0u, 0x4140);
        w[9] = __byte_perm(v[2], 0u, 0x4241);
        w[10] = __byte_perm(v[2], 0u, 0x4342);
#pragma unroll
        for (int i = 0; i < WW; ++i) {
            const int p = n - 1 - (j * WW + i);  // code bit of this window offset
            const int q = p & 7;
            const uint32_t pos = (0x100u << q) | (0x1000000u << q);
            accA[p >> 3] |= (w[OFF + i] * (1u << q) + KA[q]) & pos;
            accB[p >> 3] |= (w[OFF + i + 2] * (1u << q) + KB[q]) & pos;
        }
    }
    uint32_t tA[4], tB[4];  // code bytes (2q, 2q+1) of the low pixel, then of the high pixel
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        tA[q] = __byte_perm(accA[2 * q], accA[2 * q + 1], 0x7351);
        tB[q] = __byte_perm(accB[2 * q], accB[2 * q + 1], 0x7351);
    }
    c[0] = ((uint64_t)__byte_perm(tA[2], tA[3], 0x5410) << 32) | __byte_perm(tA[0], tA[1], 0x5410);
    c[1] = ((uint64_t)__byte_perm(tA[2], tA[3], 0x7632) << 32) | __byte_perm(tA[0], tA[1], 0x7632);
    c[2] = ((uint64_t)__byte_perm(tB[2], tB[3], 0x5410) << 32) | __byte_perm(tB[0], tB[1], 0x5410);
    c[3] = ((uint64_t)__byte_perm(tB[2], tB[3], 0x7632) << 32) | __byte_perm(tB[0], tB[1], 0x7632);
}

// codes4 with the compares in packed fp16 (census mode 2).  Grid pixels are
// exact fp16 integers 1024 + v (bit pattern 0x6400 | v), two per register, as
// the spread words of codes4 with 0x64 in place of the zero bytes.  One compare
// pair is one packed fused multiply-add with saturation, sat(nb * 1 - c): 1.0
// where nb > c, else +0.0 -- exact, as every operand and difference is a small
// integer.  A window row's compares accumulate as acc * 2 + r (fp16, exact below
// 1024; a row holds at most 9 bits, first neighbour highest); adding 1024 to a
// row's sum puts its bits in the low bits of each half, from where they go to
// their code bits.  Both operations run on the FMA pipe, which leaves the ALU
// pipe the byte spreading and the code assembly.
template <int WW, int WH, typename RowFn>
__device__ __forceinline__ void codes4_h(RowFn row, int sentinel, uint64_t (&c)[4])
{
    constexpr int sy = WH / 2;
    constexpr int n = WW * WH;
    constexpr int OFF = 4 - WW / 2;  // byte index of the window's left column for pixel x
    static_assert(WW <= 10, "a window row's bits must stay below 1024");
    const uint32_t H = 0x64646464u;
    uint32_t vc[3];
    row(sy, vc);
    // -(1024 + c) for the centre pixels (x, x+1) and (x+2, x+3)
    const uint32_t nA = __byte_perm(vc[1], H, 0x4140) ^ 0x80008000u;
    const uint32_t nB = __byte_perm(vc[1], H, 0x4342) ^ 0x80008000u;
    const __half2 one2 = __floats2half2_rn(1.0f, 1.0f), two2 = __floats2half2_rn(2.0f, 2.0f);
    const __half2 bias2 = __floats2half2_rn(1024.0f, 1024.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = 0ull;
#pragma unroll
    for (int j = 0; j < WH; ++j) {
        uint32_t v[3];
        row(j, v);
        uint32_t w[11];
        const uint32_t s1 = __funnelshift_r(v[0], v[1], 8);  // b1 .. b4
        const uint32_t s2 = __funnelshift_r(v[1], v[2], 8);  // b5 .. b8
        w[0] = __byte_perm(v[0], H, 0x4140);
        w[1] = __byte_perm(s1, H, 0x4140);
        w[2] = __byte_perm(v[0], H, 0x4342);
        w[3] = __byte_perm(s1, H, 0x4342);
        w[4] = __byte_perm(v[1], H, 0x4140);
        w[5] = __byte_perm(s2, H, 0x4140);
        w[6] = __byte_perm(v[1], H, 0x4342);
        w[7] = __byte_perm(s2, H, 0x4342);
        w[8] = __byte_perm(v[2], H, 0x4140);
        w[9] = __byte_perm(v[2], H, 0x4241);
        w[10] = __byte_perm(v[2], H, 0x4342);
        __half2 aA, aB;
#pragma unroll
        for (int i = 0; i < WW; ++i) {
            const __half2 rA = __hfma2_sat(as_h2(w[OFF + i]), one2, as_h2(nA));
            const __half2 rB = __hfma2_sat(as_h2(w[OFF + i + 2]), one2, as_h2(nB));
            aA = i == 0 ? rA : __hfma2(aA, two2, rA);
            aB = i == 0 ? rB : __hfma2(aB, two2, rB);
        }
        const __half2 hA = __hadd2(aA, bias2), hB = __hadd2(aB, bias2);
        const uint32_t uA = *reinterpret_cast<const uint32_t *>(&hA);
        const uint32_t uB = *reinterpret_cast<const uint32_t *>(&hB);
        constexpr uint32_t m = (1u << WW) - 1u;
        const int p_lo = n - WW * (j + 1);  // code bit of the row's last neighbour
        c[0] |= (uint64_t)(uA & m) << p_lo;
        c[1] |= (uint64_t)((uA >> 16) & m) << p_lo;
        c[2] |= (uint64_t)(uB & m) << p_lo;
        c[3] |= (uint64_t)((uB >> 16) & m) << p_lo;
    }
    if (sentinel) {
#pragma unroll
        for (int q = 0; q < 4; ++q) c[q] |= 1ull << n;
    }
}

// Store the codes of pixels x .. x+3 of grid row y (zero where the window leaves
// the grid, or for the whole row when `active` is false).
template <int WW>
__device__ __forceinline__ void store4(const PlaneDesc &d, int x, int y, bool active, uint64_t (&c)[4])
{
    constexpr int sx = WW / 2;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (!active || x + q - sx < 0 || x + q + sx >= d.Ws) c[q] = 0ull;
    uint64_t *dst = d.out + (long long)y * d.opitch + x;
    if (x + 3 < d.Ws && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
        reinterpret_cast<ulonglong2 *>(dst)[0] = make_ulonglong2(c[0], c[1]);
        reinterpret_cast<ulonglong2 *>(dst)[1] = make_ulonglong2(c[2], c[3]);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (x + q < d.Ws) dst[q] = c[q];
    }
}

// Codes of pixels x .. x+3 of row y of plane d (4 consecutive pixels per lane;
// bit layout as tile_codes), stored to the plane; `ok` false: this lane has
// no tile and stores nothing.  All 32 lanes of the warp must call it together.
// All window rows are loaded into registers before the first is used.
template <int WW, int WH, bool F16 = false>
__device__ __forceinline__ void census4(const PlaneDesc &d, int x0, int y, int hl, bool ok, int sentinel)
{
    constexpr int sy = WH / 2;
    const unsigned full = 0xffffffffu;
    const int x = x0 + 4 * hl;
    const bool active = ok && y - sy >= 0 && y + sy < d.Hs;
    // one load scheme for the whole warp where possible (a uniform branch, so
    // the other schemes are not executed predicated off): straight word loads
    // when every lane's twelve pixels lie inside the row; else, at image
    // borders, word loads where a word lies inside, 0 where it lies outside (it
    // only feeds pixels whose codes are zeroed) and bytes where it straddles the
    // end of a row whose width is not a multiple of the word
    const bool inside = d.vec_load && x >= 4 && (d.k == 1 ? x + 8 <= d.W : 2 * x + 16 <= d.W);
    uint32_t rows[WH][3];
    if (__all_sync(full, !active || (inside && d.k == 1))) {
        if (active) {
            const uint8_t *p = d.img + (long long)(y - sy) * d.pitch + (x - 4);
#pragma unroll
            for (int r = 0; r < WH; ++r) {
                const uint32_t *q = reinterpret_cast<const uint32_t *>(p + (long long)r * d.pitch);
                rows[r][0] = __ldg(q);
                rows[r][1] = __ldg(q + 1);
                rows[r][2] = __ldg(q + 2);
            }
        }
    } else if (__all_sync(full, !active || (inside && d.k == 2))) {
        if (active) {
            const uint8_t *p = d.img + 2LL * (y - sy) * d.pitch + 2 * (x - 4);
#pragma unroll
            for (int r = 0; r < WH; ++r) {
                const uint2 *q = reinterpret_cast<const uint2 *>(p + 2LL * r * d.pitch);
                const uint2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
                rows[r][0] = __byte_perm(a.x, a.y, 0x6420);
                rows[r][1] = __byte_perm(b.x, b.y, 0x6420);
                rows[r][2] = __byte_perm(c.x, c.y, 0x6420);
            }
        }
    } else if (__all_sync(full, !active || (d.vec_load && d.k == 1))) {
        if (active) {
            const uint8_t *p = d.img + (long long)(y - sy) * d.pitch;
#pragma unroll
            for (int r = 0; r < WH; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) rows[r][q] = word_k1(p + (long long)r * d.pitch, x - 4 + 4 * q, d.W);
        }
    } else if (__all_sync(full, !active || (d.vec_load && d.k == 2))) {
        if (active) {
            const uint8_t *p = d.img + 2LL * (y - sy) * d.pitch;
#pragma unroll
            for (int r = 0; r < WH; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    rows[r][q] = word_k2(p + 2LL * r * d.pitch, x - 4 + 4 * q, d.W, d.Ws);
        }
    } else if (active) {
#pragma unroll
        for (int r = 0; r < WH; ++r) load_row12(d, inside, x, y - sy + r, rows[r]);
    }
    uint64_t c[4] = {0ull, 0ull, 0ull, 0ull};
    if (active) {
        auto row = [&](int j, uint32_t (&v)[3]) { v[0] = rows[j][0]; v[1] = rows[j][1]; v[2] = rows[j][2]; };
        if constexpr (F16)
            codes4_h<WW, WH>(row, sentinel, c);
        else
            codes4<WW, WH>(row, sentinel, c);
    }
    if (ok) store4<WW>(d, x, y, active, c);
}

__device__ __forceinline__ PlaneDesc desc_of(const Plane &pl)
{
    PlaneDesc d;
    d.img = pl.img;
    d.out = pl.out;
    d.W = pl.W;
    d.pitch = pl.pitch;
    d.k = pl.k;
    d.Ws = pl.Ws;
    d.Hs = pl.Hs;
    d.opitch = (int)pl.opitch;
    d.vec_load = pl.vec_load;
    d.pad = 0;
    return d;
}

// Full image, fixed window: half-warp h of CTA (bx, by) takes tile bx of row by * 16 + h.
template <int WW, int WH>
__global__ void __launch_bounds__(256) census_full4_kernel(Plane pl, int sentinel)
{
    const int y = blockIdx.y * 16 + (threadIdx.x >> 4);
    // every lane reaches census4 (its load scheme is chosen warp-wide)
    census4<WW, WH>(desc_of(pl), blockIdx.x * kTile, y, threadIdx.x & 15, y < pl.Hs, sentinel);
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

// Region of interest.  The planner marks, per plane row, the 32-pixel tiles the
// search reads (bitmap, one bit per tile).  tile_list_kernel compacts the
// marks into a dense list (one packed entry per tile, row-major within each
// 256-word chunk of the bitmap) and clears the bitmap for the next call; the
// census kernels then take tiles from the list, so every warp gets the same
// share of work and no warp scans empty bitmap words.
//
// Entry: bits 0-9 tile (x0 / 32), 10-25 row, 26-27 plane (L1, R1, Lk, Rk), 28- frame.
__device__ __forceinline__ unsigned long long tile_entry(int f, int q, int y, int tile)
{
    return ((unsigned long long)f << 28) | ((unsigned long long)q << 26) | ((unsigned long long)y << 10) |
           (unsigned long long)tile;
}

// Plane descriptor, tile origin and row of a list entry; false if the tile lies
// outside its plane.
__device__ __forceinline__ bool tile_of(const MatchArgs &a, unsigned long long e, PlaneDesc &d, int &x0, int &y)
{
    const int tile = (int)(e & 1023u);
    y = (int)((e >> 10) & 0xffffu);
    d = a.ws.planes[e >> 26];  // frame * 4 + plane
    x0 = tile * kCensusTilePx;
    return x0 < d.Ws && y < d.Hs;
}

__global__ void __launch_bounds__(256) tile_list_kernel(MatchArgs a)
{
    __shared__ int warp_tot[8];
    __shared__ int s_base;
    int nf = a.counts_in[0];
    nf = nf < 0 ? 0 : (nf > a.caps.max_frames ? a.caps.max_frames : nf);
    const long long total = (long long)nf * a.ws.bm_frame_words;
    const long long w0 = (long long)blockIdx.x * blockDim.x;
    if (w0 >= total) return;  // uniform per CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long w = w0 + tid;
    uint32_t bits = 0u;
    if (w < total) {
        bits = a.ws.bitmap[w];
        if (bits) a.ws.bitmap[w] = 0u;  // consumed: clear for the next call
    }
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int wpre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        wpre += i < warp ? warp_tot[i] : 0;
        tot += warp_tot[i];
    }
    if (tid == 0) s_base = tot ? atomicAdd(&a.ws.counts->n_tiles, tot) : 0;
    __syncthreads();
    if (bits == 0u) return;
    const int f = (int)(w / a.ws.bm_frame_words);
    int r = (int)(w - (long long)f * a.ws.bm_frame_words);
    int q = 0;
    while (q < 3 && r >= a.ws.bm_plane_off[q + 1]) ++q;
    r -= a.ws.bm_plane_off[q];
    const int y = r / a.ws.bm_row_words[q];
    const int wi = r - y * a.ws.bm_row_words[q];
    int pos = s_base + wpre + incl - cnt;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        a.ws.tiles[pos++] = tile_entry(f, q, y, wi * 32 + b);
    }
}

// Fixed windows: warp w takes list entries kPer p .. kPer p + kPer - 1 (p = w,
// w + warps, ...), one per group of kLanes lanes, so all groups run the same
// instructions in lockstep.  MODE: 0 = 4 CTAs per SM (64 registers),
// otherwise 3 CTAs per SM.
template <int WW, int WH, int MODE>
__global__ void __launch_bounds__(256, MODE == 1 ? 3 : 4) census_roi4_kernel(MatchArgs a)
{
    constexpr int kLanes = kCensusTilePx / 4;  // lanes per tile (4 pixels each)
    constexpr int kPer = 32 / kLanes;          // tiles per warp step
    const int lane = threadIdx.x & 31, hl = lane % kLanes;
    const int n = a.ws.counts->n_tiles;
    const int nsteps = (n + kPer - 1) / kPer;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int sentinel = a.p.sentinel;
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < nsteps; p += nw) {
        const int t = kPer * p + lane / kLanes;
        PlaneDesc d;
        int x0, y;
        const bool ok = tile_of(a, a.ws.tiles[t < n ? t : kPer * p], d, x0, y) && t < n;
        census4<WW, WH, MODE == 2>(d, x0, y, hl, ok, sentinel);
    }
}

// Any other window: a warp per listed tile, rows staged in shared memory.
__global__ void __launch_bounds__(32 * kWarpsPerCta) census_roi_kernel(MatchArgs a)
{
    extern __shared__ __align__(16) uint32_t stage_mem[];
    const int warp = threadIdx.x >> 5;
    const WarpStage st = warp_stage(stage_mem, warp, a.p.win_h);
    const int n = a.ws.counts->n_tiles;
    const int nw = gridDim.x * kWarpsPerCta;
    for (int t = blockIdx.x * kWarpsPerCta + warp; t < n; t += nw) {
        PlaneDesc d;
        int x0, y;
        if (!tile_of(a, a.ws.tiles[t], d, x0, y)) continue;
        Plane pl;
        pl.img = d.img;
        pl.W = d.W;
        pl.H = 0;
        pl.pitch = d.pitch;
        pl.k = d.k;
        pl.Ws = d.Ws;
        pl.Hs = d.Hs;
        pl.out = d.out;
        pl.opitch = d.opitch;
        pl.vec_ok = 1;  // workspace planes: 256-byte aligned, pitch a multiple of 32
        pl.vec_load = d.vec_load;
        census_tile<0, 0>(pl, x0, y, a.p.win_w, a.p.win_h, a.p.sentinel, st);
    }
}

template <typename K>
int resident_ctas(K kernel, int threads, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
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
    const dim3 grid4(ceil_div_nn(pl.Ws, kTile), ceil_div_nn(pl.Hs, 16));
    if (win_w == 9 && win_h == 7) {
        census_full4_kernel<9, 7><<<grid4, 256, 0, s>>>(pl, sentinel);
    } else if (win_w == 7 && win_h == 7) {
        census_full4_kernel<7, 7><<<grid4, 256, 0, s>>>(pl, sentinel);
    } else if (win_w == 5 && win_h == 5) {
        census_full4_kernel<5, 5><<<grid4, 256, 0, s>>>(pl, sentinel);
    } else {
        dim3 grid(ceil_div_nn(pl.Ws, kTile), ceil_div_nn(pl.Hs, kWarpsPerCta));
        census_full_kernel<<<grid, 32 * kWarpsPerCta, census_smem_bytes(win_h), s>>>(pl, win_w, win_h, sentinel);
    }
    return cudaGetLastError();
}

template <int WW, int WH>
static int roi4_ctas(int mode)
{
    static const int n0 = resident_ctas(census_roi4_kernel<WW, WH, 0>, 256, 0);
    static const int n1 = resident_ctas(census_roi4_kernel<WW, WH, 1>, 256, 0);
    static const int n2 = resident_ctas(census_roi4_kernel<WW, WH, 2>, 256, 0);
    return mode == 0 ? n0 : (mode == 1 ? n1 : n2);
}

int census_roi_ctas_per_sm(int win_w, int win_h, int mode)
{
    if (win_w == 9 && win_h == 7) return roi4_ctas<9, 7>(mode);
    if (win_w == 7 && win_h == 7) return roi4_ctas<7, 7>(mode);
    if (win_w == 5 && win_h == 5) return roi4_ctas<5, 5>(mode);
    static const int ng = resident_ctas(census_roi_kernel, 32 * kWarpsPerCta, census_smem_bytes(kMaxWin));
    return ng;
}

template <int WW, int WH>
static void launch_roi4(const MatchArgs &a, int grid, cudaStream_t s)
{
    if (a.census_mode == 0)
        census_roi4_kernel<WW, WH, 0><<<grid, 256, 0, s>>>(a);
    else if (a.census_mode == 1)
        census_roi4_kernel<WW, WH, 1><<<grid, 256, 0, s>>>(a);
    else
        census_roi4_kernel<WW, WH, 2><<<grid, 256, 0, s>>>(a);
}

cudaError_t launch_census_roi(const MatchArgs &a, int sm_count, cudaStream_t s)
{
    const long long words = (long long)a.caps.max_frames * a.ws.bm_frame_words;
    const int list_grid = (int)((words + 255) / 256);
    if (list_grid > 0) tile_list_kernel<<<list_grid, 256, 0, s>>>(a);
    const int ww = a.p.win_w, wh = a.p.win_h;
    const int grid = sm_count * census_roi_ctas_per_sm(ww, wh, a.census_mode);
    // the fixed windows' kernel reads grid columns [x0 - 4, x0 + 36) of a tile, the
    // generic one [x0 - 8, x0 + 76): census_reach_left/right, which the mapped
    // entry point's gather copies, follow census_fixed_window's choice made here
    if (!census_fixed_window(ww, wh)) {
        census_roi_kernel<<<grid, 32 * kWarpsPerCta, census_smem_bytes(wh), s>>>(a);
    } else if (ww == 9 && wh == 7) {
        launch_roi4<9, 7>(a, grid, s);
    } else if (ww == 7 && wh == 7) {
        launch_roi4<7, 7>(a, grid, s);
    } else {
        launch_roi4<5, 5>(a, grid, s);
    }
    return cudaGetLastError();
}

}  // namespace ctm
