// census.cu -- census transform kernels (Sec. 4.3.1, Algorithm 1).
//
// One CTA computes a 32 x 16 tile of codes.  The tile's source patch with its
// window halo is staged in shared memory once (Algorithm 1's shared patch), read
// from the image at stride k when the census is taken on the decimated grid
// I_k(x, y) = I(k x, k y) (the multi-resolution census of Sec. 4.3.1).  Codes
// are built in raster window order, first neighbour in the highest comparison
// bit, after an optional leading sentinel 1; pixels whose window leaves the
// grid are stored as 0.
#include "ctm_internal.cuh"

namespace ctm {
namespace {

struct CensusJob {
    const uint8_t *img;
    int W, H, pitch, k;
    uint64_t *out;
    long long opitch;
};

constexpr int kPatchW = kCensusTileW + kMaxWin - 1;
constexpr int kPatchH = kCensusTileH + kMaxWin - 1;

// Window bits of one pixel from the shared patch; `pc` points at its centre.
template <int WW, int WH>
__device__ __forceinline__ uint64_t census_code_fixed(const uint8_t *pc, int pw, int sentinel)
{
    constexpr int sx = WW / 2, sy = WH / 2;
    const unsigned centre = pc[0];
    uint64_t c = sentinel ? 1ull : 0ull;
#pragma unroll
    for (int j = -sy; j <= sy; ++j) {
#pragma unroll
        for (int i = -sx; i <= sx; ++i) {
            const unsigned v = pc[j * pw + i];
            c = (c << 1) | (uint64_t)(v > centre);
        }
    }
    return c;
}

__device__ __forceinline__ uint64_t census_code_any(const uint8_t *pc, int pw, int win_w,
                                                    int win_h, int sentinel)
{
    const int sx = win_w / 2, sy = win_h / 2;
    const unsigned centre = pc[0];
    uint64_t c = sentinel ? 1ull : 0ull;
    for (int j = -sy; j <= sy; ++j)
        for (int i = -sx; i <= sx; ++i) {
            const unsigned v = pc[j * pw + i];
            c = (c << 1) | (uint64_t)(v > centre);
        }
    return c;
}

template <int WW, int WH>
__device__ void census_tile(const CensusJob &job, int win_w, int win_h, int sentinel,
                            int tile_x, int tile_y, uint8_t *patch)
{
    const int sx = win_w / 2, sy = win_h / 2;
    const int Ws = ceil_div_nn(job.W, job.k), Hs = ceil_div_nn(job.H, job.k);
    const int tx0 = tile_x * kCensusTileW, ty0 = tile_y * kCensusTileH;
    if (tx0 >= Ws || ty0 >= Hs) return;  // uniform over the CTA
    const int PW = kCensusTileW + 2 * sx, PH = kCensusTileH + 2 * sy;
    for (int i = threadIdx.x; i < PW * PH; i += blockDim.x) {
        const int r = i / PW, c = i - r * PW;
        const int xs = tx0 - sx + c, ys = ty0 - sy + r;
        uint8_t v = 0;
        if (xs >= 0 && xs < Ws && ys >= 0 && ys < Hs)
            v = job.img[(long long)job.k * ys * job.pitch + (long long)job.k * xs];
        patch[r * PW + c] = v;
    }
    __syncthreads();
    const int lx = threadIdx.x & 31;
    for (int ly = threadIdx.x >> 5; ly < kCensusTileH; ly += blockDim.x >> 5) {
        const int x = tx0 + lx, y = ty0 + ly;
        if (x >= Ws || y >= Hs) continue;
        uint64_t c = 0;
        if (x - sx >= 0 && x + sx < Ws && y - sy >= 0 && y + sy < Hs) {
            const uint8_t *pc = patch + (ly + sy) * PW + (lx + sx);
            if (WW > 0)
                c = census_code_fixed<WW, WH>(pc, PW, sentinel);
            else
                c = census_code_any(pc, PW, win_w, win_h, sentinel);
        }
        job.out[(long long)y * job.opitch + x] = c;
    }
}

__device__ void census_tile_dispatch(const CensusJob &job, int win_w, int win_h, int sentinel,
                                     int tx, int ty, uint8_t *patch)
{
    if (win_w == 9 && win_h == 7)
        census_tile<9, 7>(job, win_w, win_h, sentinel, tx, ty, patch);
    else if (win_w == 7 && win_h == 7)
        census_tile<7, 7>(job, win_w, win_h, sentinel, tx, ty, patch);
    else if (win_w == 5 && win_h == 5)
        census_tile<5, 5>(job, win_w, win_h, sentinel, tx, ty, patch);
    else
        census_tile<0, 0>(job, win_w, win_h, sentinel, tx, ty, patch);
}

__global__ void __launch_bounds__(256) census_single_kernel(CensusJob job, int win_w, int win_h,
                                                            int sentinel)
{
    __shared__ uint8_t patch[kPatchW * kPatchH];
    census_tile_dispatch(job, win_w, win_h, sentinel, blockIdx.x, blockIdx.y, patch);
}

// z = frame * 4 + {0: left full, 1: right full, 2: left decimated, 3: right decimated}
__global__ void __launch_bounds__(256) census_batch_kernel(MatchArgs a)
{
    __shared__ uint8_t patch[kPatchW * kPatchH];
    const int f = blockIdx.z >> 2, which = blockIdx.z & 3;
    int nf = a.counts_in[0];
    nf = nf < 0 ? 0 : (nf > a.caps.max_frames ? a.caps.max_frames : nf);
    if (f >= nf) return;
    if (which >= 2 && a.p.close_factor == 1) return;  // CLOSE boxes then use the full planes
    const ctm_frame fr = a.frames[f];
    if (fr.width > a.caps.max_width || fr.height > a.caps.max_height || fr.width < 1 ||
        fr.height < 1 || fr.pitch < fr.width)
        return;  // rejected frame: its boxes are flagged by the planner
    CensusJob job;
    job.img = (which & 1) ? fr.right : fr.left;
    job.W = fr.width;
    job.H = fr.height;
    job.pitch = fr.pitch;
    job.k = which < 2 ? 1 : a.p.close_factor;
    uint64_t *base = a.ws.census + (long long)f * a.ws.frame_stride;
    if (which < 2) {
        job.out = base + which * a.ws.plane1_elems;
        job.opitch = a.ws.pitch1;
    } else {
        job.out = base + 2 * a.ws.plane1_elems + (which - 2) * a.ws.planek_elems;
        job.opitch = a.ws.pitchk;
    }
    census_tile_dispatch(job, a.p.win_w, a.p.win_h, a.p.sentinel, blockIdx.x, blockIdx.y, patch);
}

}  // namespace

cudaError_t launch_census_single(const uint8_t *img, int W, int H, int pitch, int k, int win_w,
                                 int win_h, int sentinel, uint64_t *out, long long out_pitch,
                                 cudaStream_t s)
{
    CensusJob job{img, W, H, pitch, k, out, out_pitch};
    const int Ws = ceil_div_nn(W, k), Hs = ceil_div_nn(H, k);
    dim3 grid(ceil_div_nn(Ws, kCensusTileW), ceil_div_nn(Hs, kCensusTileH));
    census_single_kernel<<<grid, 256, 0, s>>>(job, win_w, win_h, sentinel);
    return cudaGetLastError();
}

cudaError_t launch_census_batch(const MatchArgs &a, cudaStream_t s)
{
    dim3 grid(ceil_div_nn(a.caps.max_width, kCensusTileW),
              ceil_div_nn(a.caps.max_height, kCensusTileH), a.caps.max_frames * 4);
    census_batch_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ctm
