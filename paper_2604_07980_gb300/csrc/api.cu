// api.cu -- the C ABI (include/ctm.h): context, workspace and launch sequences.
//
// A match call is six launches on one stream (seven with the two-pass
// matcher): device planning, point sampling with census demand marking, the
// census tile list, census of the listed tiles (both images, both
// resolutions), the matching kernel, and the per-box aggregation that writes
// the outputs.  The batch entry point reads its frame and box counts
// from device memory, so the whole sequence can be captured once into a CUDA
// graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "ctm_internal.cuh"

using namespace ctm;

struct GraphKey {
    const void *frames, *counts, *boxes, *disp, *depth, *flags, *dbg_blocks, *dbg_cf, *dbg_cb, *gather;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

// Sub-batches of the host entry point: the copies of sub-batch g + 1 run
// while sub-batch g is matched.
constexpr int kHostGroups = 4;

struct ctm_ctx {
    int device = 0;
    int sm_count = 0;
    int ctas_per_sm = 0;
    int match_threads = 128;
    ctm_params p{};
    Caps caps{};
    Workspace ws{};
    int nc_stride = 0;
    int strip_cols = 0;
    int strip_rows = 0;
    int census_mode = 0;
    int queue_rounds = 1;
    int match_mode = 0;
    int nd_max = 0;
    int inject_expiry = 0;  // armed by ctm_inject_wait_expiry (tests)
    int split_ways = 0;
    bool maps_ok = false;    // ws.tmaps hold the planes' maps
    int pageable_access = 0; // the device reads pageable host memory (mapped calls need no page-locking)
    void *dev_mem = nullptr;
    size_t dev_bytes = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    // host end-to-end staging (allocated on first use)
    uint8_t *img_dev = nullptr;
    long long img_pitch = 0;
    ctm_box *boxes_dev = nullptr;
    float *disp_dev = nullptr;
    float *depth_dev = nullptr;
    uint8_t *flags_dev = nullptr;
    ctm_frame *frames_host_pinned = nullptr;
    int32_t *counts_host_pinned = nullptr;
    ctm_frame *frames_dev2 = nullptr;
    int32_t *counts_dev2 = nullptr;
    cudaStream_t copy_stream = nullptr;         // host-to-device copies of the sub-batches
    cudaEvent_t host_ev[kHostGroups + 1] = {};  // sub-batch g copied; [kHostGroups]: start
};

namespace {

inline long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

// The driver's tensor-map encoder, through the runtime's entry-point lookup (the
// library does not link the driver library itself); null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

}  // namespace

// Each census plane of each frame slot as a 2-D tensor of uint64 codes (pitch x
// rows of the workspace plane), once per box width of one row of 32, 64, ... 256
// codes: a strip chunk's rows load four at a time by tile::gather4 with the
// narrowest box that holds them.  Columns beyond the pitch and rows beyond the
// workspace plane read as zero; codes between a frame's width and the pitch are
// zeroed by the matcher after landing, as for 1-D copies.
bool ctm::encode_plane_maps(const Workspace &ws, const Caps &caps, int k, CUtensorMap *dev_maps)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !dev_maps || caps.max_frames > kMaxMapFrames) return false;
    std::vector<CUtensorMap> maps((size_t)4 * kBoxClasses * caps.max_frames);
    memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    const long long rows1 = caps.max_height, rowsk = (caps.max_height + k - 1) / k;
    for (int f = 0; f < caps.max_frames; ++f) {
        for (int q = 0; q < 4; ++q) {
            if (k == 1 && q >= 2) continue;  // no decimated planes
            uint64_t *base = ws.census + (long long)f * ws.frame_stride +
                             (q < 2 ? q * ws.plane1_elems : 2 * ws.plane1_elems + (q - 2) * ws.planek_elems);
            const long long pitch = q < 2 ? ws.pitch1 : ws.pitchk;
            const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)(q < 2 ? rows1 : rowsk)};
            const cuuint64_t strides[1] = {(cuuint64_t)pitch * 8u};
            const cuuint32_t estr[2] = {1u, 1u};
            for (int c = 0; c < kBoxClasses; ++c) {
                const cuuint32_t box[2] = {(cuuint32_t)(32 * (c + 1)), 1u};
                if (enc(&maps[((size_t)4 * f + q) * kBoxClasses + c], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base,
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return false;
            }
        }
    }
    if (cudaMemcpy(dev_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Parameter limits of include/ctm.h, plus the shared-memory budget of the
// matcher's strip (shared by ctm_create and ctm_match_boxes_noalloc).
bool ctm::params_valid(const ctm_params &p)
{
    if (p.win_w < 1 || p.win_h < 1 || (p.win_w & 1) == 0 || (p.win_h & 1) == 0) return false;
    if (p.win_w > kMaxWin || p.win_h > kMaxWin) return false;
    if (p.win_w * p.win_h + (p.sentinel ? 1 : 0) > 64) return false;
    if (p.sentinel != 0 && p.sentinel != 1) return false;
    if (p.close_factor < 1 || p.close_factor > 8) return false;
    if (p.far_dmin > p.far_dmax || p.close_dmin > p.close_dmax || p.dy_min > p.dy_max) return false;
    const long long ndy = (long long)p.dy_max - p.dy_min + 1;
    if (((long long)p.far_dmax - p.far_dmin + 1) * ndy > kMaxCand) return false;
    if (((long long)p.close_dmax - p.close_dmin + 1) * ndy > kMaxCand) return false;
    if (p.grid_g < 1 || p.grid_g > kMaxGrid) return false;
    if (p.pts_side < 1 || p.pts_side > kMaxPtsSide) return false;
    if (p.min_pts < 1 || p.fb_tol < 0 || p.agg_nmin < 1) return false;
    if (p.agg_mode != 0 && p.agg_mode != 1) return false;
    if (!(p.trim_frac >= 0.0f && p.trim_frac < 0.5f)) return false;
    if (!(p.agg_tau_d == p.agg_tau_d)) return false;
    if (p.max_occluders < 0 || p.max_occluders > kMaxOcc) return false;
    if (!(p.frontal_crop >= 0.0f && p.frontal_crop <= 1.0f)) return false;
    const int nd_max = std::max(p.far_dmax - p.far_dmin + 1, p.close_dmax - p.close_dmin + 1);
    if ((long long)2 * ndy * default_strip_cols(nd_max) * 8 * 4 > 160 * 1024) return false;
    return true;
}

// Default strip width (one sampled row per piece): the disparity range plus a
// 64-column span of points, at least 128 codes, in multiples of 32; wider
// blocks are chunked.
int ctm::default_strip_cols(int nd_max) { return (int)round_up(std::max(nd_max + 64, 128), 32); }

namespace {

MatchArgs make_args(const ctm_ctx *ctx, const ctm_frame *frames, const int32_t *counts,
                    const ctm_box *boxes, float *disp, float *depth, uint8_t *flags,
                    const ctm_debug *dbg)
{
    MatchArgs a;
    a.ws = ctx->ws;
    a.caps = ctx->caps;
    a.p = ctx->p;
    a.frames = frames;
    a.counts_in = counts;
    a.boxes = boxes;
    a.disp = disp;
    a.depth = depth;
    a.flags = flags;
    a.dbg.blocks = dbg ? dbg->blocks : nullptr;
    a.dbg.cost_f = dbg ? dbg->cost_f : nullptr;
    a.dbg.cost_b = dbg ? dbg->cost_b : nullptr;
    a.nc_stride = ctx->nc_stride;
    a.strip_cols = ctx->strip_cols;
    a.strip_rows = ctx->strip_rows;
    a.queue_rounds = ctx->queue_rounds;
    a.sm_count = ctx->sm_count;
    a.census_mode = ctx->census_mode;
    a.match_mode = ctx->match_mode;
    a.split_ways = ctx->split_ways;
    if (!ctx->maps_ok) a.ws.tmaps = nullptr;
    a.stats_accumulate = 0;
    a.inject_expiry = 0;
    a.gather_src = nullptr;
    return a;
}

// The launch sequence of one match call after the frame descriptors and counts
// are in device memory: planning, census demand marking, census of the marked
// tiles, matching.  direct: launched now, not captured into a graph (an armed
// fault injection applies to such a launch of the fused persistent matcher
// only, and is then disarmed).
int enqueue_match(ctm_ctx *ctx, const MatchArgs &a, int frames_grid, int match_grid, cudaStream_t s,
                  bool plain, int n_boxes_host, bool direct = true)
{
    MatchArgs b = a;
    b.caps.max_frames = std::min(ctx->caps.max_frames, frames_grid);
    if (direct && !plain && ctx->match_mode == 0 && ctx->inject_expiry) {
        b.inject_expiry = 1;
        ctx->inject_expiry = 0;
    }
    cudaError_t e = launch_plan(b, s);
    if (e == cudaSuccess) e = launch_sample(b, s);
    if (e == cudaSuccess && b.gather_src) e = launch_gather(b, ctx->sm_count, s);
    if (e == cudaSuccess) e = launch_census_roi(b, ctx->sm_count, s);
    if (!plain) {
        if (e == cudaSuccess)
            e = ctx->match_mode == 1 ? launch_match_pipe(b, ctx->match_threads, match_grid, s)
                                     : launch_match_persistent(b, ctx->match_threads, match_grid, s);
    } else {
        for (int i = 0; i < n_boxes_host && e == cudaSuccess; ++i)
            e = launch_match_box(b, ctx->match_threads, i, s);
    }
    if (e == cudaSuccess) e = launch_aggregate(b, s);
    return e == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

int set_device(const ctm_ctx *ctx)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CTM_ENODEV;
    if (cur != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return CTM_ENODEV;
    return CTM_OK;
}

}  // namespace

namespace {
// armed by ctm_inject_alloc_failures (tests): allocations to let through, then to fail
std::mutex g_inject_mu;
int g_alloc_skip = 0, g_alloc_fail = 0;
}  // namespace

cudaError_t ctm::dev_alloc(void **ptr, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_inject_mu);
        if (g_alloc_skip > 0) {
            --g_alloc_skip;
        } else if (g_alloc_fail > 0) {
            --g_alloc_fail;
            *ptr = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(ptr, bytes);
}

size_t ctm::context_device_bytes(const ctm_ctx *ctx) { return ctx ? ctx->dev_bytes : 0; }
const int32_t *ctm::context_error_flag(const ctm_ctx *ctx) { return &ctx->ws.stats->error; }

extern "C" {

const char *ctm_status_str(int status)
{
    switch (status) {
    case CTM_OK: return "ok";
    case CTM_EINVAL: return "invalid argument";
    case CTM_ENOMEM: return "out of memory or beyond context capacity";
    case CTM_ECUDA: return "CUDA error";
    case CTM_ENODEV: return "no usable CUDA device";
    case CTM_ETOOBIG: return "request exceeds a fixed limit (no-allocation maxima, server frame size or arena)";
    case CTM_EAGAIN: return "admission queue full, try again";
    case CTM_ETIMEOUT: return "a bounded device wait expired (outputs incomplete)";
    default: return "unknown status";
    }
}

int ctm_default_params(ctm_params *p)
{
    if (!p) return CTM_EINVAL;
    p->win_w = 9;
    p->win_h = 7;
    p->sentinel = 1;
    p->far_side_px = 40;
    p->close_factor = 2;
    p->far_dmin = 0;
    p->far_dmax = 31;
    p->close_dmin = 0;
    p->close_dmax = 127;
    p->dy_min = 0;
    p->dy_max = 0;
    p->grid_g = 4;
    p->pts_side = 16;
    p->min_pts = 16;
    p->fb_tol = 1;
    p->agg_tau_d = 1.0f;
    p->agg_nmin = 6;
    p->agg_mode = 0;
    p->trim_frac = 0.2f;
    p->max_occluders = 16;
    p->frontal_crop = 0.0f;
    return CTM_OK;
}

int ctm_create(ctm_ctx **out, const ctm_params *p, int max_frames, int max_width, int max_height,
               int max_boxes)
{
    if (!out || !p) return CTM_EINVAL;
    *out = nullptr;
    if (!params_valid(*p)) return CTM_EINVAL;
    if (max_frames < 1 || max_frames > 16383 || max_width < 1 || max_height < 1 ||
        max_width > 32768 || max_height > 32768 || max_boxes < 1 || max_boxes > (1 << 22))
        return CTM_EINVAL;
    int dev = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) return CTM_ENODEV;
    if (cudaGetDevice(&dev) != cudaSuccess) return CTM_ENODEV;

    ctm_ctx *ctx = new (std::nothrow) ctm_ctx();
    if (!ctx) return CTM_ENOMEM;
    ctx->device = dev;
    ctx->p = *p;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&ctx->pageable_access, cudaDevAttrPageableMemoryAccess, dev);
    const int slots = p->grid_g * p->grid_g;
    ctx->caps.max_frames = max_frames;
    ctx->caps.max_width = max_width;
    ctx->caps.max_height = max_height;
    ctx->caps.max_boxes = max_boxes;
    ctx->caps.max_blocks = max_boxes * std::max(slots, 1);
    const int ndy = p->dy_max - p->dy_min + 1;
    const int nd_max = std::max(p->far_dmax - p->far_dmin + 1, p->close_dmax - p->close_dmin + 1);
    ctx->nc_stride = nd_max * ndy;
    ctx->nd_max = nd_max;
    ctx->strip_rows = (int)round_up((long long)p->pts_side * ndy, 4);  // gather4 fills rows four at a time
    ctx->strip_cols = default_strip_cols(nd_max);

    // workspace layout (one allocation)
    const long long pitch1 = round_up(max_width, 32);
    const int k = p->close_factor;
    const long long Wk = (max_width + k - 1) / k, Hk = (max_height + k - 1) / k;
    const long long pitchk = k == 1 ? 0 : round_up(Wk, 32);
    const long long plane1 = pitch1 * max_height;
    const long long planek = k == 1 ? 0 : pitchk * Hk;
    const long long frame_stride = 2 * plane1 + 2 * planek;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up(off + bytes, 256); return o; };
    const size_t o_census = take(sizeof(uint64_t) * (size_t)frame_stride * max_frames);
    const size_t o_plans = take(sizeof(BoxPlan) * (size_t)max_boxes);
    const size_t o_occ = take(sizeof(int4) * (size_t)max_boxes * kMaxOcc);
    const size_t o_nblk = take(sizeof(int) * (size_t)max_boxes);
    const size_t o_base = take(sizeof(int) * (size_t)max_boxes);
    const size_t o_blocks = take(sizeof(int2) * (size_t)ctx->caps.max_blocks);
    const size_t o_blkres = take(sizeof(BlockResult) * (size_t)ctx->caps.max_blocks);
    const size_t o_chunk = take(sizeof(ChunkState) * (size_t)ctx->caps.max_blocks);
    const size_t o_tmaps =
        take(max_frames <= kMaxMapFrames ? sizeof(CUtensorMap) * 4 * kBoxClasses * (size_t)max_frames : 0);
    const size_t o_ccost = take(sizeof(int32_t) * (size_t)ctx->caps.max_blocks * ctx->nc_stride);
    const size_t o_geom = take(sizeof(BlockGeom) * (size_t)ctx->caps.max_blocks);
    const size_t o_queue = take(sizeof(int) * (size_t)ctx->caps.max_blocks);
    const size_t o_queue_w = take(sizeof(int) * kQueueClasses * (size_t)ctx->caps.max_blocks);
    const size_t o_sched = take(sizeof(int) * kSchedInts);
    const size_t o_counts = take(sizeof(Counts));
    const size_t o_stats = take(sizeof(Counts));
    const size_t o_frames = take(sizeof(ctm_frame) * (size_t)max_frames);
    const size_t o_cin = take(sizeof(int) * 4);
    // census demand bitmap
    const int rows_q[4] = {max_height, max_height, k == 1 ? 0 : (int)Hk, k == 1 ? 0 : (int)Hk};
    const int wq1 = (int)((((long long)max_width + kCensusTilePx - 1) / kCensusTilePx + 31) / 32);
    const int wqk = (int)(((Wk + kCensusTilePx - 1) / kCensusTilePx + 31) / 32);
    const int words_q[4] = {wq1, wq1, wqk, wqk};
    int plane_off[5];
    plane_off[0] = 0;
    for (int q = 0; q < 4; ++q) plane_off[q + 1] = plane_off[q] + rows_q[q] * words_q[q];
    const size_t o_bm = take(sizeof(uint32_t) * (size_t)plane_off[4] * max_frames);
    const size_t o_tiles = take(sizeof(unsigned long long) * 32 * (size_t)plane_off[4] * max_frames);
    const size_t o_planes = take(sizeof(PlaneDesc) * 4 * (size_t)max_frames);
    if (dev_alloc(&ctx->dev_mem, off) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return CTM_ENOMEM;
    }
    ctx->dev_bytes = off;
    char *base = static_cast<char *>(ctx->dev_mem);
    Workspace &ws = ctx->ws;
    ws.census = reinterpret_cast<uint64_t *>(base + o_census);
    ws.frame_stride = frame_stride;
    ws.plane1_elems = plane1;
    ws.planek_elems = planek;
    ws.pitch1 = pitch1;
    ws.pitchk = pitchk;
    ws.plans = reinterpret_cast<BoxPlan *>(base + o_plans);
    ws.occ = reinterpret_cast<int4 *>(base + o_occ);
    ws.nblk = reinterpret_cast<int *>(base + o_nblk);
    ws.blk_base = reinterpret_cast<int *>(base + o_base);
    ws.blocks = reinterpret_cast<int2 *>(base + o_blocks);
    ws.blkres = reinterpret_cast<BlockResult *>(base + o_blkres);
    ws.chunk = reinterpret_cast<ChunkState *>(base + o_chunk);
    ws.tmaps = reinterpret_cast<const CUtensorMap *>(base + o_tmaps);
    ws.chunk_cost = reinterpret_cast<int32_t *>(base + o_ccost);
    ws.geom = reinterpret_cast<BlockGeom *>(base + o_geom);
    ws.queue = reinterpret_cast<int *>(base + o_queue);
    ws.queue_w = reinterpret_cast<int *>(base + o_queue_w);
    ws.sched = reinterpret_cast<int *>(base + o_sched);
    ws.counts = reinterpret_cast<Counts *>(base + o_counts);
    ws.stats = reinterpret_cast<Counts *>(base + o_stats);
    ws.frames = reinterpret_cast<ctm_frame *>(base + o_frames);
    ws.counts_in = reinterpret_cast<int *>(base + o_cin);
    ws.bitmap = reinterpret_cast<uint32_t *>(base + o_bm);
    ws.tiles = reinterpret_cast<unsigned long long *>(base + o_tiles);
    ws.planes = reinterpret_cast<PlaneDesc *>(base + o_planes);
    ws.bm_frame_words = plane_off[4];
    for (int q = 0; q < 5; ++q) ws.bm_plane_off[q] = plane_off[q];
    for (int q = 0; q < 4; ++q) ws.bm_row_words[q] = words_q[q];
    if (cudaMemset(ctx->dev_mem, 0, off) != cudaSuccess) {
        ctm_destroy(ctx);
        return CTM_ECUDA;
    }
    ctx->maps_ok = encode_plane_maps(ws, ctx->caps, k, const_cast<CUtensorMap *>(ws.tmaps));
    MatchArgs a = make_args(ctx, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (match_configure(a, ctx->match_threads, &ctx->ctas_per_sm) != cudaSuccess || ctx->ctas_per_sm < 1) {
        cudaGetLastError();
        ctm_destroy(ctx);
        return CTM_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ctm_destroy(ctx);
        return CTM_ECUDA;
    }
    for (int m = 0; m < 3; ++m) census_roi_ctas_per_sm(p->win_w, p->win_h, m);  // outside any capture
    *out = ctx;
    return CTM_OK;
}

void ctm_destroy(ctm_ctx *ctx)
{
    if (!ctx) return;
    set_device(ctx);
    cudaDeviceSynchronize();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->dev_mem) cudaFree(ctx->dev_mem);
    if (ctx->img_dev) cudaFree(ctx->img_dev);
    if (ctx->frames_host_pinned) cudaFreeHost(ctx->frames_host_pinned);
    if (ctx->counts_host_pinned) cudaFreeHost(ctx->counts_host_pinned);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t ev : ctx->host_ev)
        if (ev) cudaEventDestroy(ev);
    cudaGetLastError();
    delete ctx;
}

int ctm_census_build(const uint8_t *img_dev, int width, int height, int pitch, int factor,
                     int win_w, int win_h, int sentinel, uint64_t *codes_dev, int64_t codes_pitch,
                     ctm_stream stream)
{
    if (!img_dev || !codes_dev || width < 1 || height < 1 || pitch < width) return CTM_EINVAL;
    if (factor < 1 || factor > 64) return CTM_EINVAL;
    if (win_w < 1 || win_h < 1 || (win_w & 1) == 0 || (win_h & 1) == 0 || win_w > kMaxWin ||
        win_h > kMaxWin || win_w * win_h + (sentinel ? 1 : 0) > 64 || (sentinel != 0 && sentinel != 1))
        return CTM_EINVAL;
    const int Ws = (width + factor - 1) / factor;
    if (codes_pitch < Ws) return CTM_EINVAL;
    cudaError_t e = launch_census_single(img_dev, width, height, pitch, factor, win_w, win_h,
                                         sentinel, codes_dev, codes_pitch, (cudaStream_t)stream);
    return e == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

static int check_frame_args(const ctm_ctx *ctx, const uint8_t *l, const uint8_t *r, int width,
                            int height, int pitch, const ctm_box *boxes, int n_boxes, const float *disp,
                            const float *depth, const uint8_t *flags)
{
    if (!ctx || !l || !r || width < 1 || height < 1 || pitch < width || n_boxes < 0) return CTM_EINVAL;
    if (n_boxes > 0 && (!boxes || !disp || !depth || !flags)) return CTM_EINVAL;
    if (width > ctx->caps.max_width || height > ctx->caps.max_height || n_boxes > ctx->caps.max_boxes)
        return CTM_ENOMEM;
    return CTM_OK;
}

int ctm_match_boxes(ctm_ctx *ctx, const uint8_t *left_dev, const uint8_t *right_dev, int width,
                    int height, int pitch, const ctm_box *boxes_dev, int n_boxes, float f_px,
                    float baseline_m, float *disp_dev, float *depth_dev, uint8_t *flags_dev,
                    const ctm_debug *dbg, ctm_stream stream)
{
    int st = check_frame_args(ctx, left_dev, right_dev, width, height, pitch, boxes_dev, n_boxes,
                              disp_dev, depth_dev, flags_dev);
    if (st != CTM_OK) return st;
    if ((st = set_device(ctx)) != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ctm_frame fr{left_dev, right_dev, width, height, pitch, 0, n_boxes, f_px, baseline_m};
    MatchArgs a = make_args(ctx, ctx->ws.frames, ctx->ws.counts_in, boxes_dev, disp_dev, depth_dev,
                            flags_dev, dbg);
    if (launch_stage_frame(a, fr, n_boxes, s) != cudaSuccess) return CTM_ECUDA;
    const int slots = std::max(1, ctx->p.grid_g * ctx->p.grid_g);
    const long long blocks_ub = (long long)std::max(n_boxes, 1) * slots;
    const int grid = (int)std::min<long long>((long long)ctx->sm_count * ctx->ctas_per_sm, blocks_ub);
    return enqueue_match(ctx, a, 1, grid, s, false, n_boxes);
}

int ctm_match_boxes_plain(ctm_ctx *ctx, const uint8_t *left_dev, const uint8_t *right_dev,
                          int width, int height, int pitch, const ctm_box *boxes_dev, int n_boxes,
                          float f_px, float baseline_m, float *disp_dev, float *depth_dev,
                          uint8_t *flags_dev, ctm_stream stream)
{
    int st = check_frame_args(ctx, left_dev, right_dev, width, height, pitch, boxes_dev, n_boxes,
                              disp_dev, depth_dev, flags_dev);
    if (st != CTM_OK) return st;
    if ((st = set_device(ctx)) != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ctm_frame fr{left_dev, right_dev, width, height, pitch, 0, n_boxes, f_px, baseline_m};
    MatchArgs a = make_args(ctx, ctx->ws.frames, ctx->ws.counts_in, boxes_dev, disp_dev, depth_dev,
                            flags_dev, nullptr);
    if (launch_stage_frame(a, fr, n_boxes, s) != cudaSuccess) return CTM_ECUDA;
    return enqueue_match(ctx, a, 1, 0, s, true, n_boxes);
}

int ctm_match_batch(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                    const ctm_box *boxes_dev, float *disp_dev, float *depth_dev, uint8_t *flags_dev,
                    const ctm_debug *dbg, int use_graph, ctm_stream stream)
{
    return ctm::match_batch_dev(ctx, frames_dev, nullptr, counts_dev, boxes_dev, disp_dev, depth_dev, flags_dev,
                                dbg, use_graph, stream);
}

}  // extern "C"

namespace ctm {

int match_batch_dev(ctm_ctx *ctx, const ctm_frame *frames_dev, const ctm_frame *gather_src_dev,
                    const int32_t *counts_dev, const ctm_box *boxes_dev, float *disp_dev, float *depth_dev,
                    uint8_t *flags_dev, const ctm_debug *dbg, int use_graph, ctm_stream stream)
{
    if (!ctx || !frames_dev || !counts_dev || !boxes_dev || !disp_dev || !depth_dev || !flags_dev)
        return CTM_EINVAL;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    MatchArgs a = make_args(ctx, frames_dev, counts_dev, boxes_dev, disp_dev, depth_dev, flags_dev, dbg);
    a.gather_src = gather_src_dev;
    const int grid = ctx->sm_count * ctx->ctas_per_sm;
    if (!use_graph) return enqueue_match(ctx, a, ctx->caps.max_frames, grid, s, false, 0);

    GraphKey key{frames_dev, counts_dev, boxes_dev, disp_dev, depth_dev, flags_dev,
                 dbg ? (const void *)dbg->blocks : nullptr, dbg ? (const void *)dbg->cost_f : nullptr,
                 dbg ? (const void *)dbg->cost_b : nullptr, gather_src_dev};
    if (!ctx->gexec || !(key == ctx->gkey)) {
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return CTM_ECUDA;
        const int r = enqueue_match(ctx, a, ctx->caps.max_frames, grid, ctx->capture_stream, false, 0, false);
        const cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (r != CTM_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return CTM_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            ctx->gexec = nullptr;
            cudaGetLastError();
            return CTM_ECUDA;
        }
        ctx->gkey = key;
    }
    return cudaGraphLaunch(ctx->gexec, s) == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

}  // namespace ctm

extern "C" {

int ctm_match_batch_profiled(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                             const ctm_box *boxes_dev, float *disp_dev, float *depth_dev,
                             uint8_t *flags_dev, void *const events[8], ctm_stream stream)
{
    if (!ctx || !frames_dev || !counts_dev || !boxes_dev || !disp_dev || !depth_dev || !flags_dev || !events)
        return CTM_EINVAL;
    for (int i = 0; i < 8; ++i)
        if (!events[i]) return CTM_EINVAL;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    MatchArgs a = make_args(ctx, frames_dev, counts_dev, boxes_dev, disp_dev, depth_dev, flags_dev,
                            nullptr);
    const int grid = ctx->sm_count * ctx->ctas_per_sm;
    cudaEvent_t const *ev = reinterpret_cast<cudaEvent_t const *>(events);
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = launch_plan(a, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = launch_sample(a, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = launch_census_roi(a, ctx->sm_count, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess)
        e = ctx->match_mode == 1 ? launch_match_pipe(a, ctx->match_threads, grid, s)
                                 : launch_match_persistent(a, ctx->match_threads, grid, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], s);
    if (e == cudaSuccess) e = launch_aggregate(a, s);
    for (int i = 5; i < 8 && e == cudaSuccess; ++i) e = cudaEventRecord(ev[i], s);
    if (e != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    return CTM_OK;
}

// Staging of the host entry points (allocated on first use): device images at
// a pitch of 128 bytes, boxes and outputs, two frame tables (the staging images'
// and, for mapped calls, the caller's) in device and page-locked memory, per
// sub-batch counts, a copy stream and its events.
static int ensure_host_staging(ctm_ctx *ctx)
{
    if (ctx->img_dev) return CTM_OK;
    ctx->img_pitch = round_up(ctx->caps.max_width, 128);
    const size_t img_bytes = (size_t)ctx->img_pitch * ctx->caps.max_height * 2 * ctx->caps.max_frames;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up(off + bytes, 256); return o; };
    const size_t o_img = take(img_bytes);
    const size_t o_boxes = take(sizeof(ctm_box) * (size_t)ctx->caps.max_boxes);
    const size_t o_disp = take(sizeof(float) * (size_t)ctx->caps.max_boxes);
    const size_t o_depth = take(sizeof(float) * (size_t)ctx->caps.max_boxes);
    const size_t o_flags = take((size_t)ctx->caps.max_boxes);
    const size_t o_frames = take(sizeof(ctm_frame) * 2 * (size_t)ctx->caps.max_frames);
    const size_t o_counts = take(sizeof(int32_t) * 4 * kHostGroups);
    void *mem = nullptr;
    if (dev_alloc(&mem, off) != cudaSuccess) { cudaGetLastError(); return CTM_ENOMEM; }
    bool okh = cudaMallocHost(&ctx->frames_host_pinned, sizeof(ctm_frame) * 2 * ctx->caps.max_frames) == cudaSuccess &&
               cudaMallocHost(&ctx->counts_host_pinned, sizeof(int32_t) * 4 * kHostGroups) == cudaSuccess &&
               cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t &ev : ctx->host_ev)
        okh = okh && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (!okh) {
        cudaFree(mem);
        if (ctx->frames_host_pinned) cudaFreeHost(ctx->frames_host_pinned);
        if (ctx->counts_host_pinned) cudaFreeHost(ctx->counts_host_pinned);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        ctx->copy_stream = nullptr;
        for (cudaEvent_t &ev : ctx->host_ev)
            if (ev) { cudaEventDestroy(ev); ev = nullptr; }
        ctx->frames_host_pinned = nullptr;
        ctx->counts_host_pinned = nullptr;
        cudaGetLastError();
        return CTM_ENOMEM;
    }
    char *b = static_cast<char *>(mem);
    ctx->img_dev = reinterpret_cast<uint8_t *>(b + o_img);
    ctx->boxes_dev = reinterpret_cast<ctm_box *>(b + o_boxes);
    ctx->disp_dev = reinterpret_cast<float *>(b + o_disp);
    ctx->depth_dev = reinterpret_cast<float *>(b + o_depth);
    ctx->flags_dev = reinterpret_cast<uint8_t *>(b + o_flags);
    ctx->frames_dev2 = reinterpret_cast<ctm_frame *>(b + o_frames);
    ctx->counts_dev2 = reinterpret_cast<int32_t *>(b + o_counts);
    return CTM_OK;
}

// The end of a host call, after its kernels are queued on s: outputs and the
// call's bounded-wait flag back to host memory, then wait for s.
static int host_results(ctm_ctx *ctx, cudaStream_t s, int n_boxes, float *disp_host, float *depth_host,
                        uint8_t *flags_host)
{
    cudaError_t e = cudaSuccess;
    if (n_boxes > 0) {
        e = cudaMemcpyAsync(disp_host, ctx->disp_dev, sizeof(float) * n_boxes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(depth_host, ctx->depth_dev, sizeof(float) * n_boxes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(flags_host, ctx->flags_dev, (size_t)n_boxes, cudaMemcpyDeviceToHost, s);
    }
    int32_t *err_h = ctx->counts_host_pinned + 4 * kHostGroups - 1;  // a slot no sub-batch uses
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(err_h, &ctx->ws.stats->error, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    return *err_h ? CTM_ETIMEOUT : CTM_OK;
}

// Host memory a kernel may read at the same address: page-locked (allocated or
// registered) memory, with unified addressing.
static bool device_readable(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

int ctm_match_batch_host(ctm_ctx *ctx, const ctm_frame *frames_host, int n_frames,
                         const ctm_box *boxes_host, int n_boxes, float *disp_host,
                         float *depth_host, uint8_t *flags_host, ctm_stream stream)
{
    if (!ctx || !frames_host || n_frames < 1 || n_boxes < 0) return CTM_EINVAL;
    if (n_boxes > 0 && (!boxes_host || !disp_host || !depth_host || !flags_host)) return CTM_EINVAL;
    if (n_frames > ctx->caps.max_frames || n_boxes > ctx->caps.max_boxes) return CTM_ENOMEM;
    for (int i = 0; i < n_frames; ++i) {
        const ctm_frame &f = frames_host[i];
        if (!f.left || !f.right || f.width < 1 || f.height < 1 || f.pitch < f.width) return CTM_EINVAL;
        if (f.width > ctx->caps.max_width || f.height > ctx->caps.max_height) return CTM_ENOMEM;
    }
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_host_staging(ctx);
    if (st != CTM_OK) return st;
    // Sub-batches of consecutive frames when each frame's boxes follow the previous
    // frame's (each sub-batch then owns one slice of the boxes and outputs); else
    // one batch.  Sub-batch g + 1's copies, on the copy stream, overlap sub-batch
    // g's kernels on `stream`; the kernels of all sub-batches run in order on
    // `stream` over the one workspace, so the results equal one call's.
    bool chained = frames_host[0].box_begin >= 0;
    for (int i = 0; i < n_frames && chained; ++i) {
        const ctm_frame &f = frames_host[i];
        if (f.box_count < 0 || (i > 0 && f.box_begin != frames_host[i - 1].box_begin + frames_host[i - 1].box_count))
            chained = false;
    }
    if (chained && frames_host[n_frames - 1].box_begin + frames_host[n_frames - 1].box_count > n_boxes) chained = false;
    const int groups = chained ? std::min(kHostGroups, n_frames) : 1;

    const size_t plane = (size_t)ctx->img_pitch * ctx->caps.max_height;
    cudaStream_t cs = ctx->copy_stream;
    cudaError_t e = cudaEventRecord(ctx->host_ev[kHostGroups], s);  // work already queued on `stream`
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->host_ev[kHostGroups], 0);
    // Images go to the staging planes in as few copies as possible: an image
    // packed at the staging pitch is one linear run, and runs that continue one
    // another in both host and device memory are merged (one large copy moves
    // about 210 GB/s on GB300, the host link's rate; 64 copies of 2.3 MB about
    // 155 GB/s, and two copy streams were slower too).
    const uint8_t *run_src = nullptr;
    uint8_t *run_dst = nullptr;
    size_t run_bytes = 0;
    auto flush = [&]() {
        if (run_bytes > 0 && e == cudaSuccess)
            e = cudaMemcpyAsync(run_dst, run_src, run_bytes, cudaMemcpyHostToDevice, cs);
        run_bytes = 0;
    };
    auto image = [&](uint8_t *dst, const uint8_t *src, const ctm_frame &f) {
        if (f.pitch == f.width && (long long)f.width == ctx->img_pitch) {
            const size_t bytes = (size_t)f.pitch * f.height;
            if (run_bytes > 0 && run_src + run_bytes == src && run_dst + run_bytes == dst) {
                run_bytes += bytes;
            } else {
                flush();
                run_src = src;
                run_dst = dst;
                run_bytes = bytes;
            }
        } else {
            flush();
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(dst, ctx->img_pitch, src, f.pitch, f.width, f.height, cudaMemcpyHostToDevice, cs);
        }
    };
    if (e == cudaSuccess && n_boxes > 0)
        e = cudaMemcpyAsync(ctx->boxes_dev, boxes_host, sizeof(ctm_box) * n_boxes, cudaMemcpyHostToDevice, cs);
    const int grid = ctx->sm_count * ctx->ctas_per_sm;
    // Shrinking sub-batches (12, 10, 6, 4 of 32 frames): each sub-batch's kernels stay
    // shorter than the next sub-batch's copy, and the last one, which nothing
    // hides, is the smallest.  Below 8 frames, equal parts.
    auto bound = [&](int g) -> int {
        static const int k64ths[kHostGroups + 1] = {0, 24, 44, 56, 64};  // sub-batch bounds in 64ths
        if (groups < kHostGroups || n_frames < 8) return (int)((long long)g * n_frames / groups);
        return (int)(((long long)k64ths[g] * n_frames + 32) / 64);
    };
    for (int g = 0; g < groups && e == cudaSuccess; ++g) {
        const int f0 = bound(g), f1 = bound(g + 1);
        const int box0 = groups > 1 ? frames_host[f0].box_begin : 0;
        const int nb = groups > 1 ? frames_host[f1 - 1].box_begin + frames_host[f1 - 1].box_count - box0 : n_boxes;
        for (int i = f0; i < f1 && e == cudaSuccess; ++i) {
            const ctm_frame &f = frames_host[i];
            uint8_t *dl = ctx->img_dev + plane * (2 * (size_t)i);
            uint8_t *dr = dl + plane;
            image(dl, f.left, f);
            image(dr, f.right, f);
            ctm_frame t = f;
            t.left = dl;
            t.right = dr;
            t.pitch = (int32_t)ctx->img_pitch;
            t.box_begin = f.box_begin - box0;
            ctx->frames_host_pinned[i] = t;
        }
        flush();
        int32_t *cnt = ctx->counts_host_pinned + 4 * g;
        cnt[0] = f1 - f0;
        cnt[1] = nb;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->frames_dev2 + f0, ctx->frames_host_pinned + f0, sizeof(ctm_frame) * (f1 - f0),
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->counts_dev2 + 4 * g, cnt, sizeof(int32_t) * 2, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->host_ev[g], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->host_ev[g], 0);
        if (e != cudaSuccess) break;
        MatchArgs a = make_args(ctx, ctx->frames_dev2 + f0, ctx->counts_dev2 + 4 * g, ctx->boxes_dev + box0,
                                ctx->disp_dev + box0, ctx->depth_dev + box0, ctx->flags_dev + box0, nullptr);
        a.stats_accumulate = g > 0;  // ctm_get_stats then covers the whole call
        if (enqueue_match(ctx, a, f1 - f0, grid, s, false, 0) != CTM_OK) e = cudaErrorLaunchFailure;
    }
    if (e != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    return host_results(ctx, s, n_boxes, disp_host, depth_host, flags_host);
}

int ctm_match_batch_mapped(ctm_ctx *ctx, const ctm_frame *frames_host, int n_frames,
                           const ctm_box *boxes_host, int n_boxes, float *disp_host,
                           float *depth_host, uint8_t *flags_host, ctm_stream stream)
{
    if (!ctx || !frames_host || n_frames < 1 || n_boxes < 0) return CTM_EINVAL;
    if (n_boxes > 0 && (!boxes_host || !disp_host || !depth_host || !flags_host)) return CTM_EINVAL;
    if (n_frames > ctx->caps.max_frames || n_boxes > ctx->caps.max_boxes) return CTM_ENOMEM;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    for (int i = 0; i < n_frames; ++i) {
        const ctm_frame &f = frames_host[i];
        if (!f.left || !f.right || f.width < 1 || f.height < 1 || f.pitch < f.width) return CTM_EINVAL;
        if (f.width > ctx->caps.max_width || f.height > ctx->caps.max_height) return CTM_ENOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_host_staging(ctx);
    if (st != CTM_OK) return st;
    // the staging images' frame table and the caller's (second half of the tables); a
    // frame the gather cannot read in place (rows or width off 16-byte multiples, or
    // memory the device cannot read at its host address) is copied whole on s and gets
    // height 0 in the gather's table
    const size_t plane = (size_t)ctx->img_pitch * ctx->caps.max_height;
    ctm_frame *stage = ctx->frames_host_pinned, *src = ctx->frames_host_pinned + ctx->caps.max_frames;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_frames && e == cudaSuccess; ++i) {
        const ctm_frame &f = frames_host[i];
        ctm_frame t = f;
        src[i] = t;
        t.left = ctx->img_dev + plane * (2 * (size_t)i);
        t.right = t.left + plane;
        t.pitch = (int32_t)ctx->img_pitch;
        stage[i] = t;
        const bool aligned = ((reinterpret_cast<uintptr_t>(f.left) | reinterpret_cast<uintptr_t>(f.right) |
                               (uintptr_t)f.pitch | (uintptr_t)f.width) & 15u) == 0;
        if (!aligned || (!ctx->pageable_access && (!device_readable(f.left) || !device_readable(f.right)))) {
            src[i].height = 0;
            e = cudaMemcpy2DAsync(const_cast<uint8_t *>(t.left), ctx->img_pitch, f.left, f.pitch, f.width, f.height,
                                  cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(const_cast<uint8_t *>(t.right), ctx->img_pitch, f.right, f.pitch, f.width,
                                      f.height, cudaMemcpyHostToDevice, s);
        }
    }
    int32_t *cnt = ctx->counts_host_pinned;
    cnt[0] = n_frames;
    cnt[1] = n_boxes;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->frames_dev2, stage, sizeof(ctm_frame) * n_frames, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->frames_dev2 + ctx->caps.max_frames, src, sizeof(ctm_frame) * n_frames,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_boxes > 0)
        e = cudaMemcpyAsync(ctx->boxes_dev, boxes_host, sizeof(ctm_box) * n_boxes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->counts_dev2, cnt, sizeof(int32_t) * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        MatchArgs a = make_args(ctx, ctx->frames_dev2, ctx->counts_dev2, ctx->boxes_dev, ctx->disp_dev,
                                ctx->depth_dev, ctx->flags_dev, nullptr);
        a.gather_src = ctx->frames_dev2 + ctx->caps.max_frames;
        const int grid = ctx->sm_count * ctx->ctas_per_sm;
        if (enqueue_match(ctx, a, n_frames, grid, s, false, 0) != CTM_OK) e = cudaErrorLaunchFailure;
    }
    if (e != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    return host_results(ctx, s, n_boxes, disp_host, depth_host, flags_host);
}

int ctm_get_tuning(const ctm_ctx *ctx, ctm_tuning *out)
{
    if (!ctx || !out) return CTM_EINVAL;
    out->match_threads = ctx->match_threads;
    out->strip_cols = ctx->strip_cols;
    out->census_mode = ctx->census_mode;
    out->queue_rounds = ctx->queue_rounds;
    out->match_mode = ctx->match_mode;
    out->split_ways = ctx->split_ways;
    return CTM_OK;
}

int ctm_set_tuning(ctm_ctx *ctx, const ctm_tuning *t)
{
    if (!ctx || !t) return CTM_EINVAL;
    if (t->match_threads != 128 && t->match_threads != 256) return CTM_EINVAL;
    if (t->strip_cols < ctx->nd_max + 2 || (t->strip_cols & 7) != 0 || t->strip_cols > 4096) return CTM_EINVAL;
    if (t->census_mode < 0 || t->census_mode > 2) return CTM_EINVAL;
    if (t->queue_rounds != 0 && t->queue_rounds != 1) return CTM_EINVAL;
    if (t->match_mode != 0 && t->match_mode != 1) return CTM_EINVAL;
    if (t->split_ways != 0 && t->split_ways != 1 && t->split_ways != 2 && t->split_ways != 4 &&
        t->split_ways != 8)
        return CTM_EINVAL;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    ctm_ctx trial = *ctx;  // shallow: only the tuning fields are read below
    trial.match_threads = t->match_threads;
    trial.strip_cols = t->strip_cols;
    MatchArgs a = make_args(&trial, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    int ctas = 0;
    // the fused kernels stay configured either way (the per-box path uses them)
    if (match_smem_bytes(a) > 227 * 1024) return CTM_EINVAL;
    if (match_configure(a, t->match_threads, &ctas) != cudaSuccess || ctas < 1) {
        cudaGetLastError();
        return CTM_EINVAL;
    }
    if (t->match_mode == 1) {
        if (match_pipe_smem_bytes(a) > 227 * 1024) return CTM_EINVAL;
        if (match_pipe_configure(a, t->match_threads, &ctas) != cudaSuccess || ctas < 1) {
            cudaGetLastError();
            return CTM_EINVAL;
        }
    }
    const bool changed = t->match_threads != ctx->match_threads || t->strip_cols != ctx->strip_cols ||
                         t->census_mode != ctx->census_mode || t->queue_rounds != ctx->queue_rounds ||
                         t->match_mode != ctx->match_mode || t->split_ways != ctx->split_ways;
    ctx->match_threads = t->match_threads;
    ctx->strip_cols = t->strip_cols;
    ctx->census_mode = t->census_mode;
    ctx->queue_rounds = t->queue_rounds;
    ctx->match_mode = t->match_mode;
    ctx->split_ways = t->split_ways;
    ctx->ctas_per_sm = ctas;
    if (changed && ctx->gexec) {  // the captured graph holds the old launch shapes
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return CTM_OK;
}

int ctm_autotune(ctm_ctx *ctx, const ctm_frame *frames_dev, const int32_t *counts_dev,
                 const ctm_box *boxes_dev, float *disp_dev, float *depth_dev, uint8_t *flags_dev, int reps,
                 ctm_tuning *best, float *best_ms, ctm_stream stream)
{
    if (!ctx || !frames_dev || !counts_dev || !boxes_dev || !disp_dev || !depth_dev || !flags_dev || reps < 1)
        return CTM_EINVAL;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ctm_tuning cur;
    ctm_get_tuning(ctx, &cur);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return CTM_ECUDA;
    }
    // time one configuration: one warm-up call, then `reps` calls between events
    auto measure = [&](const ctm_tuning &t, float *ms) -> int {
        int r = ctm_set_tuning(ctx, &t);
        if (r != CTM_OK) return r;
        MatchArgs a = make_args(ctx, frames_dev, counts_dev, boxes_dev, disp_dev, depth_dev, flags_dev, nullptr);
        const int grid = ctx->sm_count * ctx->ctas_per_sm;
        r = enqueue_match(ctx, a, ctx->caps.max_frames, grid, s, false, 0, false);
        if (r == CTM_OK && cudaEventRecord(e0, s) != cudaSuccess) r = CTM_ECUDA;
        for (int i = 0; i < reps && r == CTM_OK; ++i)
            r = enqueue_match(ctx, a, ctx->caps.max_frames, grid, s, false, 0, false);
        if (r == CTM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            r = CTM_ECUDA;
        float t_ms = 0.0f;
        if (r == CTM_OK && cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess) r = CTM_ECUDA;
        *ms = t_ms / (float)reps;
        return r;
    };
    ctm_tuning bt = cur;
    float bms = 3.4e38f;
    int status = CTM_OK;
    // 1. matcher x CTA size x strip chunk width (joint), at the current census mode and split
    // strip widths: the narrowest a point column fits (N_d + 2, rounded up to 8),
    // then multiples of 32 above it
    int widths[10];
    int nw = 0;
    widths[nw++] = (int)round_up(ctx->nd_max + 2, 8);
    for (int w = (int)round_up(ctx->nd_max + 2, 32); nw < 10; w += 32)
        if (w > widths[0]) widths[nw++] = w;
    for (int mode = 0; mode <= 1 && status == CTM_OK; ++mode) {
      for (int th = 128; th <= 256 && status == CTM_OK; th *= 2) {
        for (int wi = 0; wi < nw; ++wi) {
            ctm_tuning t = bt;
            t.match_mode = mode;
            t.match_threads = th;
            t.strip_cols = widths[wi];
            float ms = 0.0f;
            const int r = measure(t, &ms);
            if (r == CTM_EINVAL) continue;  // does not fit shared memory
            if (r != CTM_OK) { status = r; break; }
            if (ms < bms) { bms = ms; bt = t; }
        }
      }
    }
    // 2. census variant, 3. per-SM rounds, one at a time around the best so far
    const int modes[3] = {0, 1, 2};
    for (int i = 0; i < 3 && status == CTM_OK; ++i) {
        ctm_tuning t = bt;
        t.census_mode = modes[i];
        float ms = 0.0f;
        const int r = measure(t, &ms);
        if (r != CTM_OK) { status = r; break; }
        if (ms < bms) { bms = ms; bt = t; }
    }
    for (int i = 0; i < 2 && status == CTM_OK; ++i) {
        ctm_tuning t = bt;
        t.queue_rounds = i;
        float ms = 0.0f;
        const int r = measure(t, &ms);
        if (r != CTM_OK) { status = r; break; }
        if (ms < bms) { bms = ms; bt = t; }
    }
    // 4. disparity-chunk tiles of the fused matcher: automatic or never
    for (int sw = 0; sw <= 1 && status == CTM_OK && bt.match_mode == 0; ++sw) {
        ctm_tuning t = bt;
        t.split_ways = sw;
        float ms = 0.0f;
        const int r = measure(t, &ms);
        if (r != CTM_OK) { status = r; break; }
        if (ms < bms) { bms = ms; bt = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != CTM_OK) {
        ctm_set_tuning(ctx, &cur);
        return status;
    }
    st = ctm_set_tuning(ctx, &bt);
    if (st != CTM_OK) return st;
    if (best) *best = bt;
    if (best_ms) *best_ms = bms;
    return CTM_OK;
}

int ctm_get_stats(ctm_ctx *ctx, ctm_stats *out, ctm_stream stream)
{
    if (!ctx || !out) return CTM_EINVAL;
    int st = set_device(ctx);
    if (st != CTM_OK) return st;
    Counts c;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&c, ctx->ws.stats, sizeof(Counts), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CTM_ECUDA;
    }
    out->cost_evals = c.evals;
    out->n_blocks = c.n_blocks;
    out->n_boxes = c.n_boxes;
    out->error = c.error;
    out->census_tiles = c.n_tiles;
    out->host_bytes = c.host_bytes;
    return CTM_OK;
}

int ctm_probe_int_rate(int kind, int iters, double *ops_per_clk_per_sm)
{
    if (kind < 0 || kind > 5 || iters < 1 || !ops_per_clk_per_sm) return CTM_EINVAL;
    return run_int_probe(kind, iters, ops_per_clk_per_sm) == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

int ctm_inject_alloc_failures(int skip, int n)
{
    if (skip < 0 || n < 0) return CTM_EINVAL;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_alloc_skip = n > 0 ? skip : 0;
    g_alloc_fail = n;
    return CTM_OK;
}

int ctm_inject_wait_expiry(ctm_ctx *ctx)
{
    if (!ctx) return CTM_EINVAL;
    ctx->inject_expiry = 1;
    return CTM_OK;
}

int ctm_probe_bounded_wait(int *expired, float *waited_ms)
{
    if (!expired || !waited_ms) return CTM_EINVAL;
    return run_wait_probe(expired, waited_ms) == cudaSuccess ? CTM_OK : CTM_ECUDA;
}

}  // extern "C"
