// noalloc.cu -- single-frame matching that allocates no device memory.
//
// Some callers of this library cannot call cudaMalloc while they run: a
// real-time control loop must not enter the device allocator, because an
// allocation can synchronize the device and take an unbounded time; and a host
// that gives the library a fixed memory budget when it starts does not let it
// grow its footprint later.  For them ctm_match_boxes_noalloc runs the same
// launch sequence as ctm_match_boxes, but its workspace is carved from one
// file-scope __device__ array of a fixed 8 MiB, which every GPU that loads the
// library holds until the process exits; frames up to 640x480 with 64 boxes fit.
//
// Set-up happens on the first call on each device (with that device current):
// the array's device address is taken with cudaGetSymbolAddress -- in host code
// the array's name is only a host-side stand-in, not a device address -- and
// the matching kernel's shared-memory limit is raised, and the census kernels'
// occupancy is looked up, so later calls make no attribute or occupancy query
// for the fixed windows.  All calls share the one array and
// it keeps the previous call's contents: each call clears what must start at
// zero (the census demand bitmap, the counters, the block counts), and calls
// that overlap on the GPU race on the array.  The counters of the last call
// (its bounded-wait flag included) sit at a fixed place at the array's start,
// where ctm_noalloc_get_stats reads them.
#include <cuda_runtime.h>

#include <algorithm>

#include "ctm_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 8u << 20;  // 8 MiB per GPU
constexpr int kMaxW = 640, kMaxH = 480, kMaxBoxes = 64;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceState {
    bool ready;
    unsigned char *base;  // device address of g_noalloc_scratch on this device
    int sm_count;
    int match_need;       // matching kernel's shared-memory bytes last configured (0: none)
    int match_ctas;       // its resident CTAs per SM at that size
};
DeviceState g_state[kMaxDevices];

inline long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

// The counters of the call in progress and of the last finished call lead the
// array, so their places do not depend on the parameters.
constexpr size_t kStatsOff = (sizeof(ctm::Counts) + 255) / 256 * 256;

int setup_device(int dev)
{
    DeviceState &st = g_state[dev];
    if (st.ready) return CTM_OK;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        return CTM_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return CTM_ECUDA;
    }
    st.base = static_cast<unsigned char *>(ptr);
    st.sm_count = sms;
    for (int m = 0; m < 2; ++m) {  // occupancy queries cached here, once per process
        ctm::census_roi_ctas_per_sm(9, 7, m);
        ctm::census_roi_ctas_per_sm(7, 7, m);
        ctm::census_roi_ctas_per_sm(5, 5, m);
    }
    st.ready = true;
    return CTM_OK;
}

}  // namespace

using namespace ctm;

extern "C" int ctm_match_boxes_noalloc(const ctm_params *p, const uint8_t *left_dev,
                                       const uint8_t *right_dev, int width, int height, int pitch,
                                       const ctm_box *boxes_dev, int n_boxes, float f_px,
                                       float baseline_m, float *disp_dev, float *depth_dev,
                                       uint8_t *flags_dev, ctm_stream stream)
{
    if (!p || !params_valid(*p)) return CTM_EINVAL;
    if (!left_dev || !right_dev || width < 1 || height < 1 || pitch < width || n_boxes < 0)
        return CTM_EINVAL;
    if (n_boxes > 0 && (!boxes_dev || !disp_dev || !depth_dev || !flags_dev)) return CTM_EINVAL;
    if (width > kMaxW || height > kMaxH || n_boxes > kMaxBoxes) return CTM_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CTM_ENODEV;
    }
    int st = setup_device(dev);
    if (st != CTM_OK) return st;
    const DeviceState &ds = g_state[dev];

    // workspace sizes for one frame of at most kMaxW x kMaxH and kMaxBoxes boxes
    Caps caps;
    caps.max_frames = 1;
    caps.max_width = kMaxW;
    caps.max_height = kMaxH;
    caps.max_boxes = kMaxBoxes;
    caps.max_blocks = kMaxBoxes * std::max(p->grid_g * p->grid_g, 1);
    const int ndy = p->dy_max - p->dy_min + 1;
    const int nd_max = std::max(p->far_dmax - p->far_dmin + 1, p->close_dmax - p->close_dmin + 1);
    const int strip_cols = default_strip_cols(nd_max);
    const int k = p->close_factor;
    const long long pitch1 = round_up(kMaxW, 32);
    const long long Wk = (kMaxW + k - 1) / k, Hk = (kMaxH + k - 1) / k;
    const long long pitchk = k == 1 ? 0 : round_up(Wk, 32);
    const long long plane1 = pitch1 * kMaxH;
    const long long planek = k == 1 ? 0 : pitchk * Hk;
    const int rows_q[4] = {kMaxH, kMaxH, k == 1 ? 0 : (int)Hk, k == 1 ? 0 : (int)Hk};
    const int wq1 = (int)(((kMaxW + kCensusTilePx - 1) / kCensusTilePx + 31) / 32);
    const int wqk = (int)(((Wk + kCensusTilePx - 1) / kCensusTilePx + 31) / 32);
    const int words_q[4] = {wq1, wq1, wqk, wqk};
    int plane_off[5];
    plane_off[0] = 0;
    for (int q = 0; q < 4; ++q) plane_off[q + 1] = plane_off[q] + rows_q[q] * words_q[q];

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up(off + bytes, 256); return o; };
    const size_t o_counts = take(sizeof(Counts));  // offset 0
    const size_t o_stats = take(sizeof(Counts));   // offset kStatsOff
    const size_t o_census = take(sizeof(uint64_t) * (size_t)(2 * plane1 + 2 * planek));
    const size_t o_plans = take(sizeof(BoxPlan) * kMaxBoxes);
    const size_t o_occ = take(sizeof(int4) * (size_t)kMaxBoxes * kMaxOcc);
    const size_t o_nblk = take(sizeof(int) * kMaxBoxes);
    const size_t o_base = take(sizeof(int) * kMaxBoxes);
    const size_t o_blocks = take(sizeof(int2) * (size_t)caps.max_blocks);
    const size_t o_blkres = take(sizeof(BlockResult) * (size_t)caps.max_blocks);
    const size_t o_geom = take(sizeof(BlockGeom) * (size_t)caps.max_blocks);
    const size_t o_queue = take(sizeof(int) * (size_t)caps.max_blocks);
    const size_t o_frames = take(sizeof(ctm_frame));
    const size_t o_cin = take(sizeof(int) * 4);
    const size_t o_bm = take(sizeof(uint32_t) * (size_t)plane_off[4]);
    const size_t o_tiles = take(sizeof(unsigned long long) * 32 * (size_t)plane_off[4]);
    const size_t o_planes = take(sizeof(PlaneDesc) * 4);
    if (off > kScratchBytes) return CTM_ETOOBIG;

    unsigned char *b = ds.base;
    MatchArgs a;
    Workspace &ws = a.ws;
    ws.census = reinterpret_cast<uint64_t *>(b + o_census);
    ws.frame_stride = 2 * plane1 + 2 * planek;
    ws.plane1_elems = plane1;
    ws.planek_elems = planek;
    ws.pitch1 = pitch1;
    ws.pitchk = pitchk;
    ws.plans = reinterpret_cast<BoxPlan *>(b + o_plans);
    ws.occ = reinterpret_cast<int4 *>(b + o_occ);
    ws.nblk = reinterpret_cast<int *>(b + o_nblk);
    ws.blk_base = reinterpret_cast<int *>(b + o_base);
    ws.blocks = reinterpret_cast<int2 *>(b + o_blocks);
    ws.blkres = reinterpret_cast<BlockResult *>(b + o_blkres);
    ws.chunk = nullptr;  // no disparity-chunk tiles: their state does not fit the array
    ws.tmaps = nullptr;  // strips load by 1-D bulk copies
    ws.chunk_cost = nullptr;
    ws.geom = reinterpret_cast<BlockGeom *>(b + o_geom);
    ws.queue = reinterpret_cast<int *>(b + o_queue);
    ws.queue_w = nullptr;  // one dynamic queue in sampling order (no per-SM rounds)
    ws.sched = nullptr;
    ws.counts = reinterpret_cast<Counts *>(b + o_counts);
    ws.stats = reinterpret_cast<Counts *>(b + o_stats);
    ws.frames = reinterpret_cast<ctm_frame *>(b + o_frames);
    ws.counts_in = reinterpret_cast<int *>(b + o_cin);
    ws.bitmap = reinterpret_cast<uint32_t *>(b + o_bm);
    ws.tiles = reinterpret_cast<unsigned long long *>(b + o_tiles);
    ws.planes = reinterpret_cast<PlaneDesc *>(b + o_planes);
    ws.bm_frame_words = plane_off[4];
    for (int q = 0; q < 5; ++q) ws.bm_plane_off[q] = plane_off[q];
    for (int q = 0; q < 4; ++q) ws.bm_row_words[q] = words_q[q];
    a.caps = caps;
    a.p = *p;
    a.stats_accumulate = 0;
    a.inject_expiry = 0;
    a.gather_src = nullptr;
    a.frames = ws.frames;
    a.counts_in = ws.counts_in;
    a.boxes = boxes_dev;
    a.disp = disp_dev;
    a.depth = depth_dev;
    a.flags = flags_dev;
    a.dbg.blocks = nullptr;
    a.dbg.cost_f = nullptr;
    a.dbg.cost_b = nullptr;
    a.nc_stride = nd_max * ndy;
    a.strip_cols = strip_cols;
    a.queue_rounds = 0;
    a.sm_count = ds.sm_count;
    a.census_mode = 0;
    a.match_mode = 0;
    a.split_ways = 1;
    a.strip_rows = p->pts_side * ndy;

    const int threads = 128;
    DeviceState &dsm = g_state[dev];
    const int need = (int)match_smem_bytes(a);
    if (dsm.match_need != need) {  // attribute and occupancy queries only when the size changes
        int ctas = 0;
        if (match_configure_raise(a, threads, &ctas) != cudaSuccess || ctas < 1) {
            cudaGetLastError();
            return CTM_ECUDA;
        }
        dsm.match_need = need;
        dsm.match_ctas = ctas;
    }
    const int ctas = dsm.match_ctas;
    census_roi_ctas_per_sm(p->win_w, p->win_h, 0);  // this window's occupancy query, cached after the first
    cudaStream_t s = (cudaStream_t)stream;
    // the census demand bitmap, the counters and the block counts must start at
    // zero (a call interrupted on the device may leave them set)
    cudaError_t e = cudaMemsetAsync(ws.bitmap, 0, sizeof(uint32_t) * (size_t)plane_off[4], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.counts, 0, sizeof(Counts), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.nblk, 0, sizeof(int) * kMaxBoxes, s);
    const ctm_frame fr{left_dev, right_dev, width, height, pitch, 0, n_boxes, f_px, baseline_m};
    if (e == cudaSuccess) e = launch_stage_frame(a, fr, n_boxes, s);
    if (e == cudaSuccess) e = launch_plan(a, s);
    if (e == cudaSuccess) e = launch_sample(a, s);
    if (e == cudaSuccess) e = launch_census_roi(a, ds.sm_count, s);
    const long long blocks_ub = (long long)std::max(n_boxes, 1) * std::max(p->grid_g * p->grid_g, 1);
    const int grid = (int)std::min<long long>((long long)ds.sm_count * ctas, blocks_ub);
    if (e == cudaSuccess) e = launch_match_persistent(a, threads, grid, s);
    if (e == cudaSuccess) e = launch_aggregate(a, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CTM_ECUDA;
    }
    return CTM_OK;
}

extern "C" int ctm_noalloc_get_stats(ctm_stats *out, ctm_stream stream)
{
    if (!out) return CTM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CTM_ENODEV;
    }
    const DeviceState &ds = g_state[dev];
    if (!ds.ready) return CTM_EINVAL;  // no ctm_match_boxes_noalloc call on this device yet
    Counts c;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&c, ds.base + kStatsOff, sizeof(Counts), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
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
