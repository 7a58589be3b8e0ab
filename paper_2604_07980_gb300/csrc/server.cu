// server.cu -- the serving loop of include/ctm_server.h.
//
// One native worker thread owns the GPU side.  Submitted frames wait in an
// arrival queue; the worker admits them in arrival order while their images
// fit in a fixed device arena (admission by device memory), uploads the images
// on a copy stream (mapped servers: only frames the device cannot read in place;
// the others' batches gather the bytes their census needs from host memory into
// the arena), and keeps up to `lanes` batches in flight: an idle lane
// takes every admitted frame (up to frames_per_batch) and replays its captured
// CUDA graph of the batched launch sequence over them.  Each lane owns a
// workspace created once (census planes, plans, counters), so census buffers
// stay resident across batches.  A host callback at the end of each lane's
// stream wakes the worker, which copies the outputs to the callers' arrays and
// posts completion records.
#include <cuda_runtime.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/ctm_server.h"
#include "arena.h"
#include "ctm_internal.cuh"

namespace {

int64_t now_ns()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

constexpr int64_t kImagePitchAlign = 64;  // device image rows start 64-byte aligned

struct Job {
    ctm_request r{};
    int64_t t_submit = 0, t_admit = 0, t_launch = 0;
    int64_t arena_off = -1;
    int64_t pitch = 0;  // device image pitch
    cudaEvent_t uploaded = nullptr;  // null for a gathered frame (nothing uploaded)
    bool gather = false;             // its batch reads its images from host memory
    int status = CTM_OK;
};

struct Lane {
    int index = 0;
    ctm_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int max_boxes = 0;
    // pinned host staging
    ctm_frame *frames_h = nullptr;
    ctm_frame *src_h = nullptr;  // mapped servers: the frames' host images (height 0: uploaded)
    ctm_box *boxes_h = nullptr;
    int32_t *counts_h = nullptr;
    float *disp_h = nullptr, *depth_h = nullptr;
    uint8_t *flags_h = nullptr;
    void *host_mem = nullptr;
    // device tables and outputs (one allocation)
    void *dev_mem = nullptr;
    ctm_frame *frames_d = nullptr;
    ctm_frame *src_d = nullptr;
    int32_t *counts_d = nullptr;
    ctm_box *boxes_d = nullptr;
    float *disp_d = nullptr, *depth_d = nullptr;
    uint8_t *flags_d = nullptr;
    size_t bytes = 0;
    // current batch
    std::vector<Job *> batch;
    std::vector<int> box_off;
    int n_boxes = 0;
    bool busy = false;
    int status = CTM_OK;
};

}  // namespace

struct ctm_server {
    int device = 0;
    ctm_params p{};
    ctm_server_config cfg{};
    ctm::Arena arena;
    uint8_t *arena_d = nullptr;
    cudaStream_t upload = nullptr;
    int pageable_access = 0;  // the device reads pageable host memory
    std::vector<Lane> lanes;
    std::vector<cudaEvent_t> event_pool;  // worker only
    std::deque<Job *> admitted;           // worker only: uploaded or uploading, not yet batched
    // shared with the callers
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> arrivals;
    std::deque<ctm_completion> completions;
    bool kick = false;
    bool stopping = false;
    int64_t outstanding = 0;  // submitted, not yet polled
    int admitted_now = 0;     // frames holding arena space
    ctm_server_stats st{};
    std::thread worker;
};

namespace {

void CUDART_CB lane_done_cb(void *arg)
{
    // runs on a CUDA callback thread: no CUDA calls here, only the wake-up
    ctm_server *S = static_cast<ctm_server *>(arg);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->kick = true;
    }
    S->cv_work.notify_one();
}

cudaEvent_t take_event(ctm_server *S)
{
    if (!S->event_pool.empty()) {
        cudaEvent_t e = S->event_pool.back();
        S->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Post completion records for finished jobs (outputs already written or the
// job failed), release their arena space and recycle their events.
void complete_jobs(ctm_server *S, const std::vector<Job *> &jobs, int lane, int batch_frames, int status)
{
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Job *j : jobs) {
            ctm_completion c{};
            c.tag = j->r.tag;
            c.status = status != CTM_OK ? status : j->status;
            c.n_boxes = j->r.n_boxes;
            c.t_submit_ns = j->t_submit;
            c.t_admit_ns = j->t_admit;
            c.t_launch_ns = j->t_launch;
            c.t_done_ns = t;
            c.lane = lane;
            c.batch_frames = batch_frames;
            S->completions.push_back(c);
            if (j->arena_off >= 0) {
                S->arena.release(j->arena_off);
                --S->admitted_now;
            }
            ++S->st.completed;
        }
    }
    S->cv_done.notify_all();
    for (Job *j : jobs) {
        if (j->uploaded) S->event_pool.push_back(j->uploaded);
        delete j;
    }
}

// Copy a newly admitted frame's images into its arena block on the upload stream.
bool upload(ctm_server *S, Job *j)
{
    const ctm_request &r = j->r;
    uint8_t *dl = S->arena_d + j->arena_off;
    uint8_t *dr = dl + j->pitch * r.height;
    j->uploaded = take_event(S);
    if (!j->uploaded) return false;
    cudaError_t e = cudaMemcpy2DAsync(dl, (size_t)j->pitch, r.left_host, (size_t)r.pitch, (size_t)r.width,
                                      (size_t)r.height, cudaMemcpyHostToDevice, S->upload);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dr, (size_t)j->pitch, r.right_host, (size_t)r.pitch, (size_t)r.width,
                              (size_t)r.height, cudaMemcpyHostToDevice, S->upload);
    if (e == cudaSuccess) e = cudaEventRecord(j->uploaded, S->upload);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Form a batch from the admitted frames and enqueue it on an idle lane.
void dispatch(ctm_server *S, Lane &L)
{
    L.batch.clear();
    L.box_off.clear();
    int nb = 0;
    while (!S->admitted.empty() && (int)L.batch.size() < S->cfg.frames_per_batch) {
        Job *j = S->admitted.front();
        if (nb + j->r.n_boxes > L.max_boxes) break;
        S->admitted.pop_front();
        L.box_off.push_back(nb);
        L.batch.push_back(j);
        nb += j->r.n_boxes;
    }
    if (L.batch.empty()) return;
    const int nf = (int)L.batch.size();
    L.n_boxes = nb;
    const int64_t t = now_ns();
    for (int i = 0; i < nf; ++i) {
        Job *j = L.batch[i];
        const ctm_request &r = j->r;
        uint8_t *dl = S->arena_d + j->arena_off;
        ctm_frame &f = L.frames_h[i];
        f.left = dl;
        f.right = dl + j->pitch * r.height;
        f.width = r.width;
        f.height = r.height;
        f.pitch = (int32_t)j->pitch;
        f.box_begin = L.box_off[i];
        f.box_count = r.n_boxes;
        f.f_px = r.f_px;
        f.baseline_m = r.baseline_m;
        if (S->cfg.mapped) {  // gathered frames: their host images; uploaded ones: height 0
            ctm_frame &g = L.src_h[i];
            g = f;
            g.left = r.left_host;
            g.right = r.right_host;
            g.pitch = r.pitch;
            if (!j->gather) g.height = 0;
        }
        if (r.n_boxes > 0) memcpy(L.boxes_h + L.box_off[i], r.boxes_host, sizeof(ctm_box) * (size_t)r.n_boxes);
        for (int b = 0; b < r.n_boxes; ++b) L.boxes_h[L.box_off[i] + b].frame = i;
        j->t_launch = t;
    }
    L.counts_h[0] = nf;
    L.counts_h[1] = nb;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nf && e == cudaSuccess; ++i)
        if (L.batch[i]->uploaded) e = cudaStreamWaitEvent(L.stream, L.batch[i]->uploaded, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.frames_d, L.frames_h, sizeof(ctm_frame) * nf, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess && nb > 0)
        e = cudaMemcpyAsync(L.boxes_d, L.boxes_h, sizeof(ctm_box) * nb, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.counts_d, L.counts_h, sizeof(int32_t) * 2, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess && S->cfg.mapped)
        e = cudaMemcpyAsync(L.src_d, L.src_h, sizeof(ctm_frame) * nf, cudaMemcpyHostToDevice, L.stream);
    int st = e == cudaSuccess ? CTM_OK : CTM_ECUDA;
    if (st == CTM_OK) {
        if (S->cfg.plain) {
            for (int i = 0; i < nf && st == CTM_OK; ++i) {
                const ctm_frame &f = L.frames_h[i];
                const int o = L.box_off[i];
                st = ctm_match_boxes_plain(L.ctx, f.left, f.right, f.width, f.height, f.pitch, L.boxes_d + o,
                                           f.box_count, f.f_px, f.baseline_m, L.disp_d + o, L.depth_d + o,
                                           L.flags_d + o, (ctm_stream)L.stream);
            }
        } else {
            st = ctm::match_batch_dev(L.ctx, L.frames_d, S->cfg.mapped ? L.src_d : nullptr, L.counts_d, L.boxes_d,
                                      L.disp_d, L.depth_d, L.flags_d, nullptr, 1, (ctm_stream)L.stream);
        }
    }
    if (st == CTM_OK && nb > 0) {
        e = cudaMemcpyAsync(L.disp_h, L.disp_d, sizeof(float) * nb, cudaMemcpyDeviceToHost, L.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(L.depth_h, L.depth_d, sizeof(float) * nb, cudaMemcpyDeviceToHost, L.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(L.flags_h, L.flags_d, (size_t)nb, cudaMemcpyDeviceToHost, L.stream);
        if (e != cudaSuccess) st = CTM_ECUDA;
    }
    if (st == CTM_OK) {  // the batch's bounded-wait flag (ctm_stats.error) into counts_h[3]
        L.counts_h[3] = 0;
        e = cudaMemcpyAsync(&L.counts_h[3], ctm::context_error_flag(L.ctx), sizeof(int32_t), cudaMemcpyDeviceToHost,
                            L.stream);
        if (e != cudaSuccess) st = CTM_ECUDA;
    }
    if (st == CTM_OK) {
        e = cudaEventRecord(L.done, L.stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(L.stream, lane_done_cb, S);
        if (e != cudaSuccess) st = CTM_ECUDA;
    }
    if (st != CTM_OK) {
        // nothing may still read the lane's staging: wait for what was enqueued
        cudaGetLastError();
        cudaStreamSynchronize(L.stream);
        cudaGetLastError();
        complete_jobs(S, L.batch, L.index, nf, st);
        L.batch.clear();
        return;
    }
    L.busy = true;
    L.status = CTM_OK;
    int busy = 0;
    for (const Lane &x : S->lanes) busy += x.busy ? 1 : 0;
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->st.batches;
    S->st.batched_frames += nf;
    if (busy > S->st.max_lanes_busy) S->st.max_lanes_busy = busy;
}

// A lane's batch has finished on the device: hand the outputs to the callers.
void finish(ctm_server *S, Lane &L, int status)
{
    const int nf = (int)L.batch.size();
    const bool expired = status == CTM_OK && L.counts_h[3] != 0;
    if (status == CTM_OK) {
        for (int i = 0; i < nf; ++i) {
            const ctm_request &r = L.batch[i]->r;
            const int o = L.box_off[i], n = r.n_boxes;
            if (n <= 0) continue;
            memcpy(r.disp_host, L.disp_h + o, sizeof(float) * (size_t)n);
            memcpy(r.depth_host, L.depth_h + o, sizeof(float) * (size_t)n);
            memcpy(r.flags_host, L.flags_h + o, (size_t)n);
        }
    }
    complete_jobs(S, L.batch, L.index, nf, expired ? CTM_ETIMEOUT : status);
    L.batch.clear();
    L.busy = false;
}

void worker_main(ctm_server *S)
{
    const bool dev_ok = cudaSetDevice(S->device) == cudaSuccess;
    std::vector<Job *> newly;
    bool progress = true;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            bool any_busy = false, any_idle = false;
            for (const Lane &L : S->lanes) (L.busy ? any_busy : any_idle) = true;
            const bool can_dispatch = any_idle && !S->admitted.empty();
            if (!progress && !S->kick && !can_dispatch) {
                if (S->stopping && S->arrivals.empty() && S->admitted.empty() && !any_busy) break;
                // a lane's callback or a submit sets kick; the timeout is a safety net
                S->cv_work.wait_for(lk, any_busy ? std::chrono::microseconds(500) : std::chrono::milliseconds(5),
                                    [S] { return S->kick; });
            }
            S->kick = false;
            // admission by device memory, in arrival order
            while (!S->arrivals.empty()) {
                Job *j = S->arrivals.front();
                const int64_t off = S->arena.alloc(2 * j->pitch * (int64_t)j->r.height);
                if (off < 0) break;
                S->arrivals.pop_front();
                j->arena_off = off;
                j->t_admit = now_ns();
                ++S->admitted_now;
                if (S->admitted_now > S->st.max_admitted) S->st.max_admitted = S->admitted_now;
                newly.push_back(j);
            }
            if (S->arena.peak() > S->st.arena_peak_bytes) S->st.arena_peak_bytes = S->arena.peak();
        }
        progress = false;
        for (Job *j : newly) {
            if (dev_ok && (j->gather || upload(S, j))) {
                S->admitted.push_back(j);
            } else {
                complete_jobs(S, std::vector<Job *>{j}, -1, 0, CTM_ECUDA);
            }
        }
        newly.clear();
        for (Lane &L : S->lanes) {
            if (!L.busy) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            finish(S, L, q == cudaSuccess ? L.status : CTM_ECUDA);
            progress = true;  // arena space freed: admit again before waiting
        }
        for (Lane &L : S->lanes) {
            if (L.busy || S->admitted.empty()) continue;
            dispatch(S, L);
        }
    }
}

void destroy_lane(Lane &L)
{
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.ctx) ctm_destroy(L.ctx);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.dev_mem) cudaFree(L.dev_mem);
    if (L.host_mem) cudaFreeHost(L.host_mem);
    cudaGetLastError();
    L = Lane();
}

void destroy_resources(ctm_server *S)
{
    for (Lane &L : S->lanes) destroy_lane(L);
    for (cudaEvent_t e : S->event_pool) cudaEventDestroy(e);
    S->event_pool.clear();
    if (S->upload) {
        cudaStreamSynchronize(S->upload);
        cudaStreamDestroy(S->upload);
    }
    if (S->arena_d) cudaFree(S->arena_d);
    cudaGetLastError();
}

int create_lane(ctm_server *S, Lane &L, int index)
{
    const ctm_server_config &c = S->cfg;
    L.index = index;
    L.max_boxes = c.frames_per_batch * c.max_boxes_per_frame;
    int st = ctm_create(&L.ctx, &S->p, c.frames_per_batch, c.max_width, c.max_height, L.max_boxes);
    if (st != CTM_OK) return st;
    if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return CTM_ECUDA;
    }
    const int64_t F = c.frames_per_batch, B = L.max_boxes;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up((int64_t)(off + bytes), 256); return o; };
    const size_t o_frames = take(sizeof(ctm_frame) * F);
    const size_t o_src = take(sizeof(ctm_frame) * F);
    const size_t o_boxes = take(sizeof(ctm_box) * B);
    const size_t o_counts = take(sizeof(int32_t) * 4);
    const size_t o_disp = take(sizeof(float) * B);
    const size_t o_depth = take(sizeof(float) * B);
    const size_t o_flags = take((size_t)B);
    if (ctm::dev_alloc(&L.dev_mem, off) != cudaSuccess || cudaHostAlloc(&L.host_mem, off, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return CTM_ENOMEM;
    }
    char *d = static_cast<char *>(L.dev_mem), *h = static_cast<char *>(L.host_mem);
    L.frames_d = reinterpret_cast<ctm_frame *>(d + o_frames);
    L.src_d = reinterpret_cast<ctm_frame *>(d + o_src);
    L.boxes_d = reinterpret_cast<ctm_box *>(d + o_boxes);
    L.counts_d = reinterpret_cast<int32_t *>(d + o_counts);
    L.disp_d = reinterpret_cast<float *>(d + o_disp);
    L.depth_d = reinterpret_cast<float *>(d + o_depth);
    L.flags_d = reinterpret_cast<uint8_t *>(d + o_flags);
    L.frames_h = reinterpret_cast<ctm_frame *>(h + o_frames);
    L.src_h = reinterpret_cast<ctm_frame *>(h + o_src);
    L.boxes_h = reinterpret_cast<ctm_box *>(h + o_boxes);
    L.counts_h = reinterpret_cast<int32_t *>(h + o_counts);
    L.disp_h = reinterpret_cast<float *>(h + o_disp);
    L.depth_h = reinterpret_cast<float *>(h + o_depth);
    L.flags_h = reinterpret_cast<uint8_t *>(h + o_flags);
    L.bytes = 2 * off + ctm::context_device_bytes(L.ctx);
    // capture the lane's graph now, on an empty batch, so serving never captures
    memset(L.host_mem, 0, off);
    cudaError_t e = cudaMemcpyAsync(L.dev_mem, L.host_mem, off, cudaMemcpyHostToDevice, L.stream);
    if (e != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    if (!c.plain) {
        st = ctm::match_batch_dev(L.ctx, L.frames_d, c.mapped ? L.src_d : nullptr, L.counts_d, L.boxes_d, L.disp_d,
                                  L.depth_d, L.flags_d, nullptr, 1, (ctm_stream)L.stream);
        if (st != CTM_OK) return st;
    }
    if (cudaStreamSynchronize(L.stream) != cudaSuccess) { cudaGetLastError(); return CTM_ECUDA; }
    return CTM_OK;
}

bool config_ok(const ctm_server_config &c)
{
    return c.lanes >= 1 && c.lanes <= 8 && c.frames_per_batch >= 1 && c.frames_per_batch <= 64 &&
           c.max_width >= 1 && c.max_width <= 32768 && c.max_height >= 1 && c.max_height <= 32768 &&
           c.max_boxes_per_frame >= 1 && c.max_boxes_per_frame <= 65536 && c.max_queue >= 1 &&
           c.image_budget_bytes >= 256 && (c.plain == 0 || c.plain == 1) && (c.mapped == 0 || c.mapped == 1) &&
           (int64_t)c.frames_per_batch * c.max_boxes_per_frame <= (1 << 22);
}

// Mapped servers: a frame the gather can read in place -- 16-byte aligned rows
// and width, in memory the device reads at the host address (page-locked, or any
// memory where the device has pageable memory access).
bool gatherable(const ctm_server *S, const ctm_request &r)
{
    if ((reinterpret_cast<uintptr_t>(r.left_host) | reinterpret_cast<uintptr_t>(r.right_host) | (uintptr_t)r.pitch |
         (uintptr_t)r.width) & 15u)
        return false;
    if (S->pageable_access) return true;
    for (const void *p : {(const void *)r.left_host, (const void *)r.right_host}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer != p) return false;
    }
    return true;
}

}  // namespace

extern "C" {

int64_t ctm_server_now_ns(void) { return now_ns(); }

int ctm_server_default_config(ctm_server_config *cfg)
{
    if (!cfg) return CTM_EINVAL;
    cfg->lanes = 4;
    cfg->frames_per_batch = 8;
    cfg->max_width = 3840;
    cfg->max_height = 2160;
    cfg->max_boxes_per_frame = 256;
    cfg->max_queue = 256;
    cfg->image_budget_bytes = 1LL << 30;
    cfg->plain = 0;
    cfg->mapped = 1;
    return CTM_OK;
}

int ctm_server_create(ctm_server **out, const ctm_params *p, const ctm_server_config *cfg)
{
    if (!out || !p || !cfg) return CTM_EINVAL;
    *out = nullptr;
    if (!config_ok(*cfg)) return CTM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CTM_ENODEV; }
    ctm_server *S = new (std::nothrow) ctm_server();
    if (!S) return CTM_ENOMEM;
    S->device = dev;
    S->p = *p;
    S->cfg = *cfg;
    if (S->cfg.plain) S->cfg.mapped = 0;  // the plain path uploads
    S->arena.reset(cfg->image_budget_bytes, 256);
    cudaDeviceGetAttribute(&S->pageable_access, cudaDevAttrPageableMemoryAccess, dev);
    cudaGetLastError();
    int st = CTM_OK;
    if (ctm::dev_alloc(reinterpret_cast<void **>(&S->arena_d), (size_t)S->arena.size()) != cudaSuccess) st = CTM_ENOMEM;
    if (st == CTM_OK && cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking) != cudaSuccess) st = CTM_ECUDA;
    if (st == CTM_OK) {
        S->lanes.resize(cfg->lanes);
        for (int i = 0; i < cfg->lanes && st == CTM_OK; ++i) st = create_lane(S, S->lanes[i], i);
    }
    if (st == CTM_OK) {
        S->st.arena_bytes = S->arena.size();
        for (const Lane &L : S->lanes) S->st.workspace_bytes += (int64_t)L.bytes;
        try {
            S->worker = std::thread(worker_main, S);
        } catch (...) {
            st = CTM_ENOMEM;
        }
    }
    if (st != CTM_OK) {
        cudaGetLastError();
        destroy_resources(S);
        delete S;
        return st;
    }
    *out = S;
    return CTM_OK;
}

int ctm_server_submit(ctm_server *S, const ctm_request *r)
{
    if (!S || !r) return CTM_EINVAL;
    if (!r->left_host || !r->right_host || r->width < 1 || r->height < 1 || r->pitch < r->width ||
        r->n_boxes < 0)
        return CTM_EINVAL;
    if (r->n_boxes > 0 && (!r->boxes_host || !r->disp_host || !r->depth_host || !r->flags_host))
        return CTM_EINVAL;
    if (r->width > S->cfg.max_width || r->height > S->cfg.max_height || r->n_boxes > S->cfg.max_boxes_per_frame)
        return CTM_ETOOBIG;
    const int64_t pitch = round_up(r->width, kImagePitchAlign);
    if (S->arena.rounded(2 * pitch * (int64_t)r->height) > S->arena.size()) return CTM_ETOOBIG;
    Job *j = new (std::nothrow) Job();
    if (!j) return CTM_ENOMEM;
    j->r = *r;
    j->pitch = pitch;
    if (S->cfg.mapped) j->gather = gatherable(S, *r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete j;
            return CTM_EINVAL;
        }
        if ((int64_t)S->arrivals.size() >= S->cfg.max_queue) {
            ++S->st.rejected;
            delete j;
            return CTM_EAGAIN;
        }
        j->t_submit = now_ns();
        S->arrivals.push_back(j);
        ++S->st.submitted;
        ++S->outstanding;
        S->kick = true;
    }
    S->cv_work.notify_one();
    return CTM_OK;
}

int ctm_server_poll(ctm_server *S, ctm_completion *out, int32_t max, int64_t timeout_us, int32_t *n_out)
{
    if (!S || !n_out || max < 0 || (max > 0 && !out)) return CTM_EINVAL;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->completions.empty() && timeout_us != 0 && max > 0) {
        auto ready = [S] { return !S->completions.empty(); };
        if (timeout_us < 0)
            S->cv_done.wait(lk, ready);
        else
            S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    int n = 0;
    while (n < max && !S->completions.empty()) {
        out[n++] = S->completions.front();
        S->completions.pop_front();
    }
    S->outstanding -= n;
    *n_out = n;
    return CTM_OK;
}

int64_t ctm_server_outstanding(ctm_server *S)
{
    if (!S) return CTM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    return S->outstanding;
}

int ctm_server_get_stats(ctm_server *S, ctm_server_stats *out)
{
    if (!S || !out) return CTM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return CTM_OK;
}

int ctm_server_destroy(ctm_server *S)
{
    if (!S) return CTM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->kick = true;
    }
    S->cv_work.notify_one();
    if (S->worker.joinable()) S->worker.join();
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != S->device) cudaSetDevice(S->device);
    destroy_resources(S);
    for (Job *j : S->arrivals) delete j;  // none after the worker has drained
    delete S;
    return CTM_OK;
}

}  // extern "C"
