/*
 * ctm_server.h -- serving loop of libctm.so: continuous batching of stereo
 * frames from several camera streams onto one GPU.
 *
 * The paper's per-frame pipeline (Algorithm 2: census, per-box block search,
 * verification, aggregation, depth) runs once per frame on the cameras' own
 * cadence (Sec. 4.3); a deployment serves several stereo streams at once.
 * The paper describes no serving system, so this interface is this library's
 * own.  Every frame goes through the same launch sequence as ctm_match_batch,
 * so a frame's outputs are the same whether it ran alone or batched with
 * others.
 *
 * Model:
 *  - ctm_server_submit() queues a frame (host images, host boxes, host output
 *    arrays) and returns at once.  A native worker thread owns the GPU side.
 *  - Admission by device memory: a queued frame is admitted, in arrival order,
 *    once its two images fit in a fixed device arena (image_budget_bytes); its
 *    images are then copied to the device on an upload stream while earlier
 *    batches compute.
 *  - Continuous batching: the worker keeps `lanes` batches in flight, each on
 *    its own stream with its own workspace (census planes, plans, counters,
 *    allocated once at creation and kept resident).  Whenever a lane is idle it
 *    takes every admitted frame (up to frames_per_batch) as one batch and
 *    replays the lane's captured CUDA graph over them; frames that arrive
 *    while other batches run are admitted as arena space frees up and start on
 *    the next idle lane, overlapping with the batches still running.
 *  - A frame completes when its outputs have been written to the caller's host
 *    arrays; its completion record (with timestamps) is then returned by
 *    ctm_server_poll().
 *
 * Threading: submit, poll and stats may be called from any thread; create and
 * destroy from one.  Every call uses the device that was current at create.
 */
#ifndef CTM_SERVER_H
#define CTM_SERVER_H

#include "ctm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_server ctm_server;

/* Server configuration. */
typedef struct {
    int32_t lanes;               /* batches in flight at once, 1..8 (stream + workspace each) */
    int32_t frames_per_batch;    /* frames one batch holds, 1..64 */
    int32_t max_width, max_height;   /* largest frame accepted */
    int32_t max_boxes_per_frame;     /* largest box count accepted */
    int32_t max_queue;           /* submitted-but-not-admitted frames; beyond: CTM_EAGAIN */
    int64_t image_budget_bytes;  /* device arena for admitted frames' images */
    int32_t plain;               /* 1: run batches through the plain per-box path (comparison) */
    int32_t mapped;              /* 1: a frame whose images the device can read in host memory
                                    (page-locked, or any memory where the device reports
                                    pageable memory access) and whose left, right, pitch and
                                    width are multiples of 16 bytes is not uploaded: its batch
                                    reads only the bytes its census needs straight from the
                                    host images, as ctm_match_batch_mapped does; other frames
                                    are uploaded whole.  0: every frame uploaded whole.
                                    Ignored with plain = 1 (frames are uploaded) */
} ctm_server_config;

/* One frame to serve.  Host pointers; with mapped = 1 the device reads the
 * images in place where it can (see ctm_server_config.mapped); an uploaded
 * frame's copy runs asynchronously from pinned host memory (cudaHostAlloc or a
 * pinned torch tensor), while from pageable memory it blocks the worker thread.
 * Every pointer must stay valid, the images unchanged and the output arrays
 * untouched, until the frame's completion has been returned by ctm_server_poll().  Boxes use full-resolution pixels of
 * this frame; their `frame` field is ignored. */
typedef struct {
    const uint8_t *left_host, *right_host;  /* width x height, `pitch` bytes per row */
    int32_t width, height, pitch;
    int32_t n_boxes;
    const ctm_box *boxes_host;   /* n_boxes */
    float f_px, baseline_m;      /* Eq. 1 */
    float *disp_host;            /* n_boxes outputs, as ctm_match_boxes */
    float *depth_host;
    uint8_t *flags_host;
    uint64_t tag;                /* returned in the completion record */
} ctm_request;

/* Completion record.  Times are CLOCK_MONOTONIC nanoseconds (ctm_server_now_ns). */
typedef struct {
    uint64_t tag;
    int32_t status;        /* CTM_OK, CTM_ECUDA if the frame's batch failed, or
                              CTM_ETIMEOUT if a bounded device wait of its batch
                              expired (outputs incomplete) */
    int32_t n_boxes;
    int64_t t_submit_ns;   /* ctm_server_submit() accepted it */
    int64_t t_admit_ns;    /* arena space granted, image upload issued */
    int64_t t_launch_ns;   /* its batch was enqueued on a lane */
    int64_t t_done_ns;     /* outputs written to the host arrays */
    int32_t lane;          /* lane it ran on */
    int32_t batch_frames;  /* frames in its batch */
} ctm_completion;

typedef struct {
    int64_t submitted, completed, rejected;  /* rejected: CTM_EAGAIN returns */
    int64_t batches, batched_frames;         /* batches launched, frames over all of them */
    int64_t arena_bytes, arena_peak_bytes;   /* arena size, high-water mark */
    int64_t workspace_bytes;                 /* resident lane workspaces and staging */
    int32_t max_admitted;                    /* most frames holding arena space at once */
    int32_t max_lanes_busy;                  /* most batches in flight at once */
} ctm_server_stats;

/* Default configuration: 4 lanes, 8 frames per batch, 3840x2160, 256 boxes,
 * queue 256, arena 1 GiB, batched path, images read in place where possible
 * (mapped = 1). */
int ctm_server_default_config(ctm_server_config *cfg);

/* Create a server on the current device: validates `p` (CTM_EINVAL as
 * ctm_create) and `cfg` (CTM_EINVAL), allocates the arena, the lanes'
 * workspaces and pinned staging (CTM_ENOMEM), captures each lane's CUDA graph
 * on an empty batch, and starts the worker thread.  *out is NULL on error. */
int ctm_server_create(ctm_server **out, const ctm_params *p, const ctm_server_config *cfg);

/* Queue one frame.  CTM_EINVAL: null pointer, bad size or pitch;
 * CTM_ETOOBIG: the frame is larger than max_width x max_height, has more than
 * max_boxes_per_frame boxes, or its images alone exceed the arena;
 * CTM_EAGAIN: max_queue frames are already waiting for admission (nothing
 * queued; submit again later); CTM_EINVAL also after destroy has begun. */
int ctm_server_submit(ctm_server *srv, const ctm_request *req);

/* Move up to `max` completion records into out[], waiting up to timeout_us
 * microseconds (0: do not wait; negative: wait until at least one) for the
 * first.  *n_out receives the count. */
int ctm_server_poll(ctm_server *srv, ctm_completion *out, int32_t max, int64_t timeout_us,
                    int32_t *n_out);

/* Frames submitted and not yet returned by ctm_server_poll. */
int64_t ctm_server_outstanding(ctm_server *srv);

int ctm_server_get_stats(ctm_server *srv, ctm_server_stats *out);

/* Finish every submitted frame (their outputs are written; completion records
 * not yet polled are dropped), stop the worker and free everything. */
int ctm_server_destroy(ctm_server *srv);

/* The clock of the completion timestamps. */
int64_t ctm_server_now_ns(void);

#ifdef __cplusplus
}
#endif
#endif /* CTM_SERVER_H */
