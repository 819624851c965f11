/* Serving loop over libds.so: continuous batching of event requests.
 *
 * The paper runs the Downstream algorithm inside a trigger that processes
 * event batches as they stream in (GPU Implementation section: events in
 * parallel, one block per event, throughput per GPU).  This server is the
 * deployment form of ds_reconstruct + ds_vertex for requests that arrive over
 * time: it keeps geometry, network weights and one library context per slot
 * resident on the device, merges queued requests into one batch per launch
 * (continuous batching: requests that arrive while other batches run are
 * admitted as soon as a slot and device memory are free), runs up to n_slots
 * batches concurrently on their own streams, and returns each request's
 * tracks and vertices in the request's own numbering.  The paper has no
 * serving loop of its own; the scheduling here is this library's.
 *
 * Events are independent, so a request's results do not depend on what it is
 * batched with: they are bit-identical to running it alone.
 *
 * All functions are thread-safe.  Errors: DS_ERR_ARG for null pointers,
 * inconsistent sizes or a bad configuration; DS_ERR_CAPACITY when a request
 * can never be admitted (larger than a slot's batch limits after splitting,
 * or than the device-memory budget); DS_ERR_CUDA / DS_ERR_OOM when set-up
 * fails. */
#ifndef DS_SERVE_H
#define DS_SERVE_H

#include "ds.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ds_server ds_server;

typedef struct {
    int32_t n_slots;            /* batches in flight at once, each with its own stream and
                                   library context, 1..16 */
    int32_t max_batch_events;   /* limits of one batch (one ds_reconstruct + ds_vertex launch) */
    int32_t max_batch_seeds;
    int32_t max_batch_hits;
    int32_t events_per_launch;  /* 0: whole requests are merged up to the batch limits
                                   (continuous batching).  k > 0: every launch carries at most
                                   k events of ONE request, requests served one after the
                                   other (k = 1, n_slots = 1: the plain one-event-per-launch
                                   form). */
    int32_t vertices_per_seed;  /* vertex output capacity of a batch = this x its seeds + 4096 */
    int64_t hbm_budget;         /* bytes of device memory for the buffers of batches in flight;
                                   a batch is admitted only when its buffers fit (0: 25 % of
                                   the device memory free at creation) */
    int32_t mlp_precision;      /* DS_MLP_FP32 / DS_MLP_BF16 / DS_MLP_FP8 for every batch */
    int32_t graphs;             /* 1 (default): every slot keeps fixed device buffers sized to
                                   the batch limits, taken from hbm_budget at creation, and runs
                                   each batch's kernels as one replay of a CUDA graph captured at
                                   creation for that slot and the batch's event-count bucket
                                   (powers of two up to max_batch_events; a batch is padded with
                                   empty events to its bucket, see DS_BATCH_CAPACITY).  A batch
                                   is admitted when a slot is free.  0, or when the slots'
                                   buffers do not fit hbm_budget: buffers per batch from the
                                   budget (admission by free device memory), kernels launched
                                   one by one.  Results are identical. */
    int32_t gather_max_bytes;   /* request arrays smaller than this many bytes whose whole range
                                   the device can read at the same address (pinned memory that
                                   cudaPointerGetAttributes reports as host memory mapped into
                                   the device's address space) are read straight from host
                                   memory by one gather kernel per batch, which moves many
                                   small arrays without a copy-engine set-up for each; larger
                                   arrays and pageable memory go through cudaMemcpyAsync.
                                   0: copies only.  Default 1 MiB.  Results are identical. */
} ds_server_config;

/* One request: n_events events with their seeds and hits, HOST memory in the
 * layouts of ds_reconstruct (offsets relative to the request, starting at 0).
 * Pinned memory is read asynchronously (gathered by the device or copied,
 * see gather_max_bytes), pageable memory goes through the driver's staging.  The caller keeps inputs and outputs alive and untouched
 * until the request's completion is returned by ds_server_poll. */
typedef struct {
    int32_t n_events;
    int32_t reserved0;
    const int32_t *seed_off, *hit_off;          /* [n_events + 1] */
    const float *seed_x, *seed_y, *seed_tx, *seed_ty, *seed_qop, *seed_chi2;
    const float *hit_x0, *hit_ybeg, *hit_yend;
    const uint8_t *hit_layer;
    /* outputs: records in the request's numbering (event, seed and hit indices
       relative to the request; vertex i, j index the request's tracks) */
    ds_track *tracks;
    int32_t trk_capacity;
    int32_t vtx_capacity;
    int32_t *trk_off;                           /* [n_events + 1] */
    ds_vertex_rec *vertices;
    int32_t *vtx_off;                           /* [n_events + 1] */
    double arrival;             /* server clock (ds_server_now) at which the request arrives
                                   (<= 0: now).  Latency is counted from it, also when it is
                                   in the past.  Requests are served in submission order once
                                   arrived (trace replay for load tests). */
} ds_request;

typedef struct {
    int64_t id;                 /* as returned by ds_server_submit */
    int32_t status;             /* DS_OK, DS_ERR_CAPACITY (outputs truncated to the request's
                                   capacities; counts below are the full counts), or the
                                   ds_sync_status code of a failed batch */
    int32_t n_tracks, n_vertices;
    int32_t n_batches;          /* launches that carried this request */
    double t_arrival, t_admit, t_done;   /* server clock, seconds */
} ds_completion;

typedef struct {
    int64_t requests_done, events_done, batches;
    int64_t hbm_budget, hbm_peak;        /* bytes: budget and peak in use by batches in flight */
    int64_t context_bytes;               /* device workspaces of the slots' contexts */
    int32_t peak_inflight;               /* most batches on the device at once */
    int32_t queued;                      /* requests waiting now */
    double worker_launch_s;              /* worker thread time spent enqueueing batches */
    double worker_finish_s;              /* ... returning results to the requests */
    double worker_wall_s;                /* worker thread lifetime so far */
    int32_t graphs;                      /* 1: batches replay captured CUDA graphs */
    int32_t graphs_captured;             /* graphs instantiated at creation (slots x buckets) */
    int64_t bytes_gathered;              /* input bytes read by the gather kernel */
    int64_t bytes_copied;                /* input bytes uploaded by cudaMemcpyAsync */
} ds_server_stats;

DS_API void ds_server_default_config(ds_server_config *cfg);
/* Create a server on `device` (one worker thread; slot contexts reserved to the
 * batch limits).  weights, params and geometry are copied. */
DS_API ds_status ds_server_create(ds_server **out, int device, const ds_geometry *geom,
                                  const ds_nn_weights *weights, const ds_params *params,
                                  const ds_server_config *cfg);
/* Queue a request; *id receives its id.  Non-blocking. */
DS_API ds_status ds_server_submit(ds_server *s, const ds_request *req, int64_t *id);
/* Seconds on the server's clock (steady clock, zero at creation). */
DS_API double ds_server_now(ds_server *s);
/* Completed requests, oldest first: waits up to timeout_s seconds for at least
 * one, writes at most max_out and returns how many (0 on time-out). */
DS_API int32_t ds_server_poll(ds_server *s, ds_completion *out, int32_t max_out, double timeout_s);
/* Wait until every submitted request has completed (completions stay queued
 * for ds_server_poll). */
DS_API ds_status ds_server_drain(ds_server *s);
DS_API ds_status ds_server_stats_get(ds_server *s, ds_server_stats *out);
/* Stop the worker after the requests in flight; queued requests are dropped. */
DS_API void ds_server_destroy(ds_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DS_SERVE_H */
