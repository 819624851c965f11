/*
 * ds.h - C ABI of the B300 Downstream tracking + two-track vertexing library
 * (libds.so).
 *
 * The calls follow the paper's statement of the problem (arXiv:2503.13092):
 *   inputs   SciFi seeds not used by long tracks (x, y, tx, ty, q/p, chi2 at the
 *            last SciFi station) and decoded UT hits (Algorithm Design section);
 *   output   downstream tracks: state (x, y, tx, ty, q/p) at the UT reference
 *            plane, chi2, UT hits and ghost-killer response (Ghost-Killer Neural
 *            Network section);
 *   output   two-track vertices from opposite-charge pairs (Vertexing Two
 *            Downstream Tracks section, Eqs. 3-4; Expected Physics Impact).
 *
 * Conventions
 *   - Units: mm, MeV, MeV/c; q/p in c/MeV.  Layer order: UTaX, UTaU, UTbV, UTbX.
 *   - Batch inputs and outputs are DEVICE pointers owned by the caller (any CUDA
 *     allocator); the library never frees them.  Host structs passed by pointer
 *     are read during the call only and may be freed afterwards.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream; a context is not thread safe and
 *     must be used from one host thread at a time.  Several contexts may share a
 *     device.
 *   - Errors found on the host (bad arguments, missing geometry or weights, a
 *     failed CUDA call) are returned immediately and described by
 *     ds_last_error().  Errors found on the device (malformed offsets, hits that
 *     break the strip/sector contract, capacity overflow, a bounded wait that ran
 *     out) set bits in a device-side flag word that ds_sync_status() reads after
 *     synchronising the stream.
 *   - Workspaces are device memory owned by the context.  They are sized by
 *     ds_reserve(); a call that needs more grows them first (a synchronous
 *     allocation), so callers that capture CUDA graphs reserve beforehand.
 */
#ifndef DS_H
#define DS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DS_API __attribute__((visibility("default")))
#else
#define DS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ds_ctx ds_ctx;

typedef enum {
    DS_OK = 0,
    DS_ERR_ARG = -1,          /* invalid argument (null pointer, bad size, bad parameter) */
    DS_ERR_CUDA = -2,         /* a CUDA runtime call failed (message in ds_last_error) */
    DS_ERR_CAPACITY = -3,     /* an output capacity was exceeded; outputs truncated */
    DS_ERR_NOT_READY = -4,    /* geometry or network weights not loaded */
    DS_ERR_TIMEOUT = -5,      /* a device-side bounded wait gave up */
    DS_ERR_DEVICE_FLAG = -6,  /* the device flagged malformed input (ds_stats.device_flags) */
    DS_ERR_OOM = -7           /* device allocation failed */
} ds_status;

/* Device flag bits, reported in ds_stats.device_flags by ds_sync_status(). */
enum {
    DS_FLAG_BAD_OFFSETS = 1u << 0,   /* seed_off / hit_off not monotone or not matching totals */
    DS_FLAG_BAD_LAYER = 1u << 1,     /* a hit with layer >= 4 or a non-finite coordinate (ignored) */
    DS_FLAG_STRIP_SECTOR = 1u << 2,  /* a strip extent crosses its Y-sector boundary */
    DS_FLAG_EVENT_TOO_LARGE = 1u << 3, /* an event has more than 65535 hits (event skipped) */
    DS_FLAG_TRACK_CAPACITY = 1u << 4,  /* more tracks than ds_tracks.capacity (truncated) */
    DS_FLAG_VERTEX_CAPACITY = 1u << 5, /* more vertices than capacity, or an event with more
                                          than 4096 tracks (only its first 4096 are paired) */
    DS_FLAG_TIMEOUT = 1u << 6,         /* a bounded device-side wait ran out */
    DS_FLAG_CAND_CAPACITY = 1u << 7    /* candidate buffer full (ds_params.cand_per_seed x
                                          seeds); the seeds concerned got no track */
};

/* Geometry of the UT and of the magnet kink model (Algorithm Design section,
 * Eq. 1; Fig. 2).  Host struct, copied into the context. */
typedef struct {
    double z_layer[4];     /* z of UTaX, UTaU, UTbV, UTbX (mm), strictly increasing */
    double dxdy[4];        /* tan(stereo angle) per layer; a hit measures x0 = x - dxdy*y */
    double y_min;          /* lower edge of the first Y sector (mm) */
    double sector_h;       /* Y-sector height (mm) */
    int32_t n_sectors;     /* number of Y sectors, 1..32 */
    int32_t reserved0;
    double x_half_bins;    /* half-range of x0 covered by the per-sector x bins (mm) */
    double z_seed;         /* z of the SciFi seed state (mm) */
    double zmag[4];        /* z_magnet = zmag0 + zmag1*tx^2 + zmag2*ty^2 + zmag3*|q/p| */
    double kappa;          /* transverse momentum kick of the kink (MeV/c) */
    double mp;             /* magnet polarity, +1 or -1 */
    double gamma0, gamma1; /* Eq. 3: gamma(q/p) = -MP (gamma0 + gamma1*q/p); 0,0 = straight */
    double z_ref;          /* reference plane of output states, midpoint of the UT (mm) */
    double sigma_hit;      /* UT hit resolution (mm) */
    double sigma_mag;      /* magnet-point resolution used in the fit (mm) */
} ds_geometry;

/* Ghost-killer network (Ghost-Killer Neural Network section): n_in inputs,
 * one or two ReLU hidden layers, one sigmoid output.  Host pointers, row-major
 * [out][in] per layer, FP32.  Supported shapes: n_in <= 16, n_h1 <= 32,
 * n_h2 <= 32 (n_h2 = 0: single hidden layer, the paper's 8-14-1).  Input i is
 * normalised as (phi_i - mean_i) * scale_i. */
typedef struct {
    int32_t n_in, n_h1, n_h2, reserved0;
    const float *w1, *b1;  /* [n_h1][n_in], [n_h1] */
    const float *w2, *b2;  /* [n_h2][n_h1], [n_h2]; ignored when n_h2 = 0 */
    const float *w3;       /* [n_h2] (or [n_h1] when n_h2 = 0) */
    float b3;
    int32_t reserved1;
    const float *mean, *scale; /* [n_in] */
} ds_nn_weights;

enum { DS_MLP_FP32 = 0, DS_MLP_BF16 = 1, DS_MLP_FP8 = 2 };

/* Method parameters.  ds_default_params() fills the defaults. */
typedef struct {
    double w1a, w1b;       /* first (UTbX) window half-width: w1a + w1b*|q/p| (mm) */
    double w2;             /* refined window half-width in UTaX/UTaU/UTbV (mm) */
    double dy_tol;         /* tolerance on a strip's y extent (mm) */
    double nn_threshold;   /* keep a track if its ghost-killer response < threshold */
    double doca_max;       /* keep a vertex if DOCA < doca_max (mm) */
    double nr_tol;         /* Newton-Raphson step tolerance (mm) */
    double eps_parallel;   /* sin^2(opening angle) below which a pair is re-solved in FP64 */
    int32_t k1;            /* UTbX hits kept per seed, 1..10 (paper: 10) */
    int32_t first_window_origin; /* 1: window centred on the line (0,0,0)-magnet point (Dv0) */
    int32_t pick_chi2;     /* 0: best = lowest NN response among those < threshold;
                              1: best = lowest chi2/ndof, then the threshold cut */
    int32_t clone_kill;    /* 1: kill clones sharing more than two UT hits */
    int32_t training;      /* 1: fixed 100/10 mm windows, no clone killing */
    int32_t nr_max_iter;   /* Newton-Raphson iteration limit */
    int32_t mlp_precision; /* arithmetic of the ghost-killer network: DS_MLP_FP32 (default,
                              CUDA cores), DS_MLP_BF16 or DS_MLP_FP8 (E4M3) on the tensor
                              cores with FP32 accumulation (see ds_mlp_eval) */
    int32_t fault_inject;  /* 0 in normal use.  Tests of the failure path: bit 0 makes the
                              search kernel's bounded wait for its staged data run out, so
                              the call reports DS_ERR_TIMEOUT (flag DS_FLAG_TIMEOUT) and
                              produces no tracks; no GPU fault is involved. */
    int32_t cand_per_seed; /* candidate buffer size per seed on average (default 16, max
                              40 = 10 x 1 x 2 x 2; training mode always uses 40); exceeding
                              it raises DS_FLAG_CAND_CAPACITY.  Used only when candidates
                              go through the buffer (see fuse_network) */
    int32_t variant;       /* 0: Dv0 (default).  1: Dv1 (Algorithm Design section): every
                              UTbX hit whose implied kink |tx' - tx_seed| < dv1_dtx_max is
                              joined to the magnet point; the closest UTaX hit within
                              dv1_w_tri of that line completes a triplet; the k1 triplets
                              with the smallest residual go on to the stereo windows */
    double dv1_dtx_max;    /* Dv1 kink bound (default 0.8: p above ~1.5 GeV/c) */
    double dv1_w_tri;      /* Dv1 UTaX collinearity tolerance, mm (default 1) */
    int32_t fuse_network;  /* 0 (default): candidates are written to the candidate buffer and
                              scored and picked by separate kernels (ds_candidates can export
                              them).  1: with the FP32 two-hidden-layer network outside
                              training mode, every candidate is scored inside the search
                              kernel and only each seed's winner leaves it (no candidate
                              buffer; measured slower on B300: the network then runs at the
                              search kernel's occupancy).  Training mode, the BF16 / FP8
                              network and single-hidden-layer networks always use the
                              buffer.  Results are identical either way. */
    int32_t reserved2;
} ds_params;

/* One event batch (CSR over events).  Device pointers. */
typedef struct {
    int32_t n_events;
    int32_t n_seeds;          /* = seed_off[n_events] (host copy, used for launch sizes) */
    int32_t n_hits;           /* = hit_off[n_events] */
    int32_t flags;            /* 0, or DS_BATCH_CAPACITY */
    const int32_t *seed_off;  /* [n_events + 1], seed_off[0] = 0, non-decreasing */
    const int32_t *hit_off;   /* [n_events + 1], hit_off[0] = 0, non-decreasing */
} ds_event_batch;

/* ds_event_batch.flags: n_seeds and n_hits are the capacities of the seed and
 * hit arrays, and the totals are seed_off[n_events] <= n_seeds and
 * hit_off[n_events] <= n_hits, read on the device.  With it, one launch
 * sequence (a captured CUDA graph) serves every batch that fits those
 * capacities and n_events (events beyond the data: repeat the last offsets,
 * i.e. empty events).  Launch sizes follow the capacities. */
enum { DS_BATCH_CAPACITY = 1 };

/* SciFi seeds, device SoA float32 [n_seeds] each, grouped by event. */
typedef struct {
    const float *x, *y, *tx, *ty, *qop, *chi2;
} ds_seeds;

/* UT hits, device SoA [n_hits] each, grouped by event, any order inside an
 * event.  x0 = x at y = 0 of the strip; [ybeg, yend] = the strip's y extent,
 * which must lie inside one Y sector [y_min + k*sector_h, y_min + (k+1)*sector_h].
 * A hit's id is its index in these arrays. */
typedef struct {
    const float *x0, *ybeg, *yend;
    const uint8_t *layer;     /* 0..3 = UTaX, UTaU, UTbV, UTbX */
} ds_ut_hits;

/* Output track record, 64 bytes. */
typedef struct {
    int32_t event;            /* event index in the batch */
    int32_t seed;             /* global seed index */
    int32_t hit[4];           /* hit ids in UTaX, UTaU, UTbV, UTbX; -1 = absent */
    float x, y, tx, ty, qop;  /* state at z_ref */
    float chi2;
    int32_t ndof;
    float nn;                 /* ghost-killer response */
    uint32_t flags;           /* reserved, 0 */
    int32_t n_candidates;     /* candidates scored for this seed */
} ds_track;

/* Track output buffers (device).  Tracks are packed in (event, seed) order;
 * trk_off[e]..trk_off[e+1] are event e's tracks.  `tracks` must be 16-byte
 * aligned (DS_ERR_ARG otherwise): records are written as 16-byte chunks. */
typedef struct {
    ds_track *tracks;         /* [capacity] */
    int32_t *trk_off;         /* [n_events + 1] */
    int32_t *n_tracks;        /* device scalar: tracks produced (may exceed capacity) */
    int32_t capacity;
    int32_t n_events;         /* filled by ds_reconstruct; read by ds_vertex */
} ds_tracks;

/* Output vertex record, 32 bytes.  When the vertex capacity is exceeded the
 * counts and vtx_off are still exact but which records were stored is not
 * specified; size the capacity from *n_vertices and call again. */
typedef struct {
    int32_t event;
    int32_t i, j;             /* global indices into the track output, i < j */
    float x, y, z;            /* midpoint of the closest-approach points */
    float doca;
    uint32_t flags;           /* bit0: solved in FP64 (near-parallel pair); bit1: not converged */
} ds_vertex_rec;

/* Vertex-level quantities, 64 bytes, one per vertex record (same order):
 * masses under the K0S (pi+ pi-), Lambda (proton = positive track, pi-) and
 * anti-Lambda (pi+, antiproton = negative track) hypotheses, the parent's
 * momentum, transverse momentum and impact parameter to the beam line, the
 * opening angle, the daughters' momenta, and the trigger-line responses. */
typedef struct {
    float m_pipi, m_ppi, m_pip; /* MeV/c^2 */
    float p, pt;              /* parent |P| and P_T (MeV/c) */
    float ip;                 /* distance of the line {V + s P} to x = y = 0 (mm) */
    float one_minus_cos;      /* 1 - cos(opening angle) at the vertex */
    float p_pos, p_neg;       /* daughter momenta (MeV/c) */
    float pt_pos, pt_neg;     /* daughter transverse momenta at the vertex (MeV/c) */
    float score[4];           /* trigger-line network responses (0 for unloaded lines) */
    uint32_t flags;           /* reserved, 0 */
} ds_vertex_info;

/* Vertex output buffers (device).  `vertices` must be 16-byte aligned
 * (DS_ERR_ARG otherwise). */
typedef struct {
    ds_vertex_rec *vertices;  /* [capacity], (event, i, j) order */
    int32_t *vtx_off;         /* [n_events + 1] */
    int32_t *n_vertices;      /* device scalar: vertices produced (may exceed capacity) */
    int32_t capacity;
    int32_t reserved0;
} ds_vertices;

/* Counters of the last synchronised work (ds_sync_status fills them). */
typedef struct {
    int64_t n_candidates;     /* candidates scored */
    int64_t n_pairs;          /* opposite-charge pairs solved */
    int64_t n_pairs_fp64;     /* pairs re-solved in FP64 */
    int32_t n_tracks, n_vertices;
    uint32_t device_flags;
    int32_t reserved0;
} ds_stats;

/* Per-kernel device time collected when profiling is enabled. */
typedef struct {
    char name[32];            /* kernel name, e.g. "k_search" */
    int32_t launches;
    int32_t reserved0;
    double total_ms;          /* sum of CUDA-event durations on the launching stream */
} ds_kernel_time;

/* Launch shape of the search kernel.  The paper fixes a block per event
 * (GPU Implementation section); here work items are chunks of one event's
 * seeds pulled from a device queue by persistent CTAs, and their shape is a
 * run-time choice that changes speed only: outputs are identical for every
 * valid tuning. */
typedef struct {
    int32_t search_chunk;       /* max seeds per work item, 1..128 (default 128) */
    int32_t search_ctas_per_sm; /* persistent search CTAs per SM, 1..8 (default 5; at most 5 are
                                   resident with the default staging, larger values only queue) */
    int32_t search_group;       /* consecutive work items per queue pull, 1..16 (default 1) */
    int32_t search_stage_hits;  /* events with at most this many hits have their x0 array
                                   staged in shared memory, 0..46080 (default 5120);
                                   larger events read it from global memory */
    int32_t vertex_ctas_per_sm; /* CTAs per SM of the vertexing launch that takes one event
                                   per CTA, 1..4 (default 4) */
    int32_t vertex_small_cap;   /* events with at most this many tracks are vertexed one per
                                   CTA; larger ones as (event, 131072-pair range) work items
                                   spread over the SMs, 2..512 (default 512) */
    int32_t search_order;       /* order of the search's work items: 0 = each event's seeds in
                                   chunks of equal size (at most search_chunk), events in order;
                                   1 = every full chunk of search_chunk seeds first, then one item
                                   per event for its remaining seeds, largest first, so that the
                                   queue ends with its smallest items (default 1) */
} ds_tuning;

/* One configuration measured by ds_autotune. */
typedef struct {
    ds_tuning tuning;
    double ms;                  /* mean ds_reconstruct + ds_vertex time on the tuning batch */
} ds_tune_entry;

/* ------------------------------------------------------------------ lifetime */

/* Create a context on CUDA device `device`.  *out receives the handle. */
DS_API ds_status ds_create(ds_ctx **out, int device);
/* Release the context and its workspaces (synchronises its device). NULL ok. */
DS_API void ds_destroy(ds_ctx *ctx);
DS_API const char *ds_status_string(ds_status s);
/* Last host-side error message of this context ("" if none). */
DS_API const char *ds_last_error(const ds_ctx *ctx);
/* Fill *p with the default method parameters. */
DS_API ds_status ds_default_params(ds_params *p);

/* ----------------------------------------------------------------- state */

/* Copy the geometry into the context.  DS_ERR_ARG if z_layer is not increasing,
 * n_sectors is outside 1..32, sector_h, x_half_bins or sigmas are not > 0. */
DS_API ds_status ds_load_geometry(ds_ctx *ctx, const ds_geometry *geom);
/* Copy the ghost-killer network into the context (FP32 master; reduced-
 * precision copies are derived from it).  DS_ERR_ARG for unsupported shapes. */
DS_API ds_status ds_load_nn_weights(ds_ctx *ctx, const ds_nn_weights *w);
/* Set the method parameters.  DS_ERR_ARG if k1 is outside 1..10 or a window,
 * tolerance or limit is not positive. */
DS_API ds_status ds_set_params(ds_ctx *ctx, const ds_params *p);
/* Size the workspaces for batches up to these totals (synchronous allocation).
 * Calls on larger batches grow the workspaces themselves. */
DS_API ds_status ds_reserve(ds_ctx *ctx, int32_t max_events, int32_t max_seeds, int32_t max_hits);
/* Size the vertexing workspace for outputs of up to `capacity` vertices
 * (synchronous allocation).  ds_vertex grows it itself outside stream capture;
 * call this first to capture ds_vertex in a CUDA graph or to keep allocations
 * out of a serving loop. */
DS_API ds_status ds_reserve_vertices(ds_ctx *ctx, int32_t capacity);

/* ----------------------------------------------------------------- compute */

/* Downstream tracking (Algorithm Design and Ghost-Killer sections): for every
 * seed, magnet point -> UTbX window (k1 closest) -> refined windows (1/2/2
 * closest) -> candidates with >= 3 hits and a station-a hit -> line fit with the
 * magnet-point constraint -> ghost-killer response -> best candidate; then
 * clone killing inside each event.  Writes out->tracks, out->trk_off,
 * *out->n_tracks and sets out->n_events.  DS_ERR_NOT_READY without geometry
 * or weights; DS_ERR_ARG for null pointers or negative sizes. */
DS_API ds_status ds_reconstruct(ds_ctx *ctx, const ds_event_batch *batch, const ds_seeds *seeds,
                         const ds_ut_hits *hits, ds_tracks *out, void *stream);

/* Two-track vertexing (Vertexing section, Eqs. 3-4): for each event, every
 * pair i < j of its tracks with opposite charge, Newton-Raphson closest
 * approach of the two quadratic-in-x trajectories, vertex = midpoint, kept if
 * DOCA < doca_max.  Pairs with sin^2(opening) < eps_parallel whose FP32 DOCA
 * is near or below the cut are re-solved in FP64.  `tracks` is the output of
 * ds_reconstruct (device), with n_events set.  Events are processed in the
 * order (largest first) the last ds_reconstruct on this context laid out when
 * the event counts match, else in index order: this changes speed only, the
 * output is the same for any order. */
DS_API ds_status ds_vertex(ds_ctx *ctx, const ds_tracks *tracks, ds_vertices *out, void *stream);

/* The ghost-killer network alone (Ghost-Killer Neural Network section: inputs
 * normalised, ReLU hidden layers, output node) over n candidates, for tests
 * and for measuring the reduced-precision forms.  d_features: device, n x 16
 * FP32 row-major (the 16 inputs of one candidate contiguous, unused inputs of
 * smaller networks ignored), 16-byte aligned.  d_logit: device, n FP32, the
 * network output before the sigmoid (the response is its sigmoid).
 * precision: DS_MLP_FP32 - FP32 on the CUDA cores (bit-identical to
 * ds_reconstruct's network); DS_MLP_BF16 - inputs and first hidden layer
 * rounded to BF16, weights to BF16, products accumulated in FP32 on the
 * tensor cores (tcgen05), biases, ReLU and the output layer in FP32;
 * DS_MLP_FP8 - as BF16 with E4M3 (saturating at +-448) in place of BF16 and
 * each output neuron's weights scaled by the power of two that brings its
 * largest weight into (224, 448] before rounding (the scale undone in FP32).  The paper's network runs in FP32; the reduced forms are this
 * library's.  DS_ERR_NOT_READY without weights, DS_ERR_ARG for n < 0, null
 * or misaligned pointers or an unknown precision.  Asynchronous on `stream`;
 * a tensor-core wait that runs out raises DS_FLAG_TIMEOUT (ds_sync_status). */
DS_API ds_status ds_mlp_eval(ds_ctx *ctx, const float *d_features, int32_t n, float *d_logit,
                             int32_t precision, void *stream);

/* The candidates of the last ds_reconstruct on this context.  In training mode
 * (fixed 100 / 10 mm windows, clone killing off; Ghost-Killer Neural Network
 * section) every fitted candidate is a training example for the ghost killer.
 * Copies on `stream` up to `capacity` candidates into device arrays:
 * d_features n x 16 FP32 (the network inputs before normalisation), d_seed n
 * (global seed index), d_hits n x 4 (hit ids in UTaX, UTaU, UTbV, UTbX, -1
 * absent) and d_logit n (the network output before the sigmoid; may be NULL).
 * *d_count (device) receives the number of candidates of the call, which may
 * exceed capacity (the rest are not copied).  A seed's candidates are
 * contiguous; in training mode they are in enumeration order (its UTbX hits
 * by (|dx|, id), then the UTaU and UTbV options), otherwise grouped by UTbX
 * hit in an unspecified order of those hits.  The order of the seeds is
 * unspecified.
 * Call after ds_reconstruct on the same stream and before the next one.
 * d_features and d_hits 16-byte aligned.  DS_ERR_ARG for null pointers (other
 * than d_logit), misaligned arrays or capacity < 0. */
DS_API ds_status ds_candidates(ds_ctx *ctx, float *d_features, int32_t *d_seed, int32_t *d_hits, float *d_logit,
                               int32_t capacity, int32_t *d_count, void *stream);

/* Trigger-line networks (Expected Physics Impact section: single hidden
 * layer of 32 nodes, one output; the paper has four: K0S, Lambda, detached
 * K0S, detached Lambda).  n_lines <= 4 networks with n_in = 16, n_h1 <= 32,
 * n_h2 = 0, copied into the context.  Their 16 inputs are listed at
 * ds_vertex_physics.  DS_ERR_ARG for other shapes. */
DS_API ds_status ds_load_line_weights(ds_ctx *ctx, const ds_nn_weights *nets, int32_t n_lines);

/* Vertex-level physics for the output of ds_vertex: one ds_vertex_info per
 * vertex record (Vertexing Two Downstream Tracks and Expected Physics Impact
 * sections).  Each daughter's momentum at the vertex has magnitude 1/|q/p|
 * and the direction of its Eq. 4 trajectory there (slopes tx + 2 gamma
 * (z_v - z_ref), ty); masses use m_pi = 139.57039 and m_p = 938.27208 MeV/c^2.
 * The line networks see: vertex x/100, y/100, z/1000 (mm), DOCA; |P|/1e4,
 * P_T/1e3, ip/10; (m_pipi - 497.611)/100, (m_ppi - 1115.683)/100,
 * (m_pip - 1115.683)/100; p_pos/1e4, p_neg/1e4, pt_pos/1e3, pt_neg/1e3;
 * 1e3 (1 - cos opening); the mean chi2/ndof of the two tracks; then each
 * network's own normalisation.  With mlp_precision FP32 the networks run on
 * the CUDA cores in FP32; with BF16 or FP8 all four run as one BF16
 * tensor-core product per 128 vertices (inputs and first-layer weights, with
 * the normalisation folded in, rounded to BF16; FP32 accumulation, bias,
 * ReLU and output node).  tracks and vertices: device outputs of
 * ds_reconstruct / ds_vertex; d_info: device [capacity]; records beyond
 * capacity are not written.  Asynchronous on `stream`. */
DS_API ds_status ds_vertex_physics(ds_ctx *ctx, const ds_tracks *tracks, const ds_vertices *vertices,
                                   ds_vertex_info *d_info, int32_t capacity, void *stream);

/* Synchronise `stream`, read and clear the device flag word and counters.
 * Returns DS_ERR_CAPACITY / DS_ERR_TIMEOUT / DS_ERR_DEVICE_FLAG when the
 * corresponding flags are set, else DS_OK.  stats may be NULL. */
DS_API ds_status ds_sync_status(ds_ctx *ctx, void *stream, ds_stats *stats);

/* ds_reconstruct for callers that cannot allocate device memory (a host
 * framework that owns every device allocation through its own pool, code that
 * must not trigger an allocation's implicit device synchronisation, callers
 * that cannot create a ds_ctx).  The paper has no counterpart: this is a
 * deployment variant of the same computation.  Runs the same kernels as
 * ds_reconstruct on the CURRENT device and stream, taking geometry, parameters
 * and weights as host structs, with every scratch buffer inside one static
 * device array of about 22 MB that each GPU loading the library holds until
 * process exit.  It calls no cudaMalloc/cudaFree.  Limits per call: at most
 * 256 events, 16384 seeds and 327680 hits (DS_ERR_CAPACITY beyond, nothing
 * launched) and 8 candidates per seed on average whatever params->cand_per_seed
 * says (beyond that DS_FLAG_CAND_CAPACITY is set in *d_flags and the seeds
 * left over stay empty, so pass d_flags to see it).  Only the FP32 network
 * and non-training parameters are accepted (DS_ERR_ARG otherwise: training
 * mode gives up to 40 candidates per seed).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  Outputs as ds_reconstruct; if d_flags (device
 * pointer, may be NULL) is given, the call's device flag word (DS_FLAG_*) is
 * written there when the work completes.  Asynchronous on `stream`. */
DS_API ds_status ds_reconstruct_noalloc(const ds_geometry *geom, const ds_params *params,
                                        const ds_nn_weights *weights, const ds_event_batch *batch,
                                        const ds_seeds *seeds, const ds_ut_hits *hits, ds_tracks *out,
                                        uint32_t *d_flags, void *stream);

/* Profiling: when enabled, every kernel launch of this context is bracketed
 * by two CUDA events on its stream.  ds_profile_read() synchronises the
 * device, returns one entry per kernel name (at most max_out; *n_out = number
 * of distinct kernels) and clears the records.  Profiling adds two event
 * records per launch; leave it off for throughput measurements. */
DS_API ds_status ds_profile_enable(ds_ctx *ctx, int32_t enable);
DS_API ds_status ds_profile_read(ds_ctx *ctx, ds_kernel_time *out, int32_t max_out, int32_t *n_out);

/* Current tuning of the context / replace it (DS_ERR_ARG outside the ranges
 * above; nothing changed then).  Applies to later ds_reconstruct calls. */
DS_API ds_status ds_get_tuning(ds_ctx *ctx, ds_tuning *out);
DS_API ds_status ds_set_tuning(ds_ctx *ctx, const ds_tuning *t);

/* Autotuner: times ds_reconstruct + ds_vertex on the caller's batch (device
 * inputs as for ds_reconstruct; `out` receives the tracks of the last run, the
 * vertices go to context-owned buffers) for candidate tunings by coordinate
 * descent over the search's stage size, chunk size, CTAs per SM and queue
 * group, the search's work-item order, and the vertexing's CTAs per SM and
 * one-event-per-CTA track limit (two
 * sweeps, each configuration run `reps` times after one warm-up run, CUDA
 * events on `stream`), keeps the fastest in the context and copies it to
 * *best.  Every configuration measured is written to entries (at most
 * max_entries; *n_entries = number measured).  Synchronous; may allocate the
 * vertex buffers; must not be called while `stream` is being captured.  Errors
 * as ds_reconstruct. */
DS_API ds_status ds_autotune(ds_ctx *ctx, const ds_event_batch *batch, const ds_seeds *seeds,
                             const ds_ut_hits *hits, ds_tracks *out, int32_t reps, ds_tuning *best,
                             ds_tune_entry *entries, int32_t max_entries, int32_t *n_entries, void *stream);

/* End-to-end call with HOST buffers: copies the batch to context-owned device
 * buffers, runs ds_reconstruct and ds_vertex, copies tracks, trk_off, vertices
 * and vtx_off back, and synchronises.  Host inputs use the layouts above (SoA
 * float32, uint8 layer, int32 offsets); pinned memory is fastest.  On return
 * *n_tracks / *n_vertices hold the produced counts (outputs truncated to the
 * given capacities, DS_ERR_CAPACITY).  h_trk_off and h_vtx_off have
 * n_events + 1 entries. */
DS_API ds_status ds_process_host(ds_ctx *ctx, int32_t n_events, const int32_t *h_seed_off,
                          const float *h_seed_cols[6], const int32_t *h_hit_off,
                          const float *h_hit_cols[3], const uint8_t *h_hit_layer,
                          ds_track *h_tracks, int32_t trk_capacity, int32_t *h_trk_off,
                          int32_t *n_tracks, ds_vertex_rec *h_vertices, int32_t vtx_capacity,
                          int32_t *h_vtx_off, int32_t *n_vertices, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DS_H */
