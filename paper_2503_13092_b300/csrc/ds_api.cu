// C ABI of libds.so: contexts, device-resident state, launches.
// Declarations and the contract of every call are in include/ds.h.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ds_args.cuh"

static constexpr ds_tuning kDefaultTuning = {ds::kSearchThreads, ds::kSearchCtasPerSm, ds::kSearchGroup,
                                             ds::kStageHits,     ds::kVtxCtasPerSmMax, ds::kVtxSmallCapMax,
                                             1};

static bool tuning_valid(const ds_tuning &t)
{
    return t.search_chunk >= 1 && t.search_chunk <= ds::kSearchThreads && t.search_ctas_per_sm >= 1 &&
           t.search_ctas_per_sm <= 8 && t.search_group >= 1 && t.search_group <= 16 &&
           t.search_stage_hits >= 0 && t.search_stage_hits <= ds::kStageHitsMax && t.vertex_ctas_per_sm >= 1 &&
           t.vertex_ctas_per_sm <= ds::kVtxCtasPerSmMax && t.vertex_small_cap >= 2 &&
           t.vertex_small_cap <= ds::kVtxSmallCapMax && (t.search_order == 0 || t.search_order == 1);
}

struct ds_ctx {
    int device = 0;
    int sm_count = 148;
    bool has_geom = false, has_nn = false;
    ds::DevGeom g{};
    ds::DevParams p{};
    ds::DevNN nn{};
    int nn_in = 16, nn_h1 = 32, nn_h2 = 32;
    int mlp_precision = DS_MLP_FP32;
    int fuse_network = 0;
    ds::MlpTcWeights *d_tc = nullptr;    // tensor-core weight tiles (BF16 / FP8 network)
    ds::DevLines lines{};                // trigger-line networks (none loaded: n_lines = 0)
    ds::LineTcWeights *d_lines_tc = nullptr;   // their tensor-core operand
    ds_tuning tune{kDefaultTuning};
    ds::DevCounters *d_cnt = nullptr;
    // workspaces
    int cap_events = 0, cap_seeds = 0, cap_hits = 0, cap_pool = 0;
    uint16_t *sperm = nullptr;
    float *sx0 = nullptr;
    uint16_t *bins = nullptr;
    int *item_off = nullptr;      // search work items [2 E + 2], then the events largest first [E]
    int order_events = -1;        // events of the batch the event order was laid out for
    ds_track *trk_ws = nullptr;
    unsigned long long *key_ws = nullptr;
    int4 *hit_ws = nullptr;
    int *rank_ws = nullptr;
    float4 *cand_feat = nullptr;
    ds::CandMeta *cand_meta = nullptr;
    float *cand_logit = nullptr;
    int4 *seed_cand = nullptr;
    int cap_cand = 0;
    int cand_per_seed = 16;
    int *count_trk = nullptr;
    int *clone_next = nullptr;
    int *count_vtx = nullptr;
    int *large_vtx = nullptr;
    int *large_aux = nullptr;      // per listed event: pair count [E], first work item [E + 1]
    int *vtx_items = nullptr;      // per work item: kept count, offset inside its event
    ds_vertex_rec *pool = nullptr;
    int *pool_pos = nullptr;
    int *pool_item = nullptr;
    // host-buffer path: device copies of inputs and outputs
    struct {
        int cap_events = 0, cap_seeds = 0, cap_hits = 0, cap_trk = 0, cap_vtx = 0;
        int32_t *seed_off = nullptr, *hit_off = nullptr;
        float *seed_cols = nullptr, *hit_cols = nullptr;
        uint8_t *layer = nullptr;
        ds_track *tracks = nullptr;
        int32_t *trk_off = nullptr, *vtx_off = nullptr, *counts = nullptr;
        ds_vertex_rec *vertices = nullptr;
    } h;
    ds::Prof prof;
    std::string err;
};

namespace ds {

void Prof::begin(const char *name, cudaStream_t st)
{
    if (!on) return;
    Rec r{name, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, st);
    recs.push_back(r);
}

void Prof::end(cudaStream_t st)
{
    if (!on || recs.empty()) return;
    cudaEventRecord(recs.back().b, st);
}

}  // namespace ds

namespace {

ds_status fail(ds_ctx *c, ds_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

ds_status cuda_fail(ds_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, DS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DS_CUDA(call, what)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);    \
    } while (0)

template <class T>
ds_status grow(ds_ctx *ctx, T **p, size_t n)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (n > 0 ? n : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, DS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return DS_OK;
}

bool stream_capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

ds_status ensure_workspace(ds_ctx *ctx, int E, int S, int H, cudaStream_t st)
{
    if (E <= ctx->cap_events && S <= ctx->cap_seeds && H <= ctx->cap_hits &&
        (long long)S * ctx->cand_per_seed <= ctx->cap_cand)
        return DS_OK;
    if (stream_capturing(st))
        return fail(ctx, DS_ERR_ARG, "workspace too small during stream capture; call ds_reserve first");
    return ds_reserve(ctx, E, S, H);
}

}  // namespace

namespace ds {

// Host structs of the ABI -> device-side parameter blocks.  Each returns
// nullptr on success or a description of the invalid argument.
const char *fill_dev_geom(const ds_geometry *gm, DevGeom *out)
{
    if (!gm || !out) return "null pointer";
    for (int l = 0; l < 3; ++l)
        if (!(gm->z_layer[l] < gm->z_layer[l + 1])) return "z_layer not increasing";
    if (gm->n_sectors < 1 || gm->n_sectors > kMaxSectors) return "n_sectors outside 1..32";
    if (!(gm->sector_h > 0) || !(gm->x_half_bins > 0) || !(gm->sigma_hit > 0) || !(gm->sigma_mag > 0))
        return "sector_h, x_half_bins and sigmas must be > 0";
    DevGeom &g = *out;
    for (int l = 0; l < 4; ++l) {
        g.z[l] = (float)gm->z_layer[l];
        g.dxdy[l] = (float)gm->dxdy[l];
        g.zmag[l] = (float)gm->zmag[l];
    }
    g.y_min = (float)gm->y_min;
    g.sector_h = (float)gm->sector_h;
    g.inv_sector_h = (float)(1.0 / gm->sector_h);
    g.n_sec = gm->n_sectors;
    g.x_half = (float)gm->x_half_bins;
    g.inv_xbin = (float)(kNXB / (2.0 * gm->x_half_bins));
    g.z_seed = (float)gm->z_seed;
    g.kappa = (float)gm->kappa;
    g.mp = (float)gm->mp;
    g.gamma0 = (float)gm->gamma0;
    g.gamma1 = (float)gm->gamma1;
    g.z_ref = (float)gm->z_ref;
    g.w_hit = (float)(1.0 / (gm->sigma_hit * gm->sigma_hit));
    g.w_mag = (float)(1.0 / (gm->sigma_mag * gm->sigma_mag));
    g.inv_sigma_hit = (float)(1.0 / gm->sigma_hit);
    g.ext_off = table_ext_offset(g.n_sec);
    g.table_stride = table_stride_for(g.n_sec);
    return nullptr;
}

const char *fill_dev_nn(const ds_nn_weights *w, DevNN *out, int *n_h2_kernel)
{
    if (!w || !out || !w->w1 || !w->b1 || !w->w3 || !w->mean || !w->scale) return "null pointer";
    if (w->n_in < 1 || w->n_in > 16 || w->n_h1 < 1 || w->n_h1 > 32 || w->n_h2 < 0 || w->n_h2 > 32)
        return "unsupported network shape (n_in<=16, n_h1<=32, n_h2<=32)";
    if (w->n_h2 > 0 && (!w->w2 || !w->b2)) return "null w2/b2";
    DevNN &nn = *out;
    std::memset(&nn, 0, sizeof(nn));
    for (int o = 0; o < w->n_h1; ++o) {
        nn.b1[o] = w->b1[o];
        for (int i = 0; i < w->n_in; ++i) nn.w1[o][i] = w->w1[o * w->n_in + i];
    }
    const int nl = w->n_h2 > 0 ? w->n_h2 : w->n_h1;
    if (w->n_h2 > 0) {
        for (int o = 0; o < w->n_h2; ++o) {
            nn.b2[o] = w->b2[o];
            for (int i = 0; i < w->n_h1; ++i) nn.w2[o][i] = w->w2[o * w->n_h1 + i];
        }
    }
    for (int i = 0; i < nl; ++i) nn.w3[i] = w->w3[i];
    nn.b3 = w->b3;
    for (int i = 0; i < w->n_in; ++i) {
        nn.mean[i] = w->mean[i];
        nn.scale[i] = w->scale[i];
    }
    // the single-hidden-layer kernel is compiled for 8 inputs x 16 hidden
    if (w->n_h2 == 0 && (w->n_in > 8 || w->n_h1 > 16)) {
        // run it through the two-layer kernel: identity second layer (exact: h1 >= 0)
        for (int o = 0; o < w->n_h1; ++o) {
            nn.w2[o][o] = 1.f;
            nn.b2[o] = 0.f;
        }
        *n_h2_kernel = 32;
    } else {
        *n_h2_kernel = w->n_h2;
    }
    return nullptr;
}

const char *fill_dev_params(const ds_params *p, DevParams *out)
{
    if (!p || !out) return "null pointer";
    if (p->k1 < 1 || p->k1 > kK1Max) return "k1 outside 1..10";
    if (!(p->w1a >= 0) || !(p->w1b >= 0) || !(p->w2 > 0) || !(p->dy_tol >= 0) || !(p->doca_max > 0) ||
        !(p->nr_tol > 0) || p->nr_max_iter < 1 || !(p->eps_parallel >= 0))
        return "window, tolerance or limit not positive";
    if (p->mlp_precision != DS_MLP_FP32 && p->mlp_precision != DS_MLP_BF16 && p->mlp_precision != DS_MLP_FP8)
        return "unknown mlp_precision";
    if (p->cand_per_seed < 1 || p->cand_per_seed > 40) return "cand_per_seed outside 1..40";
    if (p->variant != 0 && p->variant != 1) return "variant must be 0 (Dv0) or 1 (Dv1)";
    if (p->variant == 1 && (!(p->dv1_dtx_max > 0) || !(p->dv1_w_tri > 0))) return "Dv1 bounds must be positive";
    if (p->fuse_network != 0 && p->fuse_network != 1) return "fuse_network must be 0 or 1";
    DevParams &d = *out;
    d.w1a = (float)p->w1a;
    d.w1b = (float)p->w1b;
    d.w2 = (float)p->w2;
    d.dy_tol = (float)p->dy_tol;
    d.nn_threshold = (float)p->nn_threshold;
    if (p->nn_threshold <= 0.0)
        d.thr_logit = -INFINITY;
    else if (p->nn_threshold >= 1.0)
        d.thr_logit = INFINITY;
    else
        d.thr_logit = (float)std::log(p->nn_threshold / (1.0 - p->nn_threshold));
    d.doca_max = (float)p->doca_max;
    d.nr_tol = (float)p->nr_tol;
    d.eps_par = (float)p->eps_parallel;
    d.k1 = p->k1;
    d.origin = p->first_window_origin ? 1 : 0;
    d.pick_chi2 = p->pick_chi2 ? 1 : 0;
    d.clone_kill = p->clone_kill ? 1 : 0;
    d.training = p->training ? 1 : 0;
    d.nr_max_iter = p->nr_max_iter;
    d.fault_inject = p->fault_inject;
    d.variant = p->variant;
    d.dv1_dtx = (float)p->dv1_dtx_max;
    d.dv1_w_tri = (float)p->dv1_w_tri;
    return nullptr;
}

}  // namespace ds

extern "C" {

const char *ds_status_string(ds_status s)
{
    switch (s) {
    case DS_OK: return "ok";
    case DS_ERR_ARG: return "invalid argument";
    case DS_ERR_CUDA: return "CUDA error";
    case DS_ERR_CAPACITY: return "output capacity exceeded";
    case DS_ERR_NOT_READY: return "geometry or network weights not loaded";
    case DS_ERR_TIMEOUT: return "device-side wait timed out";
    case DS_ERR_DEVICE_FLAG: return "device flagged malformed input";
    case DS_ERR_OOM: return "device out of memory";
    }
    return "unknown status";
}

const char *ds_last_error(const ds_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ds_status ds_default_params(ds_params *p)
{
    if (!p) return DS_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->w1a = 3.0;
    p->w1b = 1.7e5;
    p->w2 = 2.0;
    p->dy_tol = 2.0;
    p->nn_threshold = 0.5;
    p->doca_max = 2.0;
    p->nr_tol = 1e-6;
    p->eps_parallel = 1e-4;
    p->k1 = 10;
    p->first_window_origin = 0;
    p->pick_chi2 = 0;
    p->clone_kill = 1;
    p->training = 0;
    p->nr_max_iter = 10;
    p->mlp_precision = DS_MLP_FP32;
    p->cand_per_seed = 16;
    p->variant = 0;
    p->dv1_dtx_max = 0.8;
    p->dv1_w_tri = 1.0;
    return DS_OK;
}

ds_status ds_create(ds_ctx **out, int device)
{
    if (!out) return DS_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DS_ERR_CUDA;
    ds_ctx *ctx = new ds_ctx();
    ctx->device = device;
    DS_CUDA(cudaSetDevice(device), "cudaSetDevice");
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc((void **)&ctx->d_cnt, sizeof(ds::DevCounters)) != cudaSuccess) {
        delete ctx;
        return DS_ERR_OOM;
    }
    cudaMemset(ctx->d_cnt, 0, sizeof(ds::DevCounters));
    if (ds::init_vertex_attributes() != cudaSuccess || ds::init_search_attributes() != cudaSuccess ||
        ds::init_bucket_attributes() != cudaSuccess) {
        cudaFree(ctx->d_cnt);
        delete ctx;
        return DS_ERR_CUDA;
    }
    ds_params p;
    ds_default_params(&p);
    ds_set_params(ctx, &p);
    *out = ctx;
    return DS_OK;
}

void ds_destroy(ds_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    void *ptrs[] = {ctx->d_cnt, ctx->d_tc, ctx->d_lines_tc, ctx->sperm, ctx->sx0, ctx->item_off, ctx->bins, ctx->cand_feat,
                    ctx->cand_meta, ctx->cand_logit, ctx->seed_cand, ctx->trk_ws, ctx->key_ws, ctx->hit_ws,
                    ctx->rank_ws, ctx->clone_next, ctx->count_trk, ctx->count_vtx, ctx->large_vtx, ctx->large_aux, ctx->vtx_items, ctx->pool, ctx->pool_pos, ctx->pool_item,
                    ctx->h.seed_off, ctx->h.hit_off, ctx->h.seed_cols, ctx->h.hit_cols, ctx->h.layer,
                    ctx->h.tracks, ctx->h.trk_off, ctx->h.vtx_off, ctx->h.counts, ctx->h.vertices};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete ctx;
}

ds_status ds_load_geometry(ds_ctx *ctx, const ds_geometry *gm)
{
    if (!ctx || !gm) return fail(ctx, DS_ERR_ARG, "null pointer");
    const char *why = ds::fill_dev_geom(gm, &ctx->g);
    if (why) return fail(ctx, DS_ERR_ARG, why);
    ctx->has_geom = true;
    ctx->cap_events = 0;   // bin table stride may have changed
    return DS_OK;
}

ds_status ds_load_nn_weights(ds_ctx *ctx, const ds_nn_weights *w)
{
    if (!ctx) return DS_ERR_ARG;
    int n_h2 = 0;
    const char *why = ds::fill_dev_nn(w, &ctx->nn, &n_h2);
    if (why) return fail(ctx, DS_ERR_ARG, why);
    ctx->nn_h2 = n_h2;
    ctx->nn_in = w->n_in;
    ctx->nn_h1 = w->n_h1;
    ds::MlpTcWeights tc;
    ds::prepare_tc_weights(ctx->nn, n_h2, &tc);
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!ctx->d_tc) {
        cudaError_t e = cudaMalloc((void **)&ctx->d_tc, sizeof(tc));
        if (e != cudaSuccess) {
            ctx->d_tc = nullptr;
            return fail(ctx, DS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    // ordered after earlier work on every stream: no launch may still read the old tiles
    DS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    DS_CUDA(cudaMemcpy(ctx->d_tc, &tc, sizeof(tc), cudaMemcpyHostToDevice), "weight upload");
    ctx->has_nn = true;
    return DS_OK;
}

ds_status ds_set_params(ds_ctx *ctx, const ds_params *p)
{
    if (!ctx) return DS_ERR_ARG;
    const char *why = ds::fill_dev_params(p, &ctx->p);
    if (why) return fail(ctx, DS_ERR_ARG, why);
    ctx->mlp_precision = p->mlp_precision;
    ctx->fuse_network = p->fuse_network;
    // training mode (100/10 mm windows) can give every seed the maximum of 10 x 1 x 2 x 2
    ctx->cand_per_seed = p->training ? 40 : p->cand_per_seed;
    return DS_OK;
}

ds_status ds_reserve(ds_ctx *ctx, int32_t E, int32_t S, int32_t H)
{
    if (!ctx || E < 0 || S < 0 || H < 0) return fail(ctx, DS_ERR_ARG, "negative size");
    if (!ctx->has_geom) return fail(ctx, DS_ERR_NOT_READY, "load the geometry before ds_reserve");
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    DS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    ds_status st;
    if (E > ctx->cap_events || ctx->cap_events == 0) {
        E = E > ctx->cap_events ? E : ctx->cap_events;
        ctx->order_events = -1;   // the event order lives in item_off, reallocated below
        if ((st = grow(ctx, &ctx->bins, (size_t)E * ctx->g.table_stride)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->count_trk, (size_t)E)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->count_vtx, (size_t)E)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->large_vtx, (size_t)E)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->large_aux, 2 * (size_t)E + 2)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->vtx_items, 2 * (size_t)ds::kVtxItemsPerEvent * E)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->item_off, 3 * (size_t)E + 2)) != DS_OK) return st;
        ctx->cap_events = E;
    }
    const long long want_cand = (long long)(S > ctx->cap_seeds ? S : ctx->cap_seeds) * ctx->cand_per_seed;
    if (want_cand > ctx->cap_cand) {
        if (want_cand > 0x7fffffffLL / 4) return fail(ctx, DS_ERR_ARG, "candidate buffer too large");
        const size_t n = (size_t)want_cand;
        if ((st = grow(ctx, &ctx->cand_feat, 4 * n)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->cand_meta, n)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->cand_logit, n)) != DS_OK) return st;
        ctx->cap_cand = (int)n;
    }
    if (S > ctx->cap_seeds) {
        if ((st = grow(ctx, &ctx->seed_cand, (size_t)S)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->trk_ws, (size_t)S)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->key_ws, (size_t)S)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->hit_ws, (size_t)S)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->rank_ws, (size_t)S)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->clone_next, 2 * (size_t)S)) != DS_OK) return st;
        ctx->cap_seeds = S;
    }
    if (H > ctx->cap_hits) {
        if ((st = grow(ctx, &ctx->sperm, (size_t)H)) != DS_OK) return st;
        if ((st = grow(ctx, &ctx->sx0, (size_t)H + 4)) != DS_OK) return st;   // bulk-copy tail
        ctx->cap_hits = H;
    }
    return DS_OK;
}

ds_status ds_reserve_vertices(ds_ctx *ctx, int32_t capacity)
{
    if (!ctx || capacity < 0) return fail(ctx, DS_ERR_ARG, "null context or negative capacity");
    if (capacity <= ctx->cap_pool) return DS_OK;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    DS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    ds_status s;
    if ((s = grow(ctx, &ctx->pool, (size_t)capacity)) != DS_OK) return s;
    if ((s = grow(ctx, &ctx->pool_pos, (size_t)capacity)) != DS_OK) return s;
    if ((s = grow(ctx, &ctx->pool_item, (size_t)capacity)) != DS_OK) return s;
    ctx->cap_pool = capacity;
    return DS_OK;
}

ds_status ds_reconstruct(ds_ctx *ctx, const ds_event_batch *b, const ds_seeds *sd, const ds_ut_hits *ht,
                         ds_tracks *out, void *stream)
{
    if (!ctx || !b || !sd || !ht || !out) return fail(ctx, DS_ERR_ARG, "null pointer");
    if (!ctx->has_geom || !ctx->has_nn) return fail(ctx, DS_ERR_NOT_READY, "geometry or weights not loaded");
    if (b->n_events < 0 || b->n_seeds < 0 || b->n_hits < 0 || out->capacity < 0)
        return fail(ctx, DS_ERR_ARG, "negative size");
    if (b->flags & ~DS_BATCH_CAPACITY) return fail(ctx, DS_ERR_ARG, "unknown batch flags");
    if (b->n_events > 0 && (!b->seed_off || !b->hit_off || !out->trk_off || !out->n_tracks))
        return fail(ctx, DS_ERR_ARG, "null offsets or outputs");
    if (b->n_seeds > 0 && (!sd->x || !sd->y || !sd->tx || !sd->ty || !sd->qop || !sd->chi2))
        return fail(ctx, DS_ERR_ARG, "null seed column");
    if (b->n_hits > 0 && (!ht->x0 || !ht->ybeg || !ht->yend || !ht->layer))
        return fail(ctx, DS_ERR_ARG, "null hit column");
    if (out->capacity > 0 && !out->tracks) return fail(ctx, DS_ERR_ARG, "null track buffer");
    if (reinterpret_cast<uintptr_t>(out->tracks) % 16 != 0)
        return fail(ctx, DS_ERR_ARG, "track buffer must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ds_status s = ensure_workspace(ctx, b->n_events, b->n_seeds, b->n_hits, st);
    if (s != DS_OK) return s;
    out->n_events = b->n_events;
    if (b->n_events == 0) return DS_OK;
    static_assert(offsetof(ds::DevCounters, search_queue) == offsetof(ds::DevCounters, cand_used) + sizeof(int),
                  "cand_used and search_queue are cleared together");
    DS_CUDA(cudaMemsetAsync(&ctx->d_cnt->cand_used, 0, 2 * sizeof(int), st), "memset");

    ds::BucketArgs ba{};
    ba.g = ctx->g;
    ba.n_events = b->n_events;
    ba.n_hits = b->n_hits;
    ba.n_seeds = b->n_seeds;
    ba.hit_off = b->hit_off;
    ba.seed_off = b->seed_off;
    ba.x0 = ht->x0;
    ba.ybeg = ht->ybeg;
    ba.yend = ht->yend;
    ba.layer = ht->layer;
    ba.sx0 = ctx->sx0;
    ba.sperm = ctx->sperm;
    ba.bins = ctx->bins;
    ba.item_off = ctx->item_off;
    ba.chunk = ctx->tune.search_chunk;
    ba.order = ctx->tune.search_order;
    ba.ev_order = ctx->item_off + 2 * (size_t)ctx->cap_events + 2;
    ba.capacity_sizes = (b->flags & DS_BATCH_CAPACITY) ? 1 : 0;
    ba.cnt = ctx->d_cnt;
    DS_CUDA(ds::launch_bucket(ba, st, &ctx->prof), "bucket kernel");
    ctx->order_events = b->n_events;

    ds::SearchArgs sa{};
    sa.g = ctx->g;
    sa.p = ctx->p;
    sa.n_events = b->n_events;
    sa.n_seeds = b->n_seeds;
    sa.n_hits = b->n_hits;
    sa.seed_off = b->seed_off;
    sa.hit_off = b->hit_off;
    sa.sx = sd->x; sa.sy = sd->y; sa.stx = sd->tx; sa.sty = sd->ty; sa.sqop = sd->qop; sa.schi2 = sd->chi2;
    sa.ybeg = ht->ybeg;
    sa.yend = ht->yend;
    sa.sx0 = ctx->sx0;
    sa.sperm = ctx->sperm;
    sa.bins = ctx->bins;
    sa.item_off = ctx->item_off;
    sa.chunk = ctx->tune.search_chunk;
    sa.order = ctx->tune.search_order;
    sa.cand_feat = ctx->cand_feat;
    sa.cand_meta = ctx->cand_meta;
    sa.cand_cap = ctx->cap_cand;
    sa.seed_cand = ctx->seed_cand;
    sa.rank_ws = ctx->rank_ws;
    sa.sm_count = ctx->sm_count;
    sa.ctas_per_sm = ctx->tune.search_ctas_per_sm;
    sa.group = ctx->tune.search_group;
    sa.stage_hits = ctx->tune.search_stage_hits;
    sa.cnt = ctx->d_cnt;
    // the network scored inside the search (on request): FP32, the
    // two-hidden-layer kernel shape, outside training mode
    sa.fused = ctx->fuse_network && ctx->mlp_precision == DS_MLP_FP32 && !ctx->p.training && ctx->nn_h2 == 32;
    if (sa.fused) {
        sa.nn = ctx->nn;
        sa.trk_ws = ctx->trk_ws;
        sa.key_ws = ctx->key_ws;
        sa.hit_ws = ctx->hit_ws;
    }
    DS_CUDA(ds::launch_search(sa, st, &ctx->prof), "search kernel");

    ds::MlpArgs ma{};
    ma.nn = ctx->nn;
    ma.n_in = ctx->nn_in;
    ma.n_h2 = ctx->nn_h2;
    ma.precision = ctx->mlp_precision;
    ma.tc = ctx->d_tc;
    ma.feat = ctx->cand_feat;
    ma.logit = ctx->cand_logit;
    ma.cand_cap = ctx->cap_cand;
    ma.n_host = -1;
    ma.cnt = ctx->d_cnt;
    ds::PickArgs pa{};
    pa.p = ctx->p;
    pa.n_seeds = b->n_seeds;
    pa.n_events = b->n_events;
    pa.seed_off = b->seed_off;
    pa.seed_cand = ctx->seed_cand;
    pa.logit = ctx->cand_logit;
    pa.meta = ctx->cand_meta;
    pa.trk_ws = ctx->trk_ws;
    pa.key_ws = ctx->key_ws;
    pa.hit_ws = ctx->hit_ws;
    if (!sa.fused) DS_CUDA(ds::launch_mlp_pick(ma, pa, ctx->sm_count, st, &ctx->prof), "network kernel");

    ds::CloneArgs ca{};
    ca.n_events = b->n_events;
    ca.n_seeds = b->n_seeds;
    ca.clone_kill = ctx->p.clone_kill && !ctx->p.training;
    ca.seed_off = b->seed_off;
    ca.key_ws = ctx->key_ws;
    ca.hit_ws = ctx->hit_ws;
    ca.rank_ws = ctx->rank_ws;
    ca.ev_order = ba.ev_order;
    ca.next_ws = ctx->clone_next;
    ca.count_ws = ctx->count_trk;
    ca.trk_off = out->trk_off;
    ca.n_tracks = out->n_tracks;
    ca.capacity = out->capacity;
    ca.cnt = ctx->d_cnt;
    ds::ScatterTrkArgs xa{};
    xa.n_seeds = b->n_seeds;
    xa.n_events = b->n_events;
    xa.seed_off = b->seed_off;
    xa.trk_ws = ctx->trk_ws;
    xa.rank_ws = ctx->rank_ws;
    xa.trk_off = out->trk_off;
    xa.out = out->tracks;
    xa.capacity = out->capacity;
    DS_CUDA(ds::launch_clone(ca, xa, st, &ctx->prof), "clone kernel");
    return DS_OK;
}

ds_status ds_load_line_weights(ds_ctx *ctx, const ds_nn_weights *nets, int32_t n_lines)
{
    if (!ctx) return DS_ERR_ARG;
    ds::DevLines L;
    const char *why = ds::fill_dev_lines(nets, n_lines, &L);
    if (why) return fail(ctx, DS_ERR_ARG, why);
    ds::LineTcWeights tcw;
    ds::prepare_line_tc(L, &tcw);
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!ctx->d_lines_tc) {
        cudaError_t e = cudaMalloc((void **)&ctx->d_lines_tc, sizeof(tcw));
        if (e != cudaSuccess) {
            ctx->d_lines_tc = nullptr;
            return fail(ctx, DS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    DS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    DS_CUDA(cudaMemcpy(ctx->d_lines_tc, &tcw, sizeof(tcw), cudaMemcpyHostToDevice), "line weight upload");
    ctx->lines = L;
    return DS_OK;
}

ds_status ds_vertex_physics(ds_ctx *ctx, const ds_tracks *tr, const ds_vertices *vx, ds_vertex_info *d_info,
                            int32_t capacity, void *stream)
{
    if (!ctx || !tr || !vx || capacity < 0) return fail(ctx, DS_ERR_ARG, "null pointer or negative capacity");
    if (!ctx->has_geom) return fail(ctx, DS_ERR_NOT_READY, "geometry not loaded");
    if (capacity == 0 || tr->n_events == 0) return DS_OK;
    if (!d_info || !tr->tracks || !tr->n_tracks || !vx->vertices || !vx->n_vertices)
        return fail(ctx, DS_ERR_ARG, "null buffer");
    if (reinterpret_cast<uintptr_t>(d_info) % 16 != 0) return fail(ctx, DS_ERR_ARG, "d_info must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ds::VinfoArgs va{};
    va.g = ctx->g;
    va.L = ctx->lines;
    va.tracks = tr->tracks;
    va.trk_capacity = tr->capacity;
    va.n_tracks = tr->n_tracks;
    va.vtx = vx->vertices;
    va.vtx_capacity = vx->capacity;
    va.n_vertices = vx->n_vertices;
    va.out = d_info;
    va.capacity = capacity;
    va.tcw = ctx->d_lines_tc;
    va.cnt = ctx->d_cnt;
    const bool tensor_cores = ctx->mlp_precision != DS_MLP_FP32 && ctx->d_lines_tc != nullptr;
    DS_CUDA(ds::launch_vertex_info(va, tensor_cores, ctx->sm_count, st, &ctx->prof), "vertex physics kernel");
    return DS_OK;
}

ds_status ds_candidates(ds_ctx *ctx, float *d_features, int32_t *d_seed, int32_t *d_hits, float *d_logit,
                        int32_t capacity, int32_t *d_count, void *stream)
{
    if (!ctx || !d_features || !d_seed || !d_hits || !d_count || capacity < 0)
        return fail(ctx, DS_ERR_ARG, "null pointer or negative capacity");
    if ((reinterpret_cast<uintptr_t>(d_features) | reinterpret_cast<uintptr_t>(d_hits)) % 16 != 0)
        return fail(ctx, DS_ERR_ARG, "features and hits must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (ctx->cap_cand == 0) {
        DS_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int32_t), st), "memset");
        return DS_OK;
    }
    DS_CUDA(ds::launch_export_candidates(ctx->cand_feat, ctx->cand_meta, ctx->cand_logit, ctx->cap_cand, ctx->d_cnt,
                                         d_features, d_seed, d_hits, d_logit, capacity, d_count, ctx->sm_count, st),
            "candidate export");
    return DS_OK;
}

ds_status ds_mlp_eval(ds_ctx *ctx, const float *d_features, int32_t n, float *d_logit, int32_t precision,
                      void *stream)
{
    if (!ctx) return DS_ERR_ARG;
    if (!ctx->has_nn) return fail(ctx, DS_ERR_NOT_READY, "weights not loaded");
    if (n < 0) return fail(ctx, DS_ERR_ARG, "negative size");
    if (precision != DS_MLP_FP32 && precision != DS_MLP_BF16 && precision != DS_MLP_FP8)
        return fail(ctx, DS_ERR_ARG, "unknown precision");
    if (n == 0) return DS_OK;
    if (!d_features || !d_logit) return fail(ctx, DS_ERR_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(d_features) % 16 != 0)
        return fail(ctx, DS_ERR_ARG, "features must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ds::MlpArgs ma{};
    ma.nn = ctx->nn;
    ma.n_in = ctx->nn_in;
    ma.n_h2 = ctx->nn_h2;
    ma.precision = precision;
    ma.tc = ctx->d_tc;
    ma.feat = reinterpret_cast<const float4 *>(d_features);
    ma.logit = d_logit;
    ma.cand_cap = n;
    ma.n_host = n;
    ma.cnt = ctx->d_cnt;
    ctx->prof.begin("k_mlp", st);
    cudaError_t e = ds::launch_mlp(ma, ctx->sm_count, n, st);
    ctx->prof.end(st);
    DS_CUDA(e, "network kernel");
    return DS_OK;
}

ds_status ds_vertex(ds_ctx *ctx, const ds_tracks *tr, ds_vertices *out, void *stream)
{
    if (!ctx || !tr || !out) return fail(ctx, DS_ERR_ARG, "null pointer");
    if (!ctx->has_geom) return fail(ctx, DS_ERR_NOT_READY, "geometry not loaded");
    if (tr->n_events < 0 || out->capacity < 0) return fail(ctx, DS_ERR_ARG, "negative size");
    if (tr->n_events == 0) return DS_OK;
    if (!tr->trk_off || !tr->n_tracks || !out->vtx_off || !out->n_vertices)
        return fail(ctx, DS_ERR_ARG, "null offsets");
    if (tr->capacity > 0 && !tr->tracks) return fail(ctx, DS_ERR_ARG, "null track buffer");
    if (out->capacity > 0 && !out->vertices) return fail(ctx, DS_ERR_ARG, "null vertex buffer");
    if (reinterpret_cast<uintptr_t>(out->vertices) % 16 != 0)
        return fail(ctx, DS_ERR_ARG, "vertex buffer must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int E = tr->n_events;
    if (E > ctx->cap_events || ctx->cap_pool < out->capacity) {
        if (stream_capturing(st))
            return fail(ctx, DS_ERR_ARG, "workspace too small during stream capture; call ds_reserve first");
        ds_status s = ds_reserve(ctx, E, ctx->cap_seeds, ctx->cap_hits);
        if (s != DS_OK) return s;
        if (ctx->cap_pool < out->capacity) {
            if ((s = grow(ctx, &ctx->pool, (size_t)out->capacity)) != DS_OK) return s;
            if ((s = grow(ctx, &ctx->pool_pos, (size_t)out->capacity)) != DS_OK) return s;
            if ((s = grow(ctx, &ctx->pool_item, (size_t)out->capacity)) != DS_OK) return s;
            ctx->cap_pool = out->capacity;
        }
    }
    static_assert(offsetof(ds::DevCounters, vtx_queue) == offsetof(ds::DevCounters, pool_used) + sizeof(int) &&
                      offsetof(ds::DevCounters, n_large) == offsetof(ds::DevCounters, pool_used) + 3 * sizeof(int),
                  "pool_used, the vertex queues and n_large are cleared together");
    DS_CUDA(cudaMemsetAsync(&ctx->d_cnt->pool_used, 0, 4 * sizeof(int), st), "memset");
    ds::VertexArgs va{};
    va.g = ctx->g;
    va.p = ctx->p;
    va.n_events = E;
    va.trk_capacity = tr->capacity;
    va.tracks = tr->tracks;
    va.trk_off = tr->trk_off;
    va.n_tracks = tr->n_tracks;
    va.pool = ctx->pool;
    va.pool_pos = ctx->pool_pos;
    va.pool_item = ctx->pool_item;
    va.pool_cap = out->capacity;
    va.count_ws = ctx->count_vtx;
    // the events in the order the last ds_reconstruct laid out (largest
    // first): any permutation of the events gives the same output, so it is
    // used whenever the event count matches
    va.ev_order = ctx->order_events == E ? ctx->item_off + 2 * (size_t)ctx->cap_events + 2 : nullptr;
    va.large_list = ctx->large_vtx;
    va.large_pairs = ctx->large_aux;
    va.large_item_off = ctx->large_aux + ctx->cap_events;
    va.item_count = ctx->vtx_items;
    va.item_base = ctx->vtx_items + (size_t)ds::kVtxItemsPerEvent * ctx->cap_events;
    va.max_items = ds::kVtxItemsPerEvent * ctx->cap_events;
    va.vtx_off = out->vtx_off;
    va.n_vertices = out->n_vertices;
    va.capacity = out->capacity;
    va.cnt = ctx->d_cnt;
    va.small_cap = ctx->tune.vertex_small_cap;
    va.ctas_per_sm = ctx->tune.vertex_ctas_per_sm;
    ds::ScatterVtxArgs xa{};
    xa.pool = ctx->pool;
    xa.pool_pos = ctx->pool_pos;
    xa.pool_item = ctx->pool_item;
    xa.item_base = va.item_base;
    xa.pool_cap = out->capacity;
    xa.vtx_off = out->vtx_off;
    xa.out = out->vertices;
    xa.capacity = out->capacity;
    xa.cnt = ctx->d_cnt;
    DS_CUDA(ds::launch_vertex(va, xa, ctx->sm_count, st, &ctx->prof), "vertex kernel");
    return DS_OK;
}

ds_status ds_sync_status(ds_ctx *ctx, void *stream, ds_stats *stats)
{
    if (!ctx) return DS_ERR_ARG;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    // stream-ordered: no legacy-stream call that could wait for other streams
    cudaStream_t st = (cudaStream_t)stream;
    ds::DevCounters c;
    DS_CUDA(cudaMemcpyAsync(&c, ctx->d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st), "read counters");
    DS_CUDA(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(c), st), "clear counters");
    DS_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (stats) {
        stats->n_candidates = (int64_t)c.n_candidates;
        stats->n_pairs = (int64_t)c.n_pairs;
        stats->n_pairs_fp64 = (int64_t)c.n_pairs_fp64;
        stats->n_tracks = c.n_tracks;
        stats->n_vertices = c.n_vertices;
        stats->device_flags = c.flags;
    }
    if (c.flags & DS_FLAG_TIMEOUT) return fail(ctx, DS_ERR_TIMEOUT, "device wait timed out");
    if (c.flags & (DS_FLAG_BAD_OFFSETS | DS_FLAG_BAD_LAYER | DS_FLAG_STRIP_SECTOR | DS_FLAG_EVENT_TOO_LARGE)) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), "device flags 0x%x", c.flags);
        return fail(ctx, DS_ERR_DEVICE_FLAG, buf);
    }
    if (c.flags & (DS_FLAG_TRACK_CAPACITY | DS_FLAG_VERTEX_CAPACITY | DS_FLAG_CAND_CAPACITY))
        return fail(ctx, DS_ERR_CAPACITY, "output capacity exceeded");
    return DS_OK;
}

ds_status ds_get_tuning(ds_ctx *ctx, ds_tuning *out)
{
    if (!ctx || !out) return fail(ctx, DS_ERR_ARG, "null pointer");
    *out = ctx->tune;
    return DS_OK;
}

ds_status ds_set_tuning(ds_ctx *ctx, const ds_tuning *t)
{
    if (!ctx || !t) return fail(ctx, DS_ERR_ARG, "null pointer");
    if (!tuning_valid(*t)) return fail(ctx, DS_ERR_ARG, "tuning outside its ranges");
    ctx->tune = *t;
    return DS_OK;
}

ds_status ds_autotune(ds_ctx *ctx, const ds_event_batch *b, const ds_seeds *sd, const ds_ut_hits *ht,
                      ds_tracks *out, int32_t reps, ds_tuning *best, ds_tune_entry *entries, int32_t max_entries,
                      int32_t *n_entries, void *stream)
{
    if (!ctx || !b || !sd || !ht || !out || reps < 1 || max_entries < 0 || (max_entries > 0 && !entries))
        return fail(ctx, DS_ERR_ARG, "null pointer or bad count");
    cudaStream_t st = (cudaStream_t)stream;
    if (stream_capturing(st)) return fail(ctx, DS_ERR_ARG, "ds_autotune during stream capture");
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaEvent_t e0, e1;
    DS_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, DS_ERR_CUDA, "cudaEventCreate");
    }
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    int n = 0;
    ds_status rs = DS_OK;
    // the vertices of the tuning runs go to the context's host-path buffers
    const int vcap = (int)std::min<long long>(16LL * b->n_seeds + 4096, 0x7fffffffLL / 64);
    auto &h = ctx->h;
    if (b->n_events + 1 > h.cap_events) {
        if ((rs = grow(ctx, &h.seed_off, (size_t)b->n_events + 1)) != DS_OK ||
            (rs = grow(ctx, &h.hit_off, (size_t)b->n_events + 1)) != DS_OK ||
            (rs = grow(ctx, &h.trk_off, (size_t)b->n_events + 1)) != DS_OK ||
            (rs = grow(ctx, &h.vtx_off, (size_t)b->n_events + 1)) != DS_OK ||
            (rs = grow(ctx, &h.counts, (size_t)2)) != DS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rs;
        }
        h.cap_events = b->n_events + 1;
    }
    if (vcap > h.cap_vtx) {
        if ((rs = grow(ctx, &h.vertices, (size_t)vcap)) != DS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rs;
        }
        h.cap_vtx = vcap;
    }
    ds_vertices vx{h.vertices, h.vtx_off, h.counts + 1, vcap, 0};
    auto step = [&]() -> ds_status {
        ds_status s = ds_reconstruct(ctx, b, sd, ht, out, stream);
        if (s == DS_OK) s = ds_vertex(ctx, out, &vx, stream);
        return s;
    };
    auto measure = [&](const ds_tuning &t, double *ms) -> ds_status {
        ctx->tune = t;
        ds_status s = step();   // warm-up (and workspace growth)
        if (s != DS_OK) return s;
        if (cudaEventRecord(e0, st) != cudaSuccess) return fail(ctx, DS_ERR_CUDA, "cudaEventRecord");
        for (int r = 0; r < reps; ++r)
            if ((s = step()) != DS_OK) return s;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return fail(ctx, DS_ERR_CUDA, "timing event");
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = (double)f / reps;
        if (n < max_entries) entries[n] = ds_tune_entry{t, *ms};
        ++n;
        return DS_OK;
    };
    ds_tuning cur = ctx->tune;
    double cur_ms = 0.0;
    rs = measure(cur, &cur_ms);
    static const int stage_opts[] = {2048, 5120, 8192, 12288, 16384, 24576, 32768};
    static const int chunk_opts[] = {32, 64, 96, 128};
    static const int ctas_opts[] = {2, 3, 4, 5};
    static const int group_opts[] = {1, 2, 4, 8};
    static const int vctas_opts[] = {1, 2, 3, 4};
    static const int vcap_opts[] = {64, 128, 256, 512};
    static const int order_opts[] = {0, 1};
    const int *dim_opts[7] = {stage_opts, chunk_opts, ctas_opts, group_opts, vctas_opts, vcap_opts, order_opts};
    for (int sweep = 0; sweep < 2 && rs == DS_OK; ++sweep) {
        for (int dim = 0; dim < 7 && rs == DS_OK; ++dim) {
            const int *opts = dim_opts[dim];
            const int n_opts = dim == 0 ? 7 : dim == 6 ? 2 : 4;
            for (int k = 0; k < n_opts && rs == DS_OK; ++k) {
                ds_tuning t = cur;
                int32_t *fields[7] = {&t.search_stage_hits, &t.search_chunk, &t.search_ctas_per_sm, &t.search_group,
                                      &t.vertex_ctas_per_sm, &t.vertex_small_cap, &t.search_order};
                int32_t *field = fields[dim];
                if (*field == opts[k]) continue;
                *field = opts[k];
                double ms = 0.0;
                rs = measure(t, &ms);
                if (rs == DS_OK && ms < cur_ms) {
                    cur = t;
                    cur_ms = ms;
                }
            }
        }
    }
    ctx->tune = cur;
    ctx->prof.on = prof_on;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_entries) *n_entries = n;
    if (best) *best = cur;
    return rs;
}

ds_status ds_profile_enable(ds_ctx *ctx, int32_t enable)
{
    if (!ctx) return DS_ERR_ARG;
    ctx->prof.on = enable != 0;
    return DS_OK;
}

ds_status ds_profile_read(ds_ctx *ctx, ds_kernel_time *out, int32_t max_out, int32_t *n_out)
{
    if (!ctx || !n_out || max_out < 0 || (max_out > 0 && !out)) return fail(ctx, DS_ERR_ARG, "null pointer");
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    DS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    std::vector<ds_kernel_time> acc;
    for (auto &r : ctx->prof.recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, r.a, r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        if (e != cudaSuccess) continue;
        ds_kernel_time *k = nullptr;
        for (auto &q : acc)
            if (std::strncmp(q.name, r.name, sizeof(q.name)) == 0) k = &q;
        if (!k) {
            ds_kernel_time z{};
            std::strncpy(z.name, r.name, sizeof(z.name) - 1);
            acc.push_back(z);
            k = &acc.back();
        }
        k->launches += 1;
        k->total_ms += ms;
    }
    ctx->prof.recs.clear();
    *n_out = (int32_t)acc.size();
    for (int i = 0; i < (int)acc.size() && i < max_out; ++i) out[i] = acc[i];
    return DS_OK;
}

ds_status ds_process_host(ds_ctx *ctx, int32_t E, const int32_t *h_seed_off, const float *h_seed_cols[6],
                          const int32_t *h_hit_off, const float *h_hit_cols[3], const uint8_t *h_layer,
                          ds_track *h_tracks, int32_t trk_cap, int32_t *h_trk_off, int32_t *n_tracks,
                          ds_vertex_rec *h_vertices, int32_t vtx_cap, int32_t *h_vtx_off, int32_t *n_vertices,
                          void *stream)
{
    if (!ctx || E < 0 || !h_seed_off || !h_seed_cols || !h_hit_off || !h_hit_cols || !h_layer || !h_trk_off ||
        !h_vtx_off || !n_tracks || !n_vertices || trk_cap < 0 || vtx_cap < 0)
        return fail(ctx, DS_ERR_ARG, "null pointer or negative size");
    cudaStream_t st = (cudaStream_t)stream;
    DS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int S = h_seed_off[E], H = h_hit_off[E];
    if (S < 0 || H < 0) return fail(ctx, DS_ERR_ARG, "negative totals in offsets");
    auto &h = ctx->h;
    ds_status s;
    if (E + 1 > h.cap_events) {
        if ((s = grow(ctx, &h.seed_off, (size_t)E + 1)) != DS_OK) return s;
        if ((s = grow(ctx, &h.hit_off, (size_t)E + 1)) != DS_OK) return s;
        if ((s = grow(ctx, &h.trk_off, (size_t)E + 1)) != DS_OK) return s;
        if ((s = grow(ctx, &h.vtx_off, (size_t)E + 1)) != DS_OK) return s;
        if ((s = grow(ctx, &h.counts, (size_t)2)) != DS_OK) return s;
        h.cap_events = E + 1;
    }
    if (S > h.cap_seeds) {
        if ((s = grow(ctx, &h.seed_cols, (size_t)6 * S)) != DS_OK) return s;
        h.cap_seeds = S;
    }
    if (H > h.cap_hits) {
        if ((s = grow(ctx, &h.hit_cols, (size_t)3 * H)) != DS_OK) return s;
        if ((s = grow(ctx, &h.layer, (size_t)H)) != DS_OK) return s;
        h.cap_hits = H;
    }
    if (trk_cap > h.cap_trk) {
        if ((s = grow(ctx, &h.tracks, (size_t)trk_cap)) != DS_OK) return s;
        h.cap_trk = trk_cap;
    }
    if (vtx_cap > h.cap_vtx) {
        if ((s = grow(ctx, &h.vertices, (size_t)vtx_cap)) != DS_OK) return s;
        h.cap_vtx = vtx_cap;
    }
    DS_CUDA(cudaMemcpyAsync(h.seed_off, h_seed_off, sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, st), "H2D");
    DS_CUDA(cudaMemcpyAsync(h.hit_off, h_hit_off, sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, st), "H2D");
    for (int k = 0; k < 6 && S > 0; ++k)
        DS_CUDA(cudaMemcpyAsync(h.seed_cols + (size_t)k * S, h_seed_cols[k], sizeof(float) * S,
                                cudaMemcpyHostToDevice, st), "H2D");
    for (int k = 0; k < 3 && H > 0; ++k)
        DS_CUDA(cudaMemcpyAsync(h.hit_cols + (size_t)k * H, h_hit_cols[k], sizeof(float) * H,
                                cudaMemcpyHostToDevice, st), "H2D");
    if (H > 0) DS_CUDA(cudaMemcpyAsync(h.layer, h_layer, H, cudaMemcpyHostToDevice, st), "H2D");

    ds_event_batch b{E, S, H, 0, h.seed_off, h.hit_off};
    ds_seeds sd{h.seed_cols, h.seed_cols + S, h.seed_cols + 2 * (size_t)S, h.seed_cols + 3 * (size_t)S,
                h.seed_cols + 4 * (size_t)S, h.seed_cols + 5 * (size_t)S};
    ds_ut_hits ht{h.hit_cols, h.hit_cols + H, h.hit_cols + 2 * (size_t)H, h.layer};
    ds_tracks tr{h.tracks, h.trk_off, h.counts, trk_cap, 0};
    if ((s = ds_reconstruct(ctx, &b, &sd, &ht, &tr, stream)) != DS_OK) return s;
    ds_vertices vx{h.vertices, h.vtx_off, h.counts + 1, vtx_cap, 0};
    if ((s = ds_vertex(ctx, &tr, &vx, stream)) != DS_OK) return s;
    int32_t counts[2] = {0, 0};
    if (E > 0) {
        DS_CUDA(cudaMemcpyAsync(counts, h.counts, sizeof(counts), cudaMemcpyDeviceToHost, st), "D2H");
        DS_CUDA(cudaStreamSynchronize(st), "sync");
    }
    *n_tracks = counts[0];
    *n_vertices = counts[1];
    const int nt = counts[0] < trk_cap ? counts[0] : trk_cap;
    const int nv = counts[1] < vtx_cap ? counts[1] : vtx_cap;
    if (E > 0) {
        DS_CUDA(cudaMemcpyAsync(h_trk_off, h.trk_off, sizeof(int32_t) * (E + 1), cudaMemcpyDeviceToHost, st), "D2H");
        DS_CUDA(cudaMemcpyAsync(h_vtx_off, h.vtx_off, sizeof(int32_t) * (E + 1), cudaMemcpyDeviceToHost, st), "D2H");
    } else {
        h_trk_off[0] = 0;
        h_vtx_off[0] = 0;
    }
    if (nt > 0) DS_CUDA(cudaMemcpyAsync(h_tracks, h.tracks, sizeof(ds_track) * nt, cudaMemcpyDeviceToHost, st), "D2H");
    if (nv > 0)
        DS_CUDA(cudaMemcpyAsync(h_vertices, h.vertices, sizeof(ds_vertex_rec) * nv, cudaMemcpyDeviceToHost, st), "D2H");
    DS_CUDA(cudaStreamSynchronize(st), "sync");
    if (counts[0] > trk_cap || counts[1] > vtx_cap) return fail(ctx, DS_ERR_CAPACITY, "output capacity exceeded");
    return DS_OK;
}

}  // extern "C"
