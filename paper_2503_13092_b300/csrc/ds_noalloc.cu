// ds_reconstruct_noalloc: ds_reconstruct for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns every device allocation through its own pool (and forbids others),
// callers that must not trigger an allocation that could implicitly
// synchronise the device in the middle of their work, and callers that cannot
// create a ds_ctx (which allocates its workspaces).  For them this entry point
// runs the same kernels as ds_reconstruct with every scratch buffer (bucketed
// hits, bin tables, per-seed winners, ranks, counters) carved out of one
// file-scope __device__ array of kScratchBytes, which each GPU that loads the
// library holds until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine; the caller passes the inputs and the outputs.
//
// The array's name is only a host-side stand-in in host code, not a device
// address, so the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and handed to the kernels.
// The first call on a device does that set-up; make it before any stream
// capture.  Every call shares the one array: calls that overlap on the GPU
// (two streams, two host threads) race on it and must be serialised by the
// caller.
#include <cstring>
#include <mutex>

#include "ds_args.cuh"

namespace ds {
namespace {

// Size limits of one call.
constexpr int kNAEvents = 256;
constexpr int kNASeeds = 16384;
constexpr int kNAHits = 327680;
constexpr int kNACandPerSeed = 8;
constexpr int kNACand = kNASeeds * kNACandPerSeed;
constexpr int kNATableStride = table_stride_for(kMaxSectors);

constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }
constexpr size_t kOffCounters = 0;
constexpr size_t kOffPerm = align256(sizeof(DevCounters));
constexpr size_t kOffSx0 = kOffPerm + align256(sizeof(uint16_t) * (size_t)kNAHits);
constexpr size_t kOffBins = kOffSx0 + align256(sizeof(float) * ((size_t)kNAHits + 4));
constexpr size_t kOffTrk = kOffBins + align256(sizeof(uint16_t) * (size_t)kNATableStride * kNAEvents);
constexpr size_t kOffKey = kOffTrk + align256(sizeof(ds_track) * (size_t)kNASeeds);
constexpr size_t kOffHit = kOffKey + align256(sizeof(unsigned long long) * (size_t)kNASeeds);
constexpr size_t kOffRank = kOffHit + align256(sizeof(int4) * (size_t)kNASeeds);
constexpr size_t kOffCloneNext = kOffRank + align256(sizeof(int) * (size_t)kNASeeds);
constexpr size_t kOffSeedCand = kOffCloneNext + align256(2 * sizeof(int) * (size_t)kNASeeds);
constexpr size_t kOffCount = kOffSeedCand + align256(sizeof(int4) * (size_t)kNASeeds);
constexpr size_t kOffItemOff = kOffCount + align256(sizeof(int) * (size_t)kNAEvents);
constexpr size_t kOffCandFeat = kOffItemOff + align256(sizeof(int) * (size_t)(3 * kNAEvents + 2));
constexpr size_t kOffCandMeta = kOffCandFeat + align256(sizeof(float4) * 4 * (size_t)kNACand);
constexpr size_t kOffCandLogit = kOffCandMeta + align256(sizeof(CandMeta) * (size_t)kNACand);
constexpr size_t kScratchBytes = kOffCandLogit + align256(sizeof(float) * (size_t)kNACand);
static_assert(kScratchBytes <= 32u * 1024 * 1024, "scratch must stay modest");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices] = {};   // device address of g_scratch, per device

__global__ void k_noalloc_flags(const DevCounters *cnt, uint32_t *flags_out)
{
    *flags_out = cnt->flags;
}

ds_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return DS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return DS_ERR_CUDA;
        if (init_search_attributes() != cudaSuccess || init_bucket_attributes() != cudaSuccess) return DS_ERR_CUDA;
        g_scratch_dev[device] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[device];
    return DS_OK;
}

}  // namespace
}  // namespace ds

extern "C" DS_API ds_status ds_reconstruct_noalloc(const ds_geometry *geom, const ds_params *params,
                                                   const ds_nn_weights *weights, const ds_event_batch *b,
                                                   const ds_seeds *sd, const ds_ut_hits *ht, ds_tracks *out,
                                                   uint32_t *d_flags, void *stream)
{
    using namespace ds;
    if (!geom || !params || !weights || !b || !sd || !ht || !out) return DS_ERR_ARG;
    if (b->n_events < 0 || b->n_seeds < 0 || b->n_hits < 0 || out->capacity < 0) return DS_ERR_ARG;
    if (b->flags & ~DS_BATCH_CAPACITY) return DS_ERR_ARG;
    if (b->n_events > kNAEvents || b->n_seeds > kNASeeds || b->n_hits > kNAHits) return DS_ERR_CAPACITY;
    // candidates are limited to kNACandPerSeed per seed on average (DS_FLAG_CAND_CAPACITY beyond)
    if (b->n_events > 0 && (!b->seed_off || !b->hit_off || !out->trk_off || !out->n_tracks)) return DS_ERR_ARG;
    if (b->n_seeds > 0 && (!sd->x || !sd->y || !sd->tx || !sd->ty || !sd->qop || !sd->chi2)) return DS_ERR_ARG;
    if (b->n_hits > 0 && (!ht->x0 || !ht->ybeg || !ht->yend || !ht->layer)) return DS_ERR_ARG;
    if (out->capacity > 0 && !out->tracks) return DS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out->tracks) % 16 != 0) return DS_ERR_ARG;
    if (params->mlp_precision != DS_MLP_FP32) return DS_ERR_ARG;
    // training mode can give every seed 40 candidates, five times what the
    // static candidate buffer holds per seed on average
    if (params->training) return DS_ERR_ARG;

    DevGeom g;
    DevParams p;
    DevNN nn;
    int nn_h2 = 0;
    if (fill_dev_geom(geom, &g) || fill_dev_params(params, &p) || fill_dev_nn(weights, &nn, &nn_h2))
        return DS_ERR_ARG;

    int device = 0, sm_count = 148;
    if (cudaGetDevice(&device) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sm_count < 1)
        return DS_ERR_CUDA;
    unsigned char *base = nullptr;
    ds_status st = scratch_address(device, &base);
    if (st != DS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DevCounters *cnt = reinterpret_cast<DevCounters *>(base + kOffCounters);

    out->n_events = b->n_events;
    // the array keeps the previous call's contents: counters start at zero
    if (cudaMemsetAsync(cnt, 0, sizeof(DevCounters), s) != cudaSuccess) return DS_ERR_CUDA;
    if (b->n_events > 0) {
        static Prof no_prof;   // profiling stays off here
        BucketArgs ba{};
        ba.g = g;
        ba.n_events = b->n_events;
        ba.n_hits = b->n_hits;
        ba.n_seeds = b->n_seeds;
        ba.hit_off = b->hit_off;
        ba.seed_off = b->seed_off;
        ba.x0 = ht->x0; ba.ybeg = ht->ybeg; ba.yend = ht->yend; ba.layer = ht->layer;
        ba.sx0 = reinterpret_cast<float *>(base + kOffSx0);
        ba.sperm = reinterpret_cast<uint16_t *>(base + kOffPerm);
        ba.bins = reinterpret_cast<uint16_t *>(base + kOffBins);
        ba.item_off = reinterpret_cast<int *>(base + kOffItemOff);
        ba.chunk = kSearchThreads;
        ba.order = 1;
        ba.ev_order = ba.item_off + 2 * kNAEvents + 2;
        ba.capacity_sizes = (b->flags & DS_BATCH_CAPACITY) ? 1 : 0;
        ba.cnt = cnt;
        if (launch_bucket(ba, s, &no_prof) != cudaSuccess) return DS_ERR_CUDA;

        SearchArgs sa{};
        sa.g = g;
        sa.p = p;
        sa.n_events = b->n_events;
        sa.n_seeds = b->n_seeds;
        sa.n_hits = b->n_hits;
        sa.seed_off = b->seed_off;
        sa.hit_off = b->hit_off;
        sa.sx = sd->x; sa.sy = sd->y; sa.stx = sd->tx; sa.sty = sd->ty; sa.sqop = sd->qop; sa.schi2 = sd->chi2;
        sa.ybeg = ht->ybeg;
        sa.yend = ht->yend;
        sa.sx0 = ba.sx0;
        sa.sperm = ba.sperm;
        sa.bins = ba.bins;
        sa.item_off = ba.item_off;
        sa.chunk = ba.chunk;
        sa.order = ba.order;
        sa.cand_feat = reinterpret_cast<float4 *>(base + kOffCandFeat);
        sa.cand_meta = reinterpret_cast<CandMeta *>(base + kOffCandMeta);
        sa.cand_cap = kNACand;
        sa.seed_cand = reinterpret_cast<int4 *>(base + kOffSeedCand);
        sa.rank_ws = reinterpret_cast<int *>(base + kOffRank);
        sa.sm_count = sm_count;
        sa.ctas_per_sm = kSearchCtasPerSm;
        sa.group = kSearchGroup;
        sa.stage_hits = kStageHits;
        sa.cnt = cnt;
        if (launch_search(sa, s, &no_prof) != cudaSuccess) return DS_ERR_CUDA;

        MlpArgs ma{};
        ma.nn = nn;
        ma.n_in = weights->n_in;
        ma.n_h2 = nn_h2;
        ma.precision = DS_MLP_FP32;
        ma.feat = sa.cand_feat;
        ma.logit = reinterpret_cast<float *>(base + kOffCandLogit);
        ma.cand_cap = kNACand;
        ma.n_host = -1;
        ma.cnt = cnt;
        PickArgs pa{};
        pa.p = p;
        pa.n_seeds = b->n_seeds;
        pa.n_events = b->n_events;
        pa.seed_off = b->seed_off;
        pa.seed_cand = sa.seed_cand;
        pa.logit = ma.logit;
        pa.meta = sa.cand_meta;
        pa.trk_ws = reinterpret_cast<ds_track *>(base + kOffTrk);
        pa.key_ws = reinterpret_cast<unsigned long long *>(base + kOffKey);
        pa.hit_ws = reinterpret_cast<int4 *>(base + kOffHit);
        if (launch_mlp_pick(ma, pa, sm_count, s, &no_prof) != cudaSuccess) return DS_ERR_CUDA;

        CloneArgs ca{};
        ca.n_events = b->n_events;
        ca.n_seeds = b->n_seeds;
        ca.clone_kill = p.clone_kill && !p.training;
        ca.seed_off = b->seed_off;
        ca.key_ws = pa.key_ws;
        ca.hit_ws = pa.hit_ws;
        ca.rank_ws = sa.rank_ws;
        ca.ev_order = ba.ev_order;
        ca.next_ws = reinterpret_cast<int *>(base + kOffCloneNext);
        ca.count_ws = reinterpret_cast<int *>(base + kOffCount);
        ca.trk_off = out->trk_off;
        ca.n_tracks = out->n_tracks;
        ca.capacity = out->capacity;
        ca.cnt = cnt;
        ScatterTrkArgs xa{};
        xa.n_seeds = b->n_seeds;
        xa.n_events = b->n_events;
        xa.seed_off = b->seed_off;
        xa.trk_ws = pa.trk_ws;
        xa.rank_ws = sa.rank_ws;
        xa.trk_off = out->trk_off;
        xa.out = out->tracks;
        xa.capacity = out->capacity;
        if (launch_clone(ca, xa, s, &no_prof) != cudaSuccess) return DS_ERR_CUDA;
    }
    if (d_flags) {
        k_noalloc_flags<<<1, 1, 0, s>>>(cnt, d_flags);
        if (cudaGetLastError() != cudaSuccess) return DS_ERR_CUDA;
    }
    return DS_OK;
}
