// Kernel argument blocks (passed by value as __grid_constant__ parameters)
// and the launch functions of libds.so's kernels.
#pragma once

#include <vector>

#include "ds_common.cuh"

namespace ds {

// Host-side launch recorder: CUDA events around each kernel when enabled.
struct Prof {
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<Rec> recs;
    void begin(const char *name, cudaStream_t st);
    void end(cudaStream_t st);
};

struct BucketArgs {
    DevGeom g;
    int n_events;
    int n_hits;
    int n_seeds;
    const int32_t *hit_off;
    const int32_t *seed_off;
    const float *x0, *ybeg, *yend;
    const uint8_t *layer;
    float *sx0;
    uint16_t *sperm;
    uint16_t *bins;
    int *item_off;         // [2 n_events + 2] search work items (k_bucket.cu)
    int chunk;             // max seeds per search work item (<= kSearchThreads)
    int order;             // work-item order (ds_tuning.search_order)
    int *ev_order;         // [n_events]: events by seed count, largest first (NULL: not laid out)
    int capacity_sizes;    // 1: n_seeds, n_hits are capacities (DS_BATCH_CAPACITY)
    DevCounters *cnt;
};

struct SearchArgs {
    DevGeom g;
    DevParams p;
    int n_events;
    int n_seeds;
    int n_hits;
    const int32_t *seed_off, *hit_off;
    const float *sx, *sy, *stx, *sty, *sqop, *schi2;
    const float *ybeg, *yend;   // the caller's hit arrays (strip extents)
    const float *sx0;
    const uint16_t *sperm;
    const uint16_t *bins;
    const int *item_off;   // work items laid out by k_bucket
    int chunk;             // max seeds per work item
    int order;             // 0: equal chunks in event order; 1: full chunks, then remainders largest first
    float4 *cand_feat;     // [cand_cap][4]: the 16 network inputs
    CandMeta *cand_meta;   // [cand_cap]
    int cand_cap;
    int4 *seed_cand;       // per seed: first candidate, count, event
    int *rank_ws;
    // fused form (fused = 1): every candidate is scored by the FP32 network
    // (16-32-32-1) inside the search and only each seed's winner leaves it,
    // as k_pick would write it: record, pick key and hit ids per seed
    int fused;
    DevNN nn;
    ds_track *trk_ws;
    unsigned long long *key_ws;
    int4 *hit_ws;
    int sm_count;
    int ctas_per_sm;       // persistent CTAs per SM
    int group;             // work items per queue pull
    int stage_hits;        // events with at most this many hits are staged in shared memory
    DevCounters *cnt;
};

// Ghost-killer weights for the tensor-core kernels, in the K-major no-swizzle
// core-matrix layout of tcgen05 operands (8 rows x 16 bytes per core matrix,
// core matrices 128 bytes apart along K).  W1 is 32 x 16 (E4M3: padded to K =
// 32 with zeros), W2 32 x 32.  FP8 weights are stored times a power of two
// per output neuron (row) bringing its largest weight into (224, 448];
// inv_s1, inv_s2 undo that per accumulator column in the epilogue.
struct MlpTcWeights {
    uint8_t b1_bf16[1024];
    uint8_t b2_bf16[2048];
    uint8_t b1_fp8[1024];
    uint8_t b2_fp8[1024];
    float inv_s1[32], inv_s2[32];
};

struct MlpArgs {
    DevNN nn;
    int n_in, n_h2;
    int precision;               // DS_MLP_FP32 / DS_MLP_BF16 / DS_MLP_FP8
    const MlpTcWeights *tc;      // device copy (BF16 / FP8 only)
    const float4 *feat;
    float *logit;
    int cand_cap;
    int n_host;                  // >= 0: number of candidates; < 0: read cnt->cand_used
    DevCounters *cnt;
};

struct PickArgs {
    DevParams p;
    int n_seeds, n_events;
    const int32_t *seed_off;
    const int4 *seed_cand;
    const float *logit;
    const CandMeta *meta;
    ds_track *trk_ws;
    unsigned long long *key_ws;
    int4 *hit_ws;
};

struct CloneArgs {
    int n_events, n_seeds;
    int clone_kill;
    const int32_t *seed_off;
    const unsigned long long *key_ws;
    const int4 *hit_ws;
    int *rank_ws;         // per seed: rank inside its event, -1 = not output
    int *next_ws;         // 2 ints per seed: clone chains of events larger than shared memory holds
    const int *ev_order;  // events largest first (k_bucket), or NULL: CTA b takes event b
    int *count_ws;        // per event
    int32_t *trk_off;     // [n_events + 1] (caller's)
    int32_t *n_tracks;    // caller's device scalar
    int capacity;
    DevCounters *cnt;
};

struct ScatterTrkArgs {
    int n_seeds;
    int n_events;
    const int32_t *seed_off;
    const ds_track *trk_ws;
    const int *rank_ws;
    const int32_t *trk_off;
    ds_track *out;
    int capacity;
};

struct VertexArgs {
    DevGeom g;
    DevParams p;
    int n_events;
    int trk_capacity;
    const ds_track *tracks;
    const int32_t *trk_off;
    const int32_t *n_tracks;
    ds_vertex_rec *pool;
    int *pool_pos;          // slot -> rank inside its event (small launch) or work item (large)
    int *pool_item;         // slot -> work item of the large-capacity launch
    int pool_cap;
    int *count_ws;          // per event
    const int *ev_order;    // a permutation of the events to pull them in (largest first), or NULL
    int *large_list;        // events with more tracks than the small launch takes
    int *large_pairs;       // per listed event: opposite-charge pairs
    int *large_item_off;    // per listed event: first work item (pair segment); [n_large] = total
    int *item_count;        // per work item: vertices kept
    int *item_base;         // per work item: vertices of the event's earlier items
    int max_items;
    int small_cap;          // events with at most this many tracks: one per CTA (<= kVtxSmallCapMax)
    int ctas_per_sm;        // of the one-event-per-CTA launch
    int32_t *vtx_off;
    int32_t *n_vertices;
    int capacity;
    DevCounters *cnt;
};

struct ScatterVtxArgs {
    const ds_vertex_rec *pool;
    const int *pool_pos;
    const int *pool_item;
    const int *item_base;
    int pool_cap;
    const int32_t *vtx_off;
    ds_vertex_rec *out;
    int capacity;
    const DevCounters *cnt;
};

// Trigger-line networks: up to 4 of 16 -> n_h1 (<= 32, zero-padded) -> 1.
struct DevLines {
    float w1[4][32][16];
    float b1[4][32];
    float w3[4][32];
    float b3[4];
    float mean[4][16];
    float scale[4][16];
    int n_lines;
};

// The line networks for the tensor-core kernel: first layers of all four as
// one 128 x 16 BF16 operand (K-major core matrices), normalisation folded in.
struct LineTcWeights {
    uint8_t b_bf16[4096];
    float b1[128];
    float w3[128];
    float b3[4];
    int n_lines;
};

struct VinfoArgs {
    DevGeom g;
    DevLines L;
    const LineTcWeights *tcw;   // device copy (tensor-core kernel)
    DevCounters *cnt;
    const ds_track *tracks;
    int trk_capacity;
    const int32_t *n_tracks;
    const ds_vertex_rec *vtx;
    int vtx_capacity;
    const int32_t *n_vertices;
    ds_vertex_info *out;
    int capacity;
};

cudaError_t launch_vertex_info(const VinfoArgs &a, bool tensor_cores, int sm_count, cudaStream_t st, Prof *prof);
void prepare_line_tc(const DevLines &L, LineTcWeights *out);
const char *fill_dev_lines(const ds_nn_weights *nets, int n_lines, DevLines *out);

// Host ABI structs -> device parameter blocks (nullptr = ok, else the reason).
const char *fill_dev_geom(const ds_geometry *gm, DevGeom *out);
const char *fill_dev_nn(const ds_nn_weights *w, DevNN *out, int *n_h2_kernel);
const char *fill_dev_params(const ds_params *p, DevParams *out);

cudaError_t init_vertex_attributes();
cudaError_t init_bucket_attributes();
cudaError_t init_search_attributes();
cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st, Prof *prof);
cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, Prof *prof);
cudaError_t launch_mlp_pick(const MlpArgs &m, const PickArgs &p, int sm_count, cudaStream_t st, Prof *prof);
// the network alone over n_bound candidates at most (m.n_host or the device count)
cudaError_t launch_mlp(const MlpArgs &m, int sm_count, int n_bound, cudaStream_t st);
cudaError_t launch_mlp_tc(const MlpArgs &m, int sm_count, int n_bound, cudaStream_t st);
void prepare_tc_weights(const DevNN &nn, int n_h2, MlpTcWeights *out);
// copy the candidate buffer out (features, seed, hits, logit) for training
cudaError_t launch_export_candidates(const float4 *feat, const CandMeta *meta, const float *logit, int cand_cap,
                                     const DevCounters *cnt, float *o_feat, int32_t *o_seed, int32_t *o_hits,
                                     float *o_logit, int capacity, int32_t *o_count, int sm_count, cudaStream_t st);
cudaError_t launch_clone(const CloneArgs &a, const ScatterTrkArgs &sa, cudaStream_t st, Prof *prof);
cudaError_t launch_vertex(const VertexArgs &a, const ScatterVtxArgs &sa, int sm_count, cudaStream_t st,
                          Prof *prof);

}  // namespace ds
