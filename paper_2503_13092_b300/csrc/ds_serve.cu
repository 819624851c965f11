// Serving loop: continuous batching of event requests over ds_reconstruct +
// ds_vertex (contract in include/ds_serve.h).
//
// One worker thread owns every CUDA call of the server.  Requests are cut at
// submission into segments (whole requests, or runs of at most
// events_per_launch events) that fit one batch.  The worker repeatedly
//   - polls the batches in flight (two CUDA events per batch: counts ready,
//     records ready) and finishes those that are done,
//   - admits queued segments that have arrived into a free slot: continuous
//     batching merges as many as fit the slot's batch limits, and the batch is
//     admitted only if its device buffers fit the memory budget (a first-fit
//     arena carved out of one allocation made at creation).
// Each slot owns a library context (workspaces reserved at creation, so no
// allocation or device-wide synchronisation happens while serving) and a
// non-blocking stream; batches in different slots overlap on the device.
// Graph mode (default when the budget holds it): each slot also owns fixed
// device buffers for the largest batch, and a batch's kernels (reconstruct,
// vertex, renumber) are one replay of a CUDA graph captured at creation for
// the slot and the batch's event-count bucket (a power of two; the batch is
// padded with empty events and launched with its arrays' capacities,
// DS_BATCH_CAPACITY); only the copies are issued per batch.
// A batch's inputs come from the requests' host arrays: small arrays in
// device-readable pinned memory are read by one gather kernel (k_gather_host,
// many arrays per launch, no copy-engine set-up per array), the rest by one
// cudaMemcpyAsync each.
// Results are renumbered into each request's own event, seed, hit and track
// indices on the GPU (k_renumber, on the slot's stream after ds_vertex) and
// copied straight into the caller's output buffers.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "ds.h"
#include "ds_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
size_t align_up(size_t n) { return (n + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size): host-side bookkeeping of one device block.
struct Arena {
    size_t size = 0, used = 0, peak = 0;
    std::vector<std::pair<size_t, size_t>> free_list;   // (offset, size), sorted by offset, coalesced

    void init(size_t n)
    {
        size = n;
        free_list.assign(1, {0, n});
    }
    bool alloc(size_t n, size_t *off)
    {
        n = align_up(n);
        for (size_t i = 0; i < free_list.size(); ++i) {
            if (free_list[i].second >= n) {
                *off = free_list[i].first;
                free_list[i].first += n;
                free_list[i].second -= n;
                if (free_list[i].second == 0) free_list.erase(free_list.begin() + i);
                used += n;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n);
        auto it = std::lower_bound(free_list.begin(), free_list.end(), std::make_pair(off, size_t(0)));
        it = free_list.insert(it, {off, n});
        size_t i = it - free_list.begin();
        if (i + 1 < free_list.size() && free_list[i].first + free_list[i].second == free_list[i + 1].first) {
            free_list[i].second += free_list[i + 1].second;
            free_list.erase(free_list.begin() + i + 1);
        }
        if (i > 0 && free_list[i - 1].first + free_list[i - 1].second == free_list[i].first) {
            free_list[i - 1].second += free_list[i].second;
            free_list.erase(free_list.begin() + i);
        }
        used -= n;
    }
};

struct SegOut {
    std::vector<ds_track> trk;
    std::vector<int32_t> trk_cnt;      // per event of the segment
    std::vector<ds_vertex_rec> vtx;    // i, j relative to the segment's first track
    std::vector<int32_t> vtx_cnt;
    int64_t n_vtx_total = 0;           // device count (may exceed what was stored)
};

struct Req {
    int64_t id = 0;
    ds_request r{};
    int mapped = -1;                   // 1: every input array device-readable (-1: not yet checked)
    double t_arrival = 0, t_admit = -1;
    int n_segs = 0, segs_done = 0, n_batches = 0;
    ds_status status = DS_OK;
    bool truncated = false;
    int64_t n_trk_total = 0, n_vtx_total = 0;   // single-segment requests
    std::vector<SegOut> out;                    // multi-segment requests
};

struct Seg {
    Req *q;
    int idx;          // segment index in the request
    int e0, e1;       // request events [e0, e1)
    int seeds() const { return q->r.seed_off[e1] - q->r.seed_off[e0]; }
    int hits() const { return q->r.hit_off[e1] - q->r.hit_off[e0]; }
};

// Device buffers of one batch inside the arena, in this order.
struct BatchLayout {
    size_t seed_off, hit_off, seed[6], hit[3], layer, trk, trk_off, ntrk, vtx, vtx_off, nvtx, seg, nseg, bytes;
    BatchLayout(int E, int S, int H, int V)
    {
        size_t o = 0;
        auto take = [&](size_t n) { size_t r = o; o += align_up(n > 0 ? n : 1); return r; };
        seed_off = take(4 * (size_t)(E + 1));
        hit_off = take(4 * (size_t)(E + 1));
        for (int c = 0; c < 6; ++c) seed[c] = take(4 * (size_t)S);
        for (int c = 0; c < 3; ++c) hit[c] = take(4 * (size_t)H);
        layer = take((size_t)H);
        trk = take(sizeof(ds_track) * (size_t)S);
        trk_off = take(4 * (size_t)(E + 1));
        ntrk = take(4);
        vtx = take(sizeof(ds_vertex_rec) * (size_t)V);
        vtx_off = take(4 * (size_t)(E + 1));
        nvtx = take(4);
        seg = take(16 * (size_t)E);       // at most one segment per event
        nseg = take(4);                   // the number of segments (read on the device)
        bytes = o;
    }
};

// One host -> device range for k_gather_host; chunk0 = the number of
// kGatherChunk-byte chunks of the descriptors before it.
struct GatherDesc {
    unsigned long long dst, src;
    uint32_t n, chunk0;
};
static_assert(sizeof(GatherDesc) == 24, "descriptor layout");

struct Slot {
    ds_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int phase = 0;                     // 0 idle, 1 computing, 2 copying records back
    std::vector<Seg> segs;
    std::vector<int> ev_base;          // first batch event of each segment
    int E = 0, S = 0, H = 0, V = 0;
    size_t off = 0, bytes = 0;
    char *dev = nullptr;               // arena base + off
    int n_t = 0, n_v = 0;
    // graph mode: fixed buffers (layout of the largest batch) and one graph per bucket
    bool fixed = false;
    char *fixed_dev = nullptr;
    std::vector<int> buckets;          // event counts, ascending
    std::vector<cudaGraphExec_t> graphs;
    int cap_t = 0, cap_v = 0;          // track / vertex capacities of the current batch's buffers
    // pinned staging
    int32_t *h_seed_off = nullptr, *h_hit_off = nullptr, *h_trk_off = nullptr, *h_vtx_off = nullptr;
    int32_t *h_counts = nullptr;
    int4 *h_seg = nullptr;             // segment table of the batch
    int32_t *h_seg_n = nullptr;        // its length
    ds_track *h_trk = nullptr;
    ds_vertex_rec *h_vtx = nullptr;
    bool own_mapped = false;           // the offset and segment tables above are device-readable
    // gather descriptors of the batch (host staging, device copy)
    GatherDesc *h_desc = nullptr, *d_desc = nullptr;
    int desc_cap = 0;
};

constexpr int kGatherChunk = 16384;
constexpr int kGatherCtas = 64;
constexpr int kGatherThreads = 256;

// True when the device can read [p, p + n) at address p: the first and last
// bytes lie in host memory that the runtime reports mapped at the same
// address (an array is one allocation, so the bytes between lie in it too).
bool device_readable(const void *p, size_t n)
{
    if (n == 0) return true;
    const char *ends[2] = {static_cast<const char *>(p), static_cast<const char *>(p) + n - 1};
    for (const char *q : ends) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer != static_cast<const void *>(q)) return false;
    }
    return true;
}

bool request_readable(const ds_request &r)
{
    const size_t S = (size_t)r.seed_off[r.n_events], H = (size_t)r.hit_off[r.n_events];
    const void *seeds[6] = {r.seed_x, r.seed_y, r.seed_tx, r.seed_ty, r.seed_qop, r.seed_chi2};
    for (const void *a : seeds)
        if (!device_readable(a, 4 * S)) return false;
    const void *hits[3] = {r.hit_x0, r.hit_ybeg, r.hit_yend};
    for (const void *a : hits)
        if (!device_readable(a, 4 * H)) return false;
    return device_readable(r.hit_layer, H);
}

}  // namespace

struct ds_server {
    int device = 0;
    ds_server_config cfg{};
    std::vector<Slot> slots;
    Arena arena;
    char *d_arena = nullptr;
    int64_t context_bytes = 0;
    int max_vtx = 0;
    int sm_count = 148;
    bool graph_mode = false;
    int graphs_captured = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Seg> queue;
    std::unordered_set<Req *> live;    // submitted, not yet completed
    std::deque<ds_completion> done;
    int64_t next_id = 1, submitted = 0, completed = 0;
    int64_t events_done = 0, batches = 0;
    int inflight = 0, peak_inflight = 0;
    std::atomic<double> t_launch{0.0}, t_finish{0.0};
    std::atomic<int64_t> bytes_gathered{0}, bytes_copied{0};
    bool stop = false;
    std::thread worker;
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    bool admit();
    void launch(Slot &sl);
    void copy_back(Slot &sl);
    void finish(Slot &sl);
    void fail_batch(Slot &sl, ds_status st);
    BatchLayout layout(const Slot &sl) const;
    ds_status capture_graphs(Slot &sl);
    ds_completion finalize(Req *q);
    void publish(const std::vector<std::pair<ds_completion, Req *>> &fin);   // mu held
    void release();          // CUDA resources (worker stopped)
};

namespace {

bool config_valid(const ds_server_config &c)
{
    return c.n_slots >= 1 && c.n_slots <= 16 && c.max_batch_events >= 1 && c.max_batch_seeds >= 1 &&
           c.max_batch_hits >= 1 && c.events_per_launch >= 0 && c.vertices_per_seed >= 0 && c.hbm_budget >= 0 &&
           c.gather_max_bytes >= 0 &&
           (c.mlp_precision == DS_MLP_FP32 || c.mlp_precision == DS_MLP_BF16 || c.mlp_precision == DS_MLP_FP8);
}

int vtx_capacity(const ds_server_config &c, int S)
{
    return (int)std::min<long long>((long long)c.vertices_per_seed * S + 4096, 0x7fffffffLL / 64);
}

}  // namespace

// ------------------------------------------------------------------ worker

namespace {

// Batch numbering -> request numbering, in place on the device before the
// records are copied back.  seg[k] = {first batch event of segment k, event
// shift, seed shift, hit shift}; vertex track indices become relative to the
// segment's first track (trk_off at its first event).
__global__ void k_renumber(ds_track *trk, const int32_t *n_trk, int cap_t, ds_vertex_rec *vtx,
                           const int32_t *n_vtx, int cap_v, const int32_t *trk_off, const int4 *seg,
                           const int32_t *n_seg_dev)
{
    const int nt = min(max(*n_trk, 0), cap_t), nv = min(max(*n_vtx, 0), cap_v);
    const int n_seg = *n_seg_dev;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt + nv; i += gridDim.x * blockDim.x) {
        const bool is_t = i < nt;
        const int ev = is_t ? trk[i].event : vtx[i - nt].event;
        int lo = 0, hi = n_seg;          // last k with seg[k].x <= ev
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg[mid].x <= ev) lo = mid;
            else hi = mid;
        }
        const int4 sg = seg[lo];
        if (is_t) {
            ds_track &t = trk[i];
            t.event += sg.y;
            t.seed += sg.z;
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (t.hit[l] >= 0) t.hit[l] += sg.w;
        } else {
            ds_vertex_rec &v = vtx[i - nt];
            const int tb = trk_off[sg.x];
            v.event += sg.y;
            v.i -= tb;
            v.j -= tb;
        }
    }
}

// Bytes [r, r + 16) of the 32-byte concatenation a|b, r = 4 q + s / 8
// (q, s uniform over the warp).
__device__ __forceinline__ uint4 bytes_at(const uint4 &a, const uint4 &b, int q, int s)
{
    uint32_t w0, w1, w2, w3, w4;
    switch (q) {
    case 0: w0 = a.x; w1 = a.y; w2 = a.z; w3 = a.w; w4 = b.x; break;
    case 1: w0 = a.y; w1 = a.z; w2 = a.w; w3 = b.x; w4 = b.y; break;
    case 2: w0 = a.z; w1 = a.w; w2 = b.x; w3 = b.y; w4 = b.z; break;
    default: w0 = a.w; w1 = b.x; w2 = b.y; w3 = b.z; w4 = b.w; break;
    }
    return make_uint4(__funnelshift_r(w0, w1, s), __funnelshift_r(w1, w2, s), __funnelshift_r(w2, w3, s),
                      __funnelshift_r(w3, w4, s));
}

// Host -> device gather: warps take kGatherChunk-byte chunks of the
// descriptors' ranges.  A warp writes its chunk in aligned 16-byte blocks of
// the destination; lane l reads the aligned 16-byte source block under its
// output block (only blocks that hold bytes of the source range, so no read
// leaves the pages of the source array) and takes the bytes it needs from its
// own block and its right neighbour's; lane 31 only reads, so a step covers
// 31 blocks.  Partial blocks at the ends of a chunk are written byte by byte.
__global__ void __launch_bounds__(kGatherThreads) k_gather_host(const GatherDesc *__restrict__ d, int n_desc,
                                                                 int n_chunks)
{
    const int lane = threadIdx.x & 31;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += n_warps) {
        int lo = 0, hi = n_desc - 1;             // the last descriptor with chunk0 <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int)d[mid].chunk0 <= c) lo = mid;
            else hi = mid - 1;
        }
        const GatherDesc e = d[lo];
        const unsigned long long b0 = (unsigned long long)(c - (int)e.chunk0) * kGatherChunk;
        const unsigned long long b1 = min((unsigned long long)e.n, b0 + kGatherChunk);
        const unsigned long long src_end = e.src + e.n;
        const unsigned long long w_lo = e.dst + b0, w_hi = e.dst + b1;   // bytes this warp writes
        const unsigned long long D0 = w_lo & ~15ull;
        const unsigned long long S0 = D0 + (e.src - e.dst);               // source byte under D0 (mod 2^64)
        const int r = (int)(S0 & 15);
        const int q = r >> 2, sh = (r & 3) * 8;
        const unsigned long long A0 = S0 & ~15ull;
        for (unsigned long long D = D0; D < w_hi; D += 31 * 16) {
            const unsigned long long Dl = D + 16ull * lane;
            const unsigned long long Al = A0 + (D - D0) + 16ull * lane;
            uint4 a = make_uint4(0u, 0u, 0u, 0u);
            if (Al < src_end && Al + 16 > e.src) a = __ldg(reinterpret_cast<const uint4 *>(Al));
            uint4 b;
            b.x = __shfl_down_sync(0xffffffffu, a.x, 1);
            b.y = __shfl_down_sync(0xffffffffu, a.y, 1);
            b.z = __shfl_down_sync(0xffffffffu, a.z, 1);
            b.w = __shfl_down_sync(0xffffffffu, a.w, 1);
            if (lane < 31 && Dl < w_hi) {
                const uint4 v = bytes_at(a, b, q, sh);
                const unsigned long long p0 = max(Dl, w_lo), p1 = min(Dl + 16, w_hi);
                if (p0 == Dl && p1 == Dl + 16) {
                    *reinterpret_cast<uint4 *>(Dl) = v;
                } else {
                    for (unsigned long long p = p0; p < p1; ++p) {
                        const int k = (int)(p - Dl);
                        const uint32_t wk = k < 8 ? (k < 4 ? v.x : v.y) : (k < 12 ? v.z : v.w);
                        *reinterpret_cast<uint8_t *>(p) = (uint8_t)(wk >> (8 * (k & 3)));
                    }
                }
            }
        }
    }
}

}  // namespace

// Outputs of a finished request: multi-segment requests are concatenated here
// (single-segment ones were written in place); returns its completion record.
ds_completion ds_server::finalize(Req *q)
{
    ds_request &r = q->r;
    int64_t nt = 0, nv = 0;
    bool trunc = q->truncated;
    if (q->n_segs == 1) {
        nt = q->n_trk_total;
        nv = q->n_vtx_total;
    } else {
        r.trk_off[0] = 0;
        r.vtx_off[0] = 0;
        int e = 0;
        for (SegOut &o : q->out) {
            const int32_t trk_base = (int32_t)nt;
            const int64_t nt0 = nt, nv0 = nv;
            for (size_t i = 0; i < o.trk_cnt.size(); ++i) {
                nt += o.trk_cnt[i];
                nv += o.vtx_cnt[i];
                r.trk_off[e + i + 1] = (int32_t)nt;
                r.vtx_off[e + i + 1] = (int32_t)nv;
            }
            e += (int)o.trk_cnt.size();
            const int64_t kt = std::max<int64_t>(0, std::min<int64_t>((int64_t)o.trk.size(), r.trk_capacity - nt0));
            if (kt > 0) std::memcpy(r.tracks + nt0, o.trk.data(), sizeof(ds_track) * kt);
            const int64_t kv = std::max<int64_t>(0, std::min<int64_t>((int64_t)o.vtx.size(), r.vtx_capacity - nv0));
            for (int64_t i = 0; i < kv; ++i) {
                ds_vertex_rec v = o.vtx[i];
                v.i += trk_base;
                v.j += trk_base;
                r.vertices[nv0 + i] = v;
            }
            if ((int64_t)o.vtx.size() < o.n_vtx_total) trunc = true;
        }
        q->out.clear();
    }
    if (nt > r.trk_capacity || nv > r.vtx_capacity) trunc = true;
    if (trunc && q->status == DS_OK) q->status = DS_ERR_CAPACITY;
    ds_completion c{};
    c.id = q->id;
    c.status = q->status;
    c.n_tracks = (int32_t)nt;
    c.n_vertices = (int32_t)nv;
    c.n_batches = q->n_batches;
    c.t_arrival = q->t_arrival;
    c.t_admit = q->t_admit;
    c.t_done = now();
    return c;
}

void ds_server::publish(const std::vector<std::pair<ds_completion, Req *>> &fin)   // mu held
{
    for (const auto &f : fin) {
        events_done += f.second->r.n_events;
        done.push_back(f.first);
        ++completed;
        live.erase(f.second);
    }
    if (!fin.empty()) cv_done.notify_all();
}

bool ds_server::admit()
{
    Slot *sl = nullptr;
    for (Slot &s : slots)
        if (s.phase == 0) {
            sl = &s;
            break;
        }
    if (!sl) return false;
    std::unique_lock<std::mutex> lk(mu);
    if (queue.empty()) return false;
    const double t = now();
    // peek: the longest prefix of arrived segments that fits one batch
    int E = 0, S = 0, H = 0, n = 0;
    for (const Seg &g : queue) {
        if (g.q->t_arrival > t) break;
        const int e = g.e1 - g.e0, s = g.seeds(), h = g.hits();
        if (n > 0 && (cfg.events_per_launch > 0 || E + e > cfg.max_batch_events || S + s > cfg.max_batch_seeds ||
                      H + h > cfg.max_batch_hits))
            break;
        E += e; S += s; H += h; ++n;
    }
    if (n == 0) return false;
    const int V = vtx_capacity(cfg, S);
    BatchLayout L(E, S, H, V);
    size_t off = 0;
    // admission by device memory (arena mode): wait for a batch to finish;
    // graph mode: the slot's fixed buffers hold any batch
    if (!sl->fixed && !arena.alloc(L.bytes, &off)) return false;
    sl->segs.assign(queue.begin(), queue.begin() + n);
    queue.erase(queue.begin(), queue.begin() + n);
    ++inflight;
    peak_inflight = std::max(peak_inflight, inflight);
    ++batches;
    lk.unlock();
    for (Seg &g : sl->segs) {
        if (g.q->t_admit < 0) g.q->t_admit = t;
        ++g.q->n_batches;
    }
    sl->E = E; sl->S = S; sl->H = H; sl->V = V;
    sl->off = off;
    sl->bytes = sl->fixed ? 0 : L.bytes;
    sl->dev = sl->fixed ? sl->fixed_dev : d_arena + off;
    sl->cap_t = sl->fixed ? cfg.max_batch_seeds : S;
    sl->cap_v = sl->fixed ? max_vtx : V;
    const double tl = now();
    launch(*sl);
    t_launch = t_launch + (now() - tl);
    return true;
}

BatchLayout ds_server::layout(const Slot &sl) const
{
    return sl.fixed ? BatchLayout(cfg.max_batch_events, cfg.max_batch_seeds, cfg.max_batch_hits, max_vtx)
                    : BatchLayout(sl.E, sl.S, sl.H, sl.V);
}

// Graph mode, at creation: one graph per event-count bucket of the slot's
// launch sequence over its fixed buffers, with the arrays' capacities
// (DS_BATCH_CAPACITY); the batch's sizes live in the offsets and the segment
// count on the device.
ds_status ds_server::capture_graphs(Slot &sl)
{
    BatchLayout L = layout(sl);
    char *d = sl.fixed_dev;
    ds_event_batch b{};
    b.n_seeds = cfg.max_batch_seeds;
    b.n_hits = cfg.max_batch_hits;
    b.flags = DS_BATCH_CAPACITY;
    b.seed_off = reinterpret_cast<int32_t *>(d + L.seed_off);
    b.hit_off = reinterpret_cast<int32_t *>(d + L.hit_off);
    ds_seeds sd{};
    const float **sc[6] = {&sd.x, &sd.y, &sd.tx, &sd.ty, &sd.qop, &sd.chi2};
    for (int c = 0; c < 6; ++c) *sc[c] = reinterpret_cast<float *>(d + L.seed[c]);
    ds_ut_hits ht{reinterpret_cast<float *>(d + L.hit[0]), reinterpret_cast<float *>(d + L.hit[1]),
                  reinterpret_cast<float *>(d + L.hit[2]), reinterpret_cast<uint8_t *>(d + L.layer)};
    for (int eb = 1;; eb = std::min(2 * eb, cfg.max_batch_events)) {
        sl.buckets.push_back(eb);
        if (eb == cfg.max_batch_events) break;
    }
    for (int eb : sl.buckets) {
        b.n_events = eb;
        ds_tracks tr{};
        tr.tracks = reinterpret_cast<ds_track *>(d + L.trk);
        tr.trk_off = reinterpret_cast<int32_t *>(d + L.trk_off);
        tr.n_tracks = reinterpret_cast<int32_t *>(d + L.ntrk);
        tr.capacity = cfg.max_batch_seeds;
        ds_vertices vx{};
        vx.vertices = reinterpret_cast<ds_vertex_rec *>(d + L.vtx);
        vx.vtx_off = reinterpret_cast<int32_t *>(d + L.vtx_off);
        vx.n_vertices = reinterpret_cast<int32_t *>(d + L.nvtx);
        vx.capacity = max_vtx;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DS_ERR_CUDA;
        ds_status s = ds_reconstruct(sl.ctx, &b, &sd, &ht, &tr, sl.st);
        if (s == DS_OK) s = ds_vertex(sl.ctx, &tr, &vx, sl.st);
        if (s == DS_OK) {
            k_renumber<<<2 * sm_count, 256, 0, sl.st>>>(tr.tracks, tr.n_tracks, cfg.max_batch_seeds, vx.vertices,
                                                        vx.n_vertices, max_vtx, tr.trk_off,
                                                        reinterpret_cast<const int4 *>(d + L.seg),
                                                        reinterpret_cast<const int32_t *>(d + L.nseg));
            if (cudaGetLastError() != cudaSuccess) s = DS_ERR_CUDA;
        }
        const cudaError_t ec = cudaStreamEndCapture(sl.st, &g);
        if (s != DS_OK || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return s != DS_OK ? s : DS_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return DS_ERR_CUDA;
        sl.graphs.push_back(ex);
        ++graphs_captured;
    }
    return DS_OK;
}

void ds_server::launch(Slot &sl)
{
    BatchLayout L = layout(sl);
    char *d = sl.dev;
    int32_t *d_seed_off = reinterpret_cast<int32_t *>(d + L.seed_off);
    int32_t *d_hit_off = reinterpret_cast<int32_t *>(d + L.hit_off);
    float *d_seed[6], *d_hit[3];
    for (int c = 0; c < 6; ++c) d_seed[c] = reinterpret_cast<float *>(d + L.seed[c]);
    for (int c = 0; c < 3; ++c) d_hit[c] = reinterpret_cast<float *>(d + L.hit[c]);
    uint8_t *d_layer = reinterpret_cast<uint8_t *>(d + L.layer);
    int4 *d_seg = reinterpret_cast<int4 *>(d + L.seg);
    // batch offsets and the segment table
    sl.ev_base.clear();
    int eb = 0, sb = 0, hb = 0;
    sl.h_seed_off[0] = 0;
    sl.h_hit_off[0] = 0;
    cudaError_t ce = cudaSuccess;
    // inputs: device-readable ranges below gather_max_bytes become gather
    // descriptors, the others one cudaMemcpyAsync each
    const size_t gmax = (size_t)cfg.gather_max_bytes;
    int nd = 0;
    uint32_t n_chunks = 0;
    int64_t gathered = 0, copied = 0;
    auto put = [&](void *dst, const void *src, size_t n, bool readable) {
        if (!n || ce != cudaSuccess) return;
        if (readable && n < gmax && nd < sl.desc_cap) {
            sl.h_desc[nd++] = GatherDesc{(unsigned long long)dst, (unsigned long long)src, (uint32_t)n, n_chunks};
            n_chunks += (uint32_t)((n + kGatherChunk - 1) / kGatherChunk);
            gathered += (int64_t)n;
        } else {
            ce = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, sl.st);
            copied += (int64_t)n;
        }
    };
    for (size_t k = 0; k < sl.segs.size(); ++k) {
        const Seg &g = sl.segs[k];
        const ds_request &r = g.q->r;
        if (gmax > 0 && g.q->mapped < 0) g.q->mapped = request_readable(r) ? 1 : 0;
        const bool rd = gmax > 0 && g.q->mapped == 1;
        sl.ev_base.push_back(eb);
        const int s0 = r.seed_off[g.e0], h0 = r.hit_off[g.e0];
        sl.h_seg[k] = make_int4(eb, g.e0 - eb, s0 - sb, h0 - hb);
        for (int e = g.e0; e < g.e1; ++e) {
            sl.h_seed_off[eb + e - g.e0 + 1] = sb + r.seed_off[e + 1] - s0;
            sl.h_hit_off[eb + e - g.e0 + 1] = hb + r.hit_off[e + 1] - h0;
        }
        const int ns = g.seeds(), nh = g.hits();
        const float *sc[6] = {r.seed_x, r.seed_y, r.seed_tx, r.seed_ty, r.seed_qop, r.seed_chi2};
        for (int c = 0; c < 6; ++c) put(d_seed[c] + sb, sc[c] + s0, 4 * (size_t)ns, rd);
        const float *hc[3] = {r.hit_x0, r.hit_ybeg, r.hit_yend};
        for (int c = 0; c < 3; ++c) put(d_hit[c] + hb, hc[c] + h0, 4 * (size_t)nh, rd);
        put(d_layer + hb, r.hit_layer + h0, (size_t)nh, rd);
        eb += g.e1 - g.e0; sb += ns; hb += nh;
    }
    const int n_seg = (int)sl.segs.size();
    // graph mode: the batch padded with empty events to its bucket
    int bucket = -1, E_launch = sl.E;
    if (sl.fixed) {
        bucket = 0;
        while (sl.buckets[bucket] < sl.E) ++bucket;
        E_launch = sl.buckets[bucket];
        for (int e = sl.E + 1; e <= E_launch; ++e) {
            sl.h_seed_off[e] = sb;
            sl.h_hit_off[e] = hb;
        }
    }
    sl.h_seg_n[0] = n_seg;
    put(d_seed_off, sl.h_seed_off, 4 * (size_t)(E_launch + 1), sl.own_mapped);
    put(d_hit_off, sl.h_hit_off, 4 * (size_t)(E_launch + 1), sl.own_mapped);
    put(d_seg, sl.h_seg, sizeof(int4) * (size_t)n_seg, sl.own_mapped);
    put(d + L.nseg, sl.h_seg_n, 4, sl.own_mapped);
    if (nd > 0 && ce == cudaSuccess) {
        ce = cudaMemcpyAsync(sl.d_desc, sl.h_desc, sizeof(GatherDesc) * (size_t)nd, cudaMemcpyHostToDevice, sl.st);
        if (ce == cudaSuccess) {
            const int warps = kGatherThreads / 32;
            const int grid = (int)std::min<uint32_t>(kGatherCtas, (n_chunks + warps - 1) / warps);
            k_gather_host<<<grid, kGatherThreads, 0, sl.st>>>(sl.d_desc, nd, (int)n_chunks);
            ce = cudaGetLastError();
        }
    }
    bytes_gathered += gathered;
    bytes_copied += copied;
    if (ce != cudaSuccess) return fail_batch(sl, DS_ERR_CUDA);
    ds_event_batch b{};
    b.n_events = sl.E; b.n_seeds = sl.S; b.n_hits = sl.H;
    b.seed_off = d_seed_off; b.hit_off = d_hit_off;
    ds_seeds sd{d_seed[0], d_seed[1], d_seed[2], d_seed[3], d_seed[4], d_seed[5]};
    ds_ut_hits ht{d_hit[0], d_hit[1], d_hit[2], d_layer};
    ds_tracks tr{};
    tr.tracks = reinterpret_cast<ds_track *>(d + L.trk);
    tr.trk_off = reinterpret_cast<int32_t *>(d + L.trk_off);
    tr.n_tracks = reinterpret_cast<int32_t *>(d + L.ntrk);
    tr.capacity = sl.cap_t;
    ds_vertices vx{};
    vx.vertices = reinterpret_cast<ds_vertex_rec *>(d + L.vtx);
    vx.vtx_off = reinterpret_cast<int32_t *>(d + L.vtx_off);
    vx.n_vertices = reinterpret_cast<int32_t *>(d + L.nvtx);
    vx.capacity = sl.cap_v;
    if (sl.fixed) {
        ce = cudaGraphLaunch(sl.graphs[bucket], sl.st);
    } else {
        ds_status s = ds_reconstruct(sl.ctx, &b, &sd, &ht, &tr, sl.st);
        if (s == DS_OK) s = ds_vertex(sl.ctx, &tr, &vx, sl.st);
        if (s != DS_OK) return fail_batch(sl, s);
        k_renumber<<<2 * sm_count, 256, 0, sl.st>>>(tr.tracks, tr.n_tracks, sl.S, vx.vertices, vx.n_vertices, sl.V,
                                                    tr.trk_off, d_seg, reinterpret_cast<const int32_t *>(d + L.nseg));
        ce = cudaGetLastError();
    }
    auto d2h = [&](void *dst, const void *src, size_t n) {
        if (n && ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, sl.st);
    };
    d2h(sl.h_counts, tr.n_tracks, 4);
    d2h(sl.h_counts + 1, vx.n_vertices, 4);
    d2h(sl.h_trk_off, tr.trk_off, 4 * (size_t)(sl.E + 1));
    d2h(sl.h_vtx_off, vx.vtx_off, 4 * (size_t)(sl.E + 1));
    if (ce == cudaSuccess) ce = cudaEventRecord(sl.ev_a, sl.st);
    if (ce != cudaSuccess) return fail_batch(sl, DS_ERR_CUDA);
    sl.phase = 1;
}

void ds_server::copy_back(Slot &sl)
{
    // Records of a request carried whole by this batch go straight into the
    // caller's buffers (DMA when they are pinned); those of requests cut into
    // several segments go to the slot's staging and are joined on completion.
    BatchLayout L = layout(sl);
    sl.n_t = std::min(std::max(sl.h_counts[0], 0), sl.cap_t);
    sl.n_v = std::min(std::max(sl.h_counts[1], 0), sl.cap_v);
    const bool vtx_ok = sl.h_counts[1] <= sl.cap_v;
    const ds_track *d_trk = reinterpret_cast<const ds_track *>(sl.dev + L.trk);
    const ds_vertex_rec *d_vtx = reinterpret_cast<const ds_vertex_rec *>(sl.dev + L.vtx);
    cudaError_t ce = cudaSuccess;
    auto d2h = [&](void *dst, const void *src, size_t n) {
        if (n && ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, sl.st);
    };
    for (size_t k = 0; k < sl.segs.size(); ++k) {
        const Seg &g = sl.segs[k];
        const ds_request &r = g.q->r;
        const int ne = g.e1 - g.e0, be = sl.ev_base[k];
        const int tb = sl.h_trk_off[be], te = std::min(sl.h_trk_off[be + ne], sl.n_t);
        const int vb = sl.h_vtx_off[be], ve = vtx_ok ? sl.h_vtx_off[be + ne] : vb;
        if (g.q->n_segs == 1) {
            d2h(r.tracks, d_trk + tb, sizeof(ds_track) * (size_t)std::max(0, std::min(te - tb, r.trk_capacity)));
            d2h(r.vertices, d_vtx + vb, sizeof(ds_vertex_rec) * (size_t)std::max(0, std::min(ve - vb, r.vtx_capacity)));
        } else {
            d2h(sl.h_trk + tb, d_trk + tb, sizeof(ds_track) * (size_t)std::max(0, te - tb));
            d2h(sl.h_vtx + vb, d_vtx + vb, sizeof(ds_vertex_rec) * (size_t)std::max(0, ve - vb));
        }
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(sl.ev_b, sl.st);
    if (ce != cudaSuccess) return fail_batch(sl, DS_ERR_CUDA);
    sl.phase = 2;
}

void ds_server::finish(Slot &sl)
{
    ds_stats stt{};
    const ds_status bs = ds_sync_status(sl.ctx, sl.st, &stt);
    // a batch whose vertices overflowed returns no vertex records (counts only)
    const bool vtx_ok = sl.h_counts[1] <= sl.cap_v;
    std::vector<std::pair<ds_completion, Req *>> fin;
    for (size_t k = 0; k < sl.segs.size(); ++k) {
        const Seg &g = sl.segs[k];
        Req *q = g.q;
        ds_request &r = q->r;
        const int ne = g.e1 - g.e0, be = sl.ev_base[k];
        const int tb = sl.h_trk_off[be], te = sl.h_trk_off[be + ne];
        const int vb = sl.h_vtx_off[be], ve = sl.h_vtx_off[be + ne];
        const int t_have = std::max(0, std::min(te, sl.n_t) - tb);
        const int v_have = vtx_ok ? ve - vb : 0;
        if (q->n_segs == 1) {   // the whole request: records already in the caller's buffers
            for (int i = 0; i <= ne; ++i) {
                r.trk_off[i] = sl.h_trk_off[be + i] - tb;
                r.vtx_off[i] = sl.h_vtx_off[be + i] - vb;
            }
            q->n_trk_total = te - tb;
            q->n_vtx_total = ve - vb;
            if (t_have < te - tb || v_have < ve - vb) q->truncated = true;
        } else {
            SegOut &o = q->out[g.idx];
            o.trk_cnt.resize(ne);
            o.vtx_cnt.resize(ne);
            for (int i = 0; i < ne; ++i) {
                o.trk_cnt[i] = sl.h_trk_off[be + i + 1] - sl.h_trk_off[be + i];
                o.vtx_cnt[i] = sl.h_vtx_off[be + i + 1] - sl.h_vtx_off[be + i];
            }
            o.trk.assign(sl.h_trk + tb, sl.h_trk + tb + t_have);
            o.vtx.assign(sl.h_vtx + vb, sl.h_vtx + vb + v_have);
            o.n_vtx_total = ve - vb;
            if (t_have < te - tb) q->truncated = true;
        }
        if (bs != DS_OK && q->status == DS_OK) q->status = bs;
        if (++q->segs_done == q->n_segs) fin.emplace_back(finalize(q), q);
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!sl.fixed) arena.release(sl.off, sl.bytes);
        publish(fin);
        --inflight;
    }
    sl.segs.clear();
    sl.phase = 0;
    for (auto &f : fin) delete f.second;
}

void ds_server::fail_batch(Slot &sl, ds_status st)
{
    cudaStreamSynchronize(sl.st);
    ds_sync_status(sl.ctx, sl.st, nullptr);   // clear the context's counters and flags
    std::vector<std::pair<ds_completion, Req *>> fin;
    for (const Seg &g : sl.segs) {
        Req *q = g.q;
        if (q->status == DS_OK) q->status = st;
        if (q->n_segs == 1) {
            for (int i = 0; i <= q->r.n_events; ++i) q->r.trk_off[i] = q->r.vtx_off[i] = 0;
        } else {
            SegOut &o = q->out[g.idx];
            o.trk_cnt.assign(g.e1 - g.e0, 0);
            o.vtx_cnt.assign(g.e1 - g.e0, 0);
        }
        if (++q->segs_done == q->n_segs) fin.emplace_back(finalize(q), q);
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!sl.fixed) arena.release(sl.off, sl.bytes);
        publish(fin);
        --inflight;
    }
    sl.segs.clear();
    sl.phase = 0;
    for (auto &f : fin) delete f.second;
}

void ds_server::run()
{
    cudaSetDevice(device);
    for (;;) {
        bool progressed = false;
        for (Slot &sl : slots) {
            if (sl.phase == 1 && cudaEventQuery(sl.ev_a) != cudaErrorNotReady) {
                copy_back(sl);
                progressed = true;
            } else if (sl.phase == 2 && cudaEventQuery(sl.ev_b) != cudaErrorNotReady) {
                const double tf = now();
                finish(sl);
                t_finish = t_finish + (now() - tf);
                progressed = true;
            }
        }
        while (admit()) progressed = true;
        std::unique_lock<std::mutex> lk(mu);
        if (stop && inflight == 0) break;
        if (progressed) continue;
        if (inflight > 0) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(10));
        } else if (!queue.empty()) {
            // head not arrived yet (or waiting for memory with nothing in flight)
            const double wait = std::max(0.0, std::min(queue.front().q->t_arrival - now(), 1e-3));
            cv_work.wait_for(lk, std::chrono::duration<double>(wait));
        } else {
            cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

void ds_server::release()
{
    cudaSetDevice(device);
    for (Slot &sl : slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        for (cudaGraphExec_t g : sl.graphs)
            if (g) cudaGraphExecDestroy(g);
        if (sl.ctx) ds_destroy(sl.ctx);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.ev_a) cudaEventDestroy(sl.ev_a);
        if (sl.ev_b) cudaEventDestroy(sl.ev_b);
        void *hp[] = {sl.h_seed_off, sl.h_hit_off, sl.h_trk_off, sl.h_vtx_off, sl.h_counts, sl.h_seg, sl.h_trk,
                      sl.h_vtx, sl.h_seg_n, sl.h_desc};
        for (void *p : hp)
            if (p) cudaFreeHost(p);
        if (sl.d_desc) cudaFree(sl.d_desc);
        sl = Slot();
    }
    if (d_arena) cudaFree(d_arena);
    d_arena = nullptr;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

void ds_server_default_config(ds_server_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->n_slots = 4;
    c->max_batch_events = 1024;
    c->max_batch_seeds = 1024 * 256;
    c->max_batch_hits = 1024 * 2048;
    c->events_per_launch = 0;
    c->vertices_per_seed = 16;
    c->hbm_budget = 0;
    c->mlp_precision = DS_MLP_FP32;
    c->graphs = 1;
    c->gather_max_bytes = 1 << 20;
}

ds_status ds_server_create(ds_server **out, int device, const ds_geometry *geom, const ds_nn_weights *weights,
                           const ds_params *params, const ds_server_config *cfg)
{
    if (!out || !geom || !weights || !params || !cfg) return DS_ERR_ARG;
    *out = nullptr;
    if (!config_valid(*cfg)) return DS_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    struct Guard {
        ds_server *p;
        ~Guard()
        {
            if (p) {
                p->release();
                delete p;
            }
        }
    } guard{new ds_server()};
    ds_server *s = guard.p;
    s->device = device;
    s->cfg = *cfg;
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return DS_ERR_CUDA;
    const size_t free_before = free_b;
    ds_params p = *params;
    p.mlp_precision = cfg->mlp_precision;
    s->max_vtx = vtx_capacity(*cfg, cfg->max_batch_seeds);
    s->slots.resize(cfg->n_slots);
    for (Slot &sl : s->slots) {
        ds_status st;
        if ((st = ds_create(&sl.ctx, device)) != DS_OK) return st;
        if ((st = ds_load_geometry(sl.ctx, geom)) != DS_OK || (st = ds_load_nn_weights(sl.ctx, weights)) != DS_OK ||
            (st = ds_set_params(sl.ctx, &p)) != DS_OK ||
            (st = ds_reserve(sl.ctx, cfg->max_batch_events, cfg->max_batch_seeds, cfg->max_batch_hits)) != DS_OK ||
            (st = ds_reserve_vertices(sl.ctx, s->max_vtx)) != DS_OK)
            return st;
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_b, cudaEventDisableTiming) != cudaSuccess)
            return DS_ERR_CUDA;
        const size_t E1 = (size_t)cfg->max_batch_events + 1;
        sl.desc_cap = 10 * cfg->max_batch_events + 4;
        if (cudaHostAlloc((void **)&sl.h_seed_off, 4 * E1, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_hit_off, 4 * E1, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_trk_off, 4 * E1, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_vtx_off, 4 * E1, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_counts, 8, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_seg_n, 4, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_seg, sizeof(int4) * E1, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_desc, sizeof(GatherDesc) * (size_t)sl.desc_cap, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_trk, sizeof(ds_track) * (size_t)cfg->max_batch_seeds, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_vtx, sizeof(ds_vertex_rec) * (size_t)s->max_vtx, 0) != cudaSuccess)
            return DS_ERR_OOM;
        if (cudaMalloc((void **)&sl.d_desc, sizeof(GatherDesc) * (size_t)sl.desc_cap) != cudaSuccess) return DS_ERR_OOM;
        sl.own_mapped = device_readable(sl.h_seed_off, 4 * E1) && device_readable(sl.h_hit_off, 4 * E1) &&
                        device_readable(sl.h_seg, sizeof(int4) * E1) && device_readable(sl.h_seg_n, 4);
    }
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return DS_ERR_CUDA;
    s->context_bytes = (int64_t)(free_before - std::min(free_before, free_b));
    size_t budget = cfg->hbm_budget > 0 ? (size_t)cfg->hbm_budget : free_b / 4;
    if (budget > free_b) return DS_ERR_OOM;
    if (cudaMalloc((void **)&s->d_arena, budget) != cudaSuccess) return DS_ERR_OOM;
    s->arena.init(budget);
    s->cfg.hbm_budget = (int64_t)budget;
    // graph mode when every slot's fixed buffers fit the budget
    const size_t slot_bytes =
        BatchLayout(cfg->max_batch_events, cfg->max_batch_seeds, cfg->max_batch_hits, s->max_vtx).bytes;
    if (cfg->graphs && slot_bytes * s->slots.size() <= budget) {
        s->graph_mode = true;
        for (Slot &sl : s->slots) {
            size_t off = 0;
            if (!s->arena.alloc(slot_bytes, &off)) return DS_ERR_OOM;
            sl.fixed = true;
            sl.fixed_dev = s->d_arena + off;
            ds_status st = s->capture_graphs(sl);
            if (st != DS_OK) return st;
        }
        if (cudaDeviceSynchronize() != cudaSuccess) return DS_ERR_CUDA;
    }
    s->t0 = Clock::now();
    s->worker = std::thread([s] { s->run(); });
    guard.p = nullptr;
    *out = s;
    return DS_OK;
}

double ds_server_now(ds_server *s) { return s ? s->now() : 0.0; }

ds_status ds_server_submit(ds_server *s, const ds_request *req, int64_t *id)
{
    if (!s || !req || req->n_events < 0) return DS_ERR_ARG;
    const ds_request &r = *req;
    if (!r.seed_off || !r.hit_off || !r.trk_off || !r.vtx_off || r.trk_capacity < 0 || r.vtx_capacity < 0)
        return DS_ERR_ARG;
    if ((r.trk_capacity > 0 && !r.tracks) || (r.vtx_capacity > 0 && !r.vertices)) return DS_ERR_ARG;
    if (r.seed_off[0] != 0 || r.hit_off[0] != 0) return DS_ERR_ARG;
    for (int e = 0; e < r.n_events; ++e)
        if (r.seed_off[e + 1] < r.seed_off[e] || r.hit_off[e + 1] < r.hit_off[e]) return DS_ERR_ARG;
    const int S = r.seed_off[r.n_events], H = r.hit_off[r.n_events];
    if (S > 0 && (!r.seed_x || !r.seed_y || !r.seed_tx || !r.seed_ty || !r.seed_qop || !r.seed_chi2)) return DS_ERR_ARG;
    if (H > 0 && (!r.hit_x0 || !r.hit_ybeg || !r.hit_yend || !r.hit_layer)) return DS_ERR_ARG;
    std::unique_ptr<Req> q(new Req());
    q->r = r;
    // cut into segments that fit one batch (and the memory budget)
    std::vector<Seg> segs;
    const ds_server_config &c = s->cfg;
    int e = 0;
    while (e < r.n_events) {
        int e1 = e;
        while (e1 < r.n_events) {
            const int ne = e1 + 1 - e;
            const int ns = r.seed_off[e1 + 1] - r.seed_off[e], nh = r.hit_off[e1 + 1] - r.hit_off[e];
            if (ne > c.max_batch_events || ns > c.max_batch_seeds || nh > c.max_batch_hits) break;
            if (c.events_per_launch > 0 && ne > c.events_per_launch) break;
            ++e1;
        }
        if (e1 == e) return DS_ERR_CAPACITY;            // one event larger than a batch
        Seg g{q.get(), (int)segs.size(), e, e1};
        BatchLayout L(e1 - e, g.seeds(), g.hits(), vtx_capacity(c, g.seeds()));
        if (!s->graph_mode && L.bytes > s->arena.size) return DS_ERR_CAPACITY;
        segs.push_back(g);
        e = e1;
    }
    q->n_segs = (int)segs.size();
    q->out.resize(segs.size());
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = s->next_id++;
    q->t_arrival = r.arrival > 0.0 ? r.arrival : s->now();
    if (id) *id = q->id;
    ++s->submitted;
    Req *raw = q.release();
    s->live.insert(raw);
    if (segs.empty()) {                                // no events: complete at once
        raw->t_admit = raw->t_arrival;
        raw->n_segs = 1;
        raw->r.trk_off[0] = raw->r.vtx_off[0] = 0;
        std::vector<std::pair<ds_completion, Req *>> fin{{s->finalize(raw), raw}};
        s->publish(fin);
        delete raw;
        return DS_OK;
    }
    for (const Seg &g : segs) s->queue.push_back(g);
    s->cv_work.notify_all();
    return DS_OK;
}

int32_t ds_server_poll(ds_server *s, ds_completion *out, int32_t max_out, double timeout_s)
{
    if (!s || !out || max_out <= 0) return 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [s] { return !s->done.empty(); });
    int32_t n = 0;
    while (n < max_out && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

ds_status ds_server_drain(ds_server *s)
{
    if (!s) return DS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [s] { return s->completed == s->submitted; });
    return DS_OK;
}

ds_status ds_server_stats_get(ds_server *s, ds_server_stats *o)
{
    if (!s || !o) return DS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    o->requests_done = s->completed;
    o->events_done = s->events_done;
    o->batches = s->batches;
    o->hbm_budget = (int64_t)s->arena.size;
    o->hbm_peak = (int64_t)s->arena.peak;
    o->context_bytes = s->context_bytes;
    o->peak_inflight = s->peak_inflight;
    o->worker_launch_s = s->t_launch;
    o->worker_finish_s = s->t_finish;
    o->worker_wall_s = s->now();
    o->graphs = s->graph_mode ? 1 : 0;
    o->graphs_captured = s->graphs_captured;
    o->bytes_gathered = s->bytes_gathered.load();
    o->bytes_copied = s->bytes_copied.load();
    int64_t q = 0;
    const Req *last = nullptr;
    for (const Seg &g : s->queue)
        if (g.q != last) {
            ++q;
            last = g.q;
        }
    o->queued = (int32_t)q;
    return DS_OK;
}

void ds_server_destroy(ds_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.clear();            // queued segments are dropped; batches in flight finish
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Req *q : s->live) delete q;   // requests dropped before completing
    s->live.clear();
    s->release();
    delete s;
}

}  // extern "C"
