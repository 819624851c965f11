// Device-side definitions shared by the kernels of libds.so (sm_103a).
//
// Data layout in HBM (per batch):
//   seeds     caller's SoA float32 (x, y, tx, ty, qop, chi2), CSR over events
//   hits      caller's SoA (x0, ybeg, yend float32, layer u8), CSR over events
//   sx0       x0 per hit, grouped by event, then by (layer, Y sector, x bin)
//             (4 bytes per hit): staged per event in shared memory for the
//             window scans
//   sperm     the same order: uint16 index of the hit inside its event (2
//             bytes per hit), giving its id and, through the caller's arrays,
//             its strip extent when a window needs them
//   items     search work items: (event, chunk of <= 128 of its seeds)
//   bins      per event: uint16 offsets (layer, sector, xbin) -> first sorted
//             hit, relative to the event's first hit (<= 65535 hits per event),
//             then one bit per (layer, sector): set when one of its strips does
//             not cover the whole sector (otherwise a window decides the strip
//             test of the whole sector at once)
//   trk_ws    one 64-byte candidate-winner record per seed + its clone key
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ds.h"

namespace ds {

constexpr int kNXB = 64;             // x bins per (layer, Y sector)
constexpr int kMaxSectors = 32;
constexpr int kK1Max = 10;           // UTbX hits kept per seed (paper: up to 10)
constexpr int kMaxEventHits = 65535; // uint16 offsets
constexpr int kSearchThreads = 128;  // threads per CTA in the search kernel (max seeds per work item)
// run-time search shape (ds_tuning): defaults and limits
constexpr int kSearchGroup = 1;      // consecutive work items per queue pull
constexpr int kSearchCtasPerSm = 5;   // resident search CTAs per SM (shared memory and registers sized for 5)
constexpr int kStageHits = 5120;     // event x0 arrays up to this size are staged in shared memory (4 fused search CTAs per SM fit)
constexpr int kStageHitsMax = 46080; // largest staging buffer: 32-sector table + x0 + static arrays (fused form) < 227 KB
constexpr int kBucketThreads = 512;
constexpr int kBucketVecRows = 3;    // 16-byte loads (4 hits) per bucketing thread
constexpr int kBucketStage = 6144;   // events up to this many hits are sorted in shared memory
constexpr int kMaxVertexTracks = 4096; // tracks per event staged for vertexing
constexpr int kVtxCtasPerSmMax = 4;   // one-event-per-CTA vertexing: resident CTAs per SM at most (default)
constexpr int kVtxSmallCapMax = 512;  // its largest event (tracks staged per CTA); default limit
constexpr int kVtxLargeSeg = 65536;  // pairs per segment of the large-capacity vertex launch
constexpr int kVtxItemPairs = 2 * kVtxLargeSeg;   // pairs per work item there: two segments, the event's tracks staged once
// items of one event: its opposite-charge pairs, at most (4096 / 2)^2, in segments
constexpr int kVtxItemsPerEvent = (kMaxVertexTracks / 2) * (kMaxVertexTracks / 2) / kVtxItemPairs;
constexpr unsigned long long kNoKey = ~0ull;

// Per-event table: nb + 1 = 4 n_sec kNXB + 1 uint16 offsets padded to 8
// entries, then 16 bytes of flags, one bit per (layer, sector) row (<= 128).
__host__ __device__ constexpr int table_ext_offset(int n_sec) { return ((4 * n_sec * kNXB + 1) + 7) & ~7; }
__host__ __device__ constexpr int table_stride_for(int n_sec) { return table_ext_offset(n_sec) + 8; }

struct DevGeom {
    float z[4];
    float dxdy[4];
    float y_min, sector_h, inv_sector_h;
    int n_sec;
    float x_half, inv_xbin;          // xbin = floor((x0 + x_half) * inv_xbin)
    float z_seed;
    float zmag[4];
    float kappa, mp;
    float gamma0, gamma1, z_ref;
    float w_hit, w_mag;              // 1 / sigma^2
    float inv_sigma_hit;
    int table_stride;                // uint16 entries per event bin table (offsets + row bits)
    int ext_off;                     // uint16 entry where the partial-strip row bits start
};

struct DevParams {
    float w1a, w1b, w2, dy_tol;
    float nn_threshold, doca_max, nr_tol, eps_par;
    float thr_logit;                 // ln(T / (1 - T)): response < T <=> logit < thr_logit
    int k1, origin, pick_chi2, clone_kill, training, nr_max_iter;
    int fault_inject;                // tests only: bit 0 stalls the staging barrier
    int variant;                     // 0: Dv0, 1: Dv1 (triplet search)
    float dv1_dtx, dv1_w_tri;        // Dv1 kink bound and UTaX tolerance
};

// Ghost-killer weights padded to the largest supported shape 16-32-32-1.
// Padding is zero, so a smaller network gives identical results.
struct DevNN {
    float w1[32][16];
    float b1[32];
    float w2[32][32];
    float b2[32];
    float w3[32];
    float b3;
    float mean[16];
    float scale[16];
};

struct DevCounters {                 // device-side flag word and statistics
    unsigned int flags;
    unsigned int done_trk;           // last-block-done tickets
    unsigned int done_vtx;           // small-capacity vertex launch
    unsigned int done_vtx_large;     // large-capacity vertex launch
    int n_tracks;
    int n_vertices;
    int pool_used;
    int vtx_queue[2];                // event queues of the two vertex launches
    int n_large;                     // events left to the large-capacity vertex launch
    int pool_small;                  // vertex pool slots filled by the small-capacity launch
    int cand_used;                   // candidates written this call
    int search_queue;                // next search work item
    unsigned long long n_candidates;
    unsigned long long n_pairs;
    unsigned long long n_pairs_fp64;
};

// A candidate's fit, seed and hits (the network inputs are stored beside it).
struct __align__(16) CandMeta {
    float xr, yr, t, qop;
    float chi2;
    int ndof;
    int seed;
    float ty;
    int hit[4];                      // global hit ids, -1 = absent
};
static_assert(sizeof(CandMeta) == 48, "CandMeta is 48 bytes");

// Per-seed winner record in the workspace (same 64-byte layout as ds_track).
static_assert(sizeof(ds_track) == 64, "ds_track must be 64 bytes");
static_assert(sizeof(ds_vertex_rec) == 32, "ds_vertex_rec must be 32 bytes");
static_assert(sizeof(ds_vertex_info) == 64, "ds_vertex_info must be 64 bytes");

__device__ __forceinline__ void raise_flag(DevCounters *c, unsigned int bit)
{
    atomicOr(&c->flags, bit);
}

__device__ __forceinline__ int sector_of(const DevGeom &g, float y)
{
    int k = __float2int_rd((y - g.y_min) * g.inv_sector_h);
    return min(max(k, 0), g.n_sec - 1);
}

// Y extent of sector k, rounded the same way wherever it is used.
__device__ __forceinline__ float sector_lo(const DevGeom &g, int k) { return __fmaf_rn((float)k, g.sector_h, g.y_min); }
__device__ __forceinline__ float sector_hi(const DevGeom &g, int k) { return __fadd_rn(sector_lo(g, k), g.sector_h); }

// Strip test (ybeg - dy <= y && y <= yend + dy) for every hit of one (layer,
// sector) row at once.  A row whose flag bit is clear has only strips that
// cover the whole sector (ybeg <= lo, yend >= hi), so y in [lo - dy, hi + dy]
// passes for all of them (float rounding is monotonic).  Returns 1 when every
// hit of the row passes, 2 when the hits must be tested one by one.
__device__ __forceinline__ int sector_strip_class(const DevGeom &g, const uint32_t *part, int layer, int k,
                                                  float y, float dy)
{
    const int row = layer * g.n_sec + k;
    if ((part[row >> 5] >> (row & 31)) & 1u) return 2;
    return (__fsub_rn(sector_lo(g, k), dy) <= y && y <= __fadd_rn(sector_hi(g, k), dy)) ? 1 : 2;
}

__device__ __forceinline__ int xbin_of(const DevGeom &g, float x)
{
    int b = __float2int_rd((x + g.x_half) * g.inv_xbin);
    return min(max(b, 0), kNXB - 1);
}

// Largest e in [0, n) with off[e] <= s (off non-decreasing).
__device__ __forceinline__ int find_segment(const int32_t *__restrict__ off, int n, int s)
{
    int lo = 0, hi = n;          // invariant: off[lo] <= s, answer in [lo, hi)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= s) lo = mid;
        else hi = mid;
    }
    return lo;
}

// find_segment by one warp (all 32 lanes call it): 32 probes per round, so
// two or three dependent loads instead of log2(n).
__device__ __forceinline__ int warp_find_segment(const int32_t *__restrict__ off, int n, int s)
{
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n;          // invariant: off[lo] <= s, answer in [lo, hi)
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + lane * step;
        const unsigned m = __ballot_sync(0xffffffffu, idx < hi && __ldg(off + idx) <= s);
        const int k = 31 - __clz(m);   // lane 0 always qualifies
        lo += k * step;
        hi = min(hi, lo + step);
    }
    const unsigned m = __ballot_sync(0xffffffffu, lo + lane < hi && __ldg(off + lo + lane) <= s);
    return lo + 31 - __clz(m);
}

// Ghost-killer network (Ghost-Killer Neural Network section) in FP32, inputs
// normalised, ReLU hidden layer(s), output before the sigmoid.  Weights come
// from a kernel parameter block with compile-time indices (every lane reads
// the same weight: constant-bank operands of the FMAs).
template <int NIN, int NH1, int NH2>
__device__ __forceinline__ float mlp_logit_fp32(const DevNN &nn, const float (&phi)[16])
{
    float x[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) x[i] = (phi[i] - nn.mean[i]) * nn.scale[i];
    float h1[NH1];
#pragma unroll
    for (int o = 0; o < NH1; ++o) {
        float acc = nn.b1[o];
#pragma unroll
        for (int i = 0; i < NIN; ++i) acc = fmaf(nn.w1[o][i], x[i], acc);
        h1[o] = fmaxf(acc, 0.f);
    }
    float out = nn.b3;
    if (NH2 > 0) {
#pragma unroll
        for (int o = 0; o < NH2; ++o) {
            float acc = nn.b2[o];
#pragma unroll
            for (int i = 0; i < NH1; ++i) acc = fmaf(nn.w2[o][i], h1[i], acc);
            out = fmaf(nn.w3[o], fmaxf(acc, 0.f), out);
        }
    } else {
#pragma unroll
        for (int o = 0; o < NH1; ++o) out = fmaf(nn.w3[o], h1[o], out);
    }
    return out;
}

__device__ __forceinline__ float sigmoid_fast(float z) { return 1.f / (1.f + __expf(-z)); }

// Order-preserving float -> uint32 map (negative values included) and back.
__device__ __forceinline__ unsigned int ord_f32(float x)
{
    const unsigned int u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unord_f32(unsigned int o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ unsigned long long pack_key(float k1, float k2)
{
    return ((unsigned long long)ord_f32(k1) << 32) | ord_f32(k2);
}

// ---- bulk copies (TMA) into shared memory, completion on an mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned; bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr int kWaitLimit = 1 << 22;
constexpr int kMlpTcCtasPerSm = 8;        // persistent tensor-core network CTAs per SM: 8 x 64 TMEM columns = all 512, 8 x 128 threads x 64 registers = all 64K

// Exclusive scan of one int per thread over the block; returns the prefix,
// *total receives the block sum.  `scratch` holds >= 32 ints.  All threads call.
__device__ __forceinline__ int block_exclusive_scan(int v, int *scratch, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        scratch[lane] = w;         // inclusive warp totals
    }
    __syncthreads();
    int base = warp > 0 ? scratch[warp - 1] : 0;
    *total = scratch[nwarps - 1];
    __syncthreads();
    return base + x - v;
}

// block_exclusive_scan with one barrier: every warp scans the warp totals
// itself.  The caller must not hand the same scratch to another scan before
// the block has met again (the totals are read after the barrier).
__device__ __forceinline__ int block_exclusive_scan1(int v, int *scratch, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    int w = lane < nwarps ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
    }
    const int before = __shfl_sync(0xffffffffu, w, (warp + 31) & 31);   // inclusive total of the warps before
    *total = __shfl_sync(0xffffffffu, w, nwarps - 1);
    return (warp > 0 ? before : 0) + x - v;
}

// Exclusive prefix sums of n counts written by other CTAs (read from L2):
// off[i] = cnt[0] + ... + cnt[i - 1] for i < n; returns the total to every
// thread.  One contiguous chunk per thread, all of its loads issued before
// the one block scan (a single round trip instead of one per blockDim.x
// counts).  All threads call.
// count(i) gives the i-th count (block_offsets: a load).
template <class Count>
__device__ __forceinline__ int block_offsets_f(Count count, int n, int *off, int *scratch)
{
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = min((int)threadIdx.x * per, n), i1 = min(i0 + per, n);
    constexpr int R = 8;
    int v[R];
    int local = 0;
    if (per <= R) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            v[k] = i0 + k < i1 ? count(i0 + k) : 0;
            local += v[k];
        }
    } else {
        for (int i = i0; i < i1; ++i) local += count(i);
    }
    int total;
    int run = block_exclusive_scan(local, scratch, &total);
    if (per <= R) {
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (i0 + k < i1) {
                off[i0 + k] = run;
                run += v[k];
            }
    } else {
        for (int i = i0; i < i1; ++i) {
            off[i] = run;
            run += count(i);
        }
    }
    return total;
}

__device__ __forceinline__ int block_offsets(const int *cnt, int n, int *off, int *scratch)
{
    return block_offsets_f([cnt](int i) { return __ldcg(cnt + i); }, n, off, scratch);
}

}  // namespace ds
