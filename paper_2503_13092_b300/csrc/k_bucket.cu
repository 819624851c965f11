// a1: per-event bucketing of UT hits by (layer, Y sector, x bin).
//
// The paper groups UT hits into Y sectors so that a seed only visits hits of
// compatible sectors (Algorithm Design section, Dv1), and caches hits used in
// the combinatorics in shared memory (GPU Implementation section).  Here each
// event's hits are counting-sorted into 4 x n_sectors x 64 bins; a window
// |x0 - u| < w then maps to one contiguous range of the sorted array per
// sector, found from two uint16 offsets, with no binary search.
//
// One CTA per event.  Pass 1 reads the hits with 16-byte loads (4 hits per
// load; events up to 6144 hits stay in registers) and counts bins with
// shared-memory atomics, a block scan turns counts into offsets (written out
// as the event's bin table), pass 2 places each hit's x0 and its index inside
// the event at its sorted position in shared memory, and both arrays are
// written with coalesced stores.  Larger events scatter straight to global
// memory.  Pass 1 also marks the (layer, sector) rows holding a strip
// shorter than its sector (one bit per row, written beside the bin table);
// the search decides the strip test of an unmarked row from the sector's
// bounds.  Block 0 also turns the per-event seed counts into the search
// kernel's work items (chunks of at most `chunk` <= 128 seeds of one event,
// by default the full chunks first and the remainders largest first) and the
// events by seed count, largest first, the order in which the clone-killing
// and vertex kernels take them.
// The order inside a bin comes from atomics and is not deterministic; every
// consumer ranks hits by (|dx|, id), which does not depend on it.
#include "ds_args.cuh"

namespace ds {

// Events by seed count, largest first: bucket of a count (steps of 16 seeds,
// 2032 and more in the first bucket).
constexpr int kEvBuckets = 128;
__device__ __forceinline__ int ev_bucket(int ns) { return kEvBuckets - 1 - min(ns >> 4, kEvBuckets - 1); }

// Bin counters per CTA: every thread scans a run of `per` consecutive
// counters, a multiple of 4 (16-byte shared loads, 8-byte table stores).
__host__ __device__ constexpr int bucket_counters_per_thread(int n_sec)
{
    return ((4 * n_sec * kNXB + 1 + kBucketThreads - 1) / kBucketThreads + 3) & ~3;
}
__host__ __device__ constexpr int bucket_cnt_words(int n_sec) { return bucket_counters_per_thread(n_sec) * kBucketThreads; }

__device__ __forceinline__ int hit_bin(const DevGeom &g, float x0, float yb, float ye, int lay,
                                       int nb, DevCounters *cnt, uint32_t *part)
{
    // strips must lie in one Y sector; the sector is the one of the midpoint
    if (lay > 3 || !(x0 == x0) || !(yb == yb) || !(ye == ye) || fabsf(x0) > 1e30f) {
        raise_flag(cnt, DS_FLAG_BAD_LAYER);
        return nb;                    // parked after every real bin
    }
    const float ym = 0.5f * (yb + ye);
    const int k = sector_of(g, ym);
    const float lo = sector_lo(g, k), hi = sector_hi(g, k);
    const float tol = 5e-3f;
    if (yb < lo - tol || ye > hi + tol) raise_flag(cnt, DS_FLAG_STRIP_SECTOR);
    const int row = lay * g.n_sec + k;
    if (yb > lo || ye < hi) atomicOr(part + (row >> 5), 1u << (row & 31));   // strip shorter than its sector
    return row * kNXB + xbin_of(g, x0);
}

__global__ void __launch_bounds__(kBucketThreads, 3) k_bucket(const __grid_constant__ BucketArgs a)
{
    // dynamic shared memory: nb + 1 bin counters (padded to 16 bytes), then the
    // event's x0 and hit indices in sorted order (events up to kBucketStage hits)
    extern __shared__ __align__(16) unsigned int s_cnt[];
    __shared__ uint32_t s_part[4];                // rows with a strip shorter than its sector
    __shared__ int s_scan[32];
    const int e = blockIdx.x;
    const DevGeom &g = a.g;
    const int nb = 4 * g.n_sec * kNXB;
    const int tid = threadIdx.x;

    int h0 = __ldg(a.hit_off + e), h1 = __ldg(a.hit_off + e + 1);
    uint16_t *table = a.bins + (size_t)e * g.table_stride;
    bool bad = h0 < 0 || h1 < h0 || h1 > a.n_hits;
    if (e == 0 && h0 != 0) bad = true;
    if (e == a.n_events - 1 && h1 != a.n_hits && !a.capacity_sizes) bad = true;
    if (bad) {
        if (tid == 0) raise_flag(a.cnt, DS_FLAG_BAD_OFFSETS);
        h0 = h1 = 0;
    }
    int n = h1 - h0;
    if (n > kMaxEventHits) {
        if (tid == 0) raise_flag(a.cnt, DS_FLAG_EVENT_TOO_LARGE);
        n = 0;
        h1 = h0;
    }

    // search work items: chunks of at most a.chunk seeds of one event.  They
    // depend on the seed offsets only, so block 0 lays them out first.
    // Order 0: event e's seeds in ceil(ns / chunk) chunks whose sizes differ
    // by at most one, events in order; item_off[e] = e's first item.
    // Order 1 (largest first): every full chunk of `chunk` seeds, events in
    // order (item_off[e] = e's first full chunk), then one item per event for
    // its remaining ns mod chunk seeds, the largest remainders first
    // (item_off[n_events + 2 + r] = the event of remainder item r).  The
    // queue then ends with its smallest items, so the persistent CTAs run
    // out of work at nearly the same time instead of a last partial wave of
    // full-size items running on a few SMs.  item_off[n_events] = all items;
    // item_off[n_events + 1] = full chunks (order 1).
    if (e == 0) {
        const int32_t *so = a.seed_off;
        const int E = a.n_events, C = a.chunk;
        auto seeds_of = [so, &a](int k) {
            const int s0 = __ldg(so + k), s1 = __ldg(so + k + 1);
            return (s0 < 0 || s1 < s0 || s1 > a.n_seeds) ? 0 : s1 - s0;
        };
        int n_items;
        if (a.order == 0) {
            n_items = block_offsets_f([&](int k) { return (seeds_of(k) + C - 1) / C; }, E, a.item_off, s_scan);
        } else {
            const int n_full = block_offsets_f([&](int k) { return seeds_of(k) / C; }, E, a.item_off, s_scan);
            // counting sort of the remainders by size, largest first (the
            // order inside one size is free: it changes no output)
            int *s_rc = reinterpret_cast<int *>(s_cnt);   // [kSearchThreads + 1]: counts, then cursors
            for (int r = tid; r <= kSearchThreads; r += blockDim.x) s_rc[r] = 0;
            __syncthreads();
            for (int k = tid; k < E; k += blockDim.x) {
                const int r = seeds_of(k) % C;
                if (r) atomicAdd(s_rc + (C - r), 1);
            }
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int r = 0; r < kSearchThreads; ++r) {
                    const int c = s_rc[r];
                    s_rc[r] = run;
                    run += c;
                }
                s_rc[kSearchThreads] = run;
                a.item_off[E + 1] = n_full;
            }
            __syncthreads();
            for (int k = tid; k < E; k += blockDim.x) {
                const int r = seeds_of(k) % C;
                if (r) a.item_off[E + 2 + atomicAdd(s_rc + (C - r), 1)] = k;
            }
            n_items = n_full + s_rc[kSearchThreads];
            __syncthreads();   // s_cnt is cleared below
        }
        if (a.ev_order) {
            // the events by seed count, largest first (counting sort on the
            // count in steps of 16; the order inside a step is free), the
            // order in which the clone and vertex kernels take them
            __syncthreads();
            int *s_ec = reinterpret_cast<int *>(s_cnt);   // [kEvBuckets + 1]: counts, then cursors
            for (int r = tid; r <= kEvBuckets; r += blockDim.x) s_ec[r] = 0;
            __syncthreads();
            for (int k = tid; k < E; k += blockDim.x) atomicAdd(s_ec + ev_bucket(seeds_of(k)), 1);
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int r = 0; r < kEvBuckets; ++r) {
                    const int c = s_ec[r];
                    s_ec[r] = run;
                    run += c;
                }
            }
            __syncthreads();
            for (int k = tid; k < E; k += blockDim.x) a.ev_order[atomicAdd(s_ec + ev_bucket(seeds_of(k)), 1)] = k;
            __syncthreads();   // s_cnt is cleared below
        }
        if (tid == 0) {
            a.item_off[E] = n_items;
            const int s_end = __ldg(so + E);
            if (__ldg(so) != 0 || (a.capacity_sizes ? s_end > a.n_seeds : s_end != a.n_seeds))
                raise_flag(a.cnt, DS_FLAG_BAD_OFFSETS);
        }
    }

    const int per = bucket_counters_per_thread(g.n_sec);
    const int cnt_words = per * kBucketThreads;
    float *s_x = reinterpret_cast<float *>(s_cnt + cnt_words);
    uint16_t *s_pm = reinterpret_cast<uint16_t *>(s_x + kBucketStage);
    for (int w = tid; w < cnt_words / 4; w += blockDim.x) reinterpret_cast<uint4 *>(s_cnt)[w] = make_uint4(0, 0, 0, 0);
    if (tid < 4) s_part[tid] = 0u;
    __syncthreads();

    // pass 1: bins.  Events that fit the staging buffer are read with 16-byte
    // loads (4 hits per load, from the 4-aligned hit below h0) and kept in
    // registers; the rest with scalar loads.
    const int a0 = h0 & ~3;
    const bool aligned = ((reinterpret_cast<uintptr_t>(a.x0) | reinterpret_cast<uintptr_t>(a.ybeg) |
                           reinterpret_cast<uintptr_t>(a.yend)) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(a.layer) & 3) == 0;
    const bool vec = aligned && (h1 - a0) <= 4 * kBucketVecRows * (int)blockDim.x;
    const bool staged = n <= kBucketStage;
    float4 vx[kBucketVecRows], vyb[kBucketVecRows], vye[kBucketVecRows];
    int vb[kBucketVecRows][4];
    if (vec) {
#pragma unroll
        for (int r = 0; r < kBucketVecRows; ++r) {
            const int base = a0 + 4 * (r * (int)blockDim.x + tid);
#pragma unroll
            for (int j = 0; j < 4; ++j) vb[r][j] = -1;
            if (base < h1) {
                uchar4 ly;
                if (base + 4 <= a.n_hits) {      // whole group inside the arrays
                    vx[r] = __ldg(reinterpret_cast<const float4 *>(a.x0 + base));
                    vyb[r] = __ldg(reinterpret_cast<const float4 *>(a.ybeg + base));
                    vye[r] = __ldg(reinterpret_cast<const float4 *>(a.yend + base));
                    ly = __ldg(reinterpret_cast<const uchar4 *>(a.layer + base));
                } else {                         // the arrays end inside the group
                    float t[3][4];
                    unsigned char l4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = base + j < a.n_hits;
                        t[0][j] = in ? __ldg(a.x0 + base + j) : 0.f;
                        t[1][j] = in ? __ldg(a.ybeg + base + j) : 0.f;
                        t[2][j] = in ? __ldg(a.yend + base + j) : 0.f;
                        l4[j] = in ? __ldg(a.layer + base + j) : 0;
                    }
                    vx[r] = make_float4(t[0][0], t[0][1], t[0][2], t[0][3]);
                    vyb[r] = make_float4(t[1][0], t[1][1], t[1][2], t[1][3]);
                    vye[r] = make_float4(t[2][0], t[2][1], t[2][2], t[2][3]);
                    ly = make_uchar4(l4[0], l4[1], l4[2], l4[3]);
                }
                const float xs[4] = {vx[r].x, vx[r].y, vx[r].z, vx[r].w};
                const float ybs[4] = {vyb[r].x, vyb[r].y, vyb[r].z, vyb[r].w};
                const float yes[4] = {vye[r].x, vye[r].y, vye[r].z, vye[r].w};
                const int ls[4] = {ly.x, ly.y, ly.z, ly.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int h = base + j;
                    if (h >= h0 && h < h1) {
                        vb[r][j] = hit_bin(g, xs[j], ybs[j], yes[j], ls[j], nb, a.cnt, s_part);
                        atomicAdd(&s_cnt[vb[r][j]], 1u);
                    }
                }
            }
        }
    } else {
        for (int i = tid; i < n; i += blockDim.x) {
            const int h = h0 + i;
            const int b = hit_bin(g, __ldg(a.x0 + h), __ldg(a.ybeg + h), __ldg(a.yend + h), __ldg(a.layer + h),
                                  nb, a.cnt, s_part);
            atomicAdd(&s_cnt[b], 1u);
        }
    }
    __syncthreads();

    // exclusive scan over the counters (nb + 1 used, the rest zero): a run of
    // `per` consecutive counters per thread, read and written 4 at a time.
    // Every table entry below ext_off is written; those past the last bin get
    // the hit count (the padding points at the end of the valid hits).
    {
        uint4 *c4 = reinterpret_cast<uint4 *>(s_cnt + tid * per);
        int local = 0;
        for (int q = 0; q < per / 4; ++q) {
            const uint4 v = c4[q];
            local += (int)(v.x + v.y + v.z + v.w);
        }
        int tot;
        unsigned run = (unsigned)block_exclusive_scan(local, s_scan, &tot);
        for (int q = 0; q < per / 4; ++q) {
            const uint4 v = c4[q];
            uint4 o;
            o.x = run; run += v.x;
            o.y = run; run += v.y;
            o.z = run; run += v.z;
            o.w = run; run += v.w;
            c4[q] = o;
            const int b = tid * per + 4 * q;
            if (b < g.ext_off)
                *reinterpret_cast<uint2 *>(table + b) = make_uint2(o.x | (o.y << 16), o.z | (o.w << 16));
        }
    }
    // partial-strip row bits after the offsets
    if (tid < 4) reinterpret_cast<uint32_t *>(table + g.ext_off)[tid] = s_part[tid];
    __syncthreads();

    // pass 2: x0 and the index inside the event, in sorted order.  Staged
    // events are assembled in shared memory and written with coalesced stores.
    if (vec) {
#pragma unroll
        for (int r = 0; r < kBucketVecRows; ++r) {
            const int base = a0 + 4 * (r * (int)blockDim.x + tid);
            const float xs[4] = {vx[r].x, vx[r].y, vx[r].z, vx[r].w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (vb[r][j] >= 0) {
                    const unsigned int slot = atomicAdd(&s_cnt[vb[r][j]], 1u);
                    if (staged) {
                        s_x[slot] = xs[j];
                        s_pm[slot] = (uint16_t)(base + j - h0);
                    } else {
                        a.sx0[h0 + slot] = xs[j];
                        a.sperm[h0 + slot] = (uint16_t)(base + j - h0);
                    }
                }
        }
        if (staged) {
            __syncthreads();
            for (int i = tid; i < n; i += blockDim.x) {
                a.sx0[h0 + i] = s_x[i];
                a.sperm[h0 + i] = s_pm[i];
            }
        }
    } else {
        for (int i = tid; i < n; i += blockDim.x) {
            const int h = h0 + i;
            const float x0 = __ldg(a.x0 + h);
            const int b = hit_bin(g, x0, __ldg(a.ybeg + h), __ldg(a.yend + h), __ldg(a.layer + h), nb, a.cnt, s_part);
            const unsigned int slot = atomicAdd(&s_cnt[b], 1u);
            a.sx0[h0 + slot] = x0;
            a.sperm[h0 + slot] = (uint16_t)i;
        }
    }

}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st, Prof *prof)
{
    if (a.n_events <= 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned int) * (size_t)bucket_cnt_words(a.g.n_sec) +
                        (sizeof(float) + sizeof(uint16_t)) * kBucketStage;
    prof->begin("k_bucket", st);
    k_bucket<<<a.n_events, kBucketThreads, smem, st>>>(a);
    prof->end(st);
    return cudaGetLastError();
}

cudaError_t init_bucket_attributes()
{
    const size_t smem = sizeof(unsigned int) * (size_t)bucket_cnt_words(kMaxSectors) +
                        (sizeof(float) + sizeof(uint16_t)) * kBucketStage;
    // three CTAs per SM (about 52 KB each): ask for the largest shared-memory carveout
    cudaError_t e = cudaFuncSetAttribute(k_bucket, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

}  // namespace ds
