// a1: per-event bucketing of UT hits by (layer, Y sector, x bin).
//
// The paper groups UT hits into Y sectors so that a seed only visits hits of
// compatible sectors (Algorithm Design section, Dv1), and caches hits used in
// the combinatorics in shared memory (GPU Implementation section).  Here each
// event's hits are counting-sorted into 4 x n_sectors x 64 bins; a window
// |x0 - u| < w then maps to one contiguous range of the sorted array per
// sector, found from two uint16 offsets, with no binary search.
//
// One CTA per event.  Pass 1 counts bins with shared-memory atomics (hits
// stay in registers for events up to 6144 hits), a block scan turns counts into
// offsets (written out as the event's bin table), pass 2 scatters float4
// {x0, ybeg, yend, id} records and a compact x0 array in the same order.  The
// last CTA also turns per-event seed counts into the search kernel's work
// items (chunks of at most `chunk` <= 128 seeds of one event).  The order inside a bin comes
// from atomics and is not deterministic; every consumer ranks hits by
// (|dx|, id), which does not depend on it.
#include "ds_args.cuh"

namespace ds {


__device__ __forceinline__ int hit_bin(const DevGeom &g, float x0, float yb, float ye, int lay,
                                       int nb, DevCounters *cnt)
{
    // strips must lie in one Y sector; the sector is the one of the midpoint
    if (lay > 3 || !(x0 == x0) || !(yb == yb) || !(ye == ye) || fabsf(x0) > 1e30f) {
        raise_flag(cnt, DS_FLAG_BAD_LAYER);
        return nb;                    // parked after every real bin
    }
    const float ym = 0.5f * (yb + ye);
    const int k = sector_of(g, ym);
    const float lo = g.y_min + k * g.sector_h, hi = lo + g.sector_h;
    const float tol = 5e-3f;
    if (yb < lo - tol || ye > hi + tol) raise_flag(cnt, DS_FLAG_STRIP_SECTOR);
    return (lay * g.n_sec + k) * kNXB + xbin_of(g, x0);
}

__global__ void __launch_bounds__(kBucketThreads, 2) k_bucket(const __grid_constant__ BucketArgs a)
{
    extern __shared__ unsigned int s_cnt[];   // nb + 1 counters, then x0 staging
    __shared__ int s_scan[32];
    __shared__ bool s_last;
    const int e = blockIdx.x;
    const DevGeom &g = a.g;
    const int nb = 4 * g.n_sec * kNXB;

    int h0 = __ldg(a.hit_off + e), h1 = __ldg(a.hit_off + e + 1);
    uint16_t *table = a.bins + (size_t)e * g.table_stride;
    bool bad = h0 < 0 || h1 < h0 || h1 > a.n_hits;
    if (e == 0 && h0 != 0) bad = true;
    if (e == a.n_events - 1 && h1 != a.n_hits) bad = true;
    if (bad) {
        if (threadIdx.x == 0) raise_flag(a.cnt, DS_FLAG_BAD_OFFSETS);
        h0 = h1 = 0;
    }
    int n = h1 - h0;
    if (n > kMaxEventHits) {
        if (threadIdx.x == 0) raise_flag(a.cnt, DS_FLAG_EVENT_TOO_LARGE);
        n = 0;
    }

    for (int b = threadIdx.x; b <= nb; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    // pass 1: bin of every hit; small events keep their hits in registers
    const bool in_regs = n <= kBucketRegHits * (int)blockDim.x;
    int rb[kBucketRegHits];
    float rx[kBucketRegHits], ryb[kBucketRegHits], rye[kBucketRegHits];
    if (in_regs) {
#pragma unroll
        for (int k = 0; k < kBucketRegHits; ++k) {
            const int i = k * blockDim.x + threadIdx.x;
            rb[k] = -1;
            if (i < n) {
                const int h = h0 + i;
                rx[k] = __ldg(a.x0 + h);
                ryb[k] = __ldg(a.ybeg + h);
                rye[k] = __ldg(a.yend + h);
                rb[k] = hit_bin(g, rx[k], ryb[k], rye[k], __ldg(a.layer + h), nb, a.cnt);
                atomicAdd(&s_cnt[rb[k]], 1u);
            }
        }
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int h = h0 + i;
            const int b = hit_bin(g, __ldg(a.x0 + h), __ldg(a.ybeg + h), __ldg(a.yend + h), __ldg(a.layer + h),
                                  nb, a.cnt);
            atomicAdd(&s_cnt[b], 1u);
        }
    }
    __syncthreads();

    // exclusive scan over nb + 1 counters: contiguous chunk per thread
    const int total_bins = nb + 1;
    const int per = (total_bins + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    int local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < total_bins) local += s_cnt[b0 + k];
    int tot;
    int run = block_exclusive_scan(local, s_scan, &tot);
    for (int k = 0; k < per; ++k) {
        const int b = b0 + k;
        if (b < total_bins) {
            const unsigned int c = s_cnt[b];
            s_cnt[b] = run;
            table[b] = (uint16_t)run;
            run += c;
        }
    }
    // remaining table entries (padding) point at the end of the valid hits
    for (int b = total_bins + threadIdx.x; b < g.table_stride; b += blockDim.x)
        table[b] = (uint16_t)n;
    __syncthreads();

    // pass 2: scatter float4 records; the compact x0 array is assembled in
    // shared memory and written out coalesced
    float *xs = reinterpret_cast<float *>(s_cnt + ((nb + 1 + 3) & ~3));
    if (in_regs) {
#pragma unroll
        for (int k = 0; k < kBucketRegHits; ++k) {
            if (rb[k] >= 0) {
                const unsigned int slot = atomicAdd(&s_cnt[rb[k]], 1u);
                a.sorted[h0 + slot] = make_float4(rx[k], ryb[k], rye[k], __int_as_float(h0 + k * (int)blockDim.x +
                                                                                        (int)threadIdx.x));
                xs[slot] = rx[k];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) a.sx0[h0 + i] = xs[i];
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int h = h0 + i;
            const float x0 = __ldg(a.x0 + h), yb = __ldg(a.ybeg + h), ye = __ldg(a.yend + h);
            const int b = hit_bin(g, x0, yb, ye, __ldg(a.layer + h), nb, a.cnt);
            const unsigned int slot = atomicAdd(&s_cnt[b], 1u);
            a.sorted[h0 + slot] = make_float4(x0, yb, ye, __int_as_float(h));
            a.sx0[h0 + slot] = x0;
        }
    }

    // search work items of this event: chunks of at most a.chunk seeds;
    // the last CTA to finish scans them into item_off
    if (threadIdx.x == 0) {
        const int s0 = __ldg(a.seed_off + e), s1 = __ldg(a.seed_off + e + 1);
        const int ns = (s0 < 0 || s1 < s0 || s1 > a.n_seeds) ? 0 : s1 - s0;
        a.item_cnt[e] = (ns + a.chunk - 1) / a.chunk;
        __threadfence();
        const unsigned int t = atomicAdd(&a.cnt->done_bkt, 1u);
        s_last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int acc = 0;
    for (int c0 = 0; c0 < a.n_events; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int v = i < a.n_events ? __ldcg(a.item_cnt + i) : 0;
        int t;
        const int r = block_exclusive_scan(v, s_scan, &t);
        if (i < a.n_events) a.item_off[i] = acc + r;
        acc += t;
    }
    if (threadIdx.x == 0) {
        a.item_off[a.n_events] = acc;
        if (__ldg(a.seed_off) != 0 || __ldg(a.seed_off + a.n_events) != a.n_seeds)
            raise_flag(a.cnt, DS_FLAG_BAD_OFFSETS);
        a.cnt->done_bkt = 0;
    }
}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st, Prof *prof)
{
    if (a.n_events <= 0) return cudaSuccess;
    const int nb = 4 * a.g.n_sec * kNXB;
    const size_t smem = sizeof(unsigned int) * (size_t)((nb + 1 + 3) & ~3) + sizeof(float) * kBucketRegHits * kBucketThreads;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    prof->begin("k_bucket", st);
    k_bucket<<<a.n_events, kBucketThreads, smem, st>>>(a);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
