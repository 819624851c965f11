// a1: per-event bucketing of UT hits by (layer, Y sector, x bin).
//
// The paper groups UT hits into Y sectors so that a seed only visits hits of
// compatible sectors (Algorithm Design section, Dv1), and caches hits used in
// the combinatorics in shared memory (GPU Implementation section).  Here each
// event's hits are counting-sorted into 4 x n_sectors x 64 bins; a window
// |x0 - u| < w then maps to one contiguous range of the sorted array per
// sector, found from two uint16 offsets, with no binary search.
//
// One CTA per event.  Pass 1 counts bins with shared-memory atomics, a block
// scan turns counts into offsets (written out as the event's bin table), pass 2
// scatters float4 {x0, ybeg, yend, id} records.  The order inside a bin comes
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

__global__ void __launch_bounds__(512) k_bucket(const __grid_constant__ BucketArgs a)
{
    extern __shared__ unsigned int s_cnt[];   // nb + 1 counters, then scan scratch
    __shared__ int s_scan[32];
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
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int h = h0 + i;
        int b = hit_bin(g, __ldg(a.x0 + h), __ldg(a.ybeg + h), __ldg(a.yend + h), __ldg(a.layer + h),
                        nb, a.cnt);
        atomicAdd(&s_cnt[b], 1u);
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

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int h = h0 + i;
        const float x0 = __ldg(a.x0 + h), yb = __ldg(a.ybeg + h), ye = __ldg(a.yend + h);
        const int b = hit_bin(g, x0, yb, ye, __ldg(a.layer + h), nb, a.cnt);
        const unsigned int slot = atomicAdd(&s_cnt[b], 1u);
        a.sorted[h0 + slot] = make_float4(x0, yb, ye, __int_as_float(h));
    }
}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st, Prof *prof)
{
    if (a.n_events <= 0) return cudaSuccess;
    const int nb = 4 * a.g.n_sec * kNXB;
    const size_t smem = sizeof(unsigned int) * (size_t)(nb + 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    prof->begin("k_bucket", st);
    k_bucket<<<a.n_events, 512, smem, st>>>(a);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
