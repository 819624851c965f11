// a8 + a10 (tracks): clone killing and deterministic compaction.
//
// Clone killing (Algorithm Design section): among one event's per-seed winners,
// a track B is killed when another winner A shares more than two UT hits with
// it and has a lower key (response, chi2; chi2/ndof first in chi2-pick mode;
// ties by seed order).  Every decision is taken against the full set before
// killing, so the result does not depend on the order pairs are visited.
//
// One CTA per event: winners' hits and keys are staged in shared memory (up
// to kCloneSmem seeds; larger events read them from the workspace), each thread
// owns a seed and compares it with every other winner, then alive seeds get
// their rank in seed order by a chunked block scan.  The last CTA to finish
// turns the per-event counts into trk_off with one scan; a second kernel
// scatters the surviving records to the packed output in (event, seed) order.
#include "ds_args.cuh"

namespace ds {

constexpr int kCloneThreads = 256;
constexpr int kCloneSmem = 1536;


__global__ void __launch_bounds__(kCloneThreads) k_clone(const __grid_constant__ CloneArgs a)
{
    __shared__ unsigned long long s_key[kCloneSmem];
    __shared__ int4 s_hit[kCloneSmem];
    __shared__ int s_scan[32];
    __shared__ bool s_last;
    const int e = blockIdx.x;
    int s0 = __ldg(a.seed_off + e), s1 = __ldg(a.seed_off + e + 1);
    if (s0 < 0 || s1 < s0 || s1 > a.n_seeds) s0 = s1 = 0;
    const int ns = s1 - s0;
    const bool in_smem = ns <= kCloneSmem;
    const unsigned long long *K = a.key_ws + s0;
    const int4 *Hh = a.hit_ws + s0;
    if (in_smem) {
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            s_key[i] = K[i];
            s_hit[i] = Hh[i];
        }
        __syncthreads();
        K = s_key;
        Hh = s_hit;
    }

    int base = 0;
    for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
        const int b = c0 + threadIdx.x;
        int alive = 0;
        if (b < ns) {
            const unsigned long long kb = K[b];
            if (kb != kNoKey) {
                alive = 1;
                if (a.clone_kill) {
                    const int4 hb = Hh[b];
                    for (int o = 0; o < ns; ++o) {
                        const unsigned long long ko = K[o];
                        if (o == b || ko == kNoKey) continue;
                        if (!(ko < kb || (ko == kb && o < b))) continue;
                        const int4 ho = Hh[o];
                        const int shared = (ho.x >= 0 && ho.x == hb.x) + (ho.y >= 0 && ho.y == hb.y) +
                                           (ho.z >= 0 && ho.z == hb.z) + (ho.w >= 0 && ho.w == hb.w);
                        if (shared > 2) {
                            alive = 0;
                            break;
                        }
                    }
                }
            }
        }
        int tot;
        const int r = block_exclusive_scan(alive, s_scan, &tot);
        if (b < ns) a.rank_ws[s0 + b] = alive ? base + r : -1;
        base += tot;
    }

    // last CTA: scan the per-event counts into trk_off
    if (threadIdx.x == 0) {
        a.count_ws[e] = base;
        __threadfence();
        const unsigned int t = atomicAdd(&a.cnt->done_trk, 1u);
        s_last = t == (unsigned)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int run = 0;
    for (int c0 = 0; c0 < a.n_events; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int v = i < a.n_events ? __ldcg(a.count_ws + i) : 0;
        int tot;
        const int r = block_exclusive_scan(v, s_scan, &tot);
        if (i < a.n_events) a.trk_off[i] = run + r;
        run += tot;
    }
    if (threadIdx.x == 0) {
        a.trk_off[a.n_events] = run;
        *a.n_tracks = run;
        a.cnt->n_tracks = run;
        if (run > a.capacity) raise_flag(a.cnt, DS_FLAG_TRACK_CAPACITY);
        a.cnt->done_trk = 0;
    }
}


__global__ void __launch_bounds__(256) k_scatter_tracks(const __grid_constant__ ScatterTrkArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_seeds) return;
    const int r = __ldg(a.rank_ws + s);
    if (r < 0) return;
    const int4 *src = reinterpret_cast<const int4 *>(a.trk_ws + s);
    const int e = __ldg(&src[0].x);
    const int pos = __ldg(a.trk_off + e) + r;
    if (pos >= a.capacity) return;
    int4 *dst = reinterpret_cast<int4 *>(a.out + pos);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = __ldg(src + k);
}

cudaError_t launch_clone(const CloneArgs &a, const ScatterTrkArgs &sa, cudaStream_t st, Prof *prof)
{
    if (a.n_events <= 0) return cudaSuccess;
    prof->begin("k_clone", st);
    k_clone<<<a.n_events, kCloneThreads, 0, st>>>(a);
    prof->end(st);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || sa.n_seeds <= 0) return err;
    prof->begin("k_scatter_tracks", st);
    k_scatter_tracks<<<(sa.n_seeds + 255) / 256, 256, 0, st>>>(sa);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
