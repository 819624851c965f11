// a8 + a10 (tracks): clone killing and deterministic compaction.
//
// Clone killing (Algorithm Design section): among one event's per-seed winners,
// a track B is killed when another winner A shares more than two UT hits with
// it and has a lower key (response, chi2; chi2/ndof first in chi2-pick mode;
// ties by seed order).  Every decision is taken against the full set before
// killing, so the result does not depend on the order pairs are visited.
//
// One CTA per event (largest events first, in the order the bucketing
// kernel laid out): winners are chained by their UTbX and UTaU hits (hash
// heads in shared memory; hits, keys and chain links staged in shared memory
// for events up to kCloneSmem seeds, read from and kept in the workspace for
// larger ones), each thread owns a seed and compares it with the winners on
// its two chains, then alive seeds get their rank in seed order by a chunked
// block scan.  The last CTA to finish
// turns the per-event counts into trk_off with one scan; a second kernel
// scatters the surviving records to the packed output in (event, seed) order.
#include "ds_args.cuh"

namespace ds {

// 192 threads, 24 KB of shared memory and at most 40 registers: 8 CTAs per
// SM, so a batch of up to 8 x (number of SMs) events runs in one wave
constexpr int kCloneThreads = 192;
constexpr int kCloneCtasPerSm = 8;
constexpr int kCloneSmem = 512;
constexpr int kCloneHashBits = 10;


__device__ __forceinline__ int clone_hash(int id) { return (int)(((unsigned)id * 2654435761u) >> (32 - kCloneHashBits)); }

__device__ __forceinline__ bool kills(unsigned long long ko, int o, unsigned long long kb, int b, int4 ho, int4 hb)
{
    if (!(ko < kb || (ko == kb && o < b))) return false;
    const int shared = (ho.x >= 0 && ho.x == hb.x) + (ho.y >= 0 && ho.y == hb.y) + (ho.z >= 0 && ho.z == hb.z) +
                       (ho.w >= 0 && ho.w == hb.w);
    return shared > 2;
}

__global__ void __launch_bounds__(kCloneThreads, kCloneCtasPerSm) k_clone(const __grid_constant__ CloneArgs a)
{
    __shared__ unsigned long long s_key[kCloneSmem];
    __shared__ int4 s_hit[kCloneSmem];
    __shared__ int s_next_bx[kCloneSmem], s_next_au[kCloneSmem];
    __shared__ int s_head_bx[1 << kCloneHashBits], s_head_au[1 << kCloneHashBits];
    __shared__ int s_scan[32];
    __shared__ bool s_last;
    const int e = a.ev_order ? __ldg(a.ev_order + blockIdx.x) : (int)blockIdx.x;   // largest events first
    int s0 = __ldg(a.seed_off + e), s1 = __ldg(a.seed_off + e + 1);
    if (s0 < 0 || s1 < s0 || s1 > a.n_seeds) s0 = s1 = 0;
    const int ns = s1 - s0;
    const bool in_smem = ns <= kCloneSmem;
    const unsigned long long *K = a.key_ws + s0;
    const int4 *Hh = a.hit_ws + s0;
    int *g_next_bx = a.next_ws + 2 * (size_t)s0, *g_next_au = g_next_bx + ns;   // chains of larger events
    if (a.clone_kill) {
        // two winners sharing more than two of their hits share the UTbX hit or
        // the UTaU hit: chain the winners by those two hits
        for (int i = threadIdx.x; i < (1 << kCloneHashBits); i += blockDim.x) s_head_bx[i] = s_head_au[i] = -1;
        __syncthreads();
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const unsigned long long k = K[i];
            const int4 h = Hh[i];
            if (in_smem) {
                s_key[i] = k;
                s_hit[i] = h;
            }
            if (k != kNoKey) {
                const int nb = atomicExch(&s_head_bx[clone_hash(h.w)], i);
                const int na = h.y >= 0 ? atomicExch(&s_head_au[clone_hash(h.y)], i) : -1;
                if (in_smem) {
                    s_next_bx[i] = nb;
                    s_next_au[i] = na;
                } else {
                    g_next_bx[i] = nb;
                    g_next_au[i] = na;
                }
            }
        }
        __syncthreads();
    }

    int base = 0;
    for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
        const int b = c0 + threadIdx.x;
        int alive = 0;
        if (b < ns) {
            // the keys are staged in shared memory only when clone killing is on
            const unsigned long long kb = (in_smem && a.clone_kill) ? s_key[b] : K[b];
            if (kb != kNoKey) {
                alive = 1;
                if (a.clone_kill) {
                    if (in_smem) {
                        const int4 hb = s_hit[b];
                        for (int o = s_head_bx[clone_hash(hb.w)]; o >= 0 && alive; o = s_next_bx[o])
                            if (o != b && s_hit[o].w == hb.w && kills(s_key[o], o, kb, b, s_hit[o], hb)) alive = 0;
                        if (hb.y >= 0)
                            for (int o = s_head_au[clone_hash(hb.y)]; o >= 0 && alive; o = s_next_au[o])
                                if (o != b && s_hit[o].y == hb.y && kills(s_key[o], o, kb, b, s_hit[o], hb))
                                    alive = 0;
                    } else {
                        // the same chains, links in the workspace (written by this block)
                        const int4 hb = Hh[b];
                        for (int o = s_head_bx[clone_hash(hb.w)]; o >= 0 && alive; o = g_next_bx[o]) {
                            const int4 ho = Hh[o];
                            if (o != b && ho.w == hb.w && kills(K[o], o, kb, b, ho, hb)) alive = 0;
                        }
                        if (hb.y >= 0)
                            for (int o = s_head_au[clone_hash(hb.y)]; o >= 0 && alive; o = g_next_au[o]) {
                                const int4 ho = Hh[o];
                                if (o != b && ho.y == hb.y && kills(K[o], o, kb, b, ho, hb)) alive = 0;
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
    const int run = block_offsets(a.count_ws, a.n_events, a.trk_off, s_scan);
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
    // warp-cooperative copy: 32 seeds' records move as 128 contiguous 16-byte
    // chunks read, and contiguous runs written (consecutive survivors of an
    // event land next to each other)
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int warp_s0 = s - lane;
    int pos = -1;
    if (s < a.n_seeds && s >= __ldg(a.seed_off) && s < __ldg(a.seed_off + a.n_events)) {
        const int r = __ldg(a.rank_ws + s);
        if (r >= 0) {
            const int e = __ldg(&reinterpret_cast<const int *>(a.trk_ws + s)[0]);
            const int p = __ldg(a.trk_off + e) + r;
            pos = p < a.capacity ? p : -1;
        }
    }
    if (__ballot_sync(0xffffffffu, pos >= 0) == 0) return;
    const int4 *src = reinterpret_cast<const int4 *>(a.trk_ws + warp_s0);
    for (int k = lane; k < 128; k += 32) {
        const int rec = k >> 2;
        const int p = __shfl_sync(0xffffffffu, pos, rec);
        if (p >= 0) reinterpret_cast<int4 *>(a.out + p)[k & 3] = __ldg(src + k);
    }
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
