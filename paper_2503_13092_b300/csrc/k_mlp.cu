// a6-a7: ghost-killer network over all candidates of the batch, best pick.
//
// Ghost-Killer Neural Network section: inputs -> ReLU hidden layer(s) ->
// sigmoid output; the response must stay below the threshold (Ghost Rejection
// section: NN Response < 0.5).  The best candidate of each seed is the one with
// the lowest network output before the sigmoid (same order as the response,
// no saturation) among those under the threshold; chi2 then breaks ties, then
// the hit ids in layer order (absent last).  In chi2 mode the lowest chi2/ndof wins and the cut
// is applied to the winner (Algorithm Design section: score from the distance
// between expected and real hit positions).
//
// k_mlp_fp32: one candidate per thread over the whole candidate buffer (every
// lane busy); weights in the kernel's parameter bank with compile-time indices
// (the paper's static network structure, GPU Implementation section).
// k_pick: one warp per 32 consecutive seeds, its lanes over their (contiguous)
// candidates, a segmented minimum per seed.
#include "ds_args.cuh"

namespace ds {

template <int NIN, int NH1, int NH2>
__global__ void __launch_bounds__(256) k_mlp_fp32(const __grid_constant__ MlpArgs a)
{
    const int n = a.n_host >= 0 ? a.n_host : min(*(volatile const int *)&a.cnt->cand_used, a.cand_cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const float4 *fp = a.feat + 4 * (size_t)c;
        float phi[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(fp + q);
            phi[4 * q] = v.x; phi[4 * q + 1] = v.y; phi[4 * q + 2] = v.z; phi[4 * q + 3] = v.w;
        }
        a.logit[c] = mlp_logit_fp32<NIN, NH1, NH2>(a.nn, phi);
    }
}

// Last part of the pick key: hit ids in layer order, absent (-1) last.
__device__ __forceinline__ bool hits_less(const CandMeta *x, const CandMeta *y)
{
    const int4 hx = __ldg(reinterpret_cast<const int4 *>(x) + 2), hy = __ldg(reinterpret_cast<const int4 *>(y) + 2);
    const unsigned ax[4] = {(unsigned)hx.x, (unsigned)hx.y, (unsigned)hx.z, (unsigned)hx.w};
    const unsigned ay[4] = {(unsigned)hy.x, (unsigned)hy.y, (unsigned)hy.z, (unsigned)hy.w};
#pragma unroll
    for (int l = 0; l < 4; ++l)
        if (ax[l] != ay[l]) return ax[l] < ay[l];
    return false;
}

// hits_less kept out of line: only exact key ties call it, and its loads
// stay out of the common path.
__device__ __noinline__ bool hits_less_ool(const CandMeta *x, const CandMeta *y) { return hits_less(x, y); }

// One warp per 32 consecutive seeds (one per lane).  The warp's candidates
// (each seed's are contiguous) are read 32 at a time, one per lane, with the
// warp's prefix of the seeds' counts mapping a lane to its candidate; a
// segmented minimum over the lanes of one seed (contiguous lanes) leaves each
// run's best key in its first lane, which the seed's lane merges into its
// running best.  Equal keys are ordered by the hit ids.  Every lane reads one
// candidate per round, whatever the candidates per seed.
__global__ void __launch_bounds__(256) k_pick(const __grid_constant__ PickArgs a)
{
    // each warp stages its 32 winner records in shared memory and writes them
    // as contiguous 16-byte chunks (a 64-byte record per lane would scatter)
    __shared__ __align__(16) int4 s_rec[256 / 32][32 * 4];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warp_s0 = s - lane;
    const bool valid = s < a.n_seeds && s >= __ldg(a.seed_off) && s < __ldg(a.seed_off + a.n_events);
    const DevParams &P = a.p;
    const float thr = P.thr_logit;
    const int4 sc = valid ? a.seed_cand[s] : make_int4(0, 0, 0, 0);   // first candidate, count, event
    int incl = sc.y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int off = incl - sc.y;                 // this seed's first position in the warp's list
    const int n = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long best = kNoKey;
    int bi = -1;
    for (int r0 = 0; r0 < n; r0 += 32) {
        const int k = r0 + lane;
        // the seed (lane) owning list position k: the last lane starting at or before k
        int L = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1) {
            const int o = __shfl_sync(0xffffffffu, off, L + st);
            if (o <= k) L += st;
        }
        const int offL = __shfl_sync(0xffffffffu, off, L), firstL = __shfl_sync(0xffffffffu, sc.x, L);
        const bool live = k < n;
        const int c = firstL + k - offL;
        unsigned long long key = kNoKey;
        if (live) {
            const float lg = __ldg(a.logit + c);
            const float2 q = __ldg(reinterpret_cast<const float2 *>(a.meta + c) + 2);   // chi2, ndof
            if (P.pick_chi2) key = pack_key(q.x / (float)__float_as_int(q.y), lg);
            else if (lg < thr) key = pack_key(lg, q.x);
        }
        const int own = live ? L : -1 - lane;        // lanes past the end stay apart
        unsigned long long bk = key;
        int bc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long ok = __shfl_down_sync(0xffffffffu, bk, o);
            const int oc = __shfl_down_sync(0xffffffffu, bc, o);
            const int oo = __shfl_down_sync(0xffffffffu, own, o);
            const bool same = lane + o < 32 && oo == own;
            bool take = same && ok < bk;
            const bool tie = same && ok == bk && ok != kNoKey;
            if (__any_sync(0xffffffffu, tie) && tie) take = hits_less_ool(a.meta + oc, a.meta + bc);
            if (take) {
                bk = ok;
                bc = oc;
            }
        }
        // this seed's run inside the round starts at lane h
        const bool in_round = sc.y > 0 && off < r0 + 32 && off + sc.y > r0;
        const int h = max(off - r0, 0) & 31;
        const unsigned long long vk = __shfl_sync(0xffffffffu, bk, h);
        const int vc = __shfl_sync(0xffffffffu, bc, h);
        if (in_round && (vk < best || (vk == best && vk != kNoKey && hits_less_ool(a.meta + vc, a.meta + bi)))) {
            best = vk;
            bi = vc;
        }
    }
    int4 hits = make_int4(-1, -1, -1, -1);
    int4 r0 = make_int4(0, 0, -1, -1), r1 = make_int4(-1, -1, 0, 0), r2 = make_int4(0, 0, 0, 0),
         r3 = make_int4(0, 0, 0, 0);
    if (valid) {
        bool have = best != kNoKey;
        float lg_best = 0.f;
        if (have) lg_best = P.pick_chi2 ? unord_f32((unsigned)best) : unord_f32((unsigned)(best >> 32));
        if (have && P.pick_chi2 && !(lg_best < thr)) have = false;
        r0 = make_int4(sc.z, s, -1, -1);
        r3 = make_int4(0, 0, 0, sc.y);
        if (have) {
            const float4 *mp = reinterpret_cast<const float4 *>(a.meta + bi);
            const float4 m0 = __ldg(mp), m1 = __ldg(mp + 1);
            const int4 mh = __ldg(reinterpret_cast<const int4 *>(mp + 2));
            hits = mh;
            // ds_track: event, seed, hit[4], x, y, tx, ty, qop, chi2, ndof, nn, flags, n_candidates
            r0 = make_int4(sc.z, s, mh.x, mh.y);
            r1 = make_int4(mh.z, mh.w, __float_as_int(m0.x), __float_as_int(m0.y));
            r2 = make_int4(__float_as_int(m0.z), __float_as_int(m1.w), __float_as_int(m0.w), __float_as_int(m1.x));
            r3 = make_int4(__float_as_int(m1.y), __float_as_int(sigmoid_fast(lg_best)), 0, sc.y);
        } else {
            best = kNoKey;
        }
        a.key_ws[s] = best;
        a.hit_ws[s] = hits;
    } else {
        best = kNoKey;
    }
    // only winners' records are read later (the clone kernel ranks winners
    // alone, the scatter copies ranked seeds): the others are not written
    const unsigned win = __ballot_sync(0xffffffffu, best != kNoKey);
    if (win == 0) return;
    int4 *sr = s_rec[warp];
    sr[lane * 4 + 0] = r0;
    sr[lane * 4 + 1] = r1;
    sr[lane * 4 + 2] = r2;
    sr[lane * 4 + 3] = r3;
    __syncwarp();
    int4 *dst = reinterpret_cast<int4 *>(a.trk_ws + warp_s0);
    for (int k = lane; k < 128; k += 32) {
        const int rec = k >> 2;
        const int sg = warp_s0 + rec;
        if (((win >> rec) & 1u) && sg < a.n_seeds && sg >= 0) dst[k] = sr[k];
    }
}

// The candidate buffer as training examples: features, seed, hits, logit.
__global__ void __launch_bounds__(256) k_export_candidates(const float4 *__restrict__ feat,
                                                           const CandMeta *__restrict__ meta,
                                                           const float *__restrict__ logit, int cand_cap,
                                                           const DevCounters *cnt, float4 *o_feat, int32_t *o_seed,
                                                           int4 *o_hits, float *o_logit, int capacity,
                                                           int32_t *o_count)
{
    const int used = min(*(volatile const int *)&cnt->cand_used, cand_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *o_count = used;
    const int n = min(used, capacity);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < 4; ++q) o_feat[4 * (size_t)c + q] = feat[4 * (size_t)c + q];
        const CandMeta m = meta[c];
        o_seed[c] = m.seed;
        o_hits[c] = make_int4(m.hit[0], m.hit[1], m.hit[2], m.hit[3]);
        if (o_logit) o_logit[c] = logit[c];
    }
}

cudaError_t launch_export_candidates(const float4 *feat, const CandMeta *meta, const float *logit, int cand_cap,
                                     const DevCounters *cnt, float *o_feat, int32_t *o_seed, int32_t *o_hits,
                                     float *o_logit, int capacity, int32_t *o_count, int sm_count, cudaStream_t st)
{
    k_export_candidates<<<4 * sm_count, 256, 0, st>>>(feat, meta, logit, cand_cap, cnt,
                                                      reinterpret_cast<float4 *>(o_feat), o_seed,
                                                      reinterpret_cast<int4 *>(o_hits), o_logit, capacity, o_count);
    return cudaGetLastError();
}

cudaError_t launch_mlp(const MlpArgs &m, int sm_count, int n_bound, cudaStream_t st)
{
    if (m.precision != DS_MLP_FP32) return launch_mlp_tc(m, sm_count, n_bound, st);
    int grid = (n_bound + 255) / 256;
    if (grid > 8 * sm_count) grid = 8 * sm_count;
    if (grid < 1) grid = 1;
    if (m.n_in <= 8 && m.n_h2 == 0)
        k_mlp_fp32<8, 16, 0><<<grid, 256, 0, st>>>(m);
    else
        k_mlp_fp32<16, 32, 32><<<grid, 256, 0, st>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pick(const MlpArgs &m, const PickArgs &p, int sm_count, cudaStream_t st, Prof *prof)
{
    if (p.n_seeds <= 0) return cudaSuccess;
    prof->begin("k_mlp", st);
    cudaError_t e = launch_mlp(m, sm_count, m.cand_cap, st);
    prof->end(st);
    if (e != cudaSuccess) return e;
    prof->begin("k_pick", st);
    k_pick<<<(p.n_seeds + 255) / 256, 256, 0, st>>>(p);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
