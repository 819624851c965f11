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
// k_pick: one thread per seed over its contiguous candidates.
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

constexpr int kPickBatch = 8;

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
    unsigned long long best = kNoKey;
    int4 hits = make_int4(-1, -1, -1, -1);
    int4 r0 = make_int4(0, 0, -1, -1), r1 = make_int4(-1, -1, 0, 0), r2 = make_int4(0, 0, 0, 0),
         r3 = make_int4(0, 0, 0, 0);
    if (valid) {
        const int4 sc = a.seed_cand[s];        // first candidate, count, event
        const float thr = P.thr_logit;
        int bi = -1;
        // candidates in rounds of kPickBatch whose loads are all in flight
        // together: a seed with many candidates waits for a few round trips,
        // not one per candidate
        for (int k0 = 0; k0 < sc.y; k0 += kPickBatch) {
            float lg[kPickBatch];
            float2 q[kPickBatch];   // chi2, ndof
#pragma unroll
            for (int k = 0; k < kPickBatch; ++k)
                if (k0 + k < sc.y) {
                    const int c = sc.x + k0 + k;
                    lg[k] = __ldg(a.logit + c);
                    q[k] = __ldg(reinterpret_cast<const float2 *>(a.meta + c) + 2);
                }
#pragma unroll
            for (int k = 0; k < kPickBatch; ++k)
                if (k0 + k < sc.y) {
                    const int c = sc.x + k0 + k;
                    const float chi2 = q[k].x;
                    const int ndof = __float_as_int(q[k].y);
                    unsigned long long key = kNoKey;
                    if (P.pick_chi2) key = pack_key(chi2 / (float)ndof, lg[k]);
                    else if (lg[k] < thr) key = pack_key(lg[k], chi2);
                    if (key < best || (key == best && key != kNoKey && hits_less(a.meta + c, a.meta + bi))) {
                        best = key;
                        bi = c;
                    }
                }
        }
        bool have = bi >= 0;
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
