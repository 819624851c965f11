// a6: ghost-killer network over all candidates of the batch (the best pick,
// a7, is in pick.cuh, run per event with clone killing in k_clone.cu).
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

cudaError_t launch_network(const MlpArgs &m, int sm_count, cudaStream_t st, Prof *prof)
{
    prof->begin("k_mlp", st);
    const cudaError_t e = launch_mlp(m, sm_count, m.cand_cap, st);
    prof->end(st);
    return e;
}

}  // namespace ds
