// a6 on the tensor cores: the ghost-killer network over all candidates in
// BF16 or FP8 (E4M3) with FP32 accumulation (Ghost-Killer Neural Network
// section: inputs -> ReLU hidden layers -> output node).
//
// One tile = 128 candidates.  Layer 1 (16 -> 32) and layer 2 (32 -> 32) are
// tcgen05.mma instructions (M = 128, N = 32; K = 16 per BF16 instruction, 32
// per FP8 instruction) issued by one thread, operands in shared memory in the
// K-major no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix),
// accumulators in tensor memory (TMEM columns 0-31 and 32-63).  Each warp
// reads its 32 accumulator rows back with tcgen05.ld; bias, ReLU and the
// down-conversion for the next layer run there, and the 32 -> 1 output layer
// is 32 FMAs per row on the CUDA cores.  FP8 scales each output neuron's
// weights by a power of two bringing its largest weight into (224, 448] (each
// row uses the upper E4M3 range), undone exactly per accumulator column in the
// epilogue; inputs and hidden activations are converted with saturation at
// +-448.
//
// Persistent CTAs of 4 warps (one per TMEM sub-partition), 8 per SM so that
// one SM has 8 tiles in flight (all 512 TMEM columns); every mbarrier wait
// is bounded: on time-out the kernel raises DS_FLAG_TIMEOUT, releases its TMEM
// and returns.

#include <cmath>
#include <cstring>

#include "ds_args.cuh"
#include "tc_ptx.cuh"

namespace ds {

namespace {

using namespace tc;
constexpr uint32_t kIdescBF16 = idesc_f32acc(1u, 1u, 32u);   // kind::f16, BF16 x BF16, N = 32
constexpr uint32_t kIdescE4M3 = idesc_f32acc(0u, 0u, 32u);   // kind::f8f6f4, E4M3 x E4M3, N = 32

constexpr int kTcCols = 64;          // TMEM columns: layer-1 and layer-2 accumulators

}  // namespace

template <bool FP8>
__global__ void __launch_bounds__(128, kMlpTcCtasPerSm) k_mlp_tc(const __grid_constant__ MlpArgs a)
{
    // K-major no-swizzle layouts: byte(r, k) = (r/8)*SBO + (k/epr)*LBO + (r%8)*16 + (k%epr)*esize,
    // epr = 16 / esize, LBO = 128 (core matrices adjacent along K)
    constexpr int kSboA1 = 256;                 // A1: 128 x 16 BF16 or 128 x 32 E4M3 (2 K-cores)
    constexpr int kSboA2 = FP8 ? 256 : 512;     // A2: 128 x 32 (4 BF16 K-cores, 2 E4M3 K-cores)
    __shared__ __align__(1024) uint8_t sA1[4096];
    __shared__ __align__(1024) uint8_t sA2[FP8 ? 4096 : 8192];
    __shared__ __align__(128) uint8_t sB1[1024];
    __shared__ __align__(128) uint8_t sB2[FP8 ? 1024 : 2048];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_is1[32], s_is2[32];     // FP8: per-neuron inverse weight scales

    const int tid = threadIdx.x, warp = tid >> 5;
    const MlpTcWeights &W = *a.tc;
    {
        const uint4 *s1 = reinterpret_cast<const uint4 *>(FP8 ? W.b1_fp8 : W.b1_bf16);
        const uint4 *s2 = reinterpret_cast<const uint4 *>(FP8 ? W.b2_fp8 : W.b2_bf16);
        for (int i = tid; i < (int)sizeof(sB1) / 16; i += 128) reinterpret_cast<uint4 *>(sB1)[i] = __ldg(s1 + i);
        for (int i = tid; i < (int)sizeof(sB2) / 16; i += 128) reinterpret_cast<uint4 *>(sB2)[i] = __ldg(s2 + i);
        if (tid < 32) {
            s_is1[tid] = FP8 ? __ldg(W.inv_s1 + tid) : 1.f;
            s_is2[tid] = FP8 ? __ldg(W.inv_s2 + tid) : 1.f;
        }
    }
    if (tid == 0) mbar_init(&s_bar, 1);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint64_t dA1 = smem_desc(sA1, 128, kSboA1), dB1 = smem_desc(sB1, 128, 256);
    const uint64_t dA2 = smem_desc(sA2, 128, kSboA2), dB2 = smem_desc(sB2, 128, FP8 ? 256 : 512);
    const int n = a.n_host >= 0 ? a.n_host : min(*(volatile const int *)&a.cnt->cand_used, a.cand_cap);
    const int ntiles = (n + 127) >> 7;
    const int limit = kWaitLimit;
    uint32_t phase = 0;
    const int r = tid;                       // this thread's row of the tile
    uint8_t *a1row = sA1 + (r >> 3) * kSboA1 + (r & 7) * 16;
    uint8_t *a2row = sA2 + (r >> 3) * kSboA2 + (r & 7) * 16;

    bool failed = false;
    float4 nxt[4];                           // features of this thread's row of the next tile
    auto fetch = [&](int t) {
        const int c = t * 128 + r;
        if (t < ntiles && c < n) {
            const float4 *fp = a.feat + 4 * (size_t)c;
#pragma unroll
            for (int q = 0; q < 4; ++q) nxt[q] = __ldg(fp + q);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) nxt[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    fetch(blockIdx.x);

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = t * 128 + r;
        float x[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[4 * q] = nxt[q].x; x[4 * q + 1] = nxt[q].y; x[4 * q + 2] = nxt[q].z; x[4 * q + 3] = nxt[q].w;
        }
        // rows past the end hold zero features; their logits are computed and dropped
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = (x[i] - a.nn.mean[i]) * a.nn.scale[i];
        if (FP8) {   // 16 inputs + 16 zeros: K = 32, one 16-byte row per K-core
            *reinterpret_cast<uint4 *>(a1row) =
                make_uint4(pack_e4m3(x[0], x[1], x[2], x[3]), pack_e4m3(x[4], x[5], x[6], x[7]),
                           pack_e4m3(x[8], x[9], x[10], x[11]), pack_e4m3(x[12], x[13], x[14], x[15]));
            *reinterpret_cast<uint4 *>(a1row + 128) = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
                *reinterpret_cast<uint4 *>(a1row + kc * 128) =
                    make_uint4(pack_bf16(x[8 * kc], x[8 * kc + 1]), pack_bf16(x[8 * kc + 2], x[8 * kc + 3]),
                               pack_bf16(x[8 * kc + 4], x[8 * kc + 5]), pack_bf16(x[8 * kc + 6], x[8 * kc + 7]));
        }
        fetch(t + gridDim.x);                // in flight while this tile is on the tensor cores
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            if (FP8) mma_e4m3(tmem, dA1, dB1, kIdescE4M3, 0u);
            else mma_bf16(tmem, dA1, dB1, kIdescBF16, 0u);
            mma_commit(&s_bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s_bar, phase, limit))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        float v[32];
        tmem_ld32(tmem + lane_base, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(fmaf(v[j], FP8 ? s_is1[j] : 1.f, a.nn.b1[j]), 0.f);
        if (FP8) {
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
                *reinterpret_cast<uint4 *>(a2row + kc * 128) =
                    make_uint4(pack_e4m3(v[16 * kc], v[16 * kc + 1], v[16 * kc + 2], v[16 * kc + 3]),
                               pack_e4m3(v[16 * kc + 4], v[16 * kc + 5], v[16 * kc + 6], v[16 * kc + 7]),
                               pack_e4m3(v[16 * kc + 8], v[16 * kc + 9], v[16 * kc + 10], v[16 * kc + 11]),
                               pack_e4m3(v[16 * kc + 12], v[16 * kc + 13], v[16 * kc + 14], v[16 * kc + 15]));
        } else {
#pragma unroll
            for (int kc = 0; kc < 4; ++kc)
                *reinterpret_cast<uint4 *>(a2row + kc * 128) =
                    make_uint4(pack_bf16(v[8 * kc], v[8 * kc + 1]), pack_bf16(v[8 * kc + 2], v[8 * kc + 3]),
                               pack_bf16(v[8 * kc + 4], v[8 * kc + 5]), pack_bf16(v[8 * kc + 6], v[8 * kc + 7]));
        }
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            if (FP8) {
                mma_e4m3(tmem + 32, dA2, dB2, kIdescE4M3, 0u);
            } else {   // K = 32 as two K = 16 steps: start addresses advance by two K-cores (256 B)
                mma_bf16(tmem + 32, dA2, dB2, kIdescBF16, 0u);
                mma_bf16(tmem + 32, dA2 + (256u >> 4), dB2 + (256u >> 4), kIdescBF16, 1u);
            }
            mma_commit(&s_bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s_bar, phase, limit))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        tmem_ld32(tmem + lane_base + 32, v);
        float out = a.nn.b3;
#pragma unroll
        for (int j = 0; j < 32; ++j) out = fmaf(a.nn.w3[j], fmaxf(fmaf(v[j], FP8 ? s_is2[j] : 1.f, a.nn.b2[j]), 0.f), out);
        if (c < n) a.logit[c] = out;
        tc_fence_before();
        __syncthreads();     // TMEM and the A tiles are rewritten by the next tile
        tc_fence_after();
    }
    if (failed) {   // uniform over the block
        if (tid == 0) raise_flag(a.cnt, DS_FLAG_TIMEOUT);
        mbar_wait_bounded(&s_bar, phase, limit);   // let an outstanding MMA drain before releasing TMEM
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// Host: weight tiles in the K-major core-matrix layout (BF16 and E4M3).
static int kmajor_offset(int r, int k, int esize, int sbo)
{
    const int epr = 16 / esize;
    return (r / 8) * sbo + (k / epr) * 128 + (r % 8) * 16 + (k % epr) * esize;
}

void prepare_tc_weights(const DevNN &nn, int n_h2, MlpTcWeights *out)
{
    std::memset(out, 0, sizeof(*out));
    float w2[32][32];
    for (int o = 0; o < 32; ++o)
        for (int i = 0; i < 32; ++i) w2[o][i] = n_h2 > 0 ? nn.w2[o][i] : (o == i ? 1.f : 0.f);
    // FP8: each neuron's weights scaled by the largest power of two 2^k with
    // 2^k max|W| <= 448 (its largest weight lands in (224, 448]); undoing a
    // power of two is exact
    auto pow2_scale = [](float m) {
        if (!(m > 0.f)) return 1.f;
        float s = std::ldexp(1.f, (int)std::floor(std::log2(448.f / m)));
        while (m * s > 448.f) s *= 0.5f;
        while (m * s * 2.f <= 448.f) s *= 2.f;
        return s;
    };
    for (int o = 0; o < 32; ++o) {
        float m1 = 0.f, m2 = 0.f;
        for (int i = 0; i < 16; ++i) m1 = std::fmax(m1, std::fabs(nn.w1[o][i]));
        for (int i = 0; i < 32; ++i) m2 = std::fmax(m2, std::fabs(w2[o][i]));
        const float s1 = pow2_scale(m1), s2 = pow2_scale(m2);
        out->inv_s1[o] = 1.f / s1;
        out->inv_s2[o] = 1.f / s2;
        for (int i = 0; i < 16; ++i) {
            const __nv_bfloat16 h = __float2bfloat16_rn(nn.w1[o][i]);
            std::memcpy(out->b1_bf16 + kmajor_offset(o, i, 2, 256), &h, 2);
            out->b1_fp8[kmajor_offset(o, i, 1, 256)] =
                (uint8_t)__nv_cvt_float_to_fp8(nn.w1[o][i] * s1, __NV_SATFINITE, __NV_E4M3);
        }
        for (int i = 0; i < 32; ++i) {
            const __nv_bfloat16 h = __float2bfloat16_rn(w2[o][i]);
            std::memcpy(out->b2_bf16 + kmajor_offset(o, i, 2, 512), &h, 2);
            out->b2_fp8[kmajor_offset(o, i, 1, 256)] =
                (uint8_t)__nv_cvt_float_to_fp8(w2[o][i] * s2, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

cudaError_t launch_mlp_tc(const MlpArgs &a, int sm_count, int n_bound, cudaStream_t st)
{
    int grid = (n_bound + 127) / 128;
    if (grid > kMlpTcCtasPerSm * sm_count) grid = kMlpTcCtasPerSm * sm_count;
    if (grid < 1) grid = 1;
    if (a.precision == DS_MLP_FP8) k_mlp_tc<true><<<grid, 128, 0, st>>>(a);
    else k_mlp_tc<false><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ds
