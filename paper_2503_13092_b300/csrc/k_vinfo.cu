// Vertex-level physics and the trigger-line networks (Expected Physics Impact
// section: K0S and Lambda candidates from two opposite-charge downstream
// tracks; Fig. 18: their masses once the vertex is known; trigger lines
// driven by networks of one hidden layer of 32 nodes on track, vertex and
// parent-track inputs).
//
// One thread per vertex record.  Each daughter's momentum at the vertex has
// magnitude 1/|q/p| and the direction of its Eq. 4 trajectory there (slopes
// tx + 2 gamma (z_v - z_ref), ty; gamma from Eq. 3).  In FP32 the masses are
// computed without cancellation:
//   M^2 = ma^2 + mb^2 + 2 (Ea Eb - pa pb + pa pb (1 - cos)),
//   Ea Eb - pa pb = (ma^2 pb^2 + mb^2 pa^2 + ma^2 mb^2) / (Ea Eb + pa pb),
//   1 - cos = |ua - ub|^2 / 2 for unit directions ua, ub,
// algebraically the same as (Ea + Eb)^2 - |pa + pb|^2.  The line networks'
// weights sit in the kernel's parameter bank.
#include <cstring>

#include "ds_args.cuh"
#include "tc_ptx.cuh"

namespace ds {

namespace {

constexpr float kMPi = 139.57039f, kMP = 938.27208f, kMKS = 497.611f, kMLambda = 1115.683f;

__device__ __forceinline__ float pair_mass(float pa, float ma, float pb, float mb, float omc)
{
    const float ea = sqrtf(fmaf(pa, pa, ma * ma)), eb = sqrtf(fmaf(pb, pb, mb * mb));
    const float ma2 = ma * ma, mb2 = mb * mb;
    const float t = fmaf(ma2, pb * pb, fmaf(mb2, pa * pa, ma2 * mb2)) / fmaf(ea, eb, pa * pb);
    const float m2 = ma2 + mb2 + 2.f * fmaf(pa * pb, omc, t);
    return sqrtf(fmaxf(m2, 0.f));
}

struct Daughter {
    float p, ux, uy, uz;
};

__device__ __forceinline__ Daughter daughter(const DevGeom &g, const ds_track &t, float zv)
{
    const float gam = -g.mp * fmaf(g.gamma1, t.qop, g.gamma0);     // Eq. 3
    const float txv = fmaf(2.f * gam, zv - g.z_ref, t.tx), tyv = t.ty;
    const float inv_n = rsqrtf(fmaf(txv, txv, fmaf(tyv, tyv, 1.f)));
    Daughter d;
    d.p = 1.f / fabsf(t.qop);
    d.ux = txv * inv_n;
    d.uy = tyv * inv_n;
    d.uz = inv_n;
    return d;
}

}  // namespace

// The vertex's quantities r[0..10] (record order) and the 16 line inputs f;
// false when a track index is out of range.
__device__ __forceinline__ bool vertex_quantities(const VinfoArgs &a, int nt, const ds_vertex_rec &v, float (&r)[11],
                                                  float (&f)[16])
{
    if (!(v.i >= 0 && v.i < nt && v.j >= 0 && v.j < nt)) return false;
    const DevGeom &g = a.g;
    const ds_track A = a.tracks[v.i], B = a.tracks[v.j];
    const Daughter da = daughter(g, A, v.z), db = daughter(g, B, v.z);
    const bool a_pos = A.qop > 0.f;
    const Daughter &dp = a_pos ? da : db, &dn = a_pos ? db : da;
    const float px = fmaf(da.p, da.ux, db.p * db.ux), py = fmaf(da.p, da.uy, db.p * db.uy);
    const float pz = fmaf(da.p, da.uz, db.p * db.uz);
    const float pt = sqrtf(fmaf(px, px, py * py));
    const float dx = da.ux - db.ux, dy = da.uy - db.uy, dz = da.uz - db.uz;
    const float omc = 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    r[0] = pair_mass(dp.p, kMPi, dn.p, kMPi, omc);
    r[1] = pair_mass(dp.p, kMP, dn.p, kMPi, omc);
    r[2] = pair_mass(dp.p, kMPi, dn.p, kMP, omc);
    r[3] = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
    r[4] = pt;
    r[5] = pt > 0.f ? fabsf(fmaf(v.x, py, -v.y * px)) / pt : sqrtf(fmaf(v.x, v.x, v.y * v.y));
    r[6] = omc;
    r[7] = dp.p;
    r[8] = dn.p;
    r[9] = dp.p * sqrtf(fmaf(dp.ux, dp.ux, dp.uy * dp.uy));
    r[10] = dn.p * sqrtf(fmaf(dn.ux, dn.ux, dn.uy * dn.uy));
    f[0] = v.x / 100.f; f[1] = v.y / 100.f; f[2] = v.z / 1000.f; f[3] = v.doca;
    f[4] = r[3] / 1e4f; f[5] = r[4] / 1e3f; f[6] = r[5] / 10.f;
    f[7] = (r[0] - kMKS) / 100.f; f[8] = (r[1] - kMLambda) / 100.f; f[9] = (r[2] - kMLambda) / 100.f;
    f[10] = r[7] / 1e4f; f[11] = r[8] / 1e4f; f[12] = r[9] / 1e3f; f[13] = r[10] / 1e3f;
    f[14] = 1e3f * omc;
    const float ca = A.ndof > 0 ? A.chi2 / (float)A.ndof : 0.f, cb = B.ndof > 0 ? B.chi2 / (float)B.ndof : 0.f;
    f[15] = 0.5f * (ca + cb);
    return true;
}

__device__ __forceinline__ void store_info(ds_vertex_info *out, const float (&r)[16])
{
    float4 *o = reinterpret_cast<float4 *>(out);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
}

__global__ void __launch_bounds__(256) k_vertex_info(const __grid_constant__ VinfoArgs a)
{
    const int nt = min(*(volatile const int *)a.n_tracks, a.trk_capacity);
    const int nv = min(min(*(volatile const int *)a.n_vertices, a.vtx_capacity), a.capacity);
    const DevLines &L = a.L;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += gridDim.x * blockDim.x) {
        const ds_vertex_rec v = a.vtx[k];
        float r[16], q11[11], f[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = 0.f;
        if (vertex_quantities(a, nt, v, q11, f)) {
#pragma unroll
            for (int q = 0; q < 11; ++q) r[q] = q11[q];
#pragma unroll
            for (int l = 0; l < 4; ++l) {        // compile-time weight indices (parameter bank operands)
                if (l >= L.n_lines) break;
                float x[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) x[q] = (f[q] - L.mean[l][q]) * L.scale[l][q];
                float out = L.b3[l];
#pragma unroll
                for (int o = 0; o < 32; ++o) {
                    float h = L.b1[l][o];
#pragma unroll
                    for (int q = 0; q < 16; ++q) h = fmaf(L.w1[l][o][q], x[q], h);
                    out = fmaf(L.w3[l][o], fmaxf(h, 0.f), out);
                }
                r[11 + l] = 1.f / (1.f + __expf(-out));
            }
        } else {
            r[15] = __uint_as_float(1u);     // flags bit 0: track index out of range
        }
        store_info(a.out + k, r);
    }
}

// The same with the four line networks as one BF16 tensor-core product per
// 128-vertex tile: [128 vertices x 16 inputs] x [16 x (4 lines x 32 hidden)]
// -> 128 x 128 FP32 accumulators in TMEM (tcgen05.mma kind::f16, M = N = 128,
// K = 16, one instruction).  Each network's input normalisation is folded into
// its first-layer weights and biases (in FP64, on the host); the inputs and
// those weights are rounded to BF16, bias, ReLU and the output node in FP32.
// 128 threads, one per TMEM lane (vertex of the tile); persistent CTAs; every
// mbarrier wait bounded (DS_FLAG_TIMEOUT, TMEM released, return).
__global__ void __launch_bounds__(128) k_vertex_info_tc(const __grid_constant__ VinfoArgs a)
{
    using namespace tc;
    constexpr uint32_t kIdesc = idesc_f32acc(1u, 1u, 128u);
    __shared__ __align__(1024) uint8_t sA[4096];      // 128 x 16 BF16, K-major core matrices
    __shared__ __align__(1024) uint8_t sB[4096];      // 128 x 16 BF16
    __shared__ float s_b1[128], s_w3[128];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const LineTcWeights &W = *a.tcw;
    for (int i = tid; i < 4096 / 16; i += 128)
        reinterpret_cast<uint4 *>(sB)[i] = __ldg(reinterpret_cast<const uint4 *>(W.b_bf16) + i);
    s_b1[tid] = W.b1[tid];
    s_w3[tid] = W.w3[tid];
    if (tid == 0) mbar_init(&s_bar, 1);
    if (warp == 0) tmem_alloc(&s_tmem, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem, lane_base = (uint32_t)(warp * 32) << 16;
    const uint64_t dA = smem_desc(sA, 128, 256), dB = smem_desc(sB, 128, 256);
    const int nt = min(*(volatile const int *)a.n_tracks, a.trk_capacity);
    const int nv = min(min(*(volatile const int *)a.n_vertices, a.vtx_capacity), a.capacity);
    const int n_lines = W.n_lines;
    const int ntiles = (nv + 127) >> 7;
    uint32_t phase = 0;
    bool failed = false;
    uint8_t *arow = sA + (tid >> 3) * 256 + (tid & 7) * 16;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int k = t * 128 + tid;
        float r[16], q11[11], f[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) r[q] = f[q] = 0.f;
        bool ok = false;
        if (k < nv) {
            ok = vertex_quantities(a, nt, a.vtx[k], q11, f);
            if (ok) {
#pragma unroll
                for (int q = 0; q < 11; ++q) r[q] = q11[q];
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) f[q] = 0.f;
                r[15] = __uint_as_float(1u);
            }
        }
#pragma unroll
        for (int kc = 0; kc < 2; ++kc)
            *reinterpret_cast<uint4 *>(arow + kc * 128) =
                make_uint4(pack_bf16(f[8 * kc], f[8 * kc + 1]), pack_bf16(f[8 * kc + 2], f[8 * kc + 3]),
                           pack_bf16(f[8 * kc + 4], f[8 * kc + 5]), pack_bf16(f[8 * kc + 6], f[8 * kc + 7]));
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            mma_bf16(tmem, dA, dB, kIdesc, 0u);
            mma_commit(&s_bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s_bar, phase, kWaitLimit))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        for (int l = 0; l < 4; ++l) {          // uniform over the warp (tcgen05.ld is .sync.aligned)
            float acc[32];
            tmem_ld32(tmem + lane_base + 32 * l, acc);
            float out = W.b3[l];
#pragma unroll
            for (int o = 0; o < 32; ++o) out = fmaf(s_w3[32 * l + o], fmaxf(acc[o] + s_b1[32 * l + o], 0.f), out);
            if (ok && l < n_lines) r[11 + l] = 1.f / (1.f + __expf(-out));
        }
        if (k < nv) store_info(a.out + k, r);
        tc_fence_before();
        __syncthreads();       // TMEM and the A tile are rewritten by the next tile
        tc_fence_after();
    }
    if (failed) {   // uniform over the block
        if (tid == 0) raise_flag(a.cnt, DS_FLAG_TIMEOUT);
        mbar_wait_bounded(&s_bar, phase, kWaitLimit);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

const char *fill_dev_lines(const ds_nn_weights *nets, int n_lines, DevLines *out)
{
    if (n_lines < 0 || n_lines > 4) return "n_lines outside 0..4";
    if (n_lines > 0 && !nets) return "null networks";
    DevLines &L = *out;
    std::memset(&L, 0, sizeof(L));
    for (int l = 0; l < n_lines; ++l) {
        const ds_nn_weights &w = nets[l];
        if (w.n_in != 16 || w.n_h1 < 1 || w.n_h1 > 32 || w.n_h2 != 0) return "line networks are 16 -> n_h1 <= 32 -> 1";
        if (!w.w1 || !w.b1 || !w.w3 || !w.mean || !w.scale) return "null pointer";
        for (int o = 0; o < w.n_h1; ++o) {
            L.b1[l][o] = w.b1[o];
            L.w3[l][o] = w.w3[o];
            for (int q = 0; q < 16; ++q) L.w1[l][o][q] = w.w1[o * 16 + q];
        }
        L.b3[l] = w.b3;
        for (int q = 0; q < 16; ++q) {
            L.mean[l][q] = w.mean[q];
            L.scale[l][q] = w.scale[q];
        }
    }
    L.n_lines = n_lines;
    return nullptr;
}

static int kmajor_offset(int r, int k, int esize, int sbo)
{
    const int epr = 16 / esize;
    return (r / 8) * sbo + (k / epr) * 128 + (r % 8) * 16 + (k % epr) * esize;
}

void prepare_line_tc(const DevLines &L, LineTcWeights *out)
{
    std::memset(out, 0, sizeof(*out));
    for (int l = 0; l < L.n_lines; ++l) {
        for (int o = 0; o < 32; ++o) {
            const int n = 32 * l + o;
            double b = L.b1[l][o];
            for (int q = 0; q < 16; ++q) {
                const double wq = (double)L.w1[l][o][q] * (double)L.scale[l][q];
                b -= wq * (double)L.mean[l][q];
                const __nv_bfloat16 h = __float2bfloat16_rn((float)wq);
                std::memcpy(out->b_bf16 + kmajor_offset(n, q, 2, 256), &h, 2);
            }
            out->b1[n] = (float)b;
            out->w3[n] = L.w3[l][o];
        }
        out->b3[l] = L.b3[l];
    }
    out->n_lines = L.n_lines;
}

cudaError_t launch_vertex_info(const VinfoArgs &a, bool tensor_cores, int sm_count, cudaStream_t st, Prof *prof)
{
    if (tensor_cores) {
        int grid = (a.capacity + 127) / 128;
        if (grid > 4 * sm_count) grid = 4 * sm_count;
        if (grid < 1) grid = 1;
        prof->begin("k_vertex_info", st);
        k_vertex_info_tc<<<grid, 128, 0, st>>>(a);
        prof->end(st);
        return cudaGetLastError();
    }
    int grid = (a.capacity + 255) / 256;
    if (grid > 4 * sm_count) grid = 4 * sm_count;
    if (grid < 1) grid = 1;
    prof->begin("k_vertex_info", st);
    k_vertex_info<<<grid, 256, 0, st>>>(a);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
