// a9 + a10 (vertices): two-track vertexing and deterministic compaction.
//
// Vertexing Two Downstream Tracks section: each track is extrapolated with
// Eq. 4, x(z) = x + tx (z - z_ref) + gamma (z - z_ref)^2, y(z) = y + ty (z - z_ref),
// gamma from Eq. 3; the vertex is the point of closest approach found by
// Newton-Raphson; secondary tracks must have opposite charges (Expected
// Physics Impact section).  Start: the closed-form closest approach of the
// two straight lines; stop when both steps are below the tolerance; vertex =
// midpoint of the two closest points; kept if DOCA < doca_max.
//
// FP32 solve with error-free residuals and a two-float Newton iterate (below),
// so its error stays at the float32 resolution of the output coordinates;
// pairs whose opening satisfies sin^2 < eps_par and whose FP32 DOCA is near
// or below the cut are re-solved in FP64 (flag bit 0).
//
// Small-capacity launch: one CTA per event (up to 512 tracks), pulled from a
// queue in the order given (largest first when the bucketing kernel's order
// is passed).  Tracks are
// staged in shared memory; opposite-charge partner lists make every thread's
// pair valid, enumerated in (i, j) order.  Kept vertices of each segment are
// ranked by a block scan and written to a pool slice reserved with one
// atomicAdd; their position inside the event is recorded, so the scatter
// kernel places them in (event, i, j) order whatever order the pool was
// filled in.  Larger events are listed with their pair count (npos x nneg).
// Large-capacity launch: its work items are (listed event, segment of 65536
// pairs of its (i, j) enumeration), so that the pairs of one large event are
// spread over many SMs; an item ranks its kept vertices inside the item, and
// the launch's last CTA turns per-item counts into each item's offset inside
// its event.
#include "ds_args.cuh"

namespace ds {

constexpr int kVtxThreads = 256;
constexpr int kVtxLargeThreads = 1024;  // the large-capacity launch: one CTA per SM, all of its warps
constexpr int kVtxSmallCap = kVtxSmallCapMax;   // tracks staged per CTA by the small-capacity launch
constexpr int kVtxCtasPerSm = kVtxCtasPerSmMax;   // resident CTAs of the small-capacity launch per SM (at most)
// pairs per two-phase segment and candidate results kept in shared memory per
// segment: larger for the large-capacity launch (one CTA per SM), whose
// events have up to millions of pairs
template <bool LARGE> struct VtxSeg {
    static constexpr int seg = LARGE ? kVtxLargeSeg : 12288;
    static constexpr int store = LARGE ? 2048 : 1024;
};


struct Trk {
    float x, y, tx, ty, q;
};

struct PairOut {
    float x, y, z, doca;
    unsigned int flags;
};

// 1/x in FP64 from a FP32 reciprocal refined by two Newton steps r <- r (2 - x r)
// (each doubles the correct bits: 23 -> 46 -> beyond 53), a few FP64 FMAs
// instead of a full FP64 division; x outside the FP32 range takes the division.
__device__ __forceinline__ double recip_fp64(double x)
{
    const float xf = (float)x;
    double r = (double)(1.0f / xf);
    if (!(fabs(r) > 0.0 && fabs(r) < 1e38)) return 1.0 / x;
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

__device__ __noinline__ PairOut solve_fp64(const DevGeom &g, const DevParams &P, const Trk &A, const Trk &B)
{
    // two straight lines when gamma = 0 (field mode A)
    const bool line = g.gamma0 == 0.f && g.gamma1 == 0.f;
    const double gi = line ? 0.0 : -(double)g.mp * ((double)g.gamma0 + (double)g.gamma1 * (double)A.q);
    const double gj = line ? 0.0 : -(double)g.mp * ((double)g.gamma0 + (double)g.gamma1 * (double)B.q);
    const double txi = A.tx, tyi = A.ty, txj = B.tx, tyj = B.ty;
    const double wx = (double)A.x - (double)B.x, wy = (double)A.y - (double)B.y;
    const double dtx = txi - txj, dty = tyi - tyj;
    const double a = 1.0 + txi * txi + tyi * tyi, c = 1.0 + txj * txj + tyj * tyj;
    const double b = 1.0 + txi * txj + tyi * tyj;
    const double cz = txi * tyj - tyi * txj;
    const double den = dtx * dtx + dty * dty + cz * cz;
    const double d = txi * wx + tyi * wy, m = dtx * wx + dty * wy;
    // Two straight lines: F is quadratic in (u1, u2), so the first Newton step
    // lands on the closed-form closest approach from any start and later
    // steps only repeat it to within rounding.  The closed form is then the
    // converged solution whenever the lines are not parallel and at least one
    // step is allowed (every FP64 operation counts here: this part issues
    // FP64 at a small fraction of its FP32 rate).
    const bool line_conv = line && den > 0.0 && P.nr_max_iter > 0;
    double u1 = 0.0, u2 = 0.0;
    if (den > 1e-12 * a * c || line_conv) {
        const double rden = recip_fp64(den);
        u1 = ((txj * dtx + tyj * dty) * d - b * m) * rden;
        u2 = ((txi * dtx + tyi * dty) * d - a * m) * rden;
    }
    bool conv = line_conv;
    for (int it = 0; it < (line ? 0 : P.nr_max_iter); ++it) {
        const double du = u1 - u2;
        const double pi = txi + 2.0 * gi * u1, pj = txj + 2.0 * gj * u2;
        const double dx = (wx + dtx * u2) + txi * du + gi * u1 * u1 - gj * u2 * u2;
        const double dy = (wy + dty * u2) + tyi * du;
        const double dz = du;
        const double dPi = dx * pi + dy * tyi + dz, dPj = dx * pj + dy * tyj + dz;
        const double ni = pi * pi + tyi * tyi + 1.0, nj = pj * pj + tyj * tyj + 1.0;
        const double cx = tyi - tyj, cy = pj - pi, cc = pi * tyj - tyi * pj;   // Pi x Pj
        const double det = cx * cx + cy * cy + cc * cc + 2.0 * gi * dx * nj - 2.0 * gj * dx * ni -
                           4.0 * gi * gj * dx * dx;
        if (!(det > 0.0)) break;
        // (Pj x Pi).(Pj x d) and (Pi x Pj).(Pi x d)
        const double jd_x = tyj * dz - dy, jd_y = dx - pj * dz, jd_z = pj * dy - tyj * dx;
        const double id_x = tyi * dz - dy, id_y = dx - pi * dz, id_z = pi * dy - tyi * dx;
        const double n1 = -(cx * jd_x + cy * jd_y + cc * jd_z) - 2.0 * gj * dx * dPi;
        const double n2 = -(cx * id_x + cy * id_y + cc * id_z) - 2.0 * gi * dx * dPj;
        const double rdet = recip_fp64(det);
        const double s1 = -n1 * rdet, s2 = -n2 * rdet;
        u1 += s1;
        u2 += s2;
        if (fabs(s1) < (double)P.nr_tol && fabs(s2) < (double)P.nr_tol) {
            conv = true;
            break;
        }
    }
    const double du = u1 - u2;
    double dx = (wx + dtx * u2) + txi * du, x1 = (double)A.x + txi * u1;
    if (!line) {
        dx = dx + gi * u1 * u1 - gj * u2 * u2;
        x1 = x1 + gi * u1 * u1;
    }
    const double dy = (wy + dty * u2) + tyi * du;
    PairOut o;
    const double y1 = (double)A.y + tyi * u1;
    o.x = (float)(x1 - 0.5 * dx);
    o.y = (float)(y1 - 0.5 * dy);
    o.z = (float)(0.5 * (u1 + u2) + (double)g.z_ref);
    o.doca = sqrtf((float)(dx * dx + dy * dy + du * du));   // stored as FP32: a FP32 root suffices
    o.flags = 1u | (conv ? 0u : 2u);
    return o;
}

// Error-free transformations (Knuth TwoSum, FMA TwoProduct).  The _rn
// intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float t = __fadd_rn(a, b);
    const float bb = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
    return t;
}

__device__ __forceinline__ float two_prod(float a, float b, float &e)
{
    const float p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
    return p;
}

// Transverse residual T_i(u1) - T_j(u2) along one axis:
//   w + dt*u2 + t_i*du + g_i*u1^2 - g_j*u2^2,
// with w = a_i - a_j and dt = t_i - t_j carried as (value, rounding error) and
// u = uh + ul.  The large terms cancel near the solution; they are summed
// error-free so that only the small remainder is rounded.
__device__ __forceinline__ float residual(float w, float we, float dt, float dte, float ti, float gi, float gj,
                                          float u1h, float u1l, float u2h, float u2l, float du, bool curved)
{
    float pe, se;
    const float p = two_prod(dt, u2h, pe);
    float s = two_sum(w, p, se);
    float lo = we + pe + se + dte * u2h + dt * u2l + ti * du;
    if (curved) {
        float a1e, g1e, a2e, g2e, te, t2e;
        const float a1 = two_prod(gi, u1h, a1e), g1 = two_prod(a1, u1h, g1e);
        const float a2 = two_prod(gj, u2h, a2e), g2 = two_prod(a2, u2h, g2e);
        const float t = two_sum(s, g1, te);
        s = two_sum(t, -g2, t2e);
        lo += te + t2e + g1e - g2e + a1e * u1h - a2e * u2h + 2.f * a1 * u1l - 2.f * a2 * u2l;
    }
    return s + lo;
}

// FP32 solve.  The closest-approach parameters are carried as unevaluated
// sums u = uh + ul (the Newton steps accumulate in ul), so they are not
// limited to one float32 ulp of |z - z_ref|; residuals are error-free as
// above; the Hessian uses cross products of slope differences.
__device__ __forceinline__ PairOut solve_fp32(const DevGeom &g, const DevParams &P, const Trk &A,
                                              const Trk &B, float &sin2)
{
    const float gi = -g.mp * fmaf(g.gamma1, A.q, g.gamma0);
    const float gj = -g.mp * fmaf(g.gamma1, B.q, g.gamma0);
    const bool curved = gi != 0.f || gj != 0.f;
    const float txi = A.tx, tyi = A.ty, txj = B.tx, tyj = B.ty;
    float wxe, wye, dtxe, dtye;
    const float wx = two_sum(A.x, -B.x, wxe), wy = two_sum(A.y, -B.y, wye);
    const float dtx = two_sum(txi, -txj, dtxe), dty = two_sum(tyi, -tyj, dtye);
    const float a = fmaf(txi, txi, fmaf(tyi, tyi, 1.f)), c = fmaf(txj, txj, fmaf(tyj, tyj, 1.f));
    const float b = fmaf(txi, txj, fmaf(tyi, tyj, 1.f));
    const float cz = fmaf(txi, tyj, -tyi * txj);
    const float den = fmaf(dtx, dtx, fmaf(dty, dty, cz * cz));
    sin2 = den / (a * c);
    const float d = fmaf(txi, wx, tyi * wy), m = fmaf(dtx, wx, dty * wy);
    float u1h = 0.f, u2h = 0.f, u1l = 0.f, u2l = 0.f;
    if (sin2 > 1e-12f) {
        u1h = fmaf(fmaf(txj, dtx, tyj * dty), d, -b * m) / den;
        u2h = fmaf(fmaf(txi, dtx, tyi * dty), d, -a * m) / den;
    }
    const float tol = fmaxf(P.nr_tol, 1e-3f);
    bool conv = false;
    for (int it = 0; it < P.nr_max_iter; ++it) {
        const float du = (u1h - u2h) + (u1l - u2l);
        const float pi = fmaf(2.f * gi, u1h, txi), pj = fmaf(2.f * gj, u2h, txj);
        const float dx = residual(wx, wxe, dtx, dtxe, txi, gi, gj, u1h, u1l, u2h, u2l, du, curved);
        const float dy = residual(wy, wye, dty, dtye, tyi, 0.f, 0.f, u1h, u1l, u2h, u2l, du, false);
        const float dz = du;
        const float dPi = fmaf(dx, pi, fmaf(dy, tyi, dz)), dPj = fmaf(dx, pj, fmaf(dy, tyj, dz));
        const float ni = fmaf(pi, pi, fmaf(tyi, tyi, 1.f)), nj = fmaf(pj, pj, fmaf(tyj, tyj, 1.f));
        const float cx = tyi - tyj, cy = pj - pi, cc = fmaf(pi, tyj, -tyi * pj);
        const float det = fmaf(cx, cx, fmaf(cy, cy, cc * cc)) +
                          2.f * dx * (fmaf(gi, nj, -gj * ni) - 2.f * gi * gj * dx);
        if (!(det > 0.f)) break;
        const float jd_x = fmaf(tyj, dz, -dy), jd_y = fmaf(-pj, dz, dx), jd_z = fmaf(pj, dy, -tyj * dx);
        const float id_x = fmaf(tyi, dz, -dy), id_y = fmaf(-pi, dz, dx), id_z = fmaf(pi, dy, -tyi * dx);
        const float n1 = -fmaf(cx, jd_x, fmaf(cy, jd_y, cc * jd_z)) - 2.f * gj * dx * dPi;
        const float n2 = -fmaf(cx, id_x, fmaf(cy, id_y, cc * id_z)) - 2.f * gi * dx * dPj;
        const float s1 = -n1 / det, s2 = -n2 / det;
        u1h = two_sum(u1h, u1l + s1, u1l);
        u2h = two_sum(u2h, u2l + s2, u2l);
        if (fabsf(s1) < tol && fabsf(s2) < tol) {
            conv = true;
            break;
        }
    }
    const float du = (u1h - u2h) + (u1l - u2l);
    const float dx = residual(wx, wxe, dtx, dtxe, txi, gi, gj, u1h, u1l, u2h, u2l, du, curved);
    const float dy = residual(wy, wye, dty, dtye, tyi, 0.f, 0.f, u1h, u1l, u2h, u2l, du, false);
    PairOut o;
    const float x1 = fmaf(txi, u1h, A.x) + fmaf(txi, u1l, gi * u1h * u1h);
    const float y1 = fmaf(tyi, u1h, A.y) + tyi * u1l;
    o.x = fmaf(-0.5f, dx, x1);
    o.y = fmaf(-0.5f, dy, y1);
    float se;
    const float S = two_sum(u1h, u2h, se);
    o.z = fmaf(0.5f, S, g.z_ref) + 0.5f * (se + (u1l + u2l));
    o.doca = sqrtf(fmaf(dx, dx, fmaf(dy, dy, du * du)));
    o.flags = conv ? 0u : 2u;
    return o;
}

// One pair, FP32 with the FP64 re-solve for near-parallel pairs near or below
// the cut.  Not inlined: both phases must run the very same code.
__device__ __noinline__ PairOut solve_pair(const DevGeom &g, const DevParams &P, const Trk &A, const Trk &B,
                                           int &used_fp64)
{
    float sin2;
    PairOut o = solve_fp32(g, P, A, B, sin2);
    used_fp64 = 0;
    if (sin2 < P.eps_par && o.doca < P.doca_max + 0.05f) {
        o = solve_fp64(g, P, A, B);
        used_fp64 = 1;
    }
    return o;
}

template <int CAP, bool LARGE>
__global__ void __launch_bounds__(LARGE ? kVtxLargeThreads : kVtxThreads, LARGE ? 1 : kVtxCtasPerSm)
    k_vertex(const __grid_constant__ VertexArgs a)
{
    constexpr int kVtxSeg = VtxSeg<LARGE>::seg, kVtxStore = VtxSeg<LARGE>::store, kWords = kVtxSeg / 32;
    constexpr int kThreads = LARGE ? kVtxLargeThreads : kVtxThreads;
    constexpr int kTpt = CAP / kThreads;   // tracks staged per thread
    constexpr int kWarpCap = kVtxStore / (kThreads / 32);   // listed candidates per warp
    static_assert(CAP % kThreads == 0 && CAP % 2 == 0 && CAP <= 65535, "track staging layout");
    static_assert((sizeof(float4) + sizeof(unsigned)) * kVtxStore + 5 * sizeof(unsigned) * kWords >=
                      sizeof(float4) * CAP, "tracks parked below the charge-ordered copy");
    static_assert(LARGE || sizeof(float4) * kVtxStore >= sizeof(float4) * CAP + 2 * sizeof(float4) * (CAP / 4),
                  "packed shorter list inside the candidate results");
    // dynamic: candidate results, segment masks, then the event's tracks
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ int s_scan[32];
    __shared__ int s_pool_base, s_wcnt[32];
    __shared__ bool s_last;
    float4 *s_res = reinterpret_cast<float4 *>(s_dyn);          // candidate results: x, y, z, doca
    unsigned *s_resf = reinterpret_cast<unsigned *>(s_res + kVtxStore);   // and flags
    unsigned *s_cmask = s_resf + kVtxStore;                      // candidates of the segment, a bit per pair
    int *s_cbase = reinterpret_cast<int *>(s_cmask + kWords);   // their word prefix
    unsigned *s_keep = reinterpret_cast<unsigned *>(s_cbase + kWords);   // kept pairs
    int *s_wbase = reinterpret_cast<int *>(s_keep + kWords);    // their word prefix
    int *s_wrow = s_wbase + kWords;                              // row holding each mask word's first pair
    // the event's tracks in charge order (positives, then negatives): x, y, tx, ty
    float4 *s_ctr = reinterpret_cast<float4 *>(s_wrow + kWords);
    float *s_cq = reinterpret_cast<float *>(s_ctr + CAP);       // and q/p
    uint16_t *s_cidx = reinterpret_cast<uint16_t *>(s_cq + CAP);   // and the index in the event
    uint16_t *s_self = s_cidx + CAP;       // slot of track i in that order
    uint16_t *s_start = s_self + CAP;      // first partner of track i (after it) in the opposite list
    int *s_row = reinterpret_cast<int *>(s_start + CAP);   // CAP + 1 entries: first pair of row i
    // candidate list, a part of kWarpCap entries per warp: the two slots
    // (lower | upper << 16), then (pair, slot of i | slot of j << 16)
    int2 *s_clist = reinterpret_cast<int2 *>(s_row + CAP + 2);
    int *s_rowoff = reinterpret_cast<int *>(s_clist + kVtxStore);   // per slot: first pair of its row less its s_start
    // small launch: the shorter charge list packed in pairs for the tile
    // test, (x, x', -y, -y') (tx, tx', ty, ty'), in the candidate results'
    // space past the parked tracks (both free until phase 1b)
    float4 *s_pk = reinterpret_cast<float4 *>(s_dyn + sizeof(float4) * CAP);

    const DevGeom &g = a.g;
    const DevParams &P = a.p;
    const bool straight = g.gamma0 == 0.f && g.gamma1 == 0.f;
    __shared__ int s_e, s_item, s_seg;
    // the small-capacity launch pulls every event from its queue and lists the
    // larger ones; the large-capacity launch pulls (listed event, pair
    // segment) items, numbered by the small launch's last CTA
    const int n_list = LARGE ? min(*(volatile const int *)&a.cnt->n_large, a.n_events) : 0;
    // no large event: the small-capacity launch has laid out the offsets already
    if (LARGE && n_list == 0) return;
    const int n_items = LARGE ? min(__ldcg(a.large_item_off + n_list), a.max_items) : 0;
    for (;;) {
    if (LARGE) {
        if (threadIdx.x < 32) {
            int k = 0;
            if (threadIdx.x == 0) k = atomicAdd(&a.cnt->vtx_queue[1], 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < n_items) {
                const int j = warp_find_segment(a.large_item_off, n_list, k);
                if (threadIdx.x == 0) {
                    s_e = __ldcg(a.large_list + j);
                    s_item = k;
                    s_seg = k - __ldcg(a.large_item_off + j);
                }
            } else if (threadIdx.x == 0) {
                s_e = a.n_events;
            }
        }
    } else if (threadIdx.x == 0) {
        const int k = atomicAdd(&a.cnt->vtx_queue[0], 1);
        s_e = k < a.n_events ? (a.ev_order ? __ldg(a.ev_order + k) : k) : a.n_events;
    }
    __syncthreads();
    const int e = s_e;
    const int item = LARGE ? s_item : 0, seg_k = LARGE ? s_seg : 0;
    __syncthreads();
    if (e >= a.n_events) break;
    const int tcap = min(__ldg(a.n_tracks), a.trk_capacity);
    int t0 = min(__ldg(a.trk_off + e), tcap), t1 = min(__ldg(a.trk_off + e + 1), tcap);
    if (t1 < t0) t1 = t0;
    int nt = t1 - t0;
    // the small-capacity launch takes events with nt <= small_cap (at most
    // kVtxSmallCap), the large one the rest (clamped to its capacity, flagged)
    const bool mine = LARGE ? nt > a.small_cap : nt <= a.small_cap;
    if (!LARGE && !mine) {
        // list the event with its opposite-charge pair count (of the tracks
        // the large-capacity launch stages)
        const int ntc = min(nt, kMaxVertexTracks);
        int cnt = 0;
        for (int i = threadIdx.x; i < ntc; i += blockDim.x) {
            const float q = a.tracks[t0 + i].qop;
            cnt += (q > 0.f ? 1 : 0) | (q < 0.f ? 0x10000 : 0);
        }
        int tot;
        block_exclusive_scan(cnt, s_scan, &tot);
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(&a.cnt->n_large, 1);
            a.large_list[slot] = e;
            a.large_pairs[slot] = (tot & 0xffff) * (tot >> 16);
        }
    }
    if (LARGE && nt > CAP) {
        if (threadIdx.x == 0 && seg_k == 0) raise_flag(a.cnt, DS_FLAG_VERTEX_CAPACITY);
        nt = CAP;
    }
    int ev_count = 0;
    if (mine && nt >= 2) {
        // stage the tracks in charge order: thread t takes tracks kTpt t ..
        // kTpt t + kTpt - 1; one scan of packed (positive, negative) counts of
        // their charges gives each its slot, its first partner after it in the
        // opposite list, and the first pair of its row
        // (one load of each track, parked in event order in the head of the
        // dynamic shared memory, which the segment loop only uses after the
        // staging barrier)
        float4 *s_park = reinterpret_cast<float4 *>(s_dyn);
        float qv[kTpt];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kTpt; ++k) {
            const int i = kTpt * threadIdx.x + k;
            qv[k] = 0.f;
            if (i < nt) {
                const ds_track &r = a.tracks[t0 + i];
                s_park[i] = make_float4(r.x, r.y, r.tx, r.ty);
                qv[k] = r.qop;
            }
            cnt += (qv[k] > 0.f ? 1 : 0) | (qv[k] < 0.f ? 0x10000 : 0);
        }
        int tot;
        const int r0 = block_exclusive_scan(cnt, s_scan, &tot);
        const int npos = tot & 0xffff, nneg = tot >> 16;
        int pb = r0 & 0xffff, nb = r0 >> 16;   // positives and negatives before the track
#pragma unroll
        for (int k = 0; k < kTpt; ++k) {
            const int i = kTpt * threadIdx.x + k;
            if (i < nt) {
                const float q = qv[k];
                // pairs in the rows before i: the pb positives before i pair with
                // all nneg negatives and the nb negatives with all npos
                // positives, which counts the pb nb pairs of two tracks before
                // i twice
                s_row[i] = pb * nneg + nb * npos - pb * nb;
                int slot = -1;
                if (q > 0.f) {
                    s_start[i] = (uint16_t)nb;
                    slot = pb++;
                } else if (q < 0.f) {
                    s_start[i] = (uint16_t)pb;
                    slot = npos + nb++;
                } else {
                    s_start[i] = 0;   // no partner: an empty row
                }
                s_self[i] = (uint16_t)(slot < 0 ? 0xffff : slot);
                if (slot >= 0) {
                    const float4 t4 = s_park[i];   // parked by this thread
                    if (!LARGE) {
                        s_rowoff[slot] = s_row[i] - s_start[i];
                        // the shorter charge list (negatives on a tie) again,
                        // two tracks per 32 bytes for the packed tile test
                        const bool neg_short = npos >= nneg;
                        if (neg_short ? q < 0.f : q > 0.f) {
                            const int si = neg_short ? slot - npos : slot;
                            float *pk = reinterpret_cast<float *>(s_pk + 2 * (si >> 1)) + (si & 1);
                            pk[0] = t4.x;
                            pk[2] = -t4.y;
                            pk[4] = t4.z;
                            pk[6] = t4.w;
                        }
                    }
                    s_ctr[slot] = t4;
                    s_cq[slot] = q;
                    s_cidx[slot] = (uint16_t)i;
                }
            }
        }
        const int npairs = npos * nneg;
        if (threadIdx.x == 0) s_row[nt] = npairs;
        __syncthreads();
        // the pairs this CTA solves: all of the event's, or one item's segment
        const int p_begin = LARGE ? min(seg_k * kVtxItemPairs, npairs) : 0;
        const int p_end = LARGE ? min(p_begin + kVtxItemPairs, npairs) : npairs;
        if (threadIdx.x == 0 && p_end > p_begin) atomicAdd(&a.cnt->n_pairs, (unsigned long long)(p_end - p_begin));
        // pair p of the current segment (first pair seg0) -> (i, j), i < j,
        // opposite charges, (i, j) order, and their slots: from the row of p's
        // mask word, a short walk over the rows starting inside the word
        auto pair_of = [&](int p, int seg0, int &i, int &j, int &si, int &sj) {
            i = s_wrow[(p - seg0) >> 5];
            while (s_row[i + 1] <= p) ++i;
            si = s_self[i];
            sj = (si < npos ? npos : 0) + s_start[i] + (p - s_row[i]);
            j = s_cidx[sj];
        };
        auto trk = [&](int slot) {
            const float4 v = s_ctr[slot];
            return Trk{v.x, v.y, v.z, v.w, s_cq[slot]};
        };
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        const unsigned lt = (1u << lane) - 1u;
        int n64 = 0;
        // events of one segment with gamma = 0 take the tiled prefilter and a
        // candidate list; the others the per-pair enumeration and the mask
        const bool tiled = !LARGE && straight && npairs <= kVtxSeg;
        for (int seg0 = p_begin; seg0 < p_end; seg0 += kVtxSeg) {
            const int nseg = min(kVtxSeg, p_end - seg0);
            const int nwords = (nseg + 31) >> 5;
            const int seg1 = seg0 + nseg;
            // each row records the mask words whose first pair it holds; the
            // masks start empty (with gamma != 0 every pair is a candidate)
            for (int i = threadIdx.x; i < nt; i += blockDim.x) {
                const int lo = max(s_row[i], seg0), hi = min(s_row[i + 1], seg1);
                for (int w = (lo - seg0 + 31) >> 5; seg0 + (w << 5) < hi; ++w) s_wrow[w] = i;
            }
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
                s_cmask[w] = straight ? 0u : (w == nwords - 1 && (nseg & 31)) ? (1u << (nseg & 31)) - 1u : 0xffffffffu;
                s_keep[w] = 0u;
            }
            __syncthreads();
            // phase 1a: is each pair of the segment a candidate?  With gamma = 0
            // both trajectories are lines and the solve converges to their
            // closest approach, whose distance |w.(Di x Dj)| / |Di x Dj| is exact
            // in closed form: pairs more than 1 um above the cut are not
            // candidates.
            // (|num| > lim sqrt(den)) squared; the 1 um margin dwarfs the
            // rounding, so the test does not depend on the pair's order
            const float lim2 = (P.doca_max + 1e-3f) * (P.doca_max + 1e-3f);
            auto is_cand = [lim2](const float4 &A, const float4 &B) {
                const float dtx = A.z - B.z, dty = A.w - B.w;
                const float cz = fmaf(A.z, B.w, -A.w * B.z);
                const float den = fmaf(dtx, dtx, fmaf(dty, dty, cz * cz));
                const float num = fmaf(A.x - B.x, dty, -(A.y - B.y) * dtx);
                return !(den > 1e-12f && num * num > lim2 * den);
            };
            bool listed = false;
            int ncand = 0;
            if (tiled) {
                // tiles of the (positive, negative) product: the lanes hold 32
                // tracks of the longer charge list, the loop broadcasts 8 of the
                // shorter one; each warp lists its candidates' two slots in its
                // own part of the list, with a count in a register
                const bool lpos = npos >= nneg;
                const int nl = lpos ? npos : nneg, ns = lpos ? nneg : npos;
                const int lb = lpos ? 0 : npos, sb = lpos ? npos : 0;
                const int nchunk = (nl + 31) >> 5, units = nchunk * ((ns + 7) >> 3);
                int2 *wl = s_clist + warp * kWarpCap;
                int wcnt = 0;
                // two partners per packed FP32 instruction, the operations of
                // is_cand in the same order (each lane of a packed op rounds as
                // the scalar op does)
                const float2 lim2v = make_float2(lim2, lim2);
                for (int u = warp; u < units; u += nwarps) {
                    const int c = u % nchunk, s0 = (u / nchunk) << 3;
                    const int sl = lb + (c << 5) + lane;
                    const bool lv = (c << 5) + lane < nl;
                    const float4 B = s_ctr[lv ? sl : 0];
                    const float2 nBx = make_float2(-B.x, -B.x), By = make_float2(B.y, B.y);
                    const float2 nBtx = make_float2(-B.z, -B.z), nBty = make_float2(-B.w, -B.w);
                    const float2 Bty = make_float2(B.w, B.w);
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) {
                        const int pi = min((s0 >> 1) + pp, (ns - 1) >> 1);
                        const float4 P0 = s_pk[2 * pi], P1 = s_pk[2 * pi + 1];
                        const float2 wx = __fadd2_rn(make_float2(P0.x, P0.y), nBx);
                        const float2 nwy = __fadd2_rn(By, make_float2(P0.z, P0.w));
                        const float2 dtx = __fadd2_rn(make_float2(P1.x, P1.y), nBtx);
                        const float2 dty = __fadd2_rn(make_float2(P1.z, P1.w), nBty);
                        const float2 cz = __ffma2_rn(make_float2(P1.x, P1.y), Bty, __fmul2_rn(make_float2(P1.z, P1.w), nBtx));
                        const float2 den = __ffma2_rn(dtx, dtx, __ffma2_rn(dty, dty, __fmul2_rn(cz, cz)));
                        const float2 num = __ffma2_rn(wx, dty, __fmul2_rn(nwy, dtx));
                        const float2 nn = __fmul2_rn(num, num), ld = __fmul2_rn(lim2v, den);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int t = 2 * pp + h;
                            const float dh = h ? den.y : den.x, nh = h ? nn.y : nn.x, lh = h ? ld.y : ld.x;
                            const bool cand = lv && s0 + t < ns && !(dh > 1e-12f && nh > lh);
                            const unsigned m = __ballot_sync(0xffffffffu, cand);
                            const int k = wcnt + __popc(m & lt);
                            if (cand && k < kWarpCap) wl[k].x = (sb + s0 + t) | (sl << 16);
                            wcnt += __popc(m);
                        }
                    }
                }
                if (lane == 0) s_wcnt[warp] = wcnt;
                __syncthreads();
                int over = 0;
                for (int w = 0; w < nwarps; ++w) {
                    ncand += s_wcnt[w];
                    over |= s_wcnt[w] > kWarpCap;
                }
                listed = !over;
            }
            if (straight && !listed) {
                // one warp per row of the segment, one partner per lane: the
                // row's track is one broadcast load and its partners are
                // consecutive in the opposite list; a ballot covers 32
                // consecutive pairs of the enumeration
                for (int i = s_wrow[0] + warp; i < nt; i += nwarps) {
                    const int rb = s_row[i], re = min(s_row[i + 1], seg1);
                    if (rb >= seg1) break;   // rows are in pair order
                    const int k0 = max(seg0 - rb, 0), k1 = re - rb;
                    if (k0 >= k1) continue;
                    const int si = s_self[i];
                    const float4 A = s_ctr[si];
                    const int ob = (si < npos ? npos : 0) + s_start[i];
                    for (int kb = k0; kb < k1; kb += 32) {
                        const int k = kb + lane;
                        const bool cand = k < k1 && is_cand(A, s_ctr[ob + min(k, k1 - 1)]);
                        const unsigned m = __ballot_sync(0xffffffffu, cand);
                        // pairs rb + kb .. rb + kb + 31 are bits b .. b + 31 of
                        // the segment's mask (set bits all below nseg)
                        if (lane == 0 && m) {
                            const int b = rb + kb - seg0, w = b >> 5, sh = b & 31;
                            atomicOr(&s_cmask[w], m << sh);
                            if (sh && (m >> (32 - sh))) atomicOr(&s_cmask[w + 1], m >> (32 - sh));
                        }
                    }
                }
                __syncthreads();
            }
            // the k-th listed candidate: warp parts in order
            auto entry = [&](int k) -> int2 & {
                int r = 0;
                while (k >= s_wcnt[r]) k -= s_wcnt[r++];
                return s_clist[r * kWarpCap + k];
            };
            // phase 1b: solve the candidates only, one per thread; keep bits
            bool store = listed;
            if (listed) {
                for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
                    int2 &en = entry(k);
                    // order the two tracks; the pair's place in the (i, j)
                    // enumeration: the row of the first, then the partner's
                    // place in the opposite list
                    const int ss = en.x & 0xffff, sl = en.x >> 16;
                    const bool sfirst = s_cidx[ss] < s_cidx[sl];
                    const int sx = sfirst ? ss : sl, sy = sfirst ? sl : ss;
                    const int p = s_rowoff[sx] + sy - (sy >= npos ? npos : 0);
                    en = make_int2(p, sx | (sy << 16));
                    int f64;
                    const PairOut o = solve_pair(g, P, trk(sx), trk(sy), f64);
                    n64 += f64;
                    s_res[k] = make_float4(o.x, o.y, o.z, o.doca);
                    s_resf[k] = o.flags;
                    if (o.doca < P.doca_max) atomicOr(&s_keep[(p - seg0) >> 5], 1u << ((p - seg0) & 31));
                }
            } else {
                int ctot = 0;
                for (int w0 = 0; w0 < nwords; w0 += blockDim.x) {
                    const int w = w0 + threadIdx.x;
                    const int c = w < nwords ? __popc(s_cmask[w]) : 0;
                    int t;
                    const int r = block_exclusive_scan(c, s_scan, &t);
                    if (w < nwords) s_cbase[w] = ctot + r;
                    ctot += t;
                }
                __syncthreads();
                store = ctot <= kVtxStore;
                for (int k = threadIdx.x; k < ctot; k += blockDim.x) {
                    int lo = 0, hi = nwords;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_cbase[mid] <= k) lo = mid;
                        else hi = mid;
                    }
                    const int bit = __fns(s_cmask[lo], 0, k - s_cbase[lo] + 1);
                    int i, j, si, sj, f64;
                    pair_of(seg0 + (lo << 5) + bit, seg0, i, j, si, sj);
                    const PairOut o = solve_pair(g, P, trk(si), trk(sj), f64);
                    n64 += f64;
                    if (store) {
                        s_res[k] = make_float4(o.x, o.y, o.z, o.doca);
                        s_resf[k] = o.flags;
                    }
                    if (o.doca < P.doca_max) atomicOr(&s_keep[lo], 1u << bit);
                }
            }
            __syncthreads();
            // ranks of the kept pairs: one scan over the segment's mask words
            int tot = 0;
            for (int w0 = 0; w0 < nwords; w0 += blockDim.x) {
                const int w = w0 + threadIdx.x;
                const int c = w < nwords ? __popc(s_keep[w]) : 0;
                int t;
                const int r = block_exclusive_scan(c, s_scan, &t);
                if (w < nwords) s_wbase[w] = tot + r;
                tot += t;
            }
            if (threadIdx.x == 0 && tot > 0) s_pool_base = atomicAdd(&a.cnt->pool_used, tot);
            __syncthreads();
            // phase 2: write the kept pairs at their (i, j) rank: from the list,
            // or by rank from the mask (re-solved when the segment had more
            // candidates than results kept)
            auto put = [&](int rank, int i, int j, const PairOut &o) {
                const int slot = s_pool_base + rank;
                if (slot < a.pool_cap) {
                    // the 32-byte record as two 16-byte stores (the pool is 16-byte aligned)
                    int4 *dst = reinterpret_cast<int4 *>(a.pool + slot);
                    dst[0] = make_int4(e, t0 + i, t0 + j, __float_as_int(o.x));
                    dst[1] = make_int4(__float_as_int(o.y), __float_as_int(o.z), __float_as_int(o.doca), (int)o.flags);
                    a.pool_pos[slot] = ev_count + rank;
                    if (LARGE) a.pool_item[slot] = item;
                } else {
                    raise_flag(a.cnt, DS_FLAG_VERTEX_CAPACITY);
                }
            };
            if (listed) {
                for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
                    const int2 c = entry(k);
                    const int b = c.x - seg0, w = b >> 5, bit = b & 31;
                    const unsigned kw = s_keep[w];
                    if (!((kw >> bit) & 1u)) continue;
                    const float4 r4 = s_res[k];
                    PairOut o;
                    o.x = r4.x; o.y = r4.y; o.z = r4.z; o.doca = r4.w;
                    o.flags = s_resf[k];
                    put(s_wbase[w] + __popc(kw & ((1u << bit) - 1u)), s_cidx[c.y & 0xffff], s_cidx[c.y >> 16], o);
                }
            } else {
                for (int k = threadIdx.x; k < tot; k += blockDim.x) {
                    int lo = 0, hi = nwords;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_wbase[mid] <= k) lo = mid;
                        else hi = mid;
                    }
                    const int bit = __fns(s_keep[lo], 0, k - s_wbase[lo] + 1);
                    int i, j, si, sj;
                    pair_of(seg0 + (lo << 5) + bit, seg0, i, j, si, sj);
                    PairOut o;
                    if (store) {           // the candidate's result from phase 1b
                        const int kc = s_cbase[lo] + __popc(s_cmask[lo] & ((1u << bit) - 1u));
                        const float4 r4 = s_res[kc];
                        o.x = r4.x; o.y = r4.y; o.z = r4.z; o.doca = r4.w;
                        o.flags = s_resf[kc];
                    } else {               // too many candidates to keep: the same solve again
                        int f64;
                        o = solve_pair(g, P, trk(si), trk(sj), f64);
                    }
                    put(k, i, j, o);
                }
            }
            ev_count += tot;
            __syncthreads();
        }
        if (n64) atomicAdd(&a.cnt->n_pairs_fp64, (unsigned long long)n64);
    }

    if (threadIdx.x == 0 && mine) {
        if (LARGE) a.item_count[item] = ev_count;
        else a.count_ws[e] = ev_count;
    }
    }   // event / item loop

    // the last CTA of the small-capacity launch records how many pool slots
    // its vertices took and numbers the large launch's items; the last CTA of
    // the launch that finishes the batch turns the per-event counts into
    // offsets: the small-capacity launch when it listed no large event,
    // otherwise the large-capacity one, after the items' offsets
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int *done = LARGE ? &a.cnt->done_vtx_large : &a.cnt->done_vtx;
        const unsigned int t = atomicAdd(done, 1u);
        s_last = t == gridDim.x - 1;
        if (s_last) *done = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (!LARGE) {
        const int n_large = *(volatile const int *)&a.cnt->n_large;
        if (threadIdx.x == 0) a.cnt->pool_small = *(volatile const int *)&a.cnt->pool_used;
        if (n_large > 0) {
            const int tot = block_offsets_f(
                [&a](int j) { return (__ldcg(a.large_pairs + j) + kVtxItemPairs - 1) / kVtxItemPairs; },
                n_large, a.large_item_off, s_scan);
            if (threadIdx.x == 0) {
                a.large_item_off[n_large] = tot;
                if (tot > a.max_items) raise_flag(a.cnt, DS_FLAG_VERTEX_CAPACITY);
            }
            return;
        }
    } else {
        // per listed event: each item's offset inside the event, the event's count
        for (int j = threadIdx.x; j < n_list; j += blockDim.x) {
            const int i0 = min(__ldcg(a.large_item_off + j), n_items), i1 = min(__ldcg(a.large_item_off + j + 1), n_items);
            int run = 0;
            for (int it = i0; it < i1; ++it) {
                a.item_base[it] = run;
                run += __ldcg(a.item_count + it);
            }
            a.count_ws[__ldcg(a.large_list + j)] = run;
        }
        __syncthreads();
        __threadfence();
    }
    const int run = block_offsets(a.count_ws, a.n_events, a.vtx_off, s_scan);
    if (threadIdx.x == 0) {
        a.vtx_off[a.n_events] = run;
        *a.n_vertices = run;
        a.cnt->n_vertices = run;
        if (run > a.capacity) raise_flag(a.cnt, DS_FLAG_VERTEX_CAPACITY);
    }
}


__global__ void __launch_bounds__(256) k_scatter_vertices(const __grid_constant__ ScatterVtxArgs a)
{
    // records move as two 16-byte chunks (pool and output are 16-byte aligned)
    const int used = min(*(volatile const int *)&a.cnt->pool_used, a.pool_cap);
    const int small = *(volatile const int *)&a.cnt->pool_small;   // slots of the small-capacity launch
    const int4 *src = reinterpret_cast<const int4 *>(a.pool);
    int4 *dst = reinterpret_cast<int4 *>(a.out);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < used; k += gridDim.x * blockDim.x) {
        const int4 lo = __ldcs(src + 2 * k), hi = __ldcs(src + 2 * k + 1);
        int pos = __ldg(a.vtx_off + lo.x) + __ldcs(a.pool_pos + k);
        if (k >= small) pos += __ldg(a.item_base + __ldcs(a.pool_item + k));
        if (pos < a.capacity) {
            dst[2 * pos] = lo;
            dst[2 * pos + 1] = hi;
        }
    }
}

template <bool LARGE>
static size_t vtx_smem(int cap)
{
    constexpr int seg = VtxSeg<LARGE>::seg, store = VtxSeg<LARGE>::store;
    return (sizeof(float4) + sizeof(unsigned)) * store + 5 * sizeof(unsigned) * (seg / 32) +
           (sizeof(float4) + sizeof(float)) * cap + sizeof(uint16_t) * 3 * cap + sizeof(int) * (cap + 2) +
           sizeof(int2) * store + (LARGE ? 0 : sizeof(int) * cap);
}

cudaError_t init_vertex_attributes()
{
    const cudaError_t e = cudaFuncSetAttribute(k_vertex<kVtxSmallCap, false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)vtx_smem<false>(kVtxSmallCap));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_vertex<kMaxVertexTracks, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)vtx_smem<true>(kMaxVertexTracks));
}

cudaError_t launch_vertex(const VertexArgs &a0, const ScatterVtxArgs &sa, int sm_count, cudaStream_t st,
                          Prof *prof)
{
    if (a0.n_events <= 0) return cudaSuccess;
    VertexArgs a = a0;
    const size_t sm_small = vtx_smem<false>(kVtxSmallCap), sm_large = vtx_smem<true>(kMaxVertexTracks);
    if (a.small_cap < 2 || a.small_cap > kVtxSmallCap || a.ctas_per_sm < 1 || a.ctas_per_sm > kVtxCtasPerSm)
        return cudaErrorInvalidValue;
    const int g_small = a.n_events < a.ctas_per_sm * sm_count ? a.n_events : a.ctas_per_sm * sm_count;
    // persistent over (event, two-segment pair range) items: at most kVtxItemsPerEvent per event
    const long long items_max = (long long)kVtxItemsPerEvent * a.n_events;
    const int g_large = items_max < sm_count ? (int)items_max : sm_count;
    prof->begin("k_vertex_small", st);
    k_vertex<kVtxSmallCap, false><<<g_small, kVtxThreads, sm_small, st>>>(a);
    prof->end(st);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    prof->begin("k_vertex_large", st);
    k_vertex<kMaxVertexTracks, true><<<g_large, kVtxLargeThreads, sm_large, st>>>(a);
    prof->end(st);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    prof->begin("k_scatter_vertices", st);
    k_scatter_vertices<<<sm_count * 4, 256, 0, st>>>(sa);
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
