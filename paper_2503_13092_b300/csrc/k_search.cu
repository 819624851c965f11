// a2-a5: magnet point, window searches, candidate fit and network inputs.
//
// Per seed (Algorithm Design section, Dv0):
//   magnet point from the SciFi state (Eq. 1 kink model), prediction in UTbX,
//   window of half-width w1a + w1b|q/p| -> up to k1 closest hits by (|dx|, id);
//   for each of them the trajectory through the hit and the magnet point is
//   extrapolated to UTaX/UTaU/UTbV, windows of half-width w2 keep the 1/2/2
//   closest hits; candidates = the UTbX hit x one option per layer ("absent"
//   only when the layer has no hit), kept when they have >= 3 hits including
//   one in station a (Track Types section, UT reconstructibility); each
//   candidate is fitted (line x = x_r + t (z - z_ref) through its hits and the
//   magnet point) and its 16 network inputs are formed.  The network and the
//   best pick run in k_mlp.cu over all candidates of the batch.
//
// Work decomposition (B300): persistent CTAs, 5 per SM (the fused form 4, 3
// for Dv1), take work items (up to 128 seeds of one event) from a device
// queue; the last warp resolves the next item while the block finishes the
// current one.  The event's bin table (with its partial-strip row bits) and
// compact x0 array are staged in shared memory by two bulk copies (TMA) on an
// mbarrier; every x test of every window reads shared memory, and a hit
// passing it looks up its strip extent and id (through the sorted index map
// and the caller's arrays) only when its sector holds a strip shorter than
// the sector or its distance ties with another hit's; the ids of a
// candidate's hits are looked up when it is written.
// Three flattened phases keep lanes busy whatever the hits per seed: UTbX
// window (thread per seed; Dv1's triplet search a warp per seed, its lanes
// over the seed's UTbX hits), refined windows (thread per (seed, UTbX hit)
// pair, in seed-aligned chunks of at most 640 pairs), fit + features (thread
// per candidate of the chunk).  Unfused form: candidates are written to a
// compact buffer reserved with one atomicAdd per chunk, seed by seed, for
// k_mlp / k_pick.  Fused form (FP32 network): each candidate's
// thread also evaluates the network (Ghost-Killer Neural Network section: the
// network runs inside the tracking, weights in the parameter bank) and merges
// its pick key with the hit ids of its layers into its seed's running minimum
// in shared memory (a 128-bit compare-and-swap); the fit of the current
// minimum is kept beside it, and after the last candidate each seed's thread
// writes the winner record, key and hit ids as k_pick does.
#include "ds_args.cuh"

namespace ds {


constexpr uint16_t kNone = 0xFFFFu;
constexpr int T = kSearchThreads;
#ifndef DS_FUSED_CTAS
#define DS_FUSED_CTAS 4
#endif
constexpr int kSearchFusedCtas = DS_FUSED_CTAS;   // resident CTAs per SM the fused form is compiled for

// The sorted hits of one event: x0 is staged separately; the index inside the
// event (sperm) gives a hit's id and, through the caller's arrays, its strip.
struct EvHits {
    const uint16_t *perm;       // sorted position -> index inside the event
    const float *ybeg, *yend;   // caller's arrays from the event's first hit
    int h0;                     // the event's first hit (ids are h0 + index)
};

// {unused, ybeg, yend, id bits} of the hit at sorted position pos
__device__ __forceinline__ float4 hit_record(const EvHits &E, int pos)
{
    const int k = __ldg(E.perm + pos);
    return make_float4(0.f, __ldg(E.ybeg + k), __ldg(E.yend + k), __int_as_float(E.h0 + k));
}

__device__ __forceinline__ int hit_id(const EvHits &E, int pos) { return E.h0 + __ldg(E.perm + pos); }

template <int N>
__device__ __forceinline__ void topn_insert(float (&d)[N], int (&id)[N], int (&p)[N], float dn,
                                            int idn, int pn)
{
    if (dn < d[N - 1] || (dn == d[N - 1] && idn < id[N - 1])) {
        d[N - 1] = dn;
        id[N - 1] = idn;
        p[N - 1] = pn;
#pragma unroll
        for (int k = N - 1; k > 0; --k) {
            const bool sw = d[k] < d[k - 1] || (d[k] == d[k - 1] && id[k] < id[k - 1]);
            if (sw) {
                float td = d[k]; d[k] = d[k - 1]; d[k - 1] = td;
                int ti = id[k]; id[k] = id[k - 1]; id[k - 1] = ti;
                int tp = p[k]; p[k] = p[k - 1]; p[k - 1] = tp;
            }
        }
    }
}

__device__ __forceinline__ bool key_less(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

// Hits of `layer` with |x0 - u| < w whose strip extent (+- dy) contains y,
// ranked by (|dx|, id); the N best are kept.  Returns how many qualified.
// The x test reads the staged x0 array (shared memory for events that fit).
// Sectors whose strips all cover the whole sector pass the strip test as a
// whole (sector_strip_class).  Up to B hits passing the x test are collected
// during the scan; after it (one uniform point for the whole warp) their
// strip extents and ids are looked up together for the per-hit strip test,
// but only when a sector needs the per-hit test or two
// collected distances are equal (the id breaks the tie); the survivors are
// ordered by a compare-exchange network.  A window with more than B
// x-passing hits (rare) is rescanned with one insertion per hit.
template <int N, int B>
__device__ __forceinline__ int window_scan(const DevGeom &g, const float *X0, const EvHits &H,
                                           const uint16_t *Tb, const uint32_t *Part, int layer, float u, float y,
                                           float w, float dy, float (&d)[N], int (&id)[N], int (&p)[N])
{
    const int s_lo = sector_of(g, y - dy - 0.01f), s_hi = sector_of(g, y + dy + 0.01f);
    const float eps = 1e-3f;
    const int b0 = xbin_of(g, u - w - eps), b1 = xbin_of(g, u + w + eps);
    int qi[B];
    float qd[B];
    int nq = 0;
    bool per_hit = false;
    for (int s = s_lo; s <= s_hi; ++s) {
        per_hit |= sector_strip_class(g, Part, layer, s, y, dy) == 2;
        const int row = (layer * g.n_sec + s) * kNXB;
        const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
        for (int i = i0; i < i1; ++i) {
            const float dx = fabsf(X0[i] - u);
            if (dx < w) {
#pragma unroll
                for (int k = 0; k < B; ++k)
                    if (k == nq) {
                        qi[k] = i;
                        qd[k] = dx;
                    }
                ++nq;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
        d[k] = __int_as_float(0x7f800000);
        id[k] = 0x7fffffff;
        p[k] = -1;
    }
    int cnt = 0;
    if (nq <= B) {
        bool tie = false;
#pragma unroll
        for (int k = 0; k < B; ++k)
#pragma unroll
            for (int k2 = k + 1; k2 < B; ++k2)
                tie |= k2 < nq && qd[k] == qd[k2];
        int hid[B];
        if (per_hit || tie) {
            // strips and ids of the collected hits, all loads in flight together
            float4 h[B];
#pragma unroll
            for (int k = 0; k < B; ++k)
                if (k < nq) h[k] = hit_record(H, qi[k]);
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const bool ok = k < nq && h[k].y - dy <= y && y <= h[k].z + dy;
                hid[k] = ok ? __float_as_int(h[k].w) : 0x7fffffff;
                if (!ok) qd[k] = __int_as_float(0x7f800000);
                cnt += ok;
            }
        } else {
            // every collected hit passes the strip test and the distances are
            // distinct: the order is by distance alone
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const bool ok = k < nq;
                hid[k] = 0;
                if (!ok) {
                    qd[k] = __int_as_float(0x7f800000);
                    hid[k] = 0x7fffffff;
                }
                cnt += ok;
            }
        }
        // odd-even transposition sort of (dx, id) over the B slots
#pragma unroll
        for (int r = 0; r < B; ++r) {
#pragma unroll
            for (int k = r & 1; k + 1 < B; k += 2) {
                if (key_less(qd[k + 1], hid[k + 1], qd[k], hid[k])) {
                    float td = qd[k]; qd[k] = qd[k + 1]; qd[k + 1] = td;
                    int ti = hid[k]; hid[k] = hid[k + 1]; hid[k + 1] = ti;
                    int tq = qi[k]; qi[k] = qi[k + 1]; qi[k + 1] = tq;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < N && k < B; ++k)
            if (k < cnt) {
                d[k] = qd[k];
                id[k] = hid[k];
                p[k] = qi[k];
            }
        return cnt;
    }
    // more x-passing hits than slots: exact insertion over a rescan
    for (int s = s_lo; s <= s_hi; ++s) {
        const int row = (layer * g.n_sec + s) * kNXB;
        const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
        for (int i = i0; i < i1; ++i) {
            const float dx = fabsf(X0[i] - u);
            if (dx < w) {
                const float4 hh = hit_record(H, i);
                if (hh.y - dy <= y && y <= hh.z + dy) {
                    topn_insert<N>(d, id, p, dx, __float_as_int(hh.w), i);
                    ++cnt;
                }
            }
        }
    }
    return cnt;
}

// Result of a refined-window search: how many hits qualified, the best
// distance and the sorted positions of the (up to) two best.
struct WinBest {
    int cnt;
    float d0;
    int p0, p1;
};

// window_scan kept out of line for the rare windows window_best hands over.
template <int N>
__device__ __noinline__ WinBest window_best_exact(const DevGeom &g, const float *X0, const EvHits &H,
                                                  const uint16_t *Tb, const uint32_t *Part, int layer, float u,
                                                  float y, float w, float dy)
{
    float d[N];
    int id[N], p[N];
    WinBest r;
    r.cnt = window_scan<N, 3>(g, X0, H, Tb, Part, layer, u, y, w, dy, d, id, p);
    r.d0 = d[0];
    r.p0 = p[0];
    r.p1 = N > 1 ? p[1] : -1;
    return r;
}

// The sectors a seed's window in `layer` visits (those of y -+ (dy + 0.01),
// as window_scan takes them) and whether one of them needs the per-hit strip
// test, packed as lo | hi << 5 | per_hit << 10.  They depend on the seed
// only, not on the UTbX hit a refined window starts from.
__device__ __forceinline__ int window_sectors(const DevGeom &g, const uint32_t *Part, int layer, float y, float dy)
{
    const int s_lo = sector_of(g, y - dy - 0.01f), s_hi = sector_of(g, y + dy + 0.01f);
    int per_hit = 0;
    for (int s = s_lo; s <= s_hi; ++s) per_hit |= sector_strip_class(g, Part, layer, s, y, dy) == 2;
    return s_lo | (s_hi << 5) | (per_hit << 10);
}

// The N (1 or 2) best hits of a window by (|dx|, id), as window_scan ranks
// them, from one pass that keeps the running N smallest distances.  Ids are
// needed only when two x-passing distances are equal, and strips only in
// sectors with partial strips; both cases (rare) go to window_scan.  A
// distance equal to a kept one is the only tie that can change the kept set:
// a hit dropped from it is farther than every later kept hit.  sinfo is
// window_sectors(g, Part, layer, y, dy).
template <int N>
__device__ __forceinline__ WinBest window_best(const DevGeom &g, const float *X0, const EvHits &H,
                                               const uint16_t *Tb, const uint32_t *Part, int layer, float u, float y,
                                               float w, float dy, int sinfo)
{
    static_assert(N == 1 || N == 2, "one or two kept hits");
    const int s_lo = sinfo & 31, s_hi = (sinfo >> 5) & 31;
    const float eps = 1e-3f;
    const int b0 = xbin_of(g, u - w - eps), b1 = xbin_of(g, u + w + eps);
    const float inf = __int_as_float(0x7f800000);
    WinBest r{0, inf, -1, -1};
    float d1 = inf;
    bool slow = (sinfo >> 10) & 1;
    for (int s = s_lo; s <= s_hi; ++s) {
        const int row = (layer * g.n_sec + s) * kNXB;
        const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
        // two hits per iteration: both loads in flight together
        auto take = [&](float xv, int i) {
            const float dx = fabsf(xv - u);
            if (dx < w) {
                ++r.cnt;
                slow |= dx == r.d0 || (N > 1 && dx == d1);
                if (N == 1) {
                    if (dx < r.d0) {
                        r.d0 = dx;
                        r.p0 = i;
                    }
                } else if (dx < d1) {
                    if (dx < r.d0) {
                        d1 = r.d0;
                        r.p1 = r.p0;
                        r.d0 = dx;
                        r.p0 = i;
                    } else {
                        d1 = dx;
                        r.p1 = i;
                    }
                }
            }
        };
        int i = i0;
        for (; i + 1 < i1; i += 2) {
            const float xa = X0[i], xb = X0[i + 1];
            take(xa, i);
            take(xb, i + 1);
        }
        if (i < i1) take(X0[i], i);
    }
    if (slow) return window_best_exact<N>(g, X0, H, Tb, Part, layer, u, y, w, dy);
    return r;
}

// A seed's best candidate so far in the fused form: the pick key (as k_pick
// packs it) and the hits' indices inside the event in layer order (16 bits
// each, 0xFFFF = absent): as one 128-bit integer the order is the pick order,
// hit ids breaking key ties with absent last.
struct __align__(16) KeyIds {
    unsigned long long key, ids;
};

__device__ __forceinline__ bool keyids_less(const KeyIds &x, const KeyIds &y)
{
    return x.key < y.key || (x.key == y.key && x.ids < y.ids);
}

// *dst = min(*dst, v) in shared memory (compare-and-swap on all 128 bits; the
// loop ends when v is no longer smaller or the swap went through)
__device__ __forceinline__ void keyids_min(KeyIds *dst, const KeyIds &v)
{
    KeyIds old = *dst;
    while (keyids_less(v, old)) {
        const KeyIds prev = atomicCAS(dst, old, v);
        if (prev.key == old.key && prev.ids == old.ids) break;
        old = prev;
    }
}

struct SeedCtx {     // per-seed quantities reused by candidate scoring
    float zm, xm, ym, tx, ty, qop, chi2, w1, u_bx;
    float yl[4];
};

struct CandFit {
    float xr, yr, t, qop, chi2;
    int ndof, nh;
    float res[4];
};

// Weighted straight-line fit x = a + b (z - z_bX) in a frame centred on the
// UTbX hit (keeps FP32 residuals small): one row per present hit (weight
// 1/sigma_hit^2), one row for the magnet point (1/sigma_mag^2).
__device__ __forceinline__ CandFit fit_candidate(const DevGeom &g, const SeedCtx &sc, const float *X0,
                                                 const int (&loc)[4])
{
    const float x0b = X0[loc[3]];
    const float xh = x0b + g.dxdy[3] * sc.yl[3];
    float Z[5], M[5], W[5];
    int n = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        Z[l] = g.z[l] - g.z[3];
        W[l] = 0.f;
        M[l] = 0.f;
        if (loc[l] >= 0) {
            const float x0 = l == 3 ? x0b : X0[loc[l]];
            M[l] = (x0 - x0b) + (g.dxdy[l] * sc.yl[l] - g.dxdy[3] * sc.yl[3]);
            W[l] = g.w_hit;
            ++n;
        }
    }
    Z[4] = sc.zm - g.z[3];
    M[4] = sc.xm - xh;
    W[4] = g.w_mag;
    float S0 = 0.f, SZ = 0.f, SM = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        S0 += W[r];
        SZ = fmaf(W[r], Z[r], SZ);
        SM = fmaf(W[r], M[r], SM);
    }
    const float zb = SZ / S0, mb = SM / S0;
    float Szz = 0.f, Szm = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const float dz = Z[r] - zb;
        Szz = fmaf(W[r] * dz, dz, Szz);
        Szm = fmaf(W[r] * dz, M[r] - mb, Szm);
    }
    const float b = Szm / Szz;
    const float a = fmaf(-b, zb, mb);
    CandFit f;
    float chi2 = 0.f;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const float res = M[r] - fmaf(b, Z[r], a);
        if (r < 4) f.res[r] = W[r] > 0.f ? res : 0.f;
        chi2 = fmaf(W[r] * res, res, chi2);
    }
    f.chi2 = chi2;
    f.ndof = n + 1 - 2;
    f.nh = n;
    f.t = b;
    f.xr = xh + fmaf(b, g.z_ref - g.z[3], a);
    f.yr = fmaf(sc.ty, g.z_ref - sc.zm, sc.ym);
    if (g.kappa != 0.f) {
        const float qopz = g.mp * (b - sc.tx) / g.kappa;
        f.qop = qopz * rsqrtf(fmaf(b, b, fmaf(sc.ty, sc.ty, 1.f)));
    } else {
        f.qop = sc.qop;
    }
    return f;
}

// First window with more x-passing hits than the collection column holds
// (rare): the k1 closest by (|dx|, id) are found by k1 passes over the
// window, pass r keeping the smallest (|dx|, id) above the one pass r - 1
// kept; only the running minimum lives in registers.  A hit's strip and id
// are looked up only when its distance could still win the pass.  Writes the
// kept sorted positions to out[r * T] in order, returns how many were kept.
__device__ __noinline__ int wide_first_window(const DevGeom &g, const float *X0, const EvHits &H,
                                              const uint16_t *Tb, const uint32_t *Part, float u, float y, float w,
                                              float dy, int k1, uint16_t *out)
{
    const int s_lo = sector_of(g, y - dy - 0.01f), s_hi = sector_of(g, y + dy + 0.01f);
    const int b0 = xbin_of(g, u - w - 1e-3f), b1 = xbin_of(g, u + w + 1e-3f);
    const float inf = __int_as_float(0x7f800000);
    float dp = -1.f;          // the last kept (|dx|, id); every hit is above the start
    int idp = -1;
    int r = 0;
    for (; r < k1; ++r) {
        float bd = inf;
        int bid = 0x7fffffff, bpos = -1;
        for (int sct = s_lo; sct <= s_hi; ++sct) {
            const int row = (3 * g.n_sec + sct) * kNXB;
            const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
            for (int i = i0; i < i1; ++i) {
                const float dx = fabsf(X0[i] - u);
                if (!(dx < w) || dx < dp || dx > bd) continue;
                const float4 h = hit_record(H, i);
                if (!(h.y - dy <= y && y <= h.z + dy)) continue;
                const int id = __float_as_int(h.w);
                if (key_less(dx, id, dp, idp) || (dx == dp && id == idp)) continue;   // kept by an earlier pass
                if (key_less(dx, id, bd, bid)) {
                    bd = dx;
                    bid = id;
                    bpos = i;
                }
            }
        }
        if (bpos < 0) break;
        out[r * T] = (uint16_t)bpos;
        dp = bd;
        idp = bid;
    }
    return r;
}

// Dv1: rank of triplet slot k among slots [0, c) of a warp's scratch by
// (residual, UTbX id); slot = (residual bits, UTbX position | UTaX position
// << 16).  Ids are looked up only on an exact residual tie.  Eight slots per
// step, so that their shared-memory loads overlap.
__device__ __forceinline__ int tri_rank(const int2 *tri, int k, int c, const EvHits &H)
{
    const int2 me = tri[k];
    const float dm = __int_as_float(me.x);
    int r = 0;
    for (int j0 = 0; j0 < c; j0 += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + q;
            const int2 e = tri[j];
            const float de = __int_as_float(e.x);
            r += j < c && (de < dm || (de == dm && j != k && hit_id(H, e.y & 0xffff) < hit_id(H, me.y & 0xffff)));
        }
    }
    return r;
}

// Dv1: the UTaX strip coordinate predicted by the line through the magnet
// point and the UTbX hit at sorted position ib.
__device__ __forceinline__ float dv1_ua(const DevGeom &g, const SeedCtx &sc, const float *X0, int ib)
{
    const float x_h = fmaf(g.dxdy[3], sc.yl[3], X0[ib]);
    const float txp = (x_h - sc.xm) / (g.z[3] - sc.zm);
    return fmaf(txp, g.z[0] - g.z[3], x_h) - g.dxdy[0] * sc.yl[0];
}

// Static shared memory of one search CTA (per template instance).  The first
// window collects each seed's x-passing UTbX hits in a column of kColRows
// rows (row r of seed o at [r][o]); the selection leaves the kept hits in
// rows 0..k1-1, which stay until the item is done (Dv1 also keeps each
// triplet's UTaX hit in rows kK1Max..2 kK1Max-1).  The rows above the kept
// ones then hold the refined-window pairs of one chunk of consecutive seeds:
// per pair its (seed, UTbX rank), the five refined hits and its candidate
// count.  An item whose pairs exceed kPairCap is processed in several
// seed-aligned chunks.  The fused form keeps more rows (its winner records
// are staged there at the end of an item).
template <int V, bool F>
struct SearchLayout {
    static constexpr int kKeepRows = V == 1 ? 2 * kK1Max : kK1Max;
    static constexpr int kPairBytes = 2 + 5 * 2 + 1;
    static constexpr int kPairCap = F ? 784 : 640;
    static constexpr int kColRows = kKeepRows + (kPairCap * kPairBytes + 2 * T - 1) / (2 * T);
    static_assert(kPairCap >= kK1Max, "a chunk holds at least one seed's pairs");
};

// A seed's SeedCtx from its two shared-memory records, (z_m, x_m, y_m, ty)
// and (tx, q/p, w1, u_bX), and its chi2; y at each layer is recomputed as
// the first phase computed it.
__device__ __forceinline__ SeedCtx seed_ctx_of(const DevGeom &g, const float4 &A, const float4 &B, float chi2)
{
    SeedCtx sc;
    sc.zm = A.x;
    sc.xm = A.y;
    sc.ym = A.z;
    sc.ty = A.w;
    sc.tx = B.x;
    sc.qop = B.y;
    sc.w1 = B.z;
    sc.u_bx = B.w;
    sc.chi2 = chi2;
#pragma unroll
    for (int l = 0; l < 4; ++l) sc.yl[l] = fmaf(sc.ty, g.z[l] - sc.zm, sc.ym);
    return sc;
}
// first-window column in the dynamic staging area of an event too large to
// stage (at most this many rows)
constexpr int kColRowsBig = 50;

// V = 0: Dv0.  V = 1: Dv1, whose first stage is the triplet search.
// F: fused network and pick (FP32 network 16-32-32-1).
template <int V, bool F>
__global__ void __launch_bounds__(T, F ? (V == 1 ? 3 : kSearchFusedCtas) : (V == 0 ? kSearchCtasPerSm : 4))
    k_search(const __grid_constant__ SearchArgs a)
{
    using L = SearchLayout<V, F>;
    constexpr int PC = L::kPairCap;
    extern __shared__ __align__(16) unsigned char s_dyn[];   // bin table, then staged x0
    // first-window columns, kept UTbX hits, pair arrays of a chunk; in the
    // fused form also the staging area of the winner records (128 x 64 bytes)
    __shared__ __align__(16) uint16_t s_col[L::kColRows][T];
    __shared__ float4 s_sa[T];          // per seed: z_m, x_m, y_m, ty
    __shared__ float4 s_sb[T];          // per seed: tx, q/p, w1, u_bX (chi2 is re-read from the seeds)
    __shared__ uint16_t s_wsec[3][T];   // window_sectors of the refined windows (layers 0-2)
    __shared__ int s_base[T + 4];       // candidate offsets of the chunk's seeds
    __shared__ uint16_t s_j0[T + 2];    // first pair of each seed in the item, then the item's total
    __shared__ __align__(16) KeyIds s_best[F ? T : 1];   // fused: each seed's best key + hit indices
    __shared__ __align__(16) float4 s_win[F ? T : 1];    // fused: x_ref, tx, q/p, chi2 of the best
    __shared__ int s_cand0;
    __shared__ int s_scan[64];          // two scan scratch areas (first-window pairs, candidates)
    __shared__ int s_nx[6];     // next work item: index, event, seed begin, seed end, h0, h1
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ __align__(8) uint64_t s_bar_fi;   // fault injection only: a barrier no copy targets
    uint16_t *const p_oj = &s_col[L::kKeepRows][0];                     // pair: seed << 4 | rank
    uint16_t *const p_sel = p_oj + PC;                                   // [5][PC] refined hits
    uint8_t *const p_nc = reinterpret_cast<uint8_t *>(p_sel + 5 * PC);   // candidates of the pair

    const DevGeom &g = a.g;
    const DevParams &P = a.p;
    const int tid = threadIdx.x;

    // persistent CTA: work items from a device queue (a.group consecutive
    // items per pull).  The last warp resolves the next item (queue pull,
    // event lookup, offsets) into s_nx while the block works on the current
    // one, after the refined windows, where that warp has the fewest pairs;
    // the event's data is staged again only when the event changes.
    const int n_items = __ldg(a.item_off + a.n_events);
    uint16_t *Tb = reinterpret_cast<uint16_t *>(s_dyn);
    const uint32_t *Part = reinterpret_cast<const uint32_t *>(Tb + g.ext_off);
    float *xs = reinterpret_cast<float *>(s_dyn + sizeof(uint16_t) * g.table_stride);
    constexpr int kNextWarp = T / 32 - 1;
    const bool next_warp = (tid >> 5) == kNextWarp;
    int q_next = 0, q_end = 0;     // lane 0 of the next-item warp: rest of its queue group
    // work item bi (layouts in k_bucket.cu): order 0, chunk k of event e's
    // seeds (sizes differ by at most one); order 1, full chunk k of event e,
    // or, past the full chunks, the remainder of the event listed for it
    auto resolve_next = [&]() {    // the next-item warp, all 32 lanes
        int bi = 0;
        if ((tid & 31) == 0) {
            if (q_next >= q_end) {
                q_next = atomicAdd(&a.cnt->search_queue, a.group);
                q_end = q_next + a.group;
            }
            bi = q_next++;
        }
        bi = __shfl_sync(0xffffffffu, bi, 0);
        if (bi >= n_items) {
            if ((tid & 31) == 0) s_nx[0] = n_items;
            return;
        }
        const int n_full = a.order ? __ldg(a.item_off + a.n_events + 1) : n_items;
        const int e = bi < n_full ? warp_find_segment(a.item_off, a.n_events, bi)
                                  : __ldg(a.item_off + a.n_events + 2 + (bi - n_full));
        if ((tid & 31) == 0) {
            const int s0 = __ldg(a.seed_off + e), ns = __ldg(a.seed_off + e + 1) - s0;
            int h0 = __ldg(a.hit_off + e), h1 = __ldg(a.hit_off + e + 1);
            if (h0 < 0 || h1 < h0 || h1 > a.n_hits || h1 - h0 > kMaxEventHits) h1 = h0 = 0;
            int b0, b1;
            if (!a.order) {
                const int i0 = __ldg(a.item_off + e), i1 = __ldg(a.item_off + e + 1);
                const int k = bi - i0, nc = i1 - i0;
                b0 = (int)(((long long)k * ns) / nc);
                b1 = (int)(((long long)(k + 1) * ns) / nc);
            } else if (bi < n_full) {
                b0 = (bi - __ldg(a.item_off + e)) * a.chunk;
                b1 = b0 + a.chunk;
            } else {
                b0 = ns - ns % a.chunk;
                b1 = ns;
            }
            s_nx[0] = bi;
            s_nx[1] = e;
            s_nx[2] = s0 + b0;
            s_nx[3] = s0 + b1;
            s_nx[4] = h0;
            s_nx[5] = h1;
        }
    };
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        if (P.fault_inject & 1) {
            // tests: a barrier that expects 16 bytes nothing sends; the
            // staging wait below also waits on it and runs out
            mbar_init(&s_bar_fi, 1);
            mbar_expect_tx(&s_bar_fi, 16u);
        }
    }
    if (next_warp) resolve_next();
    __syncthreads();
    uint32_t phase = 0;
    int staged_e = -1;             // the event in the staging buffers (same in every thread)
    for (;;) {
    // s_nx is read by every thread here and rewritten by the next-item warp
    // only after the block has met again (first-window scan)
    if (s_nx[0] >= n_items) break;
    const int e = s_nx[1];
    const int s_begin = s_nx[2], s_end = s_nx[3];
    const int h0 = s_nx[4], h1 = s_nx[5];
    const bool restage = e != staged_e;
    staged_e = e;
    if (tid == 0 && restage) {
        // the event's bin table and (if it fits) its x0 array, by two bulk
        // copies (TMA); the x0 copy starts at the 16-byte boundary below h0.
        // The previous item's readers are done (the block met at the end of it).
        const int nh = h1 - h0, lead = h0 & 3;
        const uint32_t tb_bytes = sizeof(uint16_t) * g.table_stride;
        const uint32_t x_bytes = nh <= a.stage_hits ? (uint32_t)(((lead + nh) * 4 + 15) & ~15) : 0u;
        mbar_expect_tx(&s_bar, tb_bytes + x_bytes);
        bulk_copy_g2s(Tb, a.bins + (size_t)e * g.table_stride, tb_bytes, &s_bar);
        if (x_bytes) bulk_copy_g2s(xs, a.sx0 + (h0 - lead), x_bytes, &s_bar);
    }
    const int s = s_begin + tid;
    const bool active = s < s_end;
    const int nh = h1 - h0;
    const EvHits H{a.sperm + h0, a.ybeg + h0, a.yend + h0, h0};
    const bool staged = nh <= a.stage_hits;
    const float *X0 = staged ? xs + (h0 & 3) : a.sx0 + h0;

    // the seed's state is loaded while the staging copies are in flight
    float sd_x = 0.f, sd_y = 0.f, sd_tx = 0.f, sd_ty = 0.f, sd_qop = 0.f, sd_chi2 = 0.f;
    if (active) {
        sd_x = __ldg(a.sx + s);
        sd_y = __ldg(a.sy + s);
        sd_tx = __ldg(a.stx + s);
        sd_ty = __ldg(a.sty + s);
        sd_qop = __ldg(a.sqop + s);
        sd_chi2 = __ldg(a.schi2 + s);
        a.rank_ws[s] = -1;     // the clone kernel ranks this call's winners
    }
    if (restage) {
        // bounded wait; the decision to go on is taken by the whole block
        bool ok = mbar_wait_bounded(&s_bar, phase, kWaitLimit);
        if (P.fault_inject & 1) ok = ok && mbar_wait_bounded(&s_bar_fi, 0, 1024);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) raise_flag(a.cnt, DS_FLAG_TIMEOUT);
            // the block must not leave while bulk copies still write into its
            // shared memory: wait (bounded again) for the staging copies.  With
            // fault injection they have already landed; after a real time-out
            // they may still be in flight if this wait runs out too.
            mbar_wait_bounded(&s_bar, phase, kWaitLimit);
            __syncthreads();
            return;
        }
        phase ^= 1u;
    }

    // ---------------------------------------------------------------- search
    // the first-window column: the static rows, or for an event too large
    // to stage (its x0 is read from global memory) the unused staging area
    const int big_rows = min(kColRowsBig, (int)((sizeof(float) * (a.stage_hits + 4)) / (sizeof(uint16_t) * T)));
    const bool col_dyn = !staged && big_rows > L::kColRows;
    uint16_t *const colb = col_dyn ? reinterpret_cast<uint16_t *>(xs) : &s_col[0][0];
    const int kCap = col_dyn ? big_rows : L::kColRows;
    int nbx = 0;
    // first window (Dv0): 0 keep the survivors as collected, 1 select the k1
    // closest (warp), 2 exact sort (training mode or a distance tie), 3 done
    int sel_state = 0, sel_n = 0;
    float sel_u = 0.f;
    if (active) {
        SeedCtx sc;
        const float x = sd_x, y = sd_y;
        sc.tx = sd_tx;
        sc.ty = sd_ty;
        sc.qop = sd_qop;
        sc.chi2 = sd_chi2;
        const float aq = fabsf(sc.qop);
        // magnet point (Eq. 1 kink model): parameterised z, straight-line x, y
        sc.zm = g.zmag[0] + g.zmag[1] * sc.tx * sc.tx + g.zmag[2] * sc.ty * sc.ty + g.zmag[3] * aq;
        sc.xm = fmaf(sc.tx, sc.zm - g.z_seed, x);
        sc.ym = fmaf(sc.ty, sc.zm - g.z_seed, y);
#pragma unroll
        for (int l = 0; l < 4; ++l) sc.yl[l] = fmaf(sc.ty, g.z[l] - sc.zm, sc.ym);
        const float tx_ut = P.origin ? sc.xm / sc.zm
                                     : sc.tx + g.mp * g.kappa * sc.qop *
                                                   sqrtf(fmaf(sc.tx, sc.tx, fmaf(sc.ty, sc.ty, 1.f)));
        const float u_bx = fmaf(tx_ut, g.z[3] - sc.zm, sc.xm) - g.dxdy[3] * sc.yl[3];
        sc.w1 = P.training ? 100.f : fmaf(P.w1b, aq, P.w1a);
        sc.u_bx = u_bx;
        s_sa[tid] = make_float4(sc.zm, sc.xm, sc.ym, sc.ty);
        s_sb[tid] = make_float4(sc.tx, sc.qop, sc.w1, sc.u_bx);
#pragma unroll
        for (int l = 0; l < 3; ++l) s_wsec[l][tid] = (uint16_t)window_sectors(g, Part, l, sc.yl[l], P.dy_tol);

        uint16_t *col = colb + tid;
        if (V == 0) {
            // UTbX window: x-passing positions collected in this thread's
            // column; the hits of sectors whose strips all cover the sector
            // pass the strip test as a whole, otherwise their strips are
            // looked up together.  The kept hits are the k1 closest by
            // (|dx|, id); their order matters only for the candidate export,
            // so they are sorted in training mode only (the pick breaks exact
            // key ties by hit ids)
            const float u = u_bx, w = sc.w1, y3 = sc.yl[3], dy = P.dy_tol;
            const int s_lo = sector_of(g, y3 - dy - 0.01f), s_hi = sector_of(g, y3 + dy + 0.01f);
            const int b0 = xbin_of(g, u - w - 1e-3f), b1 = xbin_of(g, u + w + 1e-3f);
            int nq = 0;
            bool per_hit = false;     // a sector whose strips must be tested hit by hit
            for (int sct = s_lo; sct <= s_hi; ++sct) {
                per_hit |= sector_strip_class(g, Part, 3, sct, y3, dy) == 2;
                const int row = (3 * g.n_sec + sct) * kNXB;
                const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
                for (int i = i0; i < i1; ++i)
                    if (fabsf(X0[i] - u) < w) {
                        if (nq < kCap) col[nq * T] = (uint16_t)i;
                        ++nq;
                    }
            }
            if (nq > kCap) {
                nbx = wide_first_window(g, X0, H, Tb, Part, u_bx, sc.yl[3], sc.w1, P.dy_tol, P.k1, col);
                sel_state = 3;
            } else {
                int nok = per_hit ? 0 : nq;   // otherwise every collected hit passes the strip test
                for (int k0 = 0; per_hit && k0 < nq; k0 += 4) {
                    float4 h[4];
                    int ii[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        ii[k] = k0 + k < nq ? col[(k0 + k) * T] : -1;
                        if (ii[k] >= 0) h[k] = hit_record(H, ii[k]);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (ii[k] >= 0 && h[k].y - dy <= y3 && y3 <= h[k].z + dy) col[(nok++) * T] = (uint16_t)ii[k];
                }
                // the order of the kept hits matters only for the candidate
                // export (training mode: exact sort below); otherwise only the
                // k1 closest are needed, and a window with more survivors has
                // them selected by its warp below
                sel_n = nok;
                sel_u = u;
                sel_state = P.training ? 2 : (nok > P.k1 ? 1 : 0);
            }
        }
        // Dv1: the triplet search runs below, a warp per seed
    }
    if (V == 1) {
        // Dv1 triplets: every UTbX hit with a physical kink (a window of
        // half-width dtx_max (z_m - z_bX) around the seed's straight
        // extrapolation) whose magnet-point line meets a UTaX hit within
        // w_tri; the k1 best by (residual, UTbX id) are kept.  The warp takes
        // its seeds one at a time, its lanes over the seed's UTbX hits (32 per
        // step, each with its UTaX window); the triplets found are collected
        // in a scratch of the warp and ranked once per seed (below).
        __syncwarp();
        const unsigned full = 0xffffffffu;
        const int lane = tid & 31;
        const float inf = __int_as_float(0x7f800000);
        // this warp's 32-slot triplet scratch: pair-array rows, unused until
        // the refined windows
        int2 *const tri = reinterpret_cast<int2 *>(&s_col[L::kKeepRows][0]) + (tid >> 5) * 32;
        static_assert((L::kColRows - L::kKeepRows) * T * sizeof(uint16_t) >= T * sizeof(int2), "triplet scratch");
        unsigned am = __ballot_sync(full, active);
        while (am) {
            const int src = __ffs(am) - 1;
            am &= am - 1;
            const int o = tid - lane + src;
            const SeedCtx sc = seed_ctx_of(g, s_sa[o], s_sb[o], 0.f);
            const float w_b = P.dv1_dtx * (sc.zm - g.z[3]);
            const float u0 = fmaf(sc.tx, g.z[3] - sc.zm, sc.xm) - g.dxdy[3] * sc.yl[3];
            const float y3 = sc.yl[3], dy = P.dy_tol;
            const int wsec0 = s_wsec[0][o];
            const int s_lo = sector_of(g, y3 - dy - 0.01f), s_hi = sector_of(g, y3 + dy + 0.01f);
            const int b0 = xbin_of(g, u0 - w_b - 1e-3f), b1 = xbin_of(g, u0 + w_b + 1e-3f);
            // The seed's triplets are collected in this warp's scratch
            // (slots 0..cnt-1, in the order found); when 32 slots do not hold
            // the next ones, the kK1Max best so far are kept (a triplet
            // dropped then has kK1Max better ones, which stay).  At the end
            // each collected triplet's rank by (residual, UTbX id) places the
            // kK1Max best in the seed's column.
            int cnt = 0, n_tri = 0;
            for (int sct = s_lo; sct <= s_hi; ++sct) {
                // rows whose strips all span the sector pass the strip test as a whole
                const bool per_hit = sector_strip_class(g, Part, 3, sct, y3, dy) == 2;
                const int row = (3 * g.n_sec + sct) * kNXB;
                const int i0 = Tb[row + b0], i1 = Tb[row + b1 + 1];
                for (int ib = i0; ib < i1; ib += 32) {
                    const int i = ib + lane;
                    bool ok = i < i1 && fabsf(X0[i] - u0) < w_b;
                    if (ok && per_hit) {
                        const float4 hb = hit_record(H, i);
                        ok = hb.y - dy <= y3 && y3 <= hb.z + dy;
                    }
                    float dn = inf;
                    int pn = -1;
                    if (ok) {
                        const float ua = dv1_ua(g, sc, X0, i);
                        const WinBest wa = window_best<1>(g, X0, H, Tb, Part, 0, ua, sc.yl[0], P.dv1_w_tri, dy, wsec0);
                        ok = wa.cnt > 0;
                        dn = wa.d0;
                        pn = i | (wa.p0 << 16);
                    }
                    unsigned m = __ballot_sync(full, ok);
                    n_tri += __popc(m);
                    while (m) {
                        if (cnt == 32) {
                            const int r = tri_rank(tri, lane, 32, H);
                            const int2 me = tri[lane];
                            __syncwarp();
                            if (r < kK1Max) tri[r] = me;
                            __syncwarp();
                            cnt = kK1Max;
                        }
                        // the new triplets in lane order, as many as fit
                        const int nt = min(__popc(m), 32 - cnt);
                        const int k = __popc(m & ((1u << lane) - 1u));
                        const bool put = ((m >> lane) & 1u) && k < nt;
                        if (put) tri[cnt + k] = make_int2(__float_as_int(dn), pn);
                        m &= ~__ballot_sync(full, put);
                        cnt += nt;
                        __syncwarp();
                    }
                }
            }
            const int nb = min(n_tri, P.k1);
            if (lane < cnt) {
                // every triplet is kept when there are at most k1: outside
                // training mode their order is free (the pick breaks key
                // ties by hit ids), so they keep the order found
                const int r = cnt <= P.k1 && !P.training ? lane : tri_rank(tri, lane, cnt, H);
                if (r < kK1Max) {
                    const int pk = tri[lane].y;
                    colb[r * T + o] = (uint16_t)(pk & 0xffff);
                    colb[(kK1Max + r) * T + o] = r < nb ? (uint16_t)((unsigned)pk >> 16) : kNone;   // the triplet's UTaX hit
                }
            } else if (lane < kK1Max) {
                colb[lane * T + o] = kNone;
                colb[(kK1Max + lane) * T + o] = kNone;
            }
            __syncwarp();   // the scratch is refilled by the next seed
            if (lane == src) nbx = nb;
        }
    }
    if (V == 0) {
        // first windows with more than k1 survivors (outside training): the
        // warp ranks each one's hits by (|dx|, position), one or two hits per
        // lane, and the k1 first take the first k1 slots of its column.  A
        // shared distance that could change the kept set (the order is then
        // by id) sends the seed to the exact sort.
        const int lane = tid & 31;
        const float inf = __int_as_float(0x7f800000);
        unsigned wm = __ballot_sync(0xffffffffu, sel_state == 1);
        while (wm) {
            const int src = __ffs(wm) - 1;
            wm &= wm - 1;
            const int n = __shfl_sync(0xffffffffu, sel_n, src);         // <= kCap <= 64
            const float uu = __shfl_sync(0xffffffffu, sel_u, src);
            uint16_t *cc = colb + (tid - lane + src);
            const int p0 = lane < n ? cc[lane * T] : 0, p1 = lane + 32 < n ? cc[(lane + 32) * T] : 0;
            const float d0 = lane < n ? fabsf(X0[p0] - uu) : inf, d1 = lane + 32 < n ? fabsf(X0[p1] - uu) : inf;
            int r0 = 0, r1 = 0;
            bool t0 = false, t1 = false;
            for (int k = 0; k < n; ++k) {
                const float dk = __shfl_sync(0xffffffffu, k < 32 ? d0 : d1, k & 31);
                const int pk = __shfl_sync(0xffffffffu, k < 32 ? p0 : p1, k & 31);
                r0 += dk < d0 || (dk == d0 && pk < p0);
                r1 += dk < d1 || (dk == d1 && pk < p1);
                t0 |= dk == d0 && pk != p0;
                t1 |= dk == d1 && pk != p1;
            }
            const bool tie = __any_sync(0xffffffffu, (lane < n && t0 && r0 <= P.k1) ||
                                                         (lane + 32 < n && t1 && r1 <= P.k1));
            __syncwarp();
            if (!tie) {
                if (lane < n && r0 < P.k1) cc[r0 * T] = (uint16_t)p0;
                if (lane + 32 < n && r1 < P.k1) cc[r1 * T] = (uint16_t)p1;
            } else if (lane == src) {
                sel_state = 2;
            }
            __syncwarp();
        }
        if (active && sel_state != 3) {
            uint16_t *col = colb + tid;
            // exact insertion sort by (|dx|, id), ids looked up only on ties
            for (int a2 = 1; sel_state == 2 && a2 < sel_n; ++a2) {
                const int v = col[a2 * T];
                const float dv = fabsf(X0[v] - sel_u);
                int j = a2 - 1;
                while (j >= 0) {
                    const int c = col[j * T];
                    const float dc = fabsf(X0[c] - sel_u);
                    const bool before = dv < dc || (dv == dc && hit_id(H, v) < hit_id(H, c));
                    if (!before) break;
                    col[(j + 1) * T] = (uint16_t)c;
                    --j;
                }
                col[(j + 1) * T] = (uint16_t)v;
            }
            nbx = min(sel_n, P.k1);   // the kept hits are the column's first nbx rows
        }
    }
    // the item's (seed, UTbX hit) pairs in seed order, then rank order.  The
    // scan's barrier also ends every column's first-window use, so the rows
    // above the kept ones are free for the pair arrays from here on.
    int total_j;
    const int jbase = block_exclusive_scan1(nbx, s_scan, &total_j);
    s_j0[tid] = (uint16_t)jbase;
    if (tid == T - 1) s_j0[T] = (uint16_t)(jbase + nbx);
    if (F) s_best[tid] = KeyIds{kNoKey, ~0ull};
    const bool one_chunk = total_j <= PC;   // the usual case: the pairs are written here
    if (one_chunk && active)
        for (int j = 0; j < nbx; ++j) p_oj[jbase + j] = (uint16_t)((tid << 4) | j);
    __syncthreads();

    const int n_item = s_end - s_begin;
    int n_cand = 0;    // this thread's seed: its candidates (set in its chunk)
    for (int c_lo = 0; c_lo < n_item;) {
        // the chunk: seeds [c_lo, c_hi), as many as have at most PC pairs
        const int p0 = s_j0[c_lo];
        int c_hi = c_lo + 1;
        {
            int hi = n_item;
            while (c_hi < hi) {
                const int mid = (c_hi + hi + 1) >> 1;
                if ((int)s_j0[mid] - p0 <= PC) c_hi = mid;
                else hi = mid - 1;
            }
        }
        const int np = (int)s_j0[c_hi] - p0;
        const bool in_chunk = tid >= c_lo && tid < c_hi;
        if (!one_chunk) {
            if (in_chunk)
                for (int j = 0; j < nbx; ++j) p_oj[jbase - p0 + j] = (uint16_t)((tid << 4) | j);
            __syncthreads();
        }

        // refined windows, one (seed, UTbX hit) pair per thread: every lane
        // does the same three window searches whatever the hits per seed
        for (int t = tid; t < np; t += T) {
            const int o = p_oj[t] >> 4, j = p_oj[t] & 15;
            const SeedCtx sc = seed_ctx_of(g, s_sa[o], s_sb[o], 0.f);
            const float w2 = P.training ? 10.f : P.w2;
            const float x0b = X0[colb[j * T + o]];
            const float xh = x0b + g.dxdy[3] * sc.yl[3];
            const float txp = (xh - sc.xm) / (g.z[3] - sc.zm);
            int sel[5];
            if (V == 1) {
                sel[0] = colb[(kK1Max + j) * T + o];   // Dv1: the triplet's UTaX hit
                if (sel[0] == kNone) sel[0] = -1;
            } else {
                const float ul = fmaf(txp, g.z[0] - g.z[3], xh) - g.dxdy[0] * sc.yl[0];
                sel[0] = window_best<1>(g, X0, H, Tb, Part, 0, ul, sc.yl[0], w2, P.dy_tol, s_wsec[0][o]).p0;
            }
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const float ul = fmaf(txp, g.z[l] - g.z[3], xh) - g.dxdy[l] * sc.yl[l];
                const WinBest wb = window_best<2>(g, X0, H, Tb, Part, l, ul, sc.yl[l], w2, P.dy_tol, s_wsec[l][o]);
                sel[2 * l - 1] = wb.p0;
                sel[2 * l] = wb.p1;
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) p_sel[k * PC + t] = sel[k] >= 0 ? (uint16_t)sel[k] : kNone;
            const int pa = sel[0] >= 0, pu = sel[1] >= 0, pv = sel[3] >= 0;
            const int nu = sel[2] >= 0 ? 2 : 1, nv = sel[4] >= 0 ? 2 : 1;
            const int valid = (1 + pa + pu + pv >= 3) && (pa || pu);
            p_nc[t] = (uint8_t)(valid ? nu * nv : 0);
        }
        if (next_warp && c_lo == 0) resolve_next();
        __syncthreads();
        if (in_chunk)
            for (int j = 0; j < nbx; ++j) n_cand += p_nc[jbase - p0 + j];

        int total;
        const int base = block_exclusive_scan1(in_chunk ? n_cand : 0, s_scan + 32, &total);
        s_base[tid] = base;
        if (tid == T - 1) s_base[T] = total;
        if (tid == 0) {
            if (total > 0) atomicAdd(&a.cnt->n_candidates, (unsigned long long)total);
            int c0 = total > 0 && !F ? atomicAdd(&a.cnt->cand_used, total) : 0;
            if (!F && total > 0 && c0 + total > a.cand_cap) {   // candidate buffer full: flagged, seeds left empty
                raise_flag(a.cnt, DS_FLAG_CAND_CAPACITY);
                c0 = -1;
            }
            s_cand0 = c0;
        }
        __syncthreads();
        const int cand0 = s_cand0;
        if (!F && active && in_chunk)
            a.seed_cand[s] = cand0 >= 0 ? make_int4(cand0 + base, n_cand, e, 0) : make_int4(0, 0, e, 0);
        // candidate c of the chunk decodes to (seed, pair, stereo options) in
        // enumeration order
        auto decode = [&](int c, int &o, int (&loc)[4], int &jr) {
            int lo = 0, hi = T;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_base[mid] <= c) lo = mid;
                else hi = mid;
            }
            o = lo;
            int k = c - s_base[o];
            int pp = (int)s_j0[o] - p0;
            while (k >= p_nc[pp]) {
                k -= p_nc[pp];
                ++pp;
            }
            jr = p_oj[pp] & 15;
            const int nv = p_sel[4 * PC + pp] != kNone ? 2 : 1;
            const int iu = k / nv, iv = k - iu * nv;
            const uint16_t a0 = p_sel[pp], u0 = p_sel[(1 + iu) * PC + pp], v0 = p_sel[(3 + iv) * PC + pp];
            loc[0] = a0 == kNone ? -1 : a0;
            loc[1] = u0 == kNone ? -1 : u0;
            loc[2] = v0 == kNone ? -1 : v0;
            loc[3] = colb[jr * T + o];
        };
        if (F) {
            // fused: rounds of T candidates; each merges into its seed's
            // minimum, then (after the round's barrier) the candidate holding
            // the minimum keeps its fit beside it.  A later round's merge can
            // only lower the minimum, and its holder then writes its own fit
            // after that round's barrier, so the fit kept is always the minimum's.
            for (int cr = 0; cr < total; cr += T) {
                const int c = cr + tid;
                KeyIds mine{kNoKey, 0ull};
                float4 fw = make_float4(0.f, 0.f, 0.f, 0.f);
                int o = 0;
                if (c < total) {
                    int loc[4], jr;
                    decode(c, o, loc, jr);
                    const SeedCtx sc = seed_ctx_of(g, s_sa[o], s_sb[o], __ldg(a.schi2 + s_begin + o));
                    const CandFit f = fit_candidate(g, sc, X0, loc);
                    float phi[16];
                    phi[0] = f.xr * 1e-3f;
                    phi[1] = f.yr * 1e-3f;
                    phi[2] = f.t;
                    phi[3] = sc.ty;
                    phi[4] = 1e3f * f.qop;
                    phi[5] = f.chi2 / (float)f.ndof;
                    phi[6] = 1e3f * sc.qop;
                    phi[7] = sc.chi2;
#pragma unroll
                    for (int l = 0; l < 4; ++l) phi[8 + l] = f.res[l] * g.inv_sigma_hit;
                    phi[12] = 0.25f * (float)f.nh;
                    phi[13] = V == 1 ? fabsf(X0[loc[0]] - dv1_ua(g, sc, X0, loc[3])) / P.dv1_w_tri
                                     : fabsf(X0[loc[3]] - sc.u_bx) / sc.w1;
                    phi[14] = sc.tx;
                    phi[15] = sc.ty;
                    // what the pick needs is formed before the network, so that
                    // little else is live while it runs
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        mine.ids = (mine.ids << 16) | (loc[l] >= 0 ? (unsigned long long)__ldg(H.perm + loc[l]) : 0xFFFFull);
                    fw = make_float4(f.xr, f.t, f.qop, f.chi2);
                    const float chi2_ndof = phi[5];
                    const float lg = mlp_logit_fp32<16, 32, 32>(a.nn, phi);
                    if (P.pick_chi2) mine.key = pack_key(chi2_ndof, lg);
                    else if (lg < P.thr_logit) mine.key = pack_key(lg, fw.w);
                    if (mine.key != kNoKey) keyids_min(&s_best[o], mine);
                }
                __syncthreads();
                if (mine.key != kNoKey) {
                    const KeyIds b = s_best[o];
                    if (b.key == mine.key && b.ids == mine.ids) s_win[o] = fw;
                }
            }
        } else if (cand0 >= 0) {
            // fit + network inputs, one candidate per thread
            for (int c = tid; c < total; c += T) {
                int o, loc[4], jr;
                decode(c, o, loc, jr);
                const SeedCtx sc = seed_ctx_of(g, s_sa[o], s_sb[o], __ldg(a.schi2 + s_begin + o));
                const CandFit f = fit_candidate(g, sc, X0, loc);
                float phi[16];
                phi[0] = f.xr * 1e-3f;
                phi[1] = f.yr * 1e-3f;
                phi[2] = f.t;
                phi[3] = sc.ty;
                phi[4] = 1e3f * f.qop;
                phi[5] = f.chi2 / (float)f.ndof;
                phi[6] = 1e3f * sc.qop;
                phi[7] = sc.chi2;
#pragma unroll
                for (int l = 0; l < 4; ++l) phi[8 + l] = f.res[l] * g.inv_sigma_hit;
                phi[12] = 0.25f * (float)f.nh;
                phi[13] = V == 1 ? fabsf(X0[loc[0]] - dv1_ua(g, sc, X0, loc[3])) / P.dv1_w_tri
                                 : fabsf(X0[loc[3]] - sc.u_bx) / sc.w1;
                phi[14] = sc.tx;
                phi[15] = sc.ty;
                const int slot = cand0 + c;
                float4 *fd = a.cand_feat + 4 * (size_t)slot;
#pragma unroll
                for (int q = 0; q < 4; ++q) fd[q] = make_float4(phi[4 * q], phi[4 * q + 1], phi[4 * q + 2], phi[4 * q + 3]);
                CandMeta m;
                m.xr = f.xr; m.yr = f.yr; m.t = f.t; m.qop = f.qop;
                m.chi2 = f.chi2;
                m.ndof = f.ndof;
                m.seed = s_begin + o;
                m.ty = sc.ty;
#pragma unroll
                for (int l = 0; l < 4; ++l) m.hit[l] = loc[l] >= 0 ? hit_id(H, loc[l]) : -1;
                a.cand_meta[slot] = m;
            }
        }
        // the next chunk rewrites the pair arrays (after the last one the
        // item's closing barrier covers the unfused form)
        if (F || c_hi < n_item) __syncthreads();
        c_lo = c_hi;
    }
    if (F) {
        // each seed's winner as k_pick writes it: the 64-byte record (staged
        // in the column rows, written below as contiguous 16-byte chunks),
        // the pick key and the hit ids; a seed without one gets no record
        int4 *s_rec = reinterpret_cast<int4 *>(&s_col[0][0]);
        static_assert(!F || sizeof(s_col) >= 4 * T * sizeof(int4), "records fit the column rows");
        bool have = false;
        if (active) {
            const KeyIds b = s_best[tid];
            have = b.key != kNoKey;
            float lg = 0.f;
            if (have) lg = P.pick_chi2 ? unord_f32((unsigned)b.key) : unord_f32((unsigned)(b.key >> 32));
            if (have && P.pick_chi2 && !(lg < P.thr_logit)) have = false;
            int hid[4];
            int nh = 0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const unsigned q = (unsigned)(b.ids >> (16 * (3 - l))) & 0xFFFFu;
                hid[l] = have && q != 0xFFFFu ? h0 + (int)q : -1;
                nh += hid[l] >= 0;
            }
            a.key_ws[s] = have ? b.key : kNoKey;
            a.hit_ws[s] = make_int4(hid[0], hid[1], hid[2], hid[3]);
            if (have) {
                const float4 fw = s_win[tid];
                const float4 sa = s_sa[tid];
                const float yr = fmaf(sa.w, g.z_ref - sa.x, sa.z);
                // ds_track: event, seed, hit[4], x, y, tx, ty, qop, chi2, ndof, nn, flags, n_candidates
                s_rec[4 * tid + 0] = make_int4(e, s, hid[0], hid[1]);
                s_rec[4 * tid + 1] = make_int4(hid[2], hid[3], __float_as_int(fw.x), __float_as_int(yr));
                s_rec[4 * tid + 2] = make_int4(__float_as_int(fw.y), __float_as_int(sa.w), __float_as_int(fw.z),
                                               __float_as_int(fw.w));
                s_rec[4 * tid + 3] = make_int4(nh - 1, __float_as_int(sigmoid_fast(lg)), 0, n_cand);
            }
        }
        s_base[tid] = have ? 1 : 0;
        __syncthreads();
        int4 *dst = reinterpret_cast<int4 *>(a.trk_ws + s_begin);
        for (int k = tid; k < 4 * (s_end - s_begin); k += T)
            if (s_base[k >> 2]) dst[k] = s_rec[k];
    }
    __syncthreads();   // shared state is reused by the next item; s_nx is visible
    }   // work items
}

cudaError_t init_search_attributes()
{
    // shared memory, not L1, limits residency: ask for the largest carveout
    const int smem = (int)(sizeof(uint16_t) * table_stride_for(kMaxSectors) + sizeof(float) * (kStageHitsMax + 4));
    int dev = 0, optin = 0;
    size_t static_max = 0;
    cudaError_t e = cudaSuccess;
    for (auto fn : {k_search<0, false>, k_search<1, false>, k_search<0, true>, k_search<1, true>}) {
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
        if (e == cudaSuccess && fa.sharedSizeBytes > static_max) static_max = fa.sharedSizeBytes;
    }
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((size_t)smem + static_max > (size_t)optin) return cudaErrorInvalidValue;
    for (auto fn : {k_search<0, false>, k_search<1, false>, k_search<0, true>, k_search<1, true>}) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return e;
}

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, Prof *prof)
{
    if (a.n_seeds <= 0) return cudaSuccess;
    // persistent: ctas_per_sm CTAs per SM pull work items from a queue
    if (a.group < 1 || a.ctas_per_sm < 1 || a.stage_hits < 0 || a.stage_hits > kStageHitsMax)
        return cudaErrorInvalidValue;
    const int items_max = a.n_seeds + a.n_events;
    int grid = a.sm_count * a.ctas_per_sm;
    if (grid > items_max) grid = items_max;
    const size_t smem = sizeof(uint16_t) * a.g.table_stride + sizeof(float) * (a.stage_hits + 4);
    prof->begin("k_search", st);
    if (a.fused) {
        if (a.p.variant == 1) k_search<1, true><<<grid, T, smem, st>>>(a);
        else k_search<0, true><<<grid, T, smem, st>>>(a);
    } else {
        if (a.p.variant == 1) k_search<1, false><<<grid, T, smem, st>>>(a);
        else k_search<0, false><<<grid, T, smem, st>>>(a);
    }
    prof->end(st);
    return cudaGetLastError();
}

}  // namespace ds
