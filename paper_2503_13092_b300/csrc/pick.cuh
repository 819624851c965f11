// a7 (best pick + ghost cut) for one warp of 32 consecutive seeds, as used by
// the per-event pick + clone kernel (k_clone.cu).
//
// Ghost-Killer Neural Network and Ghost Rejection sections: the best
// candidate of a seed is the one with the lowest network output before the
// sigmoid (the same order as the response) among those under the threshold
// (response < 0.5); chi2 then breaks ties, then the hit ids in layer order
// (absent last).  In chi2 mode the lowest chi2/ndof wins and the cut is
// applied to the winner (Algorithm Design section: score from the distance
// between expected and real hit positions).
//
// The warp's candidates (each seed's are contiguous) are read 32 at a time,
// one per lane, the warp's prefix of the seeds' counts mapping a lane to its
// candidate; a segmented minimum over the lanes of one seed (contiguous
// lanes) leaves each run's best key in its first lane, which the seed's lane
// merges into its running best.
#pragma once

#include "ds_args.cuh"

namespace ds {

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
static __device__ __noinline__ bool hits_less_ool(const CandMeta *x, const CandMeta *y) { return hits_less(x, y); }

// One seed's pick: its key (kNoKey when it has no winner), its hit ids and,
// for a winner, its 64-byte ds_track record as four int4.
struct SeedPick {
    unsigned long long key;
    int4 hits;
    int4 rec[4];
};

// Called by all 32 lanes of a warp; lane l picks seed s (valid: s is one of
// the batch's seeds).  Reads seed_cand, the candidates' outputs and records.
__device__ __forceinline__ SeedPick warp_pick(const PickArgs &a, int s, bool valid)
{
    const int lane = threadIdx.x & 31;
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
    SeedPick out;
    out.key = kNoKey;
    out.hits = make_int4(-1, -1, -1, -1);
    out.rec[0] = make_int4(sc.z, s, -1, -1);
    out.rec[1] = make_int4(-1, -1, 0, 0);
    out.rec[2] = make_int4(0, 0, 0, 0);
    out.rec[3] = make_int4(0, 0, 0, sc.y);
    if (valid && best != kNoKey) {
        const float lg_best = P.pick_chi2 ? unord_f32((unsigned)best) : unord_f32((unsigned)(best >> 32));
        if (!P.pick_chi2 || lg_best < thr) {
            const float4 *mp = reinterpret_cast<const float4 *>(a.meta + bi);
            const float4 m0 = __ldg(mp), m1 = __ldg(mp + 1);
            const int4 mh = __ldg(reinterpret_cast<const int4 *>(mp + 2));
            out.key = best;
            out.hits = mh;
            // ds_track: event, seed, hit[4], x, y, tx, ty, qop, chi2, ndof, nn, flags, n_candidates
            out.rec[0] = make_int4(sc.z, s, mh.x, mh.y);
            out.rec[1] = make_int4(mh.z, mh.w, __float_as_int(m0.x), __float_as_int(m0.y));
            out.rec[2] = make_int4(__float_as_int(m0.z), __float_as_int(m1.w), __float_as_int(m0.w),
                                   __float_as_int(m1.x));
            out.rec[3] = make_int4(__float_as_int(m1.y), __float_as_int(sigmoid_fast(lg_best)), 0, sc.y);
        }
    }
    return out;
}

}  // namespace ds
