"""Exact pins of the oracle's selection rules (Algorithm Design section, Dv0
and Dv1): which hits a window keeps, not only how many.

- Crowded tiny events (more qualifying hits per layer than are kept, exact
  distance ties from duplicated hits, strips that miss the predicted y, finite
  windows): the oracle's kept UTbX count, its candidate set and its winner must
  equal tests/brute.seed_select, a Python restatement of the rules (|dx|
  strictly inside the window, strip extent widened by dy_tol containing y,
  ranking by (|dx|, hit id), k1 / 1 / 2 / 2 kept; Dv1 triplets ranked by
  (residual, UTbX id)).
- Hand-built events whose predictions are exact in binary floating point
  (zero field, a seed with zero slopes, axial-only geometry), with the kept
  hits written out by hand: hits exactly on a window edge are out, strips
  exactly on the y edge are in, ties go to the lower hit id, and distances are
  absolute.
- The paper's printed constants (tests/golden/paper_constants.json) against
  the configuration every test and the library use.
CPU only.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))


# ------------------------------------------------------------------ crowded events

def crowded_event(rng, seed, n_layer=(4, 6, 6, 14), variant=0):
    """One true seed with crowded UT layers, as the second event of a batch
    (the first holds only a few hits, so hit ids are not local indices)."""
    b = synth.generate(synth.spec_fixed(1, 2, 0, 8), seed)
    t = int(b["seed_track"][0])
    base = {l: int(np.nonzero((b["hit_track"] == t) & (b["hit_layer"] == l))[0][0]) for l in range(4)}
    qop = float(b["seed_qop"][0])
    w1 = 3.0 + 1.7e5 * abs(qop)
    W = synth.WORLD
    ty = float(b["seed_ty"][0])
    ym = float(b["seed_y"][0]) + ty * (W.z_kick - W.z_seed)
    x0, lo, hi, lay = [], [], [], []
    for l in range(4):
        h = base[l]
        yb, ye = float(b["hit_ybeg"][h]), float(b["hit_yend"][h])
        y_l = ym + ty * (W.z_layer[l] - W.z_kick)          # the seed's predicted y in this layer
        for k in range(n_layer[l]):
            if k == 0 and rng.uniform() < 0.85:
                dx = 0.0
            elif l == 3 and variant == 0:
                dx = rng.uniform(-1.3 * w1, 1.3 * w1)
            else:
                dx = rng.uniform(-3.0, 3.0)
            s_lo, s_hi = yb, ye
            if rng.uniform() < 0.15:       # a strip of the same sector that misses y (by > dy_tol)
                s_lo, s_hi = (yb, yb + 10.0) if y_l - yb > ye - y_l else (ye - 10.0, ye)
                assert not (s_lo - 2.0 <= y_l <= s_hi + 2.0)
            x0.append(float(b["hit_x0"][h]) + dx); lo.append(s_lo); hi.append(s_hi); lay.append(l)
            if rng.uniform() < 0.3:        # an exact duplicate: a distance tie, ranked by id
                x0.append(x0[-1]); lo.append(s_lo); hi.append(s_hi); lay.append(l)
    perm = rng.permutation(len(x0))
    pre = 5                                # first event: a few hits far from the seed
    x0 = np.concatenate([rng.uniform(-800, -700, pre), np.array(x0)[perm]]).astype(np.float32)
    lo = np.concatenate([np.full(pre, -700.0), np.array(lo)[perm]]).astype(np.float32)
    hi = np.concatenate([np.full(pre, -600.0), np.array(hi)[perm]]).astype(np.float32)
    lay = np.concatenate([np.arange(pre) % 4, np.array(lay)[perm]]).astype(np.uint8)
    ev = dict(n_events=2, seed_off=np.array([0, 0, 1], np.int32),
              hit_off=np.array([0, pre, len(x0)], np.int32),
              hit_x0=x0, hit_ybeg=lo, hit_yend=hi, hit_layer=lay)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2"):
        ev[k] = b[k][:1].copy()
    return ev


def _check_against_rules(ev, cfg, w, stats):
    kept, cands, best = brute.seed_select(ev, cfg, w, 0)
    ctx = brute._seed_ctx(ev, cfg, 0)
    r = oracle.reconstruct(ev, cfg, w)
    assert r["nbx"][0] == len(kept)
    oc = oracle.seed_candidates(ev, cfg, w, 0)
    assert oc["n"] == len(cands)
    got = {tuple(h): i for i, h in enumerate(oc["hits"].tolist())}
    assert sorted(got) == sorted(tuple(c["hits"]) for c in cands)
    for c in cands:
        i = got[tuple(c["hits"])]
        np.testing.assert_allclose(oc["state"][i], c["state"], rtol=1e-9, atol=1e-9)
        assert oc["chi2"][i] == pytest.approx(c["chi2"], rel=1e-8, abs=1e-10)
        np.testing.assert_allclose(oc["phi"][i], c["phi"], rtol=1e-8, atol=1e-9)
        assert oc["f"][i] == pytest.approx(c["f"], abs=1e-12)
    if best >= 0:
        assert r["status"][0] == 2 and r["hits"][0].tolist() == cands[best]["hits"]
    else:
        assert r["status"][0] == 0
    # how often each rule decided something (the test must exercise them)
    if int(cfg.get("variant", 0)) == 0:
        q = brute.closest(ev, cfg, ctx, 3, ctx["u_bx"], ctx["yl"][3], ctx["w1"], 1 << 30)
        stats["bx_over_k1"] += len(q) > cfg["k1"]
        stats["bx_tie_at_k1"] += len(q) > cfg["k1"] and q[cfg["k1"] - 1][0] == q[cfg["k1"]][0]
    for hb, _, _ in kept:
        for l, keep in ((0, 1), (1, 2), (2, 2)):
            q = brute.closest(ev, cfg, ctx, l, brute._x_at(ev, ctx, hb, l), ctx["yl"][l], ctx["w2"], 1 << 30)
            stats["refined_over_keep"] += len(q) > keep
            stats["refined_tie_at_keep"] += len(q) > keep and q[keep - 1][0] == q[keep][0]
    stats["winners"] += best >= 0


@pytest.mark.parametrize("mode,k1", [("nn", 10), ("chi2", 10), ("chi2", 4)])
def test_k_closest_selection_dv0(mode, k1):
    """Dv0 on crowded events: which UTbX hits are kept (k1 closest) and which
    refined-window hits (1 / 2 / 2 closest) equal the rules' restatement."""
    rng = np.random.default_rng({("nn", 10): 41, ("chi2", 10): 42, ("chi2", 4): 43}[(mode, k1)])
    w = synth.nn_weights(seed=5, out_bias=-0.5)
    over = dict(k1=k1)
    if mode == "chi2":
        over.update(pick_chi2=1, nn_threshold=0.9)
    else:
        over["nn_threshold"] = 0.7
    cfg = synth.default_config(**over)
    stats = dict(bx_over_k1=0, bx_tie_at_k1=0, refined_over_keep=0, refined_tie_at_keep=0, winners=0)
    for it in range(60):
        ev = crowded_event(rng, 500 + it, n_layer=(4, 6, 6, 14 if k1 == 10 else 8))
        _check_against_rules(ev, cfg, w, stats)
    assert stats["bx_over_k1"] >= 10 and stats["refined_over_keep"] >= 50, stats
    assert stats["refined_tie_at_keep"] >= 5 and stats["winners"] >= 20, stats


@pytest.mark.parametrize("k1", [3, 10])
def test_triplet_ranking_dv1(k1):
    """Dv1 on crowded events with several UTaX hits: triplets ranked by
    (residual, UTbX id), k1 kept, stereo windows as Dv0."""
    rng = np.random.default_rng(44 + k1)
    w = synth.nn_weights(seed=5, out_bias=-0.5)
    cfg = synth.default_config(variant=1, k1=k1, pick_chi2=1, nn_threshold=0.9)
    stats = dict(bx_over_k1=0, bx_tie_at_k1=0, refined_over_keep=0, refined_tie_at_keep=0, winners=0)
    n_over = 0
    for it in range(50):
        ev = crowded_event(rng, 700 + it, n_layer=(5, 5, 5, 12), variant=1)
        _check_against_rules(ev, cfg, w, stats)
        ctx = brute._seed_ctx(ev, cfg, 0)
        cfg_all = dict(cfg, k1=1 << 20)
        n_over += len(brute.first_stage(ev, cfg_all, ctx)) > k1
    assert stats["winners"] >= 15, stats
    if k1 == 3:
        assert n_over >= 10, n_over


# ------------------------------------------------------------- exact window edges

F32_AFTER_52 = float(np.nextafter(np.float32(52.0), np.float32(100.0)))
F32_JUST_INSIDE = float(np.float32(102.99998))      # |dx| just below 3 mm
F32_JUST_INSIDE2 = float(np.float32(101.99999))     # |dx| just below 2 mm


def edge_config(**over):
    """Zero field, axial-only geometry, fixed window half-widths: every
    prediction of a seed at x = 100 mm, y = 50 mm with zero slopes is exactly
    100 mm in every layer, and |dx| of a hit is computed without rounding."""
    kw = dict(kappa=0.0, dxdy=[0.0, 0.0, 0.0, 0.0], w1a=3.0, w1b=0.0, w2=2.0, dy_tol=2.0,
              pick_chi2=1, nn_threshold=2.0)
    kw.update(over)
    return synth.default_config(**kw)


def edge_event(layers):
    """One event, one seed (x = 100, y = 50, zero slopes, q/p = 1e-4): layers
    maps a layer to a list of (x0, ybeg, yend); ids follow the listing order
    (layer 0 first).  Strips lie inside the Y sector [0, 100) of y = 50."""
    x0, lo, hi, lay = [], [], [], []
    for l in sorted(layers):
        for x, a, b in layers[l]:
            x0.append(x); lo.append(a); hi.append(b); lay.append(l)
    ev = dict(n_events=1, seed_off=np.array([0, 1], np.int32), hit_off=np.array([0, len(x0)], np.int32),
              hit_x0=np.array(x0, np.float32), hit_ybeg=np.array(lo, np.float32),
              hit_yend=np.array(hi, np.float32), hit_layer=np.array(lay, np.uint8),
              seed_x=np.array([100.0], np.float32), seed_y=np.array([50.0], np.float32),
              seed_tx=np.zeros(1, np.float32), seed_ty=np.zeros(1, np.float32),
              seed_qop=np.array([1e-4], np.float32), seed_chi2=np.ones(1, np.float32))
    return ev


FULL = (0.0, 100.0)


def first_window_event():
    """UTbX hits around the prediction 100 (half-width 3): ids 2.. in order
    0: 100.0 in (0)          1: 103.0 out (on the edge)   2: 101.0 in, ybeg - dy = y
    3: 99.5 in (0.5)         4: 101.0 in, tie with 2      5: 99.0 strip misses y
    6: 100.25 in, yend + dy = y   7: 102.99998 in        8: 97.0 out (on the edge)
    9: 97.5 in (2.5; first by a signed distance).
    One UTaX and one UTaU hit at 100 complete a candidate for every kept hit."""
    return edge_event({
        0: [(100.0, *FULL)],
        1: [(100.0, *FULL)],
        3: [(100.0, *FULL), (103.0, *FULL), (101.0, 52.0, 100.0), (99.5, *FULL), (101.0, *FULL),
            (99.0, F32_AFTER_52, 100.0), (100.25, 0.0, 48.0), (F32_JUST_INSIDE, *FULL), (97.0, *FULL),
            (97.5, *FULL)],
    })


# hit ids of the UTbX hits above (two hits in UTaX / UTaU come first)
FIRST_WINDOW_KEPT = {4: [2, 8, 5, 4], 10: [2, 8, 5, 4, 6, 11, 9]}


def refined_window_event():
    """One UTbX hit at 100: the refined windows (half-width 2) are centred on 100.
    UTaX (keep 1): 0: 102.0 out (edge)  1: 101.0  2: 99.0 tie with 1  3: 100.5 strip misses
                   4: 98.5 (first by a signed distance)
    UTaU (keep 2): 5: 100.75  6: 99.25 tie with 5  7: 100.5 yend + dy = y  8: 98.0 out (edge)
                   9: 101.99999 in
    UTbV (keep 2): 10: 102.0 out (edge)  11: 98.0 out (edge)  12: 100.1 strip misses -> absent
    UTbX: 13: 100.0."""
    return edge_event({
        0: [(102.0, *FULL), (101.0, *FULL), (99.0, *FULL), (100.5, F32_AFTER_52, 100.0), (98.5, *FULL)],
        1: [(100.75, *FULL), (99.25, *FULL), (100.5, 0.0, 48.0), (98.0, *FULL), (F32_JUST_INSIDE2, *FULL)],
        2: [(102.0, *FULL), (98.0, *FULL), (100.1, F32_AFTER_52, 100.0)],
        3: [(100.0, *FULL)],
    })


REFINED_CANDIDATES = sorted([(1, 7, -1, 13), (1, 5, -1, 13)])


@pytest.mark.parametrize("k1", [4, 10])
def test_first_window_edges_ties_by_hand(k1):
    ev = first_window_event()
    cfg = edge_config(k1=k1, w2=10.0)
    w = synth.nn_weights()
    r = oracle.reconstruct(ev, cfg, w)
    oc = oracle.seed_candidates(ev, cfg, w, 0)
    kept = FIRST_WINDOW_KEPT[k1]
    assert r["nbx"][0] == len(kept)
    assert sorted(oc["hits"][:, 3].tolist()) == sorted(kept)
    assert all(h[:3] == [0, 1, -1] for h in oc["hits"].tolist())
    # the rules' restatement agrees, and in ranking order
    got, _, _ = brute.seed_select(ev, cfg, w, 0)
    assert [hb for hb, _, _ in got] == kept


def test_refined_window_edges_ties_by_hand():
    ev = refined_window_event()
    cfg = edge_config(k1=1)
    w = synth.nn_weights()
    oc = oracle.seed_candidates(ev, cfg, w, 0)
    assert sorted(tuple(h) for h in oc["hits"].tolist()) == REFINED_CANDIDATES
    _, cands, _ = brute.seed_select(ev, cfg, w, 0)
    assert sorted(tuple(c["hits"]) for c in cands) == REFINED_CANDIDATES


def test_edge_events_have_exact_predictions():
    """The hand-built expectations rely on predictions that are exactly 100 mm
    and window widths exactly 3 / 2 mm (no rounding anywhere)."""
    cfg = edge_config()
    p = oracle.seed_prediction(cfg, 100.0, 50.0, 0.0, 0.0, 1e-4)
    assert p["u_bx"] == 100.0 and p["w1"] == 3.0 and p["w2"] == 2.0 and p["xm"] == 100.0
    assert list(p["yl"]) == [50.0] * 4


# ---------------------------------------------------------------- paper constants

def test_eq3_constants_in_the_world_and_config():
    g = PAPER["gamma_eq3"]["value"]
    assert synth.WORLD.gamma0 == g["c0"] and synth.WORLD.gamma1 == g["c1"]
    cfg = synth.default_config(mode="B")
    assert cfg["gamma0"] == g["c0"] and cfg["gamma1"] == g["c1"]
    # Eq. 3: gamma = -MP (c0 + c1 q/p)
    qop = 2.5e-4
    assert oracle.gamma(cfg, qop) == pytest.approx(-cfg["mp"] * (g["c0"] + g["c1"] * qop), rel=1e-15)
    assert synth.default_config(mode="A")["gamma1"] == 0.0


def test_threshold_and_counts_in_the_config():
    cfg = synth.default_config()
    assert cfg["nn_threshold"] == PAPER["nn_threshold"]["value"]
    assert cfg["k1"] == PAPER["k1_utbx_hits"]["value"]
    assert list(cfg["dxdy"]) == pytest.approx([np.tan(np.radians(a)) for a in PAPER["ut_stereo_deg"]["value"]],
                                              abs=1e-15)


def test_library_defaults_are_paper_values():
    """The C ABI's default parameters (ds_default_params, host code only)."""
    from paper_2503_13092_b300 import build, ds
    build.build()
    p = ds.ds_default_params()
    assert p.nn_threshold == PAPER["nn_threshold"]["value"]
    assert p.k1 == PAPER["k1_utbx_hits"]["value"]
