"""GPU (libds.so through its C ABI) vs the FP64 oracle on the same seeded inputs.

Rules (tests/parity.py): identical hit assignments except for seeds whose
oracle decision margin is below 1e-5 (at most 0.1 % of tracks); FP32 track
parameters within 1e-4, chi2 within 1e-3, responses within 2e-5; vertices,
with the oracle fed the GPU's own track records, within 1 um.
"""
import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13092_b300 import build
    build.build()
    return torch


def make(torch_cuda, cfg, w, **over):
    from paper_2503_13092_b300 import ds
    return ds.Downstream(cfg, w, **over)


def run_both(dsx, b, cfg, w, n_threads=8, vtx=True):
    g = dsx.run(b)
    assert g["stats"]["status"] == 0, g["stats"]
    o = oracle.reconstruct(b, cfg, w, n_threads=n_threads)
    rep = parity.compare_tracks(b, o, g)
    vrep = parity.compare_vertices(cfg, g) if vtx else None
    return g, o, rep, vrep


@pytest.mark.parametrize("pick", ["nn", "chi2"])
def test_c1_parity(torch_cuda, weights, pick):
    b = synth.config_batch("c1")
    over = dict(pick_chi2=1, nn_threshold=0.9) if pick == "chi2" else {}
    cfg = synth.default_config(**over)
    d = make(torch_cuda, cfg, weights)
    g, o, rep, vrep = run_both(d, b, cfg, weights)
    assert rep["n_tracks_oracle"] > 20
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)
    # every candidate scored on the GPU is counted like the oracle's
    ok = o["margin"] >= parity.MARGIN
    assert g["stats"]["n_candidates"] == int(o["ncand"].sum()) or not ok.all()


@pytest.mark.parametrize("variant", ["origin", "training", "paper_net", "k1_3", "mode_b"])
def test_method_variants(torch_cuda, variant):
    over = {}
    w = synth.nn_weights()
    mode = "A"
    if variant == "origin":
        over = dict(first_window_origin=1, w1a=60.0)
    elif variant == "training":
        over = dict(training=1)
    elif variant == "paper_net":
        w = synth.nn_weights(8, 14, 0, seed=3)
    elif variant == "k1_3":
        over = dict(k1=3)
    elif variant == "mode_b":
        mode = "B"
    cfg = synth.default_config(mode=mode, **over)
    b = synth.config_batch("c2", n_events=12, mode=mode)
    d = make(torch_cuda, cfg, w)
    g, o, rep, vrep = run_both(d, b, cfg, w)
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)


def test_c2_sample_parity(torch_cuda, weights):
    b = synth.config_batch("c2", n_events=60)
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    g, o, rep, vrep = run_both(d, b, cfg, weights)
    assert rep["n_tracks_oracle"] > 5000
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)


@pytest.mark.parametrize("pick", ["nn", "chi2"])
def test_duplicated_hits(torch_cuda, weights, pick):
    """Every hit of the C1 event twice (a second id, the same measurement, in a
    seeded order): every window holds exact distance ties, ordered by hit id;
    wide first windows tie at the k1 boundary (the warp selection falls back to
    the exact sort); duplicated candidates have equal keys and the pick takes
    the lower hit ids.  GPU and oracle must choose the same hits seed by seed,
    with no margin excuse."""
    b = synth.config_batch("c1")
    n = len(b["hit_x0"])
    order = np.random.default_rng(5).permutation(2 * n)
    b2 = dict(b)
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        b2[k] = np.concatenate([b[k], b[k]])[order]
    b2["hit_off"] = np.array([0, 2 * n], np.int32)
    over = dict(pick_chi2=1, nn_threshold=0.9) if pick == "chi2" else {}
    cfg = synth.default_config(**over)
    d = make(torch_cuda, cfg, weights)
    g = d.run(b2)
    assert g["stats"]["status"] == 0
    o = oracle.reconstruct(b2, cfg, weights, n_threads=8)
    gp = parity.gpu_per_seed(g, len(o["status"]))
    o_has = o["status"] == 2
    same = (o_has == gp["has"]) & (~o_has | np.all(o["hits"] == gp["hits"], axis=1))
    assert o_has.sum() > 20
    bad = np.nonzero(~same)[0]
    assert same.all(), [(int(q), o["hits"][q].tolist(), gp["hits"][q].tolist(), float(o["margin"][q])) for q in bad]


@pytest.mark.parametrize("training", [0, 1])
def test_partial_strips(torch_cuda, weights, training):
    """Strips shorter than their Y sector (in the even sectors only, half of
    their hits shortened by up to 40 mm at each end, midpoint kept inside): the
    per-hit strip test decides there, while rows whose strips all span the
    sector are decided as a whole.  Both must agree with the oracle."""
    b = synth.config_batch("c2", n_events=16)
    rng = np.random.default_rng(11)
    yb, ye = b["hit_ybeg"].astype(np.float64), b["hit_yend"].astype(np.float64)
    sector = np.floor((0.5 * (yb + ye) + 700.0) / 100.0).astype(int)
    cut = (sector % 2 == 0) & (rng.random(yb.size) < 0.5)
    b = dict(b)
    b["hit_ybeg"] = np.where(cut, yb + rng.uniform(0.0, 40.0, yb.size), yb).astype(np.float32)
    b["hit_yend"] = np.where(cut, ye - rng.uniform(0.0, 40.0, ye.size), ye).astype(np.float32)
    cfg = synth.default_config(training=training)
    d = make(torch_cuda, cfg, weights)
    g, o, rep, vrep = run_both(d, b, cfg, weights)
    assert rep["n_tracks_oracle"] > 500
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)
    # the shortened strips lost hits: fewer candidates than with full strips
    full = synth.config_batch("c2", n_events=16)
    assert g["stats"]["n_candidates"] < d.run(full)["stats"]["n_candidates"]


@pytest.mark.parametrize("name,n_events,n_sample", [("c2", 1000, 24), ("c3", 2000, 16), ("c3", None, 16)])
def test_full_size_sampled(torch_cuda, weights, name, n_events, n_sample):
    """The benchmark's launch (whole batch in one call); the oracle recomputes
    sampled events one by one (events are independent), including the largest.
    n_events None: the benchmark's own batch (c3: all 10000 events, seed 3)."""
    b = synth.config_batch(name, n_events=n_events) if n_events else synth.config_batch(name, seed=3)
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    g = d.run(b)
    assert g["stats"]["status"] == 0
    E = b["n_events"]
    ns = np.diff(b["seed_off"])
    rng = np.random.default_rng(7)
    ev = sorted(set(rng.choice(E, n_sample - 2, replace=False).tolist()) | {int(np.argmax(ns)), E - 1})
    sb = parity.sub_batch(b, ev)
    o = oracle.reconstruct(sb, cfg, weights, n_threads=8)
    # GPU output restricted to the sampled events, ids mapped into the sub-batch
    t = g["tracks"]
    sel = np.isin(t["event"], ev)
    seed_new = {int(s): k for k, s in enumerate(sb["_seed_map"])}
    hit_new = np.full(int(b["hit_off"][-1]), -1, np.int64)
    hit_new[sb["_hit_map"]] = np.arange(len(sb["_hit_map"]))
    tt = t[sel].copy()
    tt["seed"] = [seed_new[int(s)] for s in tt["seed"]]
    tt["event"] = [ev.index(int(e)) for e in tt["event"]]
    trk_off = np.zeros(len(ev) + 1, np.int32)
    trk_off[1:] = np.cumsum(np.bincount(tt["event"], minlength=len(ev)))
    sub = dict(tracks=tt, trk_off=trk_off)
    rep = parity.compare_tracks(sb, o, sub, hit_map_gpu=lambda h: hit_new[h])
    parity.assert_tracks_match(rep)
    # vertices of the sampled events: GPU records vs the oracle fed the same tracks
    v = g["vertices"]
    vsel = np.isin(v["event"], ev)
    first = {e: int(g["trk_off"][e]) for e in ev}
    new_first = {e: int(trk_off[k]) for k, e in enumerate(ev)}
    vv = v[vsel].copy()
    vv["i"] = [new_first[int(e)] + int(i) - first[int(e)] for e, i in zip(vv["event"], vv["i"])]
    vv["j"] = [new_first[int(e)] + int(j) - first[int(e)] for e, j in zip(vv["event"], vv["j"])]
    vv["event"] = [ev.index(int(e)) for e in vv["event"]]
    vtx_off = np.zeros(len(ev) + 1, np.int32)
    vtx_off[1:] = np.cumsum(np.bincount(vv["event"], minlength=len(ev)))
    vrep = parity.compare_vertices(cfg, dict(tracks=tt, trk_off=trk_off, vertices=vv, vtx_off=vtx_off))
    parity.assert_vertices_match(vrep)


def test_concurrent_contexts_match_single(torch_cuda, weights):
    """The bench's launch configuration: four contexts, each with its own
    stream, outputs and CUDA graph of the full c2 batch, replayed at the same
    time.  Every context's tracks and vertices equal one context alone, byte
    for byte (that result is checked against the oracle in
    test_full_size_sampled)."""
    from paper_2503_13092_b300 import ds
    torch = torch_cuda
    b = synth.config_batch("c2", n_events=1000)
    cfg = synth.default_config()
    ref = make(torch_cuda, cfg, weights).run(b)
    assert ref["stats"]["status"] == 0
    E, S, H = b["n_events"], int(b["seed_off"][-1]), int(b["hit_off"][-1])
    lanes = []     # every buffer a graph points at stays referenced here
    for _ in range(4):
        d = make(torch_cuda, cfg, weights)
        ds.ds_reserve(d.ctx, E, S, H)
        dev = d.to_device(b)
        d.run(b, dev=dev)                       # sizes the vertex workspace
        out = d.alloc_tracks(E, S)
        vout = d.alloc_vertices(E, 2 * ref["n_vertices"] + 4096)
        st = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            cs = torch.cuda.current_stream()
            d.reconstruct(dev, out, cs)
            d.vertex(out, vout, cs)
        lanes.append(dict(d=d, dev=dev, out=out, vout=vout, st=st, g=g))
    torch.cuda.synchronize()
    for _ in range(3):
        for ln in lanes:
            with torch.cuda.stream(ln["st"]):
                ln["g"].replay()
    torch.cuda.synchronize()
    for ln in lanes:
        assert ln["d"].sync(ln["st"])["status"] == 0
        r = ds.decode(ln["out"], ln["vout"])
        assert r["n_tracks"] == ref["n_tracks"] and r["n_vertices"] == ref["n_vertices"]
        assert r["tracks"].tobytes() == ref["tracks"].tobytes()
        assert r["vertices"].tobytes() == ref["vertices"].tobytes()
        assert np.array_equal(r["trk_off"], ref["trk_off"]) and np.array_equal(r["vtx_off"], ref["vtx_off"])
    for ln in lanes:
        del ln["g"]                              # graphs go before the buffers they point at


def test_edge_cases(torch_cuda, weights):
    from paper_2503_13092_b300 import ds
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    # empty batch
    empty = dict(n_events=0, seed_off=np.zeros(1, np.int32), hit_off=np.zeros(1, np.int32),
                 **{k: np.zeros(0, np.float32) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop",
                                                         "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend")},
                 hit_layer=np.zeros(0, np.uint8))
    g = d.run(empty)
    assert g["n_tracks"] == 0 and g["n_vertices"] == 0
    # events with no seeds, no hits, a single seed; ragged sizes
    b = synth.config_batch("c2", n_events=7)
    parts = [parity.sub_batch(b, [0])]
    nohit = parity.sub_batch(b, [1]); nohit["hit_off"][:] = 0
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        nohit[k] = nohit[k][:0]
    noseed = parity.sub_batch(b, [2]); noseed["seed_off"][:] = 0
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track"):
        noseed[k] = noseed[k][:0]
    one = parity.sub_batch(b, [3]); one["seed_off"][1] = 1
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track"):
        one[k] = one[k][:1]
    parts += [nohit, noseed, one, parity.sub_batch(b, [4, 5, 6])]
    mb = concat(parts)
    g, o, rep, vrep = run_both(d, mb, cfg, weights)
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)
    # determinism: a second run is bit-identical
    g2 = d.run(mb)
    assert g2["tracks"].tobytes() == g["tracks"].tobytes()
    assert g2["vertices"].tobytes() == g["vertices"].tobytes()
    # capacity: truncation is deterministic and flagged
    full = d.run(b)
    dev = d.to_device(b)
    out = d.alloc_tracks(b["n_events"], 100)
    d.reconstruct(dev, out)
    st = d.sync(raise_on_error=False)
    assert st["status"] == ds.DS_ERR_CAPACITY and st["device_flags"] & ds.DS_FLAG_TRACK_CAPACITY
    small = ds.decode(out)
    assert small["n_tracks"] == full["n_tracks"]
    assert small["tracks"].tobytes() == full["tracks"][:100].tobytes()


def test_candidate_buffer_overflow(torch_cuda, weights):
    """A candidate buffer too small for the batch (one slot per seed, about 1.5
    candidates per seed are found) is flagged; the seeds whose candidates were
    written keep exactly the tracks of an unconstrained run, the others get none.
    Clone killing is off, so a track does not depend on which other seeds of its
    event were dropped."""
    from paper_2503_13092_b300 import ds
    cfg = synth.default_config()
    b = synth.config_batch("c2", n_events=60)
    full = make(torch_cuda, cfg, weights, clone_kill=0).run(b)
    assert full["stats"]["status"] == 0
    d = make(torch_cuda, cfg, weights, clone_kill=0, cand_per_seed=1)
    dev = d.to_device(b)
    out = d.alloc_tracks(b["n_events"], int(b["seed_off"][-1]))
    d.reconstruct(dev, out)
    st = d.sync(raise_on_error=False)
    assert st["device_flags"] & ds.DS_FLAG_CAND_CAPACITY
    got = ds.decode(out)
    assert 0 < got["n_tracks"] < full["n_tracks"]
    ref = {int(t["seed"]): t.tobytes() for t in full["tracks"]}
    for t in got["tracks"]:
        assert ref[int(t["seed"])] == t.tobytes()


@pytest.mark.parametrize("variant", [0, 1])
def test_chunked_refined_windows(torch_cuda, weights, variant):
    """An item whose (seed, UTbX hit) pairs exceed what the search keeps per
    chunk (640): one event of 128 true seeds, each of whose UTbX hits gets 11
    companions within 1.5 mm on the same strip, so every seed keeps k1 = 10
    UTbX hits (Dv0; Dv1 keeps the triplets among them whose UTaX window holds
    a hit) and the event's single work item holds far more pairs than one
    chunk, processed in seed-aligned chunks.  Tracks must match the oracle
    seed by seed."""
    cfg = synth.default_config(variant=variant)
    b = synth.generate(synth.spec_fixed(1, 128, 0, 1500), 11)
    rng = np.random.Generator(np.random.PCG64(11))
    bx = np.flatnonzero((b["hit_layer"] == 3) & (b["hit_track"] >= 0))
    extra = np.repeat(bx, 11)
    n0 = len(b["hit_x0"])
    for k in ("hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        b[k] = np.concatenate([b[k], b[k][extra]])
    b["hit_track"][n0:] = -1
    b["hit_x0"] = np.concatenate([b["hit_x0"], (b["hit_x0"][extra] +
                                                rng.uniform(-1.5, 1.5, len(extra))).astype(np.float32)])
    b["hit_off"] = np.array([0, len(b["hit_x0"])], np.int32)
    assert int(b["seed_off"][-1]) == 128 and len(bx) >= 120
    d = make(torch_cuda, cfg, weights, cand_per_seed=40)
    g, o, rep, vrep = run_both(d, b, cfg, weights)
    assert g["stats"]["n_candidates"] > (1280 if variant == 0 else 700)
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(vrep)
    # the fused form (network and pick inside the search, 784 pairs per chunk)
    # chunks the same item too and must give the same records byte for byte
    gf = make(torch_cuda, cfg, weights, fuse_network=1).run(b)
    assert gf["stats"]["status"] == 0
    assert gf["tracks"].tobytes() == g["tracks"].tobytes()
    assert gf["vertices"].tobytes() == g["vertices"].tobytes()


def concat(parts):
    out = dict(n_events=sum(p["n_events"] for p in parts))
    so, ho = [np.zeros(1, np.int32)], [np.zeros(1, np.int32)]
    s_base = h_base = 0
    for p in parts:
        so.append(p["seed_off"][1:] + s_base); ho.append(p["hit_off"][1:] + h_base)
        s_base += int(p["seed_off"][-1]); h_base += int(p["hit_off"][-1])
    out["seed_off"] = np.concatenate(so).astype(np.int32)
    out["hit_off"] = np.concatenate(ho).astype(np.int32)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track", "hit_x0",
              "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        out[k] = np.concatenate([p[k] for p in parts])
    return out


def test_hit_permutation_and_host_path(torch_cuda, weights):
    """Input hit order does not change the GPU result; the host-buffer entry
    point returns what the device path returns."""
    from paper_2503_13092_b300 import ds
    b = synth.config_batch("c2", n_events=20)
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    g = d.run(b)
    rng = np.random.default_rng(3)
    bp = dict(b)
    perm = np.concatenate([h0 + rng.permutation(h1 - h0) for h0, h1 in zip(b["hit_off"][:-1], b["hit_off"][1:])])
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        bp[k] = b[k][perm]
    gp = d.run(bp)
    t, tp = g["tracks"], gp["tracks"]
    assert np.array_equal(t["seed"], tp["seed"])
    mapped = np.where(tp["hit"] >= 0, perm[np.maximum(tp["hit"], 0)], -1)
    assert np.array_equal(mapped, t["hit"])
    for k in ("x", "y", "tx", "ty", "qop", "chi2", "nn"):
        assert np.array_equal(t[k], tp[k])
    h = ds.ds_process_host(d.ctx, b, trk_capacity=int(b["seed_off"][-1]), vtx_capacity=200000)
    assert h["n_tracks"] == g["n_tracks"] and h["n_vertices"] == g["n_vertices"]
    assert h["tracks"][: h["n_tracks"]].tobytes() == g["tracks"].tobytes()
    assert h["vertices"][: h["n_vertices"]].tobytes() == g["vertices"].tobytes()


def test_malformed_input_is_flagged(torch_cuda, weights):
    """Bad layers and strips that cross sectors are flagged, not faulted on."""
    from paper_2503_13092_b300 import ds
    b = synth.config_batch("c2", n_events=3)
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    bad = dict(b)
    bad["hit_layer"] = b["hit_layer"].copy()
    bad["hit_layer"][5] = 9
    bad["hit_yend"] = b["hit_yend"].copy()
    bad["hit_yend"][6] += 250.0
    dev = d.to_device(bad)
    out = d.alloc_tracks(3, int(b["seed_off"][-1]))
    d.reconstruct(dev, out)
    st = d.sync(raise_on_error=False)
    assert st["status"] == ds.DS_ERR_DEVICE_FLAG
    assert st["device_flags"] & ds.DS_FLAG_BAD_LAYER and st["device_flags"] & ds.DS_FLAG_STRIP_SECTOR
    # flags are cleared by the read: a clean batch afterwards is clean
    g = d.run(b)
    assert g["stats"]["status"] == 0


def test_misaligned_outputs_are_refused(torch_cuda, weights):
    """Track and vertex records are written as 16-byte chunks: output buffers
    that are not 16-byte aligned are refused with DS_ERR_ARG before any launch,
    and the context stays usable."""
    from paper_2503_13092_b300 import ds
    torch = torch_cuda
    b = synth.config_batch("c2", n_events=2)
    d = make(torch_cuda, synth.default_config(), weights)
    dev = d.to_device(b)
    S = int(b["seed_off"][-1])
    out = d.alloc_tracks(2, S)
    raw = torch.zeros(S * 64 + 16, dtype=torch.uint8, device="cuda")
    bad = dict(out, tracks=raw[4:4 + S * 64].view(S, 64))
    with pytest.raises(ds.DSError) as ei:
        d.reconstruct(dev, bad)
    assert ei.value.status == ds.DS_ERR_ARG
    d.reconstruct(dev, out)
    vout = d.alloc_vertices(2, 4096)
    rawv = torch.zeros(4096 * 32 + 16, dtype=torch.uint8, device="cuda")
    badv = dict(vout, vertices=rawv[8:8 + 4096 * 32].view(4096, 32))
    with pytest.raises(ds.DSError) as ei:
        d.vertex(out, badv)
    assert ei.value.status == ds.DS_ERR_ARG
    d.vertex(out, vout)
    st = d.sync()
    assert st["status"] == 0 and st["n_tracks"] > 0


def test_bounded_wait_reports_timeout(torch_cuda, weights):
    """Failure detection without a GPU fault: the staging wait is made to run
    out (its barrier expects bytes nothing sends); the kernel gives up after a
    bounded number of polls, flags DS_FLAG_TIMEOUT, and the context stays usable."""
    from paper_2503_13092_b300 import ds
    b = synth.config_batch("c2", n_events=4)
    cfg = synth.default_config()
    d = make(torch_cuda, cfg, weights)
    d.set_params(fault_inject=1)
    dev = d.to_device(b)
    out = d.alloc_tracks(b["n_events"], int(b["seed_off"][-1]))
    d.reconstruct(dev, out)
    st = d.sync(raise_on_error=False)
    assert st["status"] == ds.DS_ERR_TIMEOUT and st["device_flags"] & ds.DS_FLAG_TIMEOUT
    d.set_params(fault_inject=0)
    g = d.run(b)
    assert g["stats"]["status"] == 0 and g["n_tracks"] > 0


@pytest.mark.parametrize("case", ["first_k4", "first_k10", "refined"])
def test_exact_window_edges(torch_cuda, case):
    """Hand-built events whose predictions and window widths are exact in
    binary floating point (tests/test_oracle_selection.py): the GPU's
    candidates must be exactly the hand-written sets, with no margin excuse
    (hits on a window edge out, strips on the y edge in, ties to the lower
    hit id, absolute distances)."""
    from tests import test_oracle_selection as sel
    w = synth.nn_weights()
    if case == "refined":
        ev, cfg = sel.refined_window_event(), sel.edge_config(k1=1)
        want = sel.REFINED_CANDIDATES
    else:
        k1 = 4 if case == "first_k4" else 10
        ev, cfg = sel.first_window_event(), sel.edge_config(k1=k1, w2=10.0)
        want = sorted((0, 1, -1, hb) for hb in sel.FIRST_WINDOW_KEPT[k1])
    from paper_2503_13092_b300 import ds
    for fuse in (0, 1):          # candidates through the buffer, then scored inside the search
        keep = not fuse
        d = make(torch_cuda, cfg, w, fuse_network=fuse)
        dev = d.to_device(ev)
        out = d.alloc_tracks(1, 4)
        d.reconstruct(dev, out)
        if keep:
            c = d.candidates(64)          # before the counters are cleared
            assert sorted(tuple(h) for h in c["hits"].tolist()) == want
        st = d.sync()
        assert st["status"] == 0 and st["n_candidates"] == len(want), st
        g = ds.decode(out)
        o = oracle.reconstruct(ev, cfg, w)
        gp = parity.gpu_per_seed(g, 1)
        assert gp["has"][0] == (o["status"][0] == 2) and gp["hits"][0].tolist() == o["hits"][0].tolist()
        d.close()


@pytest.mark.parametrize("variant,pick", [(0, "nn"), (0, "chi2"), (1, "nn"), (1, "chi2")])
def test_fused_equals_unfused(torch_cuda, weights, variant, pick):
    """The candidate buffer with the separate network and pick kernels
    (default) against the network and the pick inside the search kernel
    (fuse_network = 1): byte-identical track records, offsets and vertices."""
    b = synth.config_batch("c2", n_events=60)
    over = dict(pick_chi2=1, nn_threshold=0.9) if pick == "chi2" else {}
    cfg = synth.default_config(variant=variant, **over)
    d = make(torch_cuda, cfg, weights)
    g0 = d.run(b)
    d.set_params(fuse_network=1)
    g1 = d.run(b)
    assert g0["stats"]["status"] == 0 and g1["stats"]["status"] == 0
    assert g0["stats"]["n_candidates"] == g1["stats"]["n_candidates"]
    assert g0["n_tracks"] == g1["n_tracks"] > 1000
    assert g0["tracks"].tobytes() == g1["tracks"].tobytes()
    assert np.array_equal(g0["trk_off"], g1["trk_off"])
    assert g0["vertices"].tobytes() == g1["vertices"].tobytes()


@pytest.mark.parametrize("pick", ["nn", "chi2"])
def test_chi2_margin_study(torch_cuda, weights, pick):
    """How many differing seeds each reading of a chi2 comparison's margin
    excuses: the oracle's margins are taken with the chi2 gap scaled by 1e-2
    (a gap in units of the 1e-3 chi2 tolerance) and by 1 (a plain relative
    gap); the GPU-vs-oracle chi2 error on identical tracks is logged beside
    them.  The parity rule itself is the one every test uses."""
    b = synth.config_batch("c2", n_events=100)
    over = dict(pick_chi2=1, nn_threshold=0.9) if pick == "chi2" else {}
    cfg = synth.default_config(**over)
    d = make(torch_cuda, cfg, weights)
    g = d.run(b)
    o = oracle.reconstruct(b, cfg, weights, n_threads=8)
    rep = parity.compare_tracks(b, o, g)
    o1 = oracle.reconstruct(b, dict(cfg, chi2_margin_scale=1.0), weights, n_threads=8)
    assert np.array_equal(o1["hits"], o["hits"]) and np.array_equal(o1["status"], o["status"])
    rep1 = parity.compare_tracks(b, o1, g)
    parity.log_report("chi2_margin", dict(pick=pick, n_tracks_oracle=rep["n_tracks_oracle"], n_diff=rep["n_diff"],
                                          n_excused=rep["n_excused"], n_excused_scale1=rep1["n_excused"],
                                          unexcused_scale1=len(rep1["unexcused"]),
                                          max_rel_chi2=rep.get("max_rel_chi2"), rel_chi2_q=rep.get("rel_chi2_q")))
    parity.assert_tracks_match(rep)


def _vertex_only(torch_cuda, cfg, weights, sizes, seed):
    """Track records written directly (events of the given track counts, each
    track from one of a few common points so that many pairs are kept) and
    ds_vertex on them; returns the decoded GPU result."""
    from paper_2503_13092_b300 import ds
    rng = np.random.default_rng(seed)
    n = int(sum(sizes))
    t = np.zeros(n, ds.TRACK_DTYPE)
    t["event"] = np.repeat(np.arange(len(sizes)), sizes)
    t["seed"] = np.arange(n)
    t["hit"] = -1
    zr = cfg["z_ref"]
    k = 0
    for e, m in enumerate(sizes):
        pts = np.stack([rng.uniform(-30, 30, 12), rng.uniform(-30, 30, 12), rng.uniform(0, 2000, 12)], 1)
        for q in range(m):
            p = pts[rng.integers(12)]
            tx, ty = rng.uniform(-0.2, 0.2, 2)
            dz = zr - p[2]
            t["x"][k] = p[0] + tx * dz + rng.normal(0, 0.3)
            t["y"][k] = p[1] + ty * dz + rng.normal(0, 0.3)
            t["tx"][k], t["ty"][k] = tx, ty
            t["qop"][k] = rng.choice([-1.0, 1.0]) * rng.uniform(1e-5, 5e-4)
            k += 1
    t["ndof"] = 2
    trk_off = np.zeros(len(sizes) + 1, np.int32)
    trk_off[1:] = np.cumsum(sizes)
    d = make(torch_cuda, cfg, weights)
    dev = f"cuda:{d.device}"
    out = d.alloc_tracks(len(sizes), n)
    out["tracks"].copy_(torch_cuda.from_numpy(t.view(np.uint8).reshape(n, 64)).to(dev))
    out["trk_off"].copy_(torch_cuda.from_numpy(trk_off).to(dev))
    out["n_tracks"].fill_(n)
    from paper_2503_13092_b300.ds import ds_tracks, _ptr
    out["_struct"] = ds_tracks(_ptr(out["tracks"]), _ptr(out["trk_off"]), _ptr(out["n_tracks"]), n, len(sizes))
    vout = d.alloc_vertices(len(sizes), 1 << 22)
    d.vertex(out, vout)
    st = d.sync()
    g = ds.decode(out, vout)
    d.close()
    return g, st


def test_large_event_vertexing(torch_cuda, weights):
    """Events above the small launch's 512 tracks are vertexed as (event, pair
    segment) work items spread over the SMs: events of 513 to 4096 tracks (1
    to 64 segments each) between small ones; the vertices, in (event, i, j)
    order, equal the oracle vertexer fed the same track records."""
    cfg = synth.default_config()
    sizes = [3, 700, 40, 1500, 0, 513, 512, 2600, 1, 4096, 90]
    g, st = _vertex_only(torch_cuda, cfg, weights, sizes, seed=3)
    assert st["status"] == 0, st
    assert st["n_pairs"] == sum((np.sum(g["tracks"]["qop"][a:b] > 0) * np.sum(g["tracks"]["qop"][a:b] < 0))
                                for a, b in zip(g["trk_off"][:-1], g["trk_off"][1:]))
    assert g["n_vertices"] > 100000
    vrep = parity.compare_vertices(cfg, g)
    parity.assert_vertices_match(vrep)
