"""Search launch shape (ds_tuning) and the autotuner: outputs must not depend on
the tuning (bit-identical tracks and vertices), invalid tunings are refused,
and the autotuner leaves a valid tuning in the context."""
import numpy as np
import pytest

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


def mixed_batch():
    """C2 events and uneven C3 events (up to 30000 hits: staged and unstaged paths)."""
    b2 = synth.config_batch("c2", seed=4, n_events=40)
    b3 = synth.config_batch("c3", seed=3, n_events=300)
    big = np.argsort(np.diff(b3["hit_off"]))[-30:]
    small = np.arange(20)
    p3 = parity.sub_batch(b3, np.concatenate([small, np.sort(big)]))
    p2 = parity.sub_batch(b2, range(40))
    out = dict(n_events=p2["n_events"] + p3["n_events"], mode="A")
    out["seed_off"] = np.concatenate([p2["seed_off"], p2["seed_off"][-1] + p3["seed_off"][1:]]).astype(np.int32)
    out["hit_off"] = np.concatenate([p2["hit_off"], p2["hit_off"][-1] + p3["hit_off"][1:]]).astype(np.int32)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend",
              "hit_layer"):
        out[k] = np.concatenate([p2[k], p3[k]])
    return out


def run_with(d, ds, dev, tuning):
    ds.ds_set_tuning(d.ctx, tuning)
    out = d.alloc_tracks(dev["n_events"], dev["n_seeds"])
    d.reconstruct(dev, out)
    vout = d.alloc_vertices(dev["n_events"], 64 * dev["n_seeds"] + 4096)
    d.vertex(out, vout)
    st = d.sync()
    n_t, n_v = int(out["n_tracks"].cpu()[0]), int(vout["n_vertices"].cpu()[0])
    return (st, out["tracks"][:n_t].cpu().numpy().tobytes(), out["trk_off"].cpu().numpy().tobytes(),
            vout["vertices"][:n_v].cpu().numpy().tobytes(), vout["vtx_off"].cpu().numpy().tobytes())


def test_outputs_do_not_depend_on_tuning(torch_cuda, weights):
    from paper_2503_13092_b300 import ds
    b = mixed_batch()
    assert np.diff(b["hit_off"]).max() > 2 * 5120      # larger than the default staging buffer
    d = ds.Downstream(synth.default_config(), weights)
    dev = d.to_device(b)
    # search: chunk, CTAs per SM, group, staging; vertexing: CTAs per SM, one-event-per-CTA
    # track limit (2: every event with two or more tracks goes to the pair-segment items);
    # work-item order (0: equal chunks in event order, 1: full chunks, then remainders largest first)
    shapes = [(128, 4, 2, 5632, 4, 512, 0), (128, 5, 1, 5120, 4, 512, 1), (32, 1, 1, 0, 1, 64, 1),
              (64, 3, 8, 32768, 2, 128, 0), (1, 2, 16, 2048, 3, 256, 1), (96, 4, 4, 46080, 4, 2, 1),
              (100, 5, 1, 5120, 4, 512, 1), (128, 5, 1, 5120, 4, 512, 0)]
    ref = None
    for shape in shapes:
        t = ds.ds_tuning(*shape)
        r = run_with(d, ds, dev, t)
        assert r[0]["status"] == 0, (t.as_dict(), r[0])
        assert r[0]["n_tracks"] > 0
        if ref is None:
            ref = r
        else:
            assert r[1:] == ref[1:], t.as_dict()


def test_invalid_tuning_refused(torch_cuda, weights):
    from paper_2503_13092_b300 import ds
    d = ds.Downstream(synth.default_config(), weights)
    before = ds.ds_get_tuning(d.ctx).as_dict()
    for bad in [(0, 4, 2, 5632), (129, 4, 2, 5632), (128, 0, 2, 5632), (128, 9, 2, 5632), (128, 4, 0, 5632),
                (128, 4, 17, 5632), (128, 4, 2, -1), (128, 4, 2, 46081), (128, 4, 2, 5632, 0, 512),
                (128, 4, 2, 5632, 5, 512), (128, 4, 2, 5632, 4, 1), (128, 4, 2, 5632, 4, 513)]:
        with pytest.raises(ds.DSError):
            ds.ds_set_tuning(d.ctx, ds.ds_tuning(*bad))
    assert ds.ds_get_tuning(d.ctx).as_dict() == before


def test_autotune(torch_cuda, weights):
    from paper_2503_13092_b300 import ds
    b = mixed_batch()
    d = ds.Downstream(synth.default_config(), weights)
    dev = d.to_device(b)
    ref = run_with(d, ds, dev, ds.ds_tuning(128, 4, 2, 5632))
    out = d.alloc_tracks(dev["n_events"], dev["n_seeds"])
    best, entries = ds.ds_autotune(d.ctx, dev, out, reps=2)
    d.sync()
    # coordinate descent from the default: one measurement, then two sweeps over
    # 7 stage sizes, 4 chunks, 4 CTA counts, 4 groups, 4 vertex CTA counts, 4
    # vertex track limits and 2 work-item orders, each skipping the value
    # current when it is reached
    assert 1 + 2 * (6 + 3 * 5 + 1) <= len(entries) <= 1 + 2 * (7 + 4 * 5 + 2)
    assert all(ms > 0 for _, ms in entries)
    cur = ds.ds_get_tuning(d.ctx).as_dict()
    assert cur == best.as_dict()
    assert min(ms for t, ms in entries if t == cur) == min(ms for _, ms in entries)
    got = run_with(d, ds, dev, best)
    assert got[1:] == ref[1:]


def seed_count_batch(counts, seed=21):
    """One event per entry of `counts` (that many SciFi seeds, 40 % true,
    1500 UT hits), concatenated into one batch."""
    parts = []
    for k, n in enumerate(counts):
        nt = 2 * ((4 * n) // 20)
        parts.append(synth.generate(synth.spec_fixed(1, nt, n - nt, 1500), seed + k))
    out = dict(n_events=len(parts), mode="A")
    so, ho = [0], [0]
    for p in parts:
        so.append(so[-1] + int(p["seed_off"][-1]))
        ho.append(ho[-1] + int(p["hit_off"][-1]))
    out["seed_off"] = np.array(so, np.int32)
    out["hit_off"] = np.array(ho, np.int32)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track", "hit_x0",
              "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        out[k] = np.concatenate([p[k] for p in parts])
    return out


def test_work_item_orders_on_uneven_seed_counts(torch_cuda, weights):
    """Events with no seeds, fewer than a chunk, exactly one or two chunks and
    a chunk plus a remainder: equal chunks in event order (order 0) and full
    chunks then remainders largest first (order 1, chunks of 128 and 100
    seeds) give the same bytes, and those match the oracle."""
    import oracle
    from paper_2503_13092_b300 import ds
    counts = [0, 1, 127, 128, 129, 256, 300, 0, 77, 200]
    b = seed_count_batch(counts)
    assert np.diff(b["seed_off"]).tolist() == counts
    cfg = synth.default_config()
    d = ds.Downstream(cfg, weights)
    dev = d.to_device(b)
    ref = None
    for shape in [(128, 5, 1, 5120, 4, 512, 0), (128, 5, 1, 5120, 4, 512, 1), (100, 5, 1, 5120, 4, 512, 1)]:
        r = run_with(d, ds, dev, ds.ds_tuning(*shape))
        assert r[0]["status"] == 0, (shape, r[0])
        if ref is None:
            ref = r
        else:
            assert r[1:] == ref[1:], shape
    g = d.run(b, dev=dev)
    o = oracle.reconstruct(b, cfg, weights, n_threads=8)
    rep = parity.compare_tracks(b, o, g)
    assert rep["n_tracks_oracle"] > 0
    parity.assert_tracks_match(rep)


def test_vertex_event_order_is_scheduling_only(torch_cuda, weights):
    """ds_vertex takes its events in the order the last ds_reconstruct on its
    context laid out (largest first).  Vertices must not depend on it: after a
    ds_reserve that reallocates the workspaces between the two calls (the
    order is dropped), and for the tracks of another batch with the same
    event count (the order of the wrong batch is still a permutation of the
    events), the vertices equal those of a plain reconstruct + vertex."""
    from paper_2503_13092_b300 import ds
    cfg = synth.default_config()
    b1 = synth.config_batch("c2", seed=31, n_events=24)
    b2 = synth.config_batch("c2", seed=32, n_events=24)

    def plain(b):
        d = ds.Downstream(cfg, weights)
        r = run_with(d, ds, d.to_device(b), ds.ds_tuning())
        d.close()
        return r

    ref1, ref2 = plain(b1), plain(b2)
    d = ds.Downstream(cfg, weights)
    dev1, dev2 = d.to_device(b1), d.to_device(b2)
    # reconstruct, grow the workspaces, vertex
    out = d.alloc_tracks(dev1["n_events"], dev1["n_seeds"])
    d.reconstruct(dev1, out)
    ds.ds_reserve(d.ctx, 4 * dev1["n_events"] + 100, dev1["n_seeds"], dev1["n_hits"])
    vout = d.alloc_vertices(dev1["n_events"], 64 * dev1["n_seeds"] + 4096)
    d.vertex(out, vout)
    assert d.sync()["status"] == 0
    n_v = int(vout["n_vertices"].cpu()[0])
    assert vout["vertices"][:n_v].cpu().numpy().tobytes() == ref1[3]
    # batch 2's tracks vertexed right after batch 1's reconstruct (same event count)
    out2 = d.alloc_tracks(dev2["n_events"], dev2["n_seeds"])
    d.reconstruct(dev2, out2)
    d.reconstruct(dev1, out)
    vout2 = d.alloc_vertices(dev2["n_events"], 64 * dev2["n_seeds"] + 4096)
    d.vertex(out2, vout2)
    assert d.sync()["status"] == 0
    n_v2 = int(vout2["n_vertices"].cpu()[0])
    assert vout2["vertices"][:n_v2].cpu().numpy().tobytes() == ref2[3]
    assert vout2["vtx_off"].cpu().numpy().tobytes() == ref2[4]
    d.close()
