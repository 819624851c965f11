"""Serving loop (include/ds_serve.h): every request's tracks and vertices are
the same alone and in a mix of concurrent, continuously batched requests
(bit for bit: events are independent), and equal to ds_reconstruct +
ds_vertex on the request as its own batch; the plain one-event-per-launch
form gives the same results; admission respects the device-memory budget."""
import time

import numpy as np
import pytest

from paper_2503_13092_b300 import synth

pytestmark = pytest.mark.gpu

MAX_EVENTS = 60


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13092_b300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def pool():
    return synth.c5_pool(400, seed=5)


def make_requests(pool, n, seed=7, max_events=MAX_EVENTS):
    sizes, starts, _ = synth.c5_trace(n, 1000.0, pool["n_events"], seed=seed, max_events=max_events)
    return [synth.slice_events(pool, int(s), int(s + k)) for k, s in zip(sizes, starts)]


def server(torch_cuda, weights, **config):
    from paper_2503_13092_b300 import ds
    base = dict(n_slots=4, max_batch_events=256, max_batch_seeds=256 * 200, max_batch_hits=256 * 1500)
    base.update(config)
    return ds.Server(synth.default_config(), weights, **base)


def collect(srv, n, timeout=60.0):
    got, t_end = {}, time.time() + timeout
    while len(got) < n and time.time() < t_end:
        for c in srv.poll(timeout=0.5):
            got[c["id"]] = c
    assert len(got) == n, (len(got), n)
    return got


def key(c):
    return (c["tracks"].tobytes(), c["trk_off"].tobytes(), c["vertices"].tobytes(), c["vtx_off"].tobytes())


def run_alone(srv, reqs):
    out = []
    for r in reqs:
        rid = srv.submit(r)
        (c,) = collect(srv, 1).values()
        assert c["id"] == rid and c["status"] == 0, c
        out.append(c)
    return out


def test_alone_equals_mix_and_library_path(torch_cuda, weights, pool):
    from paper_2503_13092_b300 import ds
    reqs = make_requests(pool, 40)
    srv = server(torch_cuda, weights)
    alone = run_alone(srv, reqs)
    ids = [srv.submit(r) for r in reqs]
    got = collect(srv, len(reqs))
    st = srv.stats()
    for rid, a, r in zip(ids, alone, reqs):
        c = got[rid]
        assert c["status"] == 0, c
        assert key(c) == key(a), rid
        assert c["trk_off"][-1] == c["n_tracks"] and c["vtx_off"][-1] == c["n_vertices"]
    assert st["batches"] < 2 * len(reqs)       # the mix was batched: fewer launches than requests
    assert st["peak_inflight"] >= 2             # and batches overlapped on the device
    # the library path on the request as its own batch gives the same records
    d = ds.Downstream(synth.default_config(), weights)
    for a, r in list(zip(alone, reqs))[:8]:
        g = d.run(r)
        assert g["tracks"].tobytes() == a["tracks"].tobytes()
        assert g["vertices"].tobytes() == a["vertices"].tobytes()
        assert np.array_equal(g["trk_off"], a["trk_off"]) and np.array_equal(g["vtx_off"], a["vtx_off"])
    srv.close()


def test_plain_form_same_results(torch_cuda, weights, pool):
    reqs = make_requests(pool, 6, seed=8, max_events=12)
    srv = server(torch_cuda, weights)
    alone = run_alone(srv, reqs)
    srv.close()
    plain = server(torch_cuda, weights, n_slots=1, events_per_launch=1)
    ids = [plain.submit(r) for r in reqs]
    got = collect(plain, len(reqs))
    for rid, a, r in zip(ids, alone, reqs):
        assert key(got[rid]) == key(a)
        assert got[rid]["n_batches"] == r["n_events"]    # one launch per event
    plain.close()


def test_admission_by_device_memory(torch_cuda, weights, pool):
    # requests of 50 events, one per batch; the budget holds one batch, not two
    reqs = [synth.slice_events(pool, 50 * k, 50 * k + 50) for k in range(6)]
    S, H = int(reqs[0]["seed_off"][-1]), int(reqs[0]["hit_off"][-1])
    vcap = 16 * S + 4096
    one = 4 * (51 * 2 + 6 * S + 3 * H) + H + 64 * S + 4 * 52 + 32 * vcap + 4 * 52 + 4096   # above the buffers of one
    srv = server(torch_cuda, weights, max_batch_events=50, hbm_budget=int(1.5 * one))
    ids = [srv.submit(r) for r in reqs]
    got = collect(srv, len(reqs))
    st = srv.stats()
    assert all(got[i]["status"] == 0 for i in ids)
    assert st["peak_inflight"] == 1 and st["hbm_peak"] <= st["hbm_budget"]
    assert st["graphs"] == 0          # the slots' fixed buffers do not fit this budget
    srv.close()


def test_request_errors_and_timing_fields(torch_cuda, weights, pool):
    from paper_2503_13092_b300 import ds
    srv = server(torch_cuda, weights, max_batch_hits=1000)
    with pytest.raises(ds.DSError):              # one event holds more hits than a batch
        srv.submit(synth.slice_events(pool, 0, 1))
    srv.close()
    srv = server(torch_cuda, weights)
    empty = synth.slice_events(pool, 3, 3)
    rid = srv.submit(empty)
    (c,) = collect(srv, 1).values()
    assert c["id"] == rid and c["status"] == 0 and c["n_tracks"] == 0
    t = srv.now() + 0.05
    rid = srv.submit(synth.slice_events(pool, 0, 5), arrival=t)
    (c,) = collect(srv, 1).values()
    assert c["t_arrival"] == pytest.approx(t) and c["t_admit"] >= t and c["t_done"] >= c["t_admit"]
    srv.close()


@pytest.mark.parametrize("split", [False, True])
def test_served_mix_matches_oracle(torch_cuda, weights, pool, split):
    """Every request of a concurrent, continuously batched mix against the
    FP64 oracle run on that request alone, under the parity rules (tracks:
    identical hits except within the decision margin, parameters to 1e-4,
    chi2 to 1e-3; vertices: the oracle vertexer fed the served tracks, to
    1 um).  split: batches of at most 7 events, so that requests are cut into
    segments and renumbered back."""
    import oracle
    from tests import parity
    reqs = make_requests(pool, 12, seed=9, max_events=20)
    cfg = synth.default_config()
    over = dict(max_batch_events=7) if split else {}
    srv = server(torch_cuda, weights, **over)
    ids = [srv.submit(r) for r in reqs]
    got = collect(srv, len(reqs))
    srv.close()
    if split:
        assert any(got[i]["n_batches"] > 1 for i in ids)
    for rid, r in zip(ids, reqs):
        c = got[rid]
        assert c["status"] == 0, c
        o = oracle.reconstruct(r, cfg, weights, n_threads=8)
        g = dict(tracks=c["tracks"], trk_off=c["trk_off"], vertices=c["vertices"], vtx_off=c["vtx_off"])
        parity.assert_tracks_match(parity.compare_tracks(r, o, g))
        parity.assert_vertices_match(parity.compare_vertices(cfg, g))


def test_graph_replay_equals_launches(torch_cuda, weights, pool):
    """Graph mode (each batch one replay of a graph captured per slot and
    event-count bucket, batches padded with empty events) against kernels
    launched batch by batch: identical records for a mix that spans several
    buckets, split requests included."""
    reqs = make_requests(pool, 30, seed=10, max_events=40)
    res = {}
    for graphs in (1, 0):
        srv = server(torch_cuda, weights, graphs=graphs, max_batch_events=64)
        ids = [srv.submit(r) for r in reqs]
        got = collect(srv, len(reqs))
        st = srv.stats()
        srv.close()
        assert st["graphs"] == graphs
        if graphs:
            assert st["graphs_captured"] == 4 * 7        # 4 slots x buckets 1, 2, 4, ..., 64
        assert all(got[i]["status"] == 0 for i in ids)
        res[graphs] = [key(got[i]) for i in ids]
    assert res[1] == res[0]


def test_gathered_inputs_equal_copies(torch_cuda, weights, pool):
    """Inputs read from pinned host memory by the gather kernel against
    inputs uploaded by cudaMemcpyAsync: identical records.  Pinned requests
    are slices of a pinned pool starting at any event (hit layers at any byte
    offset, so every source alignment occurs); pageable requests are copied
    whatever gather_max_bytes says; split requests and requests larger than
    the gather limit are in the mix."""
    torch = torch_cuda
    pinned = dict(pool)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend",
              "hit_layer"):
        pinned[k] = torch.from_numpy(np.ascontiguousarray(pool[k])).pin_memory().numpy()
    sizes, starts, _ = synth.c5_trace(36, 1000.0, pool["n_events"], seed=12, max_events=120)
    reqs = [synth.slice_events(pinned if i % 3 else pool, int(s), int(s + k))
            for i, (k, s) in enumerate(zip(sizes, starts))]
    pageable_bytes = sum(24 * int(r["seed_off"][-1]) + 13 * int(r["hit_off"][-1]) for i, r in enumerate(reqs)
                         if i % 3 == 0)
    total_bytes = sum(24 * int(r["seed_off"][-1]) + 13 * int(r["hit_off"][-1]) for r in reqs)
    res, stats = {}, {}
    for gmax in (0, 1 << 17, 1 << 30):
        srv = server(torch_cuda, weights, gather_max_bytes=gmax, max_batch_events=64)
        ids = [srv.submit(r) for r in reqs]
        got = collect(srv, len(reqs))
        stats[gmax] = srv.stats()
        srv.close()
        assert all(got[i]["status"] == 0 for i in ids)
        res[gmax] = [key(got[i]) for i in ids]
    assert res[1 << 17] == res[0] and res[1 << 30] == res[0]
    assert stats[0]["bytes_gathered"] == 0
    assert 0 < stats[1 << 17]["bytes_gathered"] and stats[1 << 17]["bytes_copied"] > pageable_bytes
    # every pinned request array gathered; pageable ones (and nothing else) copied
    assert stats[1 << 30]["bytes_copied"] == pageable_bytes
    assert stats[1 << 30]["bytes_gathered"] >= total_bytes - pageable_bytes
