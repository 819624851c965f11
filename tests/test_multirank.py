"""Multi-rank host logic on the CPU: two processes over gloo (no GPU).

Ranks shard a batch into contiguous event ranges (events are independent),
reconstruct and vertex their own range, and rank 0 joins the records with
shard.merge: the joined result must equal the same computation on the whole
batch.  The FP64 oracle stands in for each rank's GPU here, so the test
checks the partition, the index shifts of the join and the max-over-ranks
timing that bench.py reports, not the kernels.
"""
import os
import socket

import numpy as np
import pytest

TRK = np.dtype([("event", "<i4"), ("seed", "<i4"), ("hit", "<i4", 4), ("x", "<f4"), ("y", "<f4"), ("tx", "<f4"),
                ("ty", "<f4"), ("qop", "<f4")])
VTX = np.dtype([("event", "<i4"), ("i", "<i4"), ("j", "<i4"), ("pos", "<f8", 3), ("doca", "<f8")])


def records(batch, cfg, w):
    """Oracle tracks and vertices of a batch in the library's record layout."""
    import oracle
    res = oracle.reconstruct(batch, cfg, w)
    t = oracle.tracks_from(res, batch["seed_off"])
    trk = np.zeros(len(t["seed"]), TRK)
    trk["event"], trk["seed"], trk["hit"] = t["event"], t["seed"], t["hits"]
    for k, c in zip(("x", "y", "tx", "ty", "qop"), range(5)):
        trk[k] = t["state"][:, c]
    v = oracle.vertex(cfg, t["trk_off"], trk["x"], trk["y"], trk["tx"], trk["ty"], trk["qop"])
    vtx = np.zeros(len(v["i"]), VTX)
    vtx["event"], vtx["i"], vtx["j"], vtx["pos"], vtx["doca"] = v["event"], v["i"], v["j"], v["pos"], v["doca"]
    E = int(batch["n_events"])
    vtx_off = np.zeros(E + 1, np.int64)
    vtx_off[1:] = np.cumsum(np.bincount(vtx["event"], minlength=E))
    return dict(tracks=trk, trk_off=t["trk_off"], vertices=vtx, vtx_off=vtx_off)


def _worker(rank, world, port, n_events, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2503_13092_b300 import shard, synth
    t = bench.max_over_ranks(0.25 * (rank + 1))
    b = synth.config_batch("c2", seed=6, n_events=n_events)
    part, off = shard.shard(b, rank, world)
    res = records(part, synth.default_config(), synth.nn_weights())
    parts = [None] * world
    dist.all_gather_object(parts, (off, res))
    if rank == 0:
        q.put((t, bench.aggregate([t] * world, part["n_events"], 3), shard.merge(parts)))
    dist.barrier()
    dist.destroy_process_group()


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,n_events", [(2, 7), (3, 2)])
def test_sharded_equals_whole_batch(world, n_events):
    import torch.multiprocessing as mp
    from paper_2503_13092_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_events, q)) for r in range(world)]
    for p in procs:
        p.start()
    t, agg, merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == pytest.approx(0.25 * world)            # the slowest rank's time
    assert agg["ms_per_step"] == pytest.approx(1e3 * t / 3)
    whole = records(synth.config_batch("c2", seed=6, n_events=n_events), synth.default_config(), synth.nn_weights())
    assert merged["tracks"].tobytes() == whole["tracks"].tobytes()
    assert merged["vertices"].tobytes() == whole["vertices"].tobytes()
    assert np.array_equal(merged["trk_off"], whole["trk_off"])
    assert np.array_equal(merged["vtx_off"], whole["vtx_off"])


def test_partition():
    from paper_2503_13092_b300 import shard
    for n in (0, 1, 7, 1000):
        for w in (1, 2, 3, 8):
            p = shard.partition(n, w)
            assert p[0][0] == 0 and p[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
            sizes = [e1 - e0 for e0, e1 in p]
            assert max(sizes) - min(sizes) <= 1
