"""Event sharding over several GPUs (one process per GPU).

Events are independent (the paper processes them in parallel, GPU
Implementation section), so a batch is cut into contiguous event ranges, one
per rank, each rank runs ds_reconstruct + ds_vertex on its own GPU with no
exchange between ranks, and the per-rank outputs are joined on the host by
shifting their event, seed, hit and track indices.  No collective is on the
data path; the join only moves the finished records.
"""
import numpy as np

from .synth import slice_events


def partition(n_events: int, world: int) -> list:
    """Contiguous event ranges [e0, e1) for each rank, sizes differing by one at most."""
    if world < 1 or n_events < 0:
        raise ValueError("world >= 1 and n_events >= 0")
    return [(r * n_events // world, (r + 1) * n_events // world) for r in range(world)]


def shard(batch: dict, rank: int, world: int) -> tuple:
    """This rank's events as a batch of their own, and its (event, seed, hit) offsets in the full batch."""
    e0, e1 = partition(int(batch["n_events"]), world)[rank]
    part = slice_events(batch, e0, e1)
    return part, (e0, int(batch["seed_off"][e0]), int(batch["hit_off"][e0]))


def merge(parts: list) -> dict:
    """Join per-rank results in rank order.  parts: [(offsets, result)] with
    offsets = (first event, first seed, first hit) of the rank's range and
    result = {tracks, trk_off, vertices, vtx_off} in the rank's own numbering
    (tracks with fields event, seed, hit; vertices with event, i, j)."""
    trk, vtx, trk_off, vtx_off = [], [], [np.zeros(1, np.int64)], [np.zeros(1, np.int64)]
    n_t = n_v = 0
    for (e0, s0, h0), res in parts:
        t = np.array(res["tracks"], copy=True)
        t["event"] += e0
        t["seed"] += s0
        h = t["hit"]
        t["hit"] = np.where(h >= 0, h + h0, h)
        v = np.array(res["vertices"], copy=True)
        v["event"] += e0
        v["i"] += n_t
        v["j"] += n_t
        trk.append(t)
        vtx.append(v)
        trk_off.append(np.asarray(res["trk_off"][1:], np.int64) + n_t)
        vtx_off.append(np.asarray(res["vtx_off"][1:], np.int64) + n_v)
        n_t += len(t)
        n_v += len(v)
    return dict(tracks=np.concatenate(trk) if trk else np.zeros(0),
                vertices=np.concatenate(vtx) if vtx else np.zeros(0),
                trk_off=np.concatenate(trk_off), vtx_off=np.concatenate(vtx_off))
