"""Python binding of libds.so (ctypes).  Argument marshalling only.

The functions keep the C names of include/ds.h (ds_create, ds_load_geometry,
ds_load_nn_weights, ds_set_params, ds_reserve, ds_reconstruct, ds_vertex,
ds_sync_status, ds_process_host, ...).  Every step of the computation runs in
the CUDA kernels of libds.so; PyTorch only provides device memory and streams.
There is no fallback: if the library is missing or no CUDA device is present
the calls raise.

`Downstream` is a small convenience wrapper (one context, device-resident
geometry and weights) used by the tests, the benchmark and the server.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libds.so")

DS_OK, DS_ERR_ARG, DS_ERR_CUDA, DS_ERR_CAPACITY, DS_ERR_NOT_READY, DS_ERR_TIMEOUT, \
    DS_ERR_DEVICE_FLAG, DS_ERR_OOM = 0, -1, -2, -3, -4, -5, -6, -7
DS_FLAG_BAD_OFFSETS, DS_FLAG_BAD_LAYER, DS_FLAG_STRIP_SECTOR, DS_FLAG_EVENT_TOO_LARGE, \
    DS_FLAG_TRACK_CAPACITY, DS_FLAG_VERTEX_CAPACITY, DS_FLAG_TIMEOUT, DS_FLAG_CAND_CAPACITY = (1 << k for k in range(8))
DS_MLP_FP32, DS_MLP_BF16, DS_MLP_FP8 = 0, 1, 2


class ds_geometry(C.Structure):
    _fields_ = [("z_layer", C.c_double * 4), ("dxdy", C.c_double * 4), ("y_min", C.c_double),
                ("sector_h", C.c_double), ("n_sectors", C.c_int32), ("reserved0", C.c_int32),
                ("x_half_bins", C.c_double), ("z_seed", C.c_double), ("zmag", C.c_double * 4),
                ("kappa", C.c_double), ("mp", C.c_double), ("gamma0", C.c_double), ("gamma1", C.c_double),
                ("z_ref", C.c_double), ("sigma_hit", C.c_double), ("sigma_mag", C.c_double)]


class ds_nn_weights(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_h1", C.c_int32), ("n_h2", C.c_int32), ("reserved0", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_float), ("reserved1", C.c_int32),
                ("mean", C.c_void_p), ("scale", C.c_void_p)]


class ds_params(C.Structure):
    _fields_ = [("w1a", C.c_double), ("w1b", C.c_double), ("w2", C.c_double), ("dy_tol", C.c_double),
                ("nn_threshold", C.c_double), ("doca_max", C.c_double), ("nr_tol", C.c_double),
                ("eps_parallel", C.c_double), ("k1", C.c_int32), ("first_window_origin", C.c_int32),
                ("pick_chi2", C.c_int32), ("clone_kill", C.c_int32), ("training", C.c_int32),
                ("nr_max_iter", C.c_int32), ("mlp_precision", C.c_int32), ("fault_inject", C.c_int32),
                ("cand_per_seed", C.c_int32), ("variant", C.c_int32), ("dv1_dtx_max", C.c_double),
                ("dv1_w_tri", C.c_double), ("fuse_network", C.c_int32), ("reserved2", C.c_int32)]


class ds_event_batch(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_seeds", C.c_int32), ("n_hits", C.c_int32),
                ("flags", C.c_int32), ("seed_off", C.c_void_p), ("hit_off", C.c_void_p)]


class ds_seeds(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "y", "tx", "ty", "qop", "chi2")]


class ds_ut_hits(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x0", "ybeg", "yend", "layer")]


class ds_tracks(C.Structure):
    _fields_ = [("tracks", C.c_void_p), ("trk_off", C.c_void_p), ("n_tracks", C.c_void_p),
                ("capacity", C.c_int32), ("n_events", C.c_int32)]


class ds_vertices(C.Structure):
    _fields_ = [("vertices", C.c_void_p), ("vtx_off", C.c_void_p), ("n_vertices", C.c_void_p),
                ("capacity", C.c_int32), ("reserved0", C.c_int32)]


class ds_stats(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_pairs", C.c_int64), ("n_pairs_fp64", C.c_int64),
                ("n_tracks", C.c_int32), ("n_vertices", C.c_int32), ("device_flags", C.c_uint32),
                ("reserved0", C.c_int32)]


class ds_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int32), ("reserved0", C.c_int32),
                ("total_ms", C.c_double)]


class ds_tuning(C.Structure):
    _fields_ = [("search_chunk", C.c_int32), ("search_ctas_per_sm", C.c_int32), ("search_group", C.c_int32),
                ("search_stage_hits", C.c_int32), ("vertex_ctas_per_sm", C.c_int32), ("vertex_small_cap", C.c_int32),
                ("search_order", C.c_int32)]
    _defaults = dict(search_chunk=128, search_ctas_per_sm=5, search_group=1, search_stage_hits=5120,
                     vertex_ctas_per_sm=4, vertex_small_cap=512, search_order=1)

    def __init__(self, *args, **kw):
        """Positional values in field order; fields not given take the library's defaults."""
        names = [n for n, _ in self._fields_]
        vals = dict(self._defaults)
        vals.update(zip(names, args))
        vals.update(kw)
        super().__init__(**vals)

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ds_tune_entry(C.Structure):
    _fields_ = [("tuning", ds_tuning), ("ms", C.c_double)]


class ds_server_config(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("max_batch_events", C.c_int32), ("max_batch_seeds", C.c_int32),
                ("max_batch_hits", C.c_int32), ("events_per_launch", C.c_int32), ("vertices_per_seed", C.c_int32),
                ("hbm_budget", C.c_int64), ("mlp_precision", C.c_int32), ("graphs", C.c_int32),
                ("gather_max_bytes", C.c_int32)]


class ds_request(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("reserved0", C.c_int32), ("seed_off", C.c_void_p),
                ("hit_off", C.c_void_p)] + \
               [(k, C.c_void_p) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2",
                                          "hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "tracks")] + \
               [("trk_capacity", C.c_int32), ("vtx_capacity", C.c_int32), ("trk_off", C.c_void_p),
                ("vertices", C.c_void_p), ("vtx_off", C.c_void_p), ("arrival", C.c_double)]


class ds_completion(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("n_tracks", C.c_int32), ("n_vertices", C.c_int32),
                ("n_batches", C.c_int32), ("t_arrival", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class ds_server_stats(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("events_done", C.c_int64), ("batches", C.c_int64),
                ("hbm_budget", C.c_int64), ("hbm_peak", C.c_int64), ("context_bytes", C.c_int64),
                ("peak_inflight", C.c_int32), ("queued", C.c_int32), ("worker_launch_s", C.c_double),
                ("worker_finish_s", C.c_double), ("worker_wall_s", C.c_double), ("graphs", C.c_int32),
                ("graphs_captured", C.c_int32), ("bytes_gathered", C.c_int64), ("bytes_copied", C.c_int64)]


VINFO_DTYPE = np.dtype([("m_pipi", "<f4"), ("m_ppi", "<f4"), ("m_pip", "<f4"), ("p", "<f4"), ("pt", "<f4"),
                        ("ip", "<f4"), ("one_minus_cos", "<f4"), ("p_pos", "<f4"), ("p_neg", "<f4"),
                        ("pt_pos", "<f4"), ("pt_neg", "<f4"), ("score", "<f4", 4), ("flags", "<u4")])
assert VINFO_DTYPE.itemsize == 64

TRACK_DTYPE = np.dtype([("event", "<i4"), ("seed", "<i4"), ("hit", "<i4", 4), ("x", "<f4"), ("y", "<f4"),
                        ("tx", "<f4"), ("ty", "<f4"), ("qop", "<f4"), ("chi2", "<f4"), ("ndof", "<i4"),
                        ("nn", "<f4"), ("flags", "<u4"), ("n_candidates", "<i4")])
VERTEX_DTYPE = np.dtype([("event", "<i4"), ("i", "<i4"), ("j", "<i4"), ("x", "<f4"), ("y", "<f4"),
                         ("z", "<f4"), ("doca", "<f4"), ("flags", "<u4")])
assert TRACK_DTYPE.itemsize == 64 and VERTEX_DTYPE.itemsize == 32

_lib = None


class DSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib():
    """Load libds.so; raise if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libds.so not found at {LIB_PATH}; run python -m paper_2503_13092_b300.build")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "ds_create": ([C.POINTER(P), C.c_int], C.c_int),
            "ds_destroy": ([P], None),
            "ds_status_string": ([C.c_int], C.c_char_p),
            "ds_last_error": ([P], C.c_char_p),
            "ds_default_params": ([C.POINTER(ds_params)], C.c_int),
            "ds_load_geometry": ([P, C.POINTER(ds_geometry)], C.c_int),
            "ds_load_nn_weights": ([P, C.POINTER(ds_nn_weights)], C.c_int),
            "ds_set_params": ([P, C.POINTER(ds_params)], C.c_int),
            "ds_reserve": ([P, C.c_int32, C.c_int32, C.c_int32], C.c_int),
            "ds_reconstruct": ([P, C.POINTER(ds_event_batch), C.POINTER(ds_seeds), C.POINTER(ds_ut_hits),
                                C.POINTER(ds_tracks), P], C.c_int),
            "ds_vertex": ([P, C.POINTER(ds_tracks), C.POINTER(ds_vertices), P], C.c_int),
            "ds_sync_status": ([P, P, C.POINTER(ds_stats)], C.c_int),
            "ds_mlp_eval": ([P, P, C.c_int32, P, C.c_int32, P], C.c_int),
            "ds_get_tuning": ([P, C.POINTER(ds_tuning)], C.c_int),
            "ds_reserve_vertices": ([P, C.c_int32], C.c_int),
            "ds_candidates": ([P, P, P, P, P, C.c_int32, P, P], C.c_int),
            "ds_load_line_weights": ([P, P, C.c_int32], C.c_int),
            "ds_vertex_physics": ([P, C.POINTER(ds_tracks), C.POINTER(ds_vertices), P, C.c_int32, P], C.c_int),
            "ds_server_default_config": ([C.POINTER(ds_server_config)], None),
            "ds_server_create": ([C.POINTER(P), C.c_int, C.POINTER(ds_geometry), C.POINTER(ds_nn_weights),
                                  C.POINTER(ds_params), C.POINTER(ds_server_config)], C.c_int),
            "ds_server_submit": ([P, C.POINTER(ds_request), C.POINTER(C.c_int64)], C.c_int),
            "ds_server_now": ([P], C.c_double),
            "ds_server_poll": ([P, C.POINTER(ds_completion), C.c_int32, C.c_double], C.c_int32),
            "ds_server_drain": ([P], C.c_int),
            "ds_server_stats_get": ([P, C.POINTER(ds_server_stats)], C.c_int),
            "ds_server_destroy": ([P], None),
            "ds_set_tuning": ([P, C.POINTER(ds_tuning)], C.c_int),
            "ds_autotune": ([P, C.POINTER(ds_event_batch), C.POINTER(ds_seeds), C.POINTER(ds_ut_hits),
                             C.POINTER(ds_tracks), C.c_int32, C.POINTER(ds_tuning), C.POINTER(ds_tune_entry),
                             C.c_int32, C.POINTER(C.c_int32), P], C.c_int),
            "ds_reconstruct_noalloc": ([C.POINTER(ds_geometry), C.POINTER(ds_params), C.POINTER(ds_nn_weights),
                                        C.POINTER(ds_event_batch), C.POINTER(ds_seeds), C.POINTER(ds_ut_hits),
                                        C.POINTER(ds_tracks), P, P], C.c_int),
            "ds_profile_enable": ([P, C.c_int32], C.c_int),
            "ds_profile_read": ([P, C.POINTER(ds_kernel_time), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
            "ds_process_host": ([P, C.c_int32, P, C.POINTER(P), P, C.POINTER(P), P, P, C.c_int32, P,
                                 C.POINTER(C.c_int32), P, C.c_int32, P, C.POINTER(C.c_int32), P], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


EXPORTED = ("ds_create", "ds_destroy", "ds_status_string", "ds_last_error", "ds_default_params",
            "ds_load_geometry", "ds_load_nn_weights", "ds_set_params", "ds_reserve", "ds_reconstruct",
            "ds_vertex", "ds_sync_status", "ds_process_host", "ds_profile_enable", "ds_profile_read",
            "ds_reconstruct_noalloc", "ds_mlp_eval", "ds_get_tuning", "ds_set_tuning", "ds_autotune",
            "ds_reserve_vertices", "ds_candidates", "ds_load_line_weights", "ds_vertex_physics",
            "ds_server_default_config", "ds_server_create", "ds_server_submit",
            "ds_server_now", "ds_server_poll", "ds_server_drain", "ds_server_stats_get", "ds_server_destroy")


# --------------------------------------------------------------- C names, marshalled

def ds_create(device: int = 0):
    h = C.c_void_p()
    st = lib().ds_create(C.byref(h), device)
    if st != DS_OK:
        raise DSError(st, f"ds_create(device={device}) failed: {lib().ds_status_string(st).decode()}")
    return h


def ds_destroy(ctx):
    lib().ds_destroy(ctx)


def ds_status_string(st: int) -> str:
    return lib().ds_status_string(st).decode()


def ds_last_error(ctx) -> str:
    return lib().ds_last_error(ctx).decode()


def _check(ctx, st, what):
    if st != DS_OK:
        raise DSError(st, f"{what}: {ds_status_string(st)}: {ds_last_error(ctx)}")
    return st


def ds_default_params() -> ds_params:
    p = ds_params()
    lib().ds_default_params(C.byref(p))
    return p


def make_geometry(cfg: dict) -> ds_geometry:
    g = ds_geometry()
    g.z_layer[:] = cfg["z_layer"]
    g.dxdy[:] = cfg["dxdy"]
    g.zmag[:] = cfg["zmag"]
    for k in ("y_min", "sector_h", "x_half_bins", "z_seed", "kappa", "mp", "gamma0", "gamma1", "z_ref",
              "sigma_hit", "sigma_mag"):
        setattr(g, k, float(cfg[k]))
    g.n_sectors = int(cfg["n_sectors"])
    return g


def make_params(cfg: dict, **over) -> ds_params:
    p = ds_default_params()
    for k in ("w1a", "w1b", "w2", "dy_tol", "nn_threshold", "doca_max", "nr_tol"):
        setattr(p, k, float(cfg[k]))
    for k in ("k1", "first_window_origin", "pick_chi2", "clone_kill", "training", "nr_max_iter"):
        setattr(p, k, int(cfg[k]))
    p.variant = int(cfg.get("variant", 0))
    p.dv1_dtx_max = float(cfg.get("dv1_dtx_max", 0.8))
    p.dv1_w_tri = float(cfg.get("dv1_w_tri", 1.0))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def ds_load_geometry(ctx, geom: ds_geometry):
    return _check(ctx, lib().ds_load_geometry(ctx, C.byref(geom)), "ds_load_geometry")


class _NN:
    def __init__(self, w: dict):
        f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32).ravel())
        self.keep = [f(w["w1"]), f(w["b1"]), f(w["w2"]) if w["n_h2"] else np.zeros(1, np.float32),
                     f(w["b2"]) if w["n_h2"] else np.zeros(1, np.float32), f(w["w3"]), f(w["mean"]),
                     f(w["scale"])]
        s = ds_nn_weights()
        s.n_in, s.n_h1, s.n_h2 = int(w["n_in"]), int(w["n_h1"]), int(w["n_h2"])
        s.w1, s.b1, s.w2, s.b2, s.w3, s.mean, s.scale = [a.ctypes.data for a in self.keep]
        s.b3 = float(w["b3"])
        self.s = s


def ds_load_nn_weights(ctx, w: dict):
    nn = _NN(w)
    return _check(ctx, lib().ds_load_nn_weights(ctx, C.byref(nn.s)), "ds_load_nn_weights")


def ds_set_params(ctx, p: ds_params):
    return _check(ctx, lib().ds_set_params(ctx, C.byref(p)), "ds_set_params")


def ds_reserve(ctx, max_events: int, max_seeds: int, max_hits: int):
    return _check(ctx, lib().ds_reserve(ctx, max_events, max_seeds, max_hits), "ds_reserve")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def ds_reconstruct(ctx, dev: dict, out: dict, stream=None):
    """dev: device tensors of one batch (see Downstream.to_device); out: track
    output tensors {tracks (uint8 [cap, 64]), trk_off (int32 [E+1]), n_tracks (int32 [1])}."""
    b = ds_event_batch(dev["n_events"], dev["n_seeds"], dev["n_hits"], 0, _ptr(dev["seed_off"]),
                       _ptr(dev["hit_off"]))
    sd = ds_seeds(*[_ptr(dev[k]) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2")])
    ht = ds_ut_hits(*[_ptr(dev[k]) for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer")])
    tr = ds_tracks(_ptr(out["tracks"]), _ptr(out["trk_off"]), _ptr(out["n_tracks"]),
                   int(out["tracks"].shape[0]), 0)
    _check(ctx, lib().ds_reconstruct(ctx, C.byref(b), C.byref(sd), C.byref(ht), C.byref(tr), _stream(stream)),
           "ds_reconstruct")
    out["_struct"] = tr
    return tr


def ds_vertex(ctx, trk_out: dict, vout: dict, stream=None):
    tr = trk_out["_struct"]
    vx = ds_vertices(_ptr(vout["vertices"]), _ptr(vout["vtx_off"]), _ptr(vout["n_vertices"]),
                     int(vout["vertices"].shape[0]), 0)
    _check(ctx, lib().ds_vertex(ctx, C.byref(tr), C.byref(vx), _stream(stream)), "ds_vertex")
    return vx


def ds_mlp_eval(ctx, features, logit, precision: int, stream=None):
    """features: device float32 [n, 16] (contiguous); logit: device float32 [n]."""
    n = int(features.shape[0])
    if n and (features.dtype.itemsize != 4 or not features.is_contiguous() or tuple(features.shape[1:]) != (16,)):
        raise ValueError("features must be a contiguous float32 [n, 16] tensor")
    if int(logit.numel()) < n:
        raise ValueError("logit holds fewer than n values")
    _check(ctx, lib().ds_mlp_eval(ctx, _ptr(features), n, _ptr(logit), int(precision), _stream(stream)),
           "ds_mlp_eval")


def ds_get_tuning(ctx) -> ds_tuning:
    t = ds_tuning()
    _check(ctx, lib().ds_get_tuning(ctx, C.byref(t)), "ds_get_tuning")
    return t


def ds_set_tuning(ctx, t: ds_tuning):
    return _check(ctx, lib().ds_set_tuning(ctx, C.byref(t)), "ds_set_tuning")


def ds_autotune(ctx, dev: dict, out: dict, reps: int = 3, stream=None, max_entries: int = 64):
    """Autotune the search launch shape on this batch; returns (best, [(tuning dict, ms), ...])."""
    b = ds_event_batch(dev["n_events"], dev["n_seeds"], dev["n_hits"], 0, _ptr(dev["seed_off"]),
                       _ptr(dev["hit_off"]))
    sd = ds_seeds(*[_ptr(dev[k]) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2")])
    ht = ds_ut_hits(*[_ptr(dev[k]) for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer")])
    tr = ds_tracks(_ptr(out["tracks"]), _ptr(out["trk_off"]), _ptr(out["n_tracks"]),
                   int(out["tracks"].shape[0]), 0)
    best = ds_tuning()
    ent = (ds_tune_entry * max_entries)()
    n = C.c_int32(0)
    _check(ctx, lib().ds_autotune(ctx, C.byref(b), C.byref(sd), C.byref(ht), C.byref(tr), int(reps), C.byref(best),
                                  ent, max_entries, C.byref(n), _stream(stream)), "ds_autotune")
    out["_struct"] = tr
    return best, [(ent[i].tuning.as_dict(), ent[i].ms) for i in range(min(n.value, max_entries))]


def ds_candidates(ctx, features, seed, hits, logit, count, stream=None):
    """Device tensors: features float32 [cap, 16], seed int32 [cap], hits int32 [cap, 4],
    logit float32 [cap] (or None), count int32 [1] (receives the candidates of the call)."""
    cap = int(features.shape[0])
    if seed.numel() < cap or hits.numel() < 4 * cap or (logit is not None and logit.numel() < cap):
        raise ValueError("output arrays smaller than the capacity")
    _check(ctx, lib().ds_candidates(ctx, _ptr(features), _ptr(seed), _ptr(hits), _ptr(logit), cap, _ptr(count),
                                    _stream(stream)), "ds_candidates")


def ds_load_line_weights(ctx, nets: list):
    """Trigger-line networks: list of up to 4 weight dicts (16 -> n_h1 -> 1)."""
    holders = [_NN(w) for w in nets]
    arr = (ds_nn_weights * max(len(nets), 1))(*[h.s for h in holders])
    return _check(ctx, lib().ds_load_line_weights(ctx, arr, len(nets)), "ds_load_line_weights")


def ds_vertex_physics(ctx, trk_out: dict, vout: dict, info, stream=None):
    """info: device uint8 tensor [capacity, 64] (VINFO_DTYPE records)."""
    tr = trk_out["_struct"]
    vx = ds_vertices(_ptr(vout["vertices"]), _ptr(vout["vtx_off"]), _ptr(vout["n_vertices"]),
                     int(vout["vertices"].shape[0]), 0)
    _check(ctx, lib().ds_vertex_physics(ctx, C.byref(tr), C.byref(vx), _ptr(info), int(info.shape[0]),
                                        _stream(stream)), "ds_vertex_physics")


def ds_reserve_vertices(ctx, capacity: int):
    return _check(ctx, lib().ds_reserve_vertices(ctx, int(capacity)), "ds_reserve_vertices")


def ds_sync_status(ctx, stream=None, raise_on_error: bool = True):
    s = ds_stats()
    st = lib().ds_sync_status(ctx, _stream(stream), C.byref(s))
    stats = {k: getattr(s, k) for k, _ in ds_stats._fields_ if k != "reserved0"}
    stats["status"] = st
    if raise_on_error and st != DS_OK:
        raise DSError(st, f"ds_sync_status: {ds_status_string(st)}: {ds_last_error(ctx)} flags=0x{s.device_flags:x}")
    return stats


def ds_reconstruct_noalloc(geom: ds_geometry, params: ds_params, weights: dict, dev: dict, out: dict,
                           d_flags=None, stream=None) -> int:
    """Allocation-free ds_reconstruct (no context; static device scratch).
    Returns the ds_status code; outputs as ds_reconstruct."""
    nn = _NN(weights)
    b = ds_event_batch(dev["n_events"], dev["n_seeds"], dev["n_hits"], 0, _ptr(dev["seed_off"]),
                       _ptr(dev["hit_off"]))
    sd = ds_seeds(*[_ptr(dev[k]) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2")])
    ht = ds_ut_hits(*[_ptr(dev[k]) for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer")])
    tr = ds_tracks(_ptr(out["tracks"]), _ptr(out["trk_off"]), _ptr(out["n_tracks"]),
                   int(out["tracks"].shape[0]), 0)
    st = lib().ds_reconstruct_noalloc(C.byref(geom), C.byref(params), C.byref(nn.s), C.byref(b), C.byref(sd),
                                      C.byref(ht), C.byref(tr), _ptr(d_flags), _stream(stream))
    out["_struct"] = tr
    return st


def ds_profile_enable(ctx, enable: bool = True):
    return _check(ctx, lib().ds_profile_enable(ctx, int(enable)), "ds_profile_enable")


def ds_profile_read(ctx) -> dict:
    """{kernel name: (launches, total_ms)}; synchronises the device, clears the records."""
    buf = (ds_kernel_time * 32)()
    n = C.c_int32()
    _check(ctx, lib().ds_profile_read(ctx, buf, 32, C.byref(n)), "ds_profile_read")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n.value, 32))}


def ds_process_host(ctx, batch: dict, trk_capacity: int, vtx_capacity: int, stream=None, host_out=None):
    """End-to-end call with host (numpy, ideally pinned) buffers."""
    E = int(batch["n_events"])
    seed_cols = [np.ascontiguousarray(batch[k], np.float32)
                 for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2")]
    hit_cols = [np.ascontiguousarray(batch[k], np.float32) for k in ("hit_x0", "hit_ybeg", "hit_yend")]
    layer = np.ascontiguousarray(batch["hit_layer"], np.uint8)
    so = np.ascontiguousarray(batch["seed_off"], np.int32)
    ho = np.ascontiguousarray(batch["hit_off"], np.int32)
    if host_out is None:
        host_out = dict(tracks=np.zeros(trk_capacity, TRACK_DTYPE), trk_off=np.zeros(E + 1, np.int32),
                        vertices=np.zeros(vtx_capacity, VERTEX_DTYPE), vtx_off=np.zeros(E + 1, np.int32))
    sc = (C.c_void_p * 6)(*[a.ctypes.data for a in seed_cols])
    hc = (C.c_void_p * 3)(*[a.ctypes.data for a in hit_cols])
    nt = C.c_int32(); nv = C.c_int32()
    st = lib().ds_process_host(ctx, E, so.ctypes.data, sc, ho.ctypes.data, hc, layer.ctypes.data,
                               host_out["tracks"].ctypes.data, trk_capacity, host_out["trk_off"].ctypes.data,
                               C.byref(nt), host_out["vertices"].ctypes.data, vtx_capacity,
                               host_out["vtx_off"].ctypes.data, C.byref(nv), _stream(stream))
    _check(ctx, st, "ds_process_host")
    host_out["n_tracks"] = nt.value
    host_out["n_vertices"] = nv.value
    return host_out


# ------------------------------------------------------------------ convenience

class Downstream:
    """One library context with device-resident geometry and network weights."""

    def __init__(self, cfg: dict, weights: dict, device: int = 0, **param_over):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.torch = torch
        self.device = device
        self.ctx = ds_create(device)
        self.cfg = cfg
        ds_load_geometry(self.ctx, make_geometry(cfg))
        ds_load_nn_weights(self.ctx, weights)
        self.params = make_params(cfg, **param_over)
        ds_set_params(self.ctx, self.params)

    def close(self):
        if self.ctx is not None:
            ds_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **over):
        for k, v in over.items():
            setattr(self.params, k, v)
        ds_set_params(self.ctx, self.params)

    def to_device(self, batch: dict) -> dict:
        t = self.torch
        dev = f"cuda:{self.device}"
        d = dict(n_events=int(batch["n_events"]), n_seeds=int(batch["seed_off"][-1]),
                 n_hits=int(batch["hit_off"][-1]))
        for k in ("seed_off", "hit_off"):
            d[k] = t.from_numpy(np.ascontiguousarray(batch[k], np.int32)).to(dev)
        for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg",
                  "hit_yend"):
            d[k] = t.from_numpy(np.ascontiguousarray(batch[k], np.float32)).to(dev)
        d["hit_layer"] = t.from_numpy(np.ascontiguousarray(batch["hit_layer"], np.uint8)).to(dev)
        return d

    def alloc_tracks(self, n_events: int, capacity: int) -> dict:
        t = self.torch
        dev = f"cuda:{self.device}"
        return dict(tracks=t.zeros((max(capacity, 1), 64), dtype=t.uint8, device=dev),
                    trk_off=t.zeros(n_events + 1, dtype=t.int32, device=dev),
                    n_tracks=t.zeros(1, dtype=t.int32, device=dev))

    def alloc_vertices(self, n_events: int, capacity: int) -> dict:
        t = self.torch
        dev = f"cuda:{self.device}"
        return dict(vertices=t.zeros((max(capacity, 1), 32), dtype=t.uint8, device=dev),
                    vtx_off=t.zeros(n_events + 1, dtype=t.int32, device=dev),
                    n_vertices=t.zeros(1, dtype=t.int32, device=dev))

    def reconstruct(self, dev: dict, out: dict, stream=None):
        return ds_reconstruct(self.ctx, dev, out, stream)

    def vertex(self, trk_out: dict, vout: dict, stream=None):
        return ds_vertex(self.ctx, trk_out, vout, stream)

    def sync(self, stream=None, raise_on_error=True):
        return ds_sync_status(self.ctx, stream, raise_on_error)

    def candidates(self, capacity: int, stream=None) -> dict:
        """The last reconstruct's candidates as host numpy arrays (features, seed, hits, logit)."""
        t = self.torch
        dev = f"cuda:{self.device}"
        f = t.empty((max(capacity, 1), 16), dtype=t.float32, device=dev)
        sd = t.empty(max(capacity, 1), dtype=t.int32, device=dev)
        h = t.empty((max(capacity, 1), 4), dtype=t.int32, device=dev)
        lg = t.empty(max(capacity, 1), dtype=t.float32, device=dev)
        cnt = t.zeros(1, dtype=t.int32, device=dev)
        ds_candidates(self.ctx, f, sd, h, lg, cnt, stream)
        n = min(int(cnt.cpu()[0]), capacity)
        return dict(n_total=int(cnt.cpu()[0]), features=f[:n].cpu().numpy(), seed=sd[:n].cpu().numpy(),
                    hits=h[:n].cpu().numpy(), logit=lg[:n].cpu().numpy())

    def mlp_eval(self, features, precision: int = 0, stream=None):
        """Network output before the sigmoid for device features [n, 16]."""
        t = self.torch
        logit = t.empty(features.shape[0], dtype=t.float32, device=features.device)
        ds_mlp_eval(self.ctx, features, logit, precision, stream)
        return logit

    def run(self, batch: dict, trk_capacity=None, vtx_capacity=None, dev=None):
        """Upload, reconstruct, vertex, synchronise and decode (host numpy)."""
        dev = dev or self.to_device(batch)
        E = dev["n_events"]
        trk_capacity = trk_capacity if trk_capacity is not None else max(dev["n_seeds"], 1)
        out = self.alloc_tracks(E, trk_capacity)
        self.reconstruct(dev, out)
        if vtx_capacity is None:
            vtx_capacity = 16 * trk_capacity + 4096
        vout = self.alloc_vertices(E, vtx_capacity)
        self.vertex(out, vout)
        stats = self.sync()
        return decode(out, vout) | {"stats": stats}


def decode(out: dict, vout: dict | None = None) -> dict:
    n = int(out["n_tracks"].cpu()[0])
    cap = out["tracks"].shape[0]
    raw = out["tracks"][: min(n, cap)].cpu().numpy()
    res = dict(tracks=raw.view(TRACK_DTYPE).reshape(-1), trk_off=out["trk_off"].cpu().numpy(), n_tracks=n)
    if vout is not None:
        nv = int(vout["n_vertices"].cpu()[0])
        vcap = vout["vertices"].shape[0]
        vr = vout["vertices"][: min(nv, vcap)].cpu().numpy()
        res.update(vertices=vr.view(VERTEX_DTYPE).reshape(-1), vtx_off=vout["vtx_off"].cpu().numpy(),
                   n_vertices=nv)
    return res


# --------------------------------------------------------------- serving loop

def ds_server_default_config() -> ds_server_config:
    c = ds_server_config()
    lib().ds_server_default_config(C.byref(c))
    return c


class Server:
    """Continuous-batching request server (include/ds_serve.h) over host numpy
    requests.  submit() takes one request dict (host arrays of one or more
    events: seed_off, hit_off, seed_*, hit_* as in Downstream.to_device) and
    keeps it, and its output arrays, alive until poll() returns it."""

    def __init__(self, cfg: dict, weights: dict, device: int = 0, params: dict | None = None, **config):
        self.ptr = None
        c = ds_server_default_config()
        for k, v in config.items():
            setattr(c, k, v)
        self.config = c
        self._nn = _NN(weights)
        self._geom = make_geometry(cfg)
        self._params = make_params(cfg, **(params or {}))
        p = C.c_void_p()
        st = lib().ds_server_create(C.byref(p), device, C.byref(self._geom), C.byref(self._nn.s),
                                    C.byref(self._params), C.byref(c))
        if st != DS_OK:
            raise DSError(st, f"ds_server_create: {ds_status_string(st)}")
        self.ptr = p
        self._pending = {}

    def now(self) -> float:
        return lib().ds_server_now(self.ptr)

    def alloc_outputs(self, req: dict, vtx_capacity: int | None = None, pinned: bool = True) -> dict:
        """Output arrays for one request: tracks (one per seed at most), vertices
        (vtx_capacity, default 4 per seed + 4096), trk_off, vtx_off.  Pinned
        (page-locked, through torch's caching host allocator) by default: the
        server then copies the records into them by DMA."""
        E, S = int(req["n_events"]), int(req["seed_off"][-1])
        vcap = vtx_capacity if vtx_capacity is not None else 4 * S + 4096

        def buf(n, dtype):
            if pinned:
                import torch
                t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8, pin_memory=True)
                return t.numpy().view(dtype)
            return np.zeros(n, dtype)

        return dict(tracks=buf(max(S, 1), TRACK_DTYPE), vertices=buf(max(vcap, 1), VERTEX_DTYPE),
                    trk_off=np.zeros(E + 1, np.int32), vtx_off=np.zeros(E + 1, np.int32))

    def submit(self, req: dict, arrival: float = 0.0, out: dict | None = None, vtx_capacity: int | None = None) -> int:
        """Queue one request (host arrays; pinned inputs are read by the device
        directly or uploaded by DMA, pageable ones through the driver's staging).
        out: buffers from alloc_outputs (allocated here when None).  The
        request's arrays and out stay referenced until poll() returns it."""
        E = int(req["n_events"])
        keep = {}

        def arr(k, t):
            a = np.ascontiguousarray(req[k], t)
            keep[k] = a
            return a.ctypes.data

        r = ds_request()
        r.n_events = E
        r.seed_off = arr("seed_off", np.int32)
        r.hit_off = arr("hit_off", np.int32)
        for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend"):
            setattr(r, k, arr(k, np.float32))
        r.hit_layer = arr("hit_layer", np.uint8)
        o = out if out is not None else self.alloc_outputs(req, vtx_capacity)
        r.tracks, r.trk_capacity, r.trk_off = o["tracks"].ctypes.data, len(o["tracks"]), o["trk_off"].ctypes.data
        r.vertices, r.vtx_capacity, r.vtx_off = o["vertices"].ctypes.data, len(o["vertices"]), o["vtx_off"].ctypes.data
        r.arrival = float(arrival)
        rid = C.c_int64(0)
        st = lib().ds_server_submit(self.ptr, C.byref(r), C.byref(rid))
        if st != DS_OK:
            raise DSError(st, f"ds_server_submit: {ds_status_string(st)}")
        self._pending[rid.value] = (keep, o["tracks"], o["trk_off"], o["vertices"], o["vtx_off"])
        return rid.value

    def poll(self, timeout: float = 0.1, max_out: int = 256) -> list:
        """Completed requests: dicts with the completion fields and the outputs."""
        buf = (ds_completion * max_out)()
        n = lib().ds_server_poll(self.ptr, buf, max_out, float(timeout))
        res = []
        for i in range(n):
            c = buf[i]
            keep, tracks, trk_off, vertices, vtx_off = self._pending.pop(c.id)
            d = {k: getattr(c, k) for k, _ in ds_completion._fields_}
            d.update(tracks=tracks[:min(c.n_tracks, len(tracks))], trk_off=trk_off,
                     vertices=vertices[:min(c.n_vertices, len(vertices))], vtx_off=vtx_off)
            res.append(d)
        return res

    def drain(self):
        lib().ds_server_drain(self.ptr)

    def stats(self) -> dict:
        s = ds_server_stats()
        lib().ds_server_stats_get(self.ptr, C.byref(s))
        return {k: getattr(s, k) for k, _ in ds_server_stats._fields_}

    def close(self):
        if self.ptr is not None:
            lib().ds_server_destroy(self.ptr)
            self.ptr = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
