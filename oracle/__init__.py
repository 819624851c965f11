"""FP64 CPU oracle of the Downstream tracking + two-track vertexing path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg; the product package never imports it.  The C
source (oracle.c) is compiled with gcc into oracle/_build/liboracle.so on first
use.  Every function cites the section or equation of arXiv:2503.13092 it
restates (see oracle.c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, -O2, OpenMP over events)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-Wno-unused-parameter", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrConfig(C.Structure):
    _fields_ = [("z", C.c_double * 4), ("dxdy", C.c_double * 4), ("z_seed", C.c_double),
                ("zmag", C.c_double * 4), ("kappa", C.c_double), ("mp", C.c_double),
                ("gamma0", C.c_double), ("gamma1", C.c_double), ("z_ref", C.c_double),
                ("sigma_hit", C.c_double), ("sigma_mag", C.c_double),
                ("w1a", C.c_double), ("w1b", C.c_double), ("w2", C.c_double),
                ("dy_tol", C.c_double), ("nn_threshold", C.c_double), ("doca_max", C.c_double),
                ("nr_tol", C.c_double), ("k1", C.c_int), ("first_window_origin", C.c_int),
                ("pick_chi2", C.c_int), ("clone_kill", C.c_int), ("training", C.c_int),
                ("nr_max_iter", C.c_int), ("variant", C.c_int), ("dv1_dtx_max", C.c_double),
                ("dv1_w_tri", C.c_double), ("chi2_margin_scale", C.c_double)]


class OrNN(C.Structure):
    _fields_ = [("n_in", C.c_int), ("n_h1", C.c_int), ("n_h2", C.c_int), ("pad", C.c_int),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("mean", C.c_void_p), ("scale", C.c_void_p),
                ("b3", C.c_float)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_mlp.restype = C.c_double
            _lib.or_mlp_logit.restype = C.c_double
            _lib.or_gamma.restype = C.c_double
            _lib.or_poca.restype = C.c_int
            _lib.or_vertex.restype = C.c_long
            _lib.or_seed_candidates.restype = C.c_int
    return _lib


def make_config(cfg: dict) -> OrConfig:
    c = OrConfig()
    c.z[:] = cfg["z_layer"]
    c.dxdy[:] = cfg["dxdy"]
    c.zmag[:] = cfg["zmag"]
    for k in ("z_seed", "kappa", "mp", "gamma0", "gamma1", "z_ref", "sigma_hit", "sigma_mag",
              "w1a", "w1b", "w2", "dy_tol", "nn_threshold", "doca_max", "nr_tol"):
        setattr(c, k, float(cfg[k]))
    for k in ("k1", "first_window_origin", "pick_chi2", "clone_kill", "training", "nr_max_iter"):
        setattr(c, k, int(cfg[k]))
    c.variant = int(cfg.get("variant", 0))
    c.dv1_dtx_max = float(cfg.get("dv1_dtx_max", 0.8))
    c.dv1_w_tri = float(cfg.get("dv1_w_tri", 1.0))
    # margin of a chi2 key comparison per unit of its relative gap (decision
    # margins are compared with 1e-5 by the parity rules)
    c.chi2_margin_scale = float(cfg.get("chi2_margin_scale", 1e-2))
    return c


class _NNHolder:
    """Keeps the float32 arrays alive while the C struct points at them."""

    def __init__(self, w: dict):
        f = lambda a: np.ascontiguousarray(np.asarray(a, np.float32).ravel())
        self.arrays = [f(w["w1"]), f(w["b1"]), f(w["w2"]) if w["n_h2"] else np.zeros(1, np.float32),
                       f(w["b2"]) if w["n_h2"] else np.zeros(1, np.float32), f(w["w3"]),
                       f(w["mean"]), f(w["scale"])]
        s = OrNN()
        s.n_in, s.n_h1, s.n_h2 = int(w["n_in"]), int(w["n_h1"]), int(w["n_h2"])
        s.w1, s.b1, s.w2, s.b2, s.w3, s.mean, s.scale = [_p(a) for a in self.arrays]
        s.b3 = float(w["b3"])
        self.s = s


def mlp(w: dict, phi) -> np.ndarray:
    """Ghost-killer response for each row of phi (FP64)."""
    h = _NNHolder(w)
    phi = np.ascontiguousarray(np.atleast_2d(np.asarray(phi, np.float64)))
    out = np.empty(phi.shape[0])
    L = lib()
    for i in range(phi.shape[0]):
        out[i] = L.or_mlp(C.byref(h.s), _p(phi[i]))
    return out


def mlp_logit(w: dict, phi) -> np.ndarray:
    """Ghost-killer network output before the sigmoid for each row of phi (FP64)."""
    h = _NNHolder(w)
    phi = np.ascontiguousarray(np.atleast_2d(np.asarray(phi, np.float64)))
    out = np.empty(phi.shape[0])
    L = lib()
    for i in range(phi.shape[0]):
        out[i] = L.or_mlp_logit(C.byref(h.s), _p(phi[i]))
    return out


def gamma(cfg: dict, qop: float) -> float:
    return lib().or_gamma(C.byref(make_config(cfg)), C.c_double(qop))


def reconstruct(batch: dict, cfg: dict, w: dict, n_threads: int = 1) -> dict:
    """Per-seed oracle results for a whole batch (see or_reconstruct)."""
    c = make_config(cfg)
    h = _NNHolder(w)
    S = int(batch["seed_off"][-1])
    E = int(batch["n_events"])
    out = dict(status=np.zeros(S, np.int32), hits=np.full((S, 4), -1, np.int32),
               state=np.zeros((S, 5)), chi2=np.zeros(S), ndof=np.zeros(S, np.int32),
               nn=np.zeros(S), ncand=np.zeros(S, np.int32), nbx=np.zeros(S, np.int32),
               margin=np.zeros(S))
    a = lambda k, t: np.ascontiguousarray(batch[k], t)
    ins = [a("seed_off", np.int32), a("seed_x", np.float32), a("seed_y", np.float32),
           a("seed_tx", np.float32), a("seed_ty", np.float32), a("seed_qop", np.float32),
           a("seed_chi2", np.float32), a("hit_off", np.int32), a("hit_x0", np.float32),
           a("hit_ybeg", np.float32), a("hit_yend", np.float32), a("hit_layer", np.uint8)]
    lib().or_reconstruct(C.byref(c), C.byref(h.s), C.c_int(E), *[_p(x) for x in ins],
                         _p(out["status"]), _p(out["hits"]), _p(out["state"]), _p(out["chi2"]),
                         _p(out["ndof"]), _p(out["nn"]), _p(out["ncand"]), _p(out["nbx"]),
                         _p(out["margin"]), C.c_int(n_threads))
    return out


def tracks_from(res: dict, seed_off) -> dict:
    """Packed track list (alive tracks in (event, seed) order) and trk_off."""
    alive = res["status"] == 2
    E = len(seed_off) - 1
    ev = np.repeat(np.arange(E), np.diff(seed_off))
    idx = np.nonzero(alive)[0]
    trk_off = np.zeros(E + 1, np.int64)
    trk_off[1:] = np.cumsum(np.bincount(ev[idx], minlength=E))
    return dict(seed=idx.astype(np.int32), event=ev[idx].astype(np.int32), hits=res["hits"][idx],
                state=res["state"][idx], chi2=res["chi2"][idx], ndof=res["ndof"][idx],
                nn=res["nn"][idx], margin=res["margin"][idx], trk_off=trk_off)


def seed_candidates(batch: dict, cfg: dict, w: dict, s: int, max_c: int = 64) -> dict:
    """Every candidate of global seed s, in enumeration order, with the winner index."""
    c = make_config(cfg)
    h = _NNHolder(w)
    e = int(np.searchsorted(batch["seed_off"], s, side="right") - 1)
    h0, h1 = int(batch["hit_off"][e]), int(batch["hit_off"][e + 1])
    a = lambda k, t: np.ascontiguousarray(batch[k], t)
    hx = [np.ascontiguousarray(batch[k][h0:h1]) for k in ("hit_x0", "hit_ybeg", "hit_yend")]
    hl = np.ascontiguousarray(batch["hit_layer"][h0:h1], np.uint8)
    hits = np.zeros((max_c, 4), np.int32); state = np.zeros((max_c, 5)); chi2 = np.zeros(max_c)
    ndof = np.zeros(max_c, np.int32); f = np.zeros(max_c); phi = np.zeros((max_c, 16))
    win = C.c_int(-1)
    sx = [a(k, np.float32) for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2")]
    n = lib().or_seed_candidates(C.byref(c), C.byref(h.s), *[_p(x) for x in sx], C.c_int(s),
                                 C.c_int(h1 - h0), C.c_int(h0), *[_p(x) for x in hx], _p(hl),
                                 C.c_int(max_c), _p(hits), _p(state), _p(chi2), _p(ndof), _p(f),
                                 _p(phi), C.byref(win))
    k = min(n, max_c)
    return dict(n=n, hits=hits[:k], state=state[:k], chi2=chi2[:k], ndof=ndof[:k], f=f[:k],
                phi=phi[:k], winner=win.value)


def poca(cfg: dict, ti, tj) -> dict:
    """Newton-Raphson closest approach of two Eq. 4 trajectories (FP64)."""
    c = make_config(cfg)
    ti = np.ascontiguousarray(ti, np.float64); tj = np.ascontiguousarray(tj, np.float64)
    z1 = C.c_double(); z2 = C.c_double(); pos = np.zeros(3); doca = C.c_double(); it = C.c_int()
    fl = lib().or_poca(C.byref(c), _p(ti), _p(tj), C.byref(z1), C.byref(z2), _p(pos),
                       C.byref(doca), C.byref(it))
    return dict(z1=z1.value, z2=z2.value, pos=pos, doca=doca.value, iters=it.value, flags=fl)


def vertex(cfg: dict, trk_off, x, y, tx, ty, qop, cap: int | None = None) -> dict:
    """Opposite-charge two-track vertices with DOCA < doca_max, (event, i, j) order."""
    c = make_config(cfg)
    trk_off = np.ascontiguousarray(trk_off, np.int32)
    cols = [np.ascontiguousarray(v, np.float32) for v in (x, y, tx, ty, qop)]
    E = len(trk_off) - 1
    if cap is None:
        n_t = np.diff(trk_off).astype(np.int64)
        cap = int(max(1, (n_t * (n_t - 1) // 2).sum()))
    ev = np.zeros(cap, np.int32); i = np.zeros(cap, np.int32); j = np.zeros(cap, np.int32)
    pos = np.zeros((cap, 3)); doca = np.zeros(cap); fl = np.zeros(cap, np.int32)
    it = np.zeros(cap, np.int32); mg = np.zeros(cap); pairs = C.c_long()
    n = lib().or_vertex(C.byref(c), C.c_int(E), _p(trk_off), *[_p(v) for v in cols], C.c_long(cap),
                        _p(ev), _p(i), _p(j), _p(pos), _p(doca), _p(fl), _p(it), _p(mg),
                        C.byref(pairs))
    k = min(n, cap)
    return dict(n=n, event=ev[:k], i=i[:k], j=j[:k], pos=pos[:k], doca=doca[:k], flags=fl[:k],
                iters=it[:k], margin=mg[:k], pairs=pairs.value)


def vertex_info(cfg: dict, ti, tj, v) -> np.ndarray:
    """One vertex's quantities: m_pipi, m_ppi, m_pip, |P|, P_T, ip, 1 - cos, p_pos, p_neg, pt_pos, pt_neg."""
    out = np.zeros(11)
    a = lambda t: np.ascontiguousarray(t, np.float64)
    lib().or_vertex_info(C.byref(make_config(cfg)), _p(a(ti)), _p(a(tj)), _p(a(v)), _p(out))
    return out


def vertex_infos(cfg: dict, tracks: dict, vertices: dict, lines: list) -> dict:
    """Info, 16 line-network inputs and line responses for every vertex.
    tracks: arrays x, y, tx, ty, qop, chi2, ndof (output order); vertices: i, j,
    pos [n, 3] (or x, y, z), doca."""
    n = len(vertices["i"])
    f32 = lambda k: np.ascontiguousarray(tracks[k], np.float32)
    pos = vertices["pos"] if "pos" in vertices else np.stack([vertices["x"], vertices["y"], vertices["z"]], 1)
    pos = np.ascontiguousarray(pos, np.float64)
    doca = np.ascontiguousarray(vertices["doca"], np.float64)
    vi = np.ascontiguousarray(vertices["i"], np.int32)
    vj = np.ascontiguousarray(vertices["j"], np.int32)
    ndof = np.ascontiguousarray(tracks["ndof"], np.int32)
    holders = [_NNHolder(w) for w in lines]
    arr = (OrNN * max(len(lines), 1))(*[h.s for h in holders])
    info = np.zeros((n, 11)); feat = np.zeros((n, 16)); score = np.zeros((n, max(len(lines), 1)))
    cols = [f32(k) for k in ("x", "y", "tx", "ty", "qop", "chi2")]
    lib().or_vertex_infos(C.byref(make_config(cfg)), C.c_long(n), _p(vi), _p(vj), _p(pos), _p(doca), *[_p(c) for c in cols],
                          _p(ndof), C.c_int(len(lines)), arr, _p(info), _p(feat), _p(score))
    return dict(info=info, features=feat, score=score[:, :len(lines)])


def seed_prediction(cfg: dict, x, y, tx, ty, qop) -> dict:
    """Magnet point, first-window prediction and window sizes of one seed (FP64)."""
    c = make_config(cfg)
    out = np.zeros(11)
    lib().or_seed_prediction(C.byref(c), *[C.c_double(float(v)) for v in (x, y, tx, ty, qop)], _p(out))
    return dict(zm=out[0], xm=out[1], ym=out[2], u_bx=out[3], w1=out[4], yl=out[5:9].copy(),
                w2=out[9], tx_ut=out[10])


def clone_kill(hits, k1, k2, enabled: bool = True, has=None) -> np.ndarray:
    """Clone-killing step over one event's winners: 0 none, 1 killed, 2 kept."""
    hits = np.ascontiguousarray(hits, np.int32).reshape(-1, 4)
    n = hits.shape[0]
    has = np.ones(n, np.int32) if has is None else np.ascontiguousarray(has, np.int32)
    k1 = np.ascontiguousarray(k1, np.float64); k2 = np.ascontiguousarray(k2, np.float64)
    st = np.zeros(n, np.int32)
    lib().or_clone_kill(C.c_int(n), _p(has), _p(hits), _p(k1), _p(k2), C.c_int(int(enabled)),
                        C.c_int(0), C.c_double(1e-2), _p(st), None)
    return st
