"""GPU-vs-oracle comparison rules (test infrastructure).

Tracks: hit assignments must be identical, except for a seed whose oracle
decision margin (window edge, k-closest boundary, key comparison, threshold)
is below MARGIN, or whose event holds such a seed sharing a hit with it (a
flip there can change clone killing here); those excused seeds may be at most
0.1 % of the tracks.  On identical hits: x, y, tx, ty, q/p within 1e-4
relative (absolute floor 1e-6), chi2 within 1e-3 relative (absolute floor
1e-4), network response within 2e-5 absolute for the fixed-seed network
(callers pass a wider bound for a trained one, whose steeper response
amplifies the FP32 rounding of its inputs).

Vertices: the oracle vertexer is fed the GPU's own FP32 track records; kept
(i, j) sets must agree except where |DOCA - doca_max| is below MARGIN
(relative); positions within 1 um (1e-3 mm), or within 2 ulp of the vertex's
largest float32 coordinate where that is coarser (vertices beyond 8 m, whose
float32 coordinates cannot hold 1 um); DOCA within 1e-4 mm.
"""
import json
import os

import numpy as np

import oracle

MARGIN = 1e-5
RTOL_PAR, ATOL_PAR = 1e-4, 1e-6
RTOL_CHI2, ATOL_CHI2 = 1e-3, 1e-4
ATOL_NN = 2e-5
ATOL_POS = 1e-3
ATOL_DOCA = 1e-4


def sub_batch(b, events):
    """Events `events` of batch b as a new batch (hit ids renumbered)."""
    events = list(events)
    out = dict(n_events=len(events), mode=b.get("mode", "A"))
    so, ho = [0], [0]
    seed_idx, hit_idx = [], []
    for e in events:
        s0, s1 = int(b["seed_off"][e]), int(b["seed_off"][e + 1])
        h0, h1 = int(b["hit_off"][e]), int(b["hit_off"][e + 1])
        seed_idx.append(np.arange(s0, s1)); hit_idx.append(np.arange(h0, h1))
        so.append(so[-1] + s1 - s0); ho.append(ho[-1] + h1 - h0)
    si = np.concatenate(seed_idx) if seed_idx else np.zeros(0, int)
    hi = np.concatenate(hit_idx) if hit_idx else np.zeros(0, int)
    out["seed_off"] = np.array(so, np.int32)
    out["hit_off"] = np.array(ho, np.int32)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "seed_track"):
        if k in b:
            out[k] = b[k][si]
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer", "hit_track"):
        if k in b:
            out[k] = b[k][hi]
    out["_seed_map"] = si
    out["_hit_map"] = hi
    return out


def gpu_per_seed(gpu, n_seeds):
    """Scatter the GPU's packed tracks back to per-seed arrays."""
    t = gpu["tracks"]
    has = np.zeros(n_seeds, bool)
    hits = np.full((n_seeds, 4), -1, np.int64)
    state = np.zeros((n_seeds, 5))
    chi2 = np.zeros(n_seeds); nn = np.zeros(n_seeds); ndof = np.zeros(n_seeds, int)
    s = t["seed"].astype(np.int64)
    has[s] = True
    hits[s] = t["hit"]
    state[s] = np.stack([t["x"], t["y"], t["tx"], t["ty"], t["qop"]], 1)
    chi2[s] = t["chi2"]; nn[s] = t["nn"]; ndof[s] = t["ndof"]
    return dict(has=has, hits=hits, state=state, chi2=chi2, nn=nn, ndof=ndof)


def _close(a, b, rtol, atol):
    return np.abs(a - b) <= np.maximum(rtol * np.maximum(np.abs(a), np.abs(b)), atol)


def compare_tracks(batch, orc, gpu, hit_map_gpu=None, atol_nn=ATOL_NN):
    """orc: oracle.reconstruct(batch); gpu: ds.decode output for the same batch.
    hit_map_gpu: optional function mapping GPU hit ids to batch hit ids.
    atol_nn: response tolerance (a trained network amplifies the FP32 rounding
    of its inputs more than the fixed-seed one)."""
    S = len(orc["status"])
    E = int(batch["n_events"])
    g = gpu_per_seed(gpu, S)
    if hit_map_gpu is not None:
        g["hits"] = np.where(g["hits"] >= 0, hit_map_gpu(g["hits"]), -1)
    t = gpu["tracks"]
    # packed order: (event, seed) ascending, trk_off consistent with it
    assert np.all(np.diff(t["seed"].astype(np.int64)) > 0)
    ev_of_seed = np.repeat(np.arange(E), np.diff(batch["seed_off"]))
    assert np.array_equal(t["event"], ev_of_seed[t["seed"]])
    cnt = np.bincount(t["event"], minlength=E)
    assert np.array_equal(np.diff(gpu["trk_off"]), cnt)
    o_has = orc["status"] == 2
    o_hits = orc["hits"].astype(np.int64)
    diff = (o_has != g["has"]) | (o_has & g["has"] & np.any(o_hits != g["hits"], axis=1))
    small = orc["margin"] < MARGIN
    excused = np.zeros(S, bool)
    for s in np.nonzero(diff)[0]:
        if small[s]:
            excused[s] = True
            continue
        e = ev_of_seed[s]
        s0, s1 = batch["seed_off"][e], batch["seed_off"][e + 1]
        mine = set(o_hits[s][o_hits[s] >= 0]) | set(g["hits"][s][g["hits"][s] >= 0])
        for q in range(s0, s1):
            if q != s and small[q]:
                theirs = set(o_hits[q][o_hits[q] >= 0]) | set(g["hits"][q][g["hits"][q] >= 0])
                if mine & theirs:
                    excused[s] = True
                    break
    same = o_has & g["has"] & ~diff
    rep = dict(n_tracks_oracle=int(o_has.sum()), n_tracks_gpu=int(g["has"].sum()), n_diff=int(diff.sum()),
               n_excused=int(excused.sum()), unexcused=np.nonzero(diff & ~excused)[0].tolist(),
               n_same=int(same.sum()))
    if same.any():
        st_o, st_g = orc["state"][same], g["state"][same]
        ok_par = _close(st_o, st_g, RTOL_PAR, ATOL_PAR)
        ok_chi2 = _close(orc["chi2"][same], g["chi2"][same], RTOL_CHI2, ATOL_CHI2)
        ok_nn = np.abs(orc["nn"][same] - g["nn"][same]) <= atol_nn
        ok_ndof = orc["ndof"][same] == g["ndof"][same]
        rel_chi2 = np.abs(orc["chi2"][same] - g["chi2"][same]) / np.maximum(orc["chi2"][same], ATOL_CHI2 / RTOL_CHI2)
        rep.update(bad_par=int((~ok_par).sum()), bad_chi2=int((~ok_chi2).sum()), bad_nn=int((~ok_nn).sum()),
                   bad_ndof=int((~ok_ndof).sum()),
                   max_rel_par=float(np.max(np.abs(st_o - st_g) / np.maximum(np.abs(st_o), ATOL_PAR / RTOL_PAR))),
                   max_rel_chi2=float(np.max(rel_chi2)),
                   rel_chi2_q=[float(np.quantile(rel_chi2, q)) for q in (0.5, 0.99, 0.999)],
                   max_abs_nn=float(np.max(np.abs(orc["nn"][same] - g["nn"][same]))))
    log_report("tracks", rep)
    return rep


def log_report(kind, rep):
    """Append a parity report to the JSON-lines file named by DS_PARITY_LOG
    (if set), tagged with the running test, and print a one-line summary."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    keys = ("n_tracks_oracle", "n_same", "n_diff", "n_excused", "max_rel_chi2", "n_oracle", "n_gpu",
            "n_unexcused", "max_pos_err")
    print(f"parity[{kind}] {test}: " + ", ".join(f"{k}={rep[k]}" for k in keys if k in rep))
    path = os.environ.get("DS_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(kind=kind, test=test, **{k: v for k, v in rep.items()
                                                               if k not in ("unexcused", "bad_pos_pairs")})) + "\n")


def assert_tracks_match(rep):
    n = max(rep["n_tracks_oracle"], 1)
    assert rep["unexcused"] == [], rep
    assert rep["n_excused"] <= int(0.001 * n), rep
    for k in ("bad_par", "bad_chi2", "bad_nn", "bad_ndof"):
        assert rep.get(k, 0) == 0, rep


def compare_vertices(cfg, gpu):
    """Feed the GPU's FP32 track records to the FP64 oracle vertexer and compare."""
    t = gpu["tracks"]
    ov = oracle.vertex(cfg, gpu["trk_off"], t["x"], t["y"], t["tx"], t["ty"], t["qop"])
    gv = gpu["vertices"]
    # packed order and offsets
    key_g = gv["event"].astype(np.int64) * (1 << 40) + gv["i"].astype(np.int64) * (1 << 20) + gv["j"]
    assert np.all(np.diff(key_g) > 0)
    E = len(gpu["trk_off"]) - 1
    assert np.array_equal(np.diff(gpu["vtx_off"]), np.bincount(gv["event"], minlength=E))
    go = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(gv["i"], gv["j"]))}
    oo = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(ov["i"], ov["j"]))}
    unexcused, excused = [], 0
    for p in set(go) ^ set(oo):
        if p in oo:
            m = ov["margin"][oo[p]]
        else:
            i, j = p
            r = oracle.poca(cfg, [t["x"][i], t["y"][i], t["tx"][i], t["ty"][i], t["qop"][i]],
                            [t["x"][j], t["y"][j], t["tx"][j], t["ty"][j], t["qop"][j]])
            m = abs(r["doca"] - cfg["doca_max"]) / cfg["doca_max"]
        if m < MARGIN:
            excused += 1
        else:
            unexcused.append(p)
    both = sorted(set(go) & set(oo))
    gi = np.array([go[p] for p in both], int)
    oi = np.array([oo[p] for p in both], int)
    rep = dict(n_oracle=len(oo), n_gpu=len(go), n_excused=excused, unexcused=unexcused[:20],
               n_unexcused=len(unexcused), n_fp64=int(np.sum(gv["flags"] & 1)))
    if len(both):
        gpos = np.stack([gv["x"][gi], gv["y"][gi], gv["z"][gi]], 1)
        dpos = np.abs(gpos - ov["pos"][oi]).max(1)
        big = np.abs(ov["pos"][oi]).max(1).astype(np.float32)
        tol = np.maximum(ATOL_POS, 2.0 * np.spacing(big).astype(np.float64))
        bad = dpos > tol
        rep.update(max_pos_err=float(dpos.max()), n_bad_pos=int(bad.sum()),
                   max_pos_err_within_8m=float(dpos[big < 8192].max()) if np.any(big < 8192) else 0.0,
                   max_doca_err=float(np.max(np.abs(gv["doca"][gi] - ov["doca"][oi]))),
                   bad_pos_pairs=[both[k] for k in np.nonzero(bad)[0][:10]])
    log_report("vertices", rep)
    return rep


def assert_vertices_match(rep):
    assert rep["n_unexcused"] == 0, rep
    assert rep["n_excused"] <= max(int(0.001 * max(rep["n_oracle"], 1)), 0), rep
    assert rep.get("n_bad_pos", 0) == 0, rep
    assert rep.get("max_doca_err", 0.0) <= ATOL_DOCA, rep
