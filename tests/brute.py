"""Brute-force checker for tiny events (test infrastructure).

An independent route to the oracle's per-seed result: every combination of one
hit per layer (or "absent" when the layer has no hit) is fitted with
numpy.linalg.lstsq on the weighted rows, its features are formed, the network
is evaluated with torch in float64, and the winner is the lexicographic minimum
of the pick key.  seed_best is valid only when every hit of the event qualifies (windows made
huge) and no layer holds more hits than the method keeps (1 in UTaX, 2 in UTaU
and UTbV, k1 in UTbX), so that the k-closest rules admit every combination.

seed_select restates the selection rules themselves (Algorithm Design section,
Dv0 and Dv1), for events whose layers hold more hits than are kept and whose
windows are finite: a hit qualifies when its |dx| is strictly below the window
half-width and its strip extent, widened by dy_tol, contains the predicted y;
qualifying hits are ranked by (|dx|, hit id) with Python's sort and the first
k are kept (k1 in UTbX, then 1 / 2 / 2 in UTaX / UTaU / UTbV).  Dv1 replaces
the first window by triplets: every UTbX hit within the kink bound, joined to
the magnet point, takes the closest UTaX hit within dv1_w_tri of that line;
triplets are ranked by (residual, UTbX id).  Candidates are then fitted and
scored as in seed_best.
"""
import itertools

import numpy as np
import torch


@torch.no_grad()
def torch_mlp(w, phi):
    phi = torch.as_tensor(np.atleast_2d(phi), dtype=torch.float64)
    x = (phi - torch.as_tensor(w["mean"], dtype=torch.float64)) * torch.as_tensor(w["scale"], dtype=torch.float64)
    l1 = torch.nn.Linear(w["n_in"], w["n_h1"]).double()
    l1.weight.data = torch.as_tensor(w["w1"], dtype=torch.float64)
    l1.bias.data = torch.as_tensor(w["b1"], dtype=torch.float64)
    h = torch.relu(l1(x))
    if w["n_h2"]:
        l2 = torch.nn.Linear(w["n_h1"], w["n_h2"]).double()
        l2.weight.data = torch.as_tensor(w["w2"], dtype=torch.float64)
        l2.bias.data = torch.as_tensor(w["b2"], dtype=torch.float64)
        h = torch.relu(l2(h))
    l3 = torch.nn.Linear(h.shape[1], 1).double()
    l3.weight.data = torch.as_tensor(np.asarray(w["w3"])[None, :], dtype=torch.float64)
    l3.bias.data = torch.tensor([float(w["b3"])], dtype=torch.float64)
    return torch.sigmoid(l3(h))[:, 0].detach().numpy()


def seed_best(batch, cfg, w, s):
    """All candidates of seed s by exhaustive enumeration, and the winner index."""
    e = int(np.searchsorted(batch["seed_off"], s, side="right") - 1)
    h0, h1 = int(batch["hit_off"][e]), int(batch["hit_off"][e + 1])
    x_s, y_s, tx, ty, qop, chi2s = (float(batch[k][s]) for k in
                                    ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2"))
    z = np.asarray(cfg["z_layer"]); dxdy = np.asarray(cfg["dxdy"])
    zm = cfg["zmag"][0] + cfg["zmag"][1] * tx ** 2 + cfg["zmag"][2] * ty ** 2 + cfg["zmag"][3] * abs(qop)
    xm = x_s + tx * (zm - cfg["z_seed"])
    ym = y_s + ty * (zm - cfg["z_seed"])
    yl = ym + ty * (z - zm)
    tx_ut = tx + cfg["mp"] * cfg["kappa"] * qop * np.sqrt(1 + tx * tx + ty * ty)
    u_bx = xm + tx_ut * (z[3] - zm) - dxdy[3] * yl[3]
    w1 = cfg["w1a"] + cfg["w1b"] * abs(qop)
    per_layer = [[h for h in range(h0, h1) if batch["hit_layer"][h] == l] for l in range(4)]
    opts = [(p if p else [-1]) for p in per_layer[:3]]
    dv1 = int(cfg.get("variant", 0)) == 1
    if dv1:                                  # Dv1: the UTaX hit is part of every triplet
        assert len(per_layer[0]) == 1
    cands = []
    for hb in per_layer[3]:
        for combo in itertools.product(*opts):
            hits = list(combo) + [hb]
            present = [l for l in range(4) if hits[l] >= 0]
            if len(present) < 3 or (hits[0] < 0 and hits[1] < 0):
                continue
            if dv1 and hits[0] < 0:
                continue
            rows_z = [z[l] - cfg["z_ref"] for l in present] + [zm - cfg["z_ref"]]
            meas = [float(batch["hit_x0"][hits[l]]) + dxdy[l] * yl[l] for l in present] + [xm]
            sw = [1 / cfg["sigma_hit"]] * len(present) + [1 / cfg["sigma_mag"]]
            A = np.array([[1.0, dz] for dz in rows_z]) * np.array(sw)[:, None]
            bvec = np.array(meas) * np.array(sw)
            sol, *_ = np.linalg.lstsq(A, bvec, rcond=None)
            xr, t = sol
            r = bvec - A @ sol
            chi2 = float(r @ r)
            ndof = len(present) - 1
            res = np.zeros(4)
            for l in present:
                res[l] = float(batch["hit_x0"][hits[l]]) + dxdy[l] * yl[l] - (xr + t * (z[l] - cfg["z_ref"]))
            yr = ym + ty * (cfg["z_ref"] - zm)
            q = cfg["mp"] * (t - tx) / cfg["kappa"] / np.sqrt(1 + t * t + ty * ty) if cfg["kappa"] != 0 else qop
            if dv1:
                x_h = float(batch["hit_x0"][hb]) + dxdy[3] * yl[3]
                u_a = x_h + (x_h - xm) / (z[3] - zm) * (z[0] - z[3]) - dxdy[0] * yl[0]
                p13 = abs(float(batch["hit_x0"][hits[0]]) - u_a) / cfg["dv1_w_tri"]
            else:
                p13 = abs(float(batch["hit_x0"][hb]) - u_bx) / w1
            phi = np.array([xr / 1e3, yr / 1e3, t, ty, 1e3 * q, chi2 / ndof, 1e3 * qop, chi2s,
                            *(res / cfg["sigma_hit"]), len(present) / 4, p13, tx, ty])
            cands.append(dict(hits=[h if h >= 0 else -1 for h in hits], state=[xr, yr, t, ty, q],
                              chi2=chi2, ndof=ndof, phi=phi))
    if not cands:
        return cands, -1
    f = torch_mlp(w, np.array([c["phi"][: w["n_in"]] for c in cands]))
    for c, fv in zip(cands, f):
        c["f"] = float(fv)
    T = cfg["nn_threshold"]

    def key(c):
        ids = tuple(h if h >= 0 else 1 << 40 for h in c["hits"])
        if cfg["pick_chi2"]:
            return (c["chi2"] / c["ndof"], c["f"], ids)
        return (c["f"], c["chi2"], ids)

    elig = [i for i, c in enumerate(cands) if cfg["pick_chi2"] or c["f"] < T]
    if not elig:
        return cands, -1
    best = min(elig, key=lambda i: key(cands[i]))
    if cfg["pick_chi2"] and not cands[best]["f"] < T:
        return cands, -1
    return cands, best


def _seed_ctx(batch, cfg, s):
    """Magnet point, y at the layers and the predictions of seed s (float64)."""
    e = int(np.searchsorted(batch["seed_off"], s, side="right") - 1)
    x_s, y_s, tx, ty, qop, chi2s = (float(batch[k][s]) for k in
                                    ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2"))
    z = np.asarray(cfg["z_layer"], float)
    dxdy = np.asarray(cfg["dxdy"], float)
    zm = cfg["zmag"][0] + cfg["zmag"][1] * tx ** 2 + cfg["zmag"][2] * ty ** 2 + cfg["zmag"][3] * abs(qop)
    xm = x_s + tx * (zm - cfg["z_seed"])
    ym = y_s + ty * (zm - cfg["z_seed"])
    yl = [ym + ty * (z[l] - zm) for l in range(4)]
    if cfg["first_window_origin"]:
        tx_ut = xm / zm
    else:
        tx_ut = tx + cfg["mp"] * cfg["kappa"] * qop * np.sqrt(1 + tx * tx + ty * ty)
    return dict(e=e, h0=int(batch["hit_off"][e]), h1=int(batch["hit_off"][e + 1]), x_s=x_s, y_s=y_s, tx=tx,
                ty=ty, qop=qop, chi2s=chi2s, z=z, dxdy=dxdy, zm=zm, xm=xm, ym=ym, yl=yl,
                u_bx=xm + tx_ut * (z[3] - zm) - dxdy[3] * yl[3],
                w1=100.0 if cfg["training"] else cfg["w1a"] + cfg["w1b"] * abs(qop),
                w2=10.0 if cfg["training"] else cfg["w2"])


def closest(batch, cfg, ctx, layer, u, y, w, keep):
    """Hits of `layer` in the seed's event with |x0 - u| < w and a strip that,
    widened by dy_tol, contains y; the `keep` first by (|dx|, hit id), as
    (|dx|, id) pairs."""
    q = []
    for h in range(ctx["h0"], ctx["h1"]):
        if int(batch["hit_layer"][h]) != layer:
            continue
        d = abs(float(batch["hit_x0"][h]) - u)
        lo = float(batch["hit_ybeg"][h]) - cfg["dy_tol"]
        hi = float(batch["hit_yend"][h]) + cfg["dy_tol"]
        if d < w and lo <= y <= hi:
            q.append((d, h))
    return sorted(q)[:keep]


def _x_at(batch, ctx, hb, layer):
    """Strip coordinate in `layer` of the line through UTbX hit hb and the magnet point."""
    z, dxdy, yl = ctx["z"], ctx["dxdy"], ctx["yl"]
    x_h = float(batch["hit_x0"][hb]) + dxdy[3] * yl[3]
    txp = (x_h - ctx["xm"]) / (z[3] - ctx["zm"])
    return x_h + txp * (z[layer] - z[3]) - dxdy[layer] * yl[layer]


def first_stage(batch, cfg, ctx):
    """The kept UTbX hits, each with its fixed UTaX hit (Dv1, else None) and
    the value behind network input 13."""
    k1 = int(cfg["k1"])
    if int(cfg.get("variant", 0)) == 1:
        z, dxdy, yl = ctx["z"], ctx["dxdy"], ctx["yl"]
        w_b = cfg["dv1_dtx_max"] * (ctx["zm"] - z[3])
        u0 = ctx["xm"] + ctx["tx"] * (z[3] - ctx["zm"]) - dxdy[3] * yl[3]
        trip = []
        for _, hb in closest(batch, cfg, ctx, 3, u0, yl[3], w_b, 1 << 30):
            a = closest(batch, cfg, ctx, 0, _x_at(batch, ctx, hb, 0), yl[0], cfg["dv1_w_tri"], 1)
            if a:
                trip.append((a[0][0], hb, a[0][1]))
        trip.sort()
        return [(hb, ha, d / cfg["dv1_w_tri"]) for d, hb, ha in trip[:k1]]
    return [(hb, None, d / ctx["w1"])
            for d, hb in closest(batch, cfg, ctx, 3, ctx["u_bx"], ctx["yl"][3], ctx["w1"], k1)]


def _fit_record(batch, cfg, ctx, hits, p13):
    z, dxdy, yl = ctx["z"], ctx["dxdy"], ctx["yl"]
    present = [l for l in range(4) if hits[l] >= 0]
    rows_z = [z[l] - cfg["z_ref"] for l in present] + [ctx["zm"] - cfg["z_ref"]]
    meas = [float(batch["hit_x0"][hits[l]]) + dxdy[l] * yl[l] for l in present] + [ctx["xm"]]
    sw = [1 / cfg["sigma_hit"]] * len(present) + [1 / cfg["sigma_mag"]]
    A = np.array([[1.0, dz] for dz in rows_z]) * np.array(sw)[:, None]
    bvec = np.array(meas) * np.array(sw)
    sol, *_ = np.linalg.lstsq(A, bvec, rcond=None)
    xr, t = sol
    r = bvec - A @ sol
    chi2 = float(r @ r)
    ndof = len(present) - 1
    res = np.zeros(4)
    for l in present:
        res[l] = float(batch["hit_x0"][hits[l]]) + dxdy[l] * yl[l] - (xr + t * (z[l] - cfg["z_ref"]))
    yr = ctx["ym"] + ctx["ty"] * (cfg["z_ref"] - ctx["zm"])
    ty, tx, qop = ctx["ty"], ctx["tx"], ctx["qop"]
    q = cfg["mp"] * (t - tx) / cfg["kappa"] / np.sqrt(1 + t * t + ty * ty) if cfg["kappa"] != 0 else qop
    phi = np.array([xr / 1e3, yr / 1e3, t, ty, 1e3 * q, chi2 / ndof, 1e3 * qop, ctx["chi2s"],
                    *(res / cfg["sigma_hit"]), len(present) / 4, p13, tx, ty])
    return dict(hits=list(hits), state=[xr, yr, t, ty, q], chi2=chi2, ndof=ndof, phi=phi)


def pick(cands, cfg, w):
    """Network responses and the winner index (-1: none) by the pick key."""
    if not cands:
        return -1
    f = torch_mlp(w, np.array([c["phi"][: w["n_in"]] for c in cands]))
    for c, fv in zip(cands, f):
        c["f"] = float(fv)
    T = cfg["nn_threshold"]

    def key(c):
        ids = tuple(h if h >= 0 else 1 << 40 for h in c["hits"])
        if cfg["pick_chi2"]:
            return (c["chi2"] / c["ndof"], c["f"], ids)
        return (c["f"], c["chi2"], ids)

    elig = [i for i, c in enumerate(cands) if cfg["pick_chi2"] or c["f"] < T]
    if not elig:
        return -1
    best = min(elig, key=lambda i: key(cands[i]))
    if cfg["pick_chi2"] and not cands[best]["f"] < T:
        return -1
    return best


def seed_select(batch, cfg, w, s):
    """Seed s through the k-closest selection rules (module docstring):
    (kept UTbX hits, candidates, winner index)."""
    ctx = _seed_ctx(batch, cfg, s)
    kept = first_stage(batch, cfg, ctx)
    cands = []
    for hb, ha, p13 in kept:
        opts = []
        for l, keep in ((0, 1), (1, 2), (2, 2)):
            if l == 0 and ha is not None:
                opts.append([ha])
                continue
            sel = closest(batch, cfg, ctx, l, _x_at(batch, ctx, hb, l), ctx["yl"][l], ctx["w2"], keep)
            opts.append([h for _, h in sel] or [-1])      # absent only when nothing qualifies
        for combo in itertools.product(*opts):
            hits = list(combo) + [hb]
            n = sum(h >= 0 for h in hits)
            if n < 3 or (hits[0] < 0 and hits[1] < 0):
                continue
            cands.append(_fit_record(batch, cfg, ctx, hits, p13))
    return kept, cands, pick(cands, cfg, w)
