"""Vertex-level physics on the GPU (ds_vertex_physics) against the FP64
oracle fed the GPU's own FP32 track and vertex records, and against boosted
two-body decays of known mass built directly as records."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth
from tests.test_oracle_physics import M_KS, M_LAMBDA, M_P, M_PI, decay, track_through

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13092_b300 import build
    build.build()
    return torch


def physics(torch, d, out, vout, cap=None):
    from paper_2503_13092_b300 import ds
    n_v = int(vout["n_vertices"].cpu()[0])
    cap = n_v if cap is None else cap
    info = torch.zeros((max(cap, 1), 64), dtype=torch.uint8, device="cuda")
    ds.ds_vertex_physics(d.ctx, out, vout, info)
    d.sync()
    return info.cpu().numpy().view(ds.VINFO_DTYPE).reshape(-1)[:min(cap, n_v)]


@pytest.mark.parametrize("mode", ["A", "B"])
def test_matches_oracle_on_reconstructed_vertices(torch_cuda, weights, mode):
    from paper_2503_13092_b300 import ds
    cfg = synth.default_config(mode=mode)
    b = synth.config_batch("c2", seed=31, n_events=30, mode=mode)
    nets = synth.line_weights()
    d = ds.Downstream(cfg, weights)
    ds.ds_load_line_weights(d.ctx, nets)
    dev = d.to_device(b)
    out = d.alloc_tracks(dev["n_events"], dev["n_seeds"])
    d.reconstruct(dev, out)
    vout = d.alloc_vertices(dev["n_events"], 16 * dev["n_seeds"] + 4096)
    d.vertex(out, vout)
    got = physics(torch_cuda, d, out, vout)
    g = ds.decode(out, vout)
    t, v = g["tracks"], g["vertices"]
    assert len(v) > 100 and len(got) == len(v)
    o = oracle.vertex_infos(cfg, dict(x=t["x"], y=t["y"], tx=t["tx"], ty=t["ty"], qop=t["qop"], chi2=t["chi2"],
                                      ndof=t["ndof"]),
                            dict(i=v["i"], j=v["j"], x=v["x"], y=v["y"], z=v["z"], doca=v["doca"]), nets)
    I = o["info"]
    close = lambda a, b, r, at: np.all(np.abs(a - b) <= np.maximum(r * np.abs(b), at))
    for k, name in enumerate(("m_pipi", "m_ppi", "m_pip")):
        assert close(got[name], I[:, k], 2e-5, 1e-3), (name, np.max(np.abs(got[name] - I[:, k]) / I[:, k]))
    assert close(got["p"], I[:, 3], 1e-5, 1e-3) and close(got["pt"], I[:, 4], 1e-5, 1e-2)
    vt = np.hypot(v["x"], v["y"])
    assert np.all(np.abs(got["ip"] - I[:, 5]) <= 1e-5 * vt + 1e-3)
    assert close(got["one_minus_cos"], I[:, 6], 1e-4, 1e-10)
    for k, name in ((7, "p_pos"), (8, "p_neg"), (9, "pt_pos"), (10, "pt_neg")):
        assert close(got[name], I[:, k], 1e-5, 1e-3), name
    assert np.max(np.abs(got["score"] - o["score"])) < 1e-4
    assert np.all(got["flags"] == 0)


def test_boosted_decays_give_their_mass(torch_cuda):
    """Records built from K0S, Lambda and anti-Lambda decays boosted up to 60 GeV."""
    from paper_2503_13092_b300 import ds
    t = torch_cuda
    cfg = synth.default_config(mode="B")
    rng = np.random.default_rng(5)
    cases = [(M_KS, M_PI, M_PI, "m_pipi"), (M_LAMBDA, M_P, M_PI, "m_ppi"), (M_LAMBDA, M_PI, M_P, "m_pip")]
    trk, vtx, want = [], [], []
    for M, m_pos, m_neg, name in cases:
        for _ in range(300):
            P = np.array([rng.uniform(-900, 900), rng.uniform(-900, 900), rng.uniform(2e3, 6e4)])
            a, bb = decay(M, m_pos, m_neg, P, rng)
            if a[3] <= 0 or bb[3] <= 0:
                continue
            vpos = np.array([rng.uniform(-60, 60), rng.uniform(-60, 60), rng.uniform(100, 2200)])
            tp, tn = track_through(cfg, vpos, a[1:], 1.0), track_through(cfg, vpos, bb[1:], -1.0)
            i = len(trk)
            for s in (tp, tn):
                r = np.zeros(1, ds.TRACK_DTYPE)
                r["x"], r["y"], r["tx"], r["ty"], r["qop"], r["ndof"] = s[0], s[1], s[2], s[3], s[4], 2
                trk.append(r)
            vr = np.zeros(1, ds.VERTEX_DTYPE)
            vr["i"], vr["j"], vr["x"], vr["y"], vr["z"] = i, i + 1, vpos[0], vpos[1], vpos[2]
            vtx.append(vr)
            want.append((name, M, float(np.linalg.norm(P))))
    trk = np.concatenate(trk); vtx = np.concatenate(vtx)
    d = ds.Downstream(cfg, synth.nn_weights())
    out = dict(tracks=t.from_numpy(trk.view(np.uint8).reshape(-1, 64).copy()).cuda(),
               trk_off=t.tensor([0, len(trk)], dtype=t.int32, device="cuda"),
               n_tracks=t.tensor([len(trk)], dtype=t.int32, device="cuda"))
    out["_struct"] = ds.ds_tracks(ds._ptr(out["tracks"]), ds._ptr(out["trk_off"]), ds._ptr(out["n_tracks"]),
                                  len(trk), 1)
    vout = dict(vertices=t.from_numpy(vtx.view(np.uint8).reshape(-1, 32).copy()).cuda(),
                vtx_off=t.tensor([0, len(vtx)], dtype=t.int32, device="cuda"),
                n_vertices=t.tensor([len(vtx)], dtype=t.int32, device="cuda"))
    got = physics(t, d, out, vout)
    for k, (name, M, p) in enumerate(want):
        assert got[name][k] == pytest.approx(M, rel=2e-5), (k, name, p)
        assert got["p"][k] == pytest.approx(p, rel=2e-6)
    # no line networks loaded: responses are zero; a capacity below the count writes a prefix
    assert np.all(got["score"] == 0)
    part = physics(t, d, out, vout, cap=7)
    assert len(part) == 7 and np.array_equal(part.view(np.uint8), got[:7].view(np.uint8))


def _bf16(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def test_tensor_core_lines_match_their_specified_arithmetic(torch_cuda, weights):
    """BF16 line networks (one N = 128 tcgen05 product per 128 vertices)
    against the same arithmetic restated on the CPU from the kernel's own FP32
    vertex quantities; and close to the FP32 networks."""
    from paper_2503_13092_b300 import ds
    t = torch_cuda
    cfg = synth.default_config()
    b = synth.config_batch("c2", seed=33, n_events=40)
    nets = synth.line_weights()
    for k, w in enumerate(nets):        # non-trivial normalisation, folded into the weights on the GPU
        w["mean"] = np.linspace(-0.5, 0.5, 16).astype(np.float32) * (k + 1)
        w["scale"] = np.linspace(0.5, 2.0, 16).astype(np.float32)
        w["b1"] = np.linspace(-0.2, 0.2, 32).astype(np.float32)
    d = ds.Downstream(cfg, weights)
    ds.ds_load_line_weights(d.ctx, nets)
    dev = d.to_device(b)
    out = d.alloc_tracks(dev["n_events"], dev["n_seeds"])
    d.reconstruct(dev, out)
    vout = d.alloc_vertices(dev["n_events"], 16 * dev["n_seeds"] + 4096)
    d.vertex(out, vout)
    fp32 = physics(t, d, out, vout)
    d.set_params(mlp_precision=ds.DS_MLP_BF16)
    tc = physics(t, d, out, vout)
    g = ds.decode(out, vout)
    tr, v = g["tracks"], g["vertices"]
    n = len(v)
    assert n > 300 and len(tc) == n
    names = ("m_pipi", "m_ppi", "m_pip", "p", "pt", "ip", "one_minus_cos", "p_pos", "p_neg", "pt_pos", "pt_neg")
    for k in names:                      # the physics is the same code in both kernels
        assert np.array_equal(tc[k], fp32[k]), k
    f32 = np.float32
    ca = tr["chi2"][v["i"]] / tr["ndof"][v["i"]].astype(f32)
    cb = tr["chi2"][v["j"]] / tr["ndof"][v["j"]].astype(f32)
    F = np.stack([v["x"] / f32(100), v["y"] / f32(100), v["z"] / f32(1000), v["doca"], tc["p"] / f32(1e4),
                  tc["pt"] / f32(1e3), tc["ip"] / f32(10), (tc["m_pipi"] - f32(497.611)) / f32(100),
                  (tc["m_ppi"] - f32(1115.683)) / f32(100), (tc["m_pip"] - f32(1115.683)) / f32(100),
                  tc["p_pos"] / f32(1e4), tc["p_neg"] / f32(1e4), tc["pt_pos"] / f32(1e3), tc["pt_neg"] / f32(1e3),
                  f32(1e3) * tc["one_minus_cos"], f32(0.5) * (ca + cb)], 1).astype(np.float32)
    Fq = _bf16(t, F).astype(np.float64)
    for k, w in enumerate(nets):
        W = w["w1"].astype(np.float64).reshape(32, 16) * w["scale"].astype(np.float64)
        b1 = (w["b1"].astype(np.float64) - W @ w["mean"].astype(np.float64)).astype(np.float32).astype(np.float64)
        Wq = _bf16(t, W.astype(np.float32)).astype(np.float64)
        acc = Fq @ Wq.T
        h = np.maximum(acc + b1, 0.0)
        terms = h * w["w3"].astype(np.float64)
        z = float(w["b3"]) + terms.sum(1)
        want = 1 / (1 + np.exp(-z))
        bound = 0.25 * (1e-5 * (np.abs(terms).sum(1) + np.abs(acc) @ np.abs(w["w3"].astype(np.float64))) + 1e-6)
        err = np.abs(tc["score"][:, k] - want)
        assert np.all(err <= bound + 2e-7), (k, err.max())
        # and the BF16 networks stay close to the FP32 ones
        assert np.max(np.abs(tc["score"][:, k] - fp32["score"][:, k])) < 0.05
