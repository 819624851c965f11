"""Ghost-killer training on synthetic events: the candidates exported by the
GPU path in training mode equal the oracle's enumeration; a network trained
on them (BCE + Adam, FP64) rejects more ghosts than the fixed-seed one at no
loss of efficiency; the GPU path with trained weights still matches the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth, train
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


@pytest.fixture(scope="module")
def trained(torch_cuda):
    cfg = synth.default_config()
    b = synth.config_batch("c2", seed=11, n_events=80)
    x, y, _ = train.training_set(cfg, b, synth.nn_weights())
    hist = []
    w = train.train(x, y, epochs=12, seed=0, history=hist)
    return w, hist, len(y), float(y.mean())


def test_exported_candidates_match_oracle(torch_cuda, weights):
    cfg = synth.default_config(training=1)
    b = synth.config_batch("c2", seed=12, n_events=6)
    x, y, c = train.training_set(synth.default_config(), b, weights)
    assert c["n_total"] == len(c["seed"]) > 0
    rng = np.random.default_rng(0)
    seeds = rng.choice(np.unique(c["seed"]), 60, replace=False)
    differ = []
    for s in seeds:
        mine = np.nonzero(c["seed"] == s)[0]
        assert np.all(np.diff(mine) == 1)                # a seed's candidates are contiguous
        o = oracle.seed_candidates(b, cfg, weights, int(s))
        if o["n"] != len(mine) or not np.array_equal(o["hits"], c["hits"][mine]):
            differ.append(int(s))                       # a hit within float rounding of a window edge
            continue
        # FP32 inputs against FP64: chi2 to 1e-3 relative, pulls to 1e-3 absolute
        assert np.allclose(c["features"][mine], o["phi"], rtol=2e-3, atol=2e-3), s
    assert len(differ) <= 1, differ


def test_training_reduces_ghosts(torch_cuda, trained):
    from paper_2503_13092_b300 import ds
    w, hist, n, ghost_frac = trained
    print(f"training: {n} candidates, ghost fraction {ghost_frac:.3f}, loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    assert hist[-1] < 0.8 * hist[0]
    cfg = synth.default_config()
    b = synth.config_batch("c2", seed=13, n_events=80)

    def score(weights):
        g = ds.Downstream(cfg, weights).run(b)
        t = g["tracks"]
        st = b["seed_track"][t["seed"]]
        h = t["hit"]
        own = ((h >= 0) & (b["hit_track"][np.clip(h, 0, None)] == st[:, None])).sum(1)
        good = (st >= 0) & (own >= 3)
        return good.sum() / max((b["seed_track"] >= 0).sum(), 1), 1 - good.mean()

    eff0, ghost0 = score(synth.nn_weights())
    eff1, ghost1 = score(w)
    print(f"fixed-seed weights: efficiency {eff0:.3f} ghost rate {ghost0:.3f}; "
          f"trained: efficiency {eff1:.3f} ghost rate {ghost1:.3f}")
    assert ghost1 < 0.5 * ghost0
    assert eff1 > eff0 - 0.02


def test_parity_with_trained_weights(torch_cuda, trained):
    from paper_2503_13092_b300 import ds
    w = trained[0]
    cfg = synth.default_config()
    b = synth.config_batch("c2", seed=14, n_events=30)
    g = ds.Downstream(cfg, w).run(b)
    o = oracle.reconstruct(b, cfg, w, n_threads=8)
    # The trained network is far steeper than the fixed-seed one: its response
    # moves by up to ~1e-4 when its FP32 inputs move by their rounding, so the
    # response is compared to 1e-3 here (hits, parameters and chi2 as always).
    rep = parity.compare_tracks(b, o, g, atol_nn=1e-3)
    print("trained-weight parity:", {k: rep[k] for k in ("n_tracks_oracle", "n_diff", "max_abs_nn")})
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(parity.compare_vertices(cfg, g))
