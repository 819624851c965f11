"""Dv1 (triplet search) on the GPU against the FP64 oracle, same rules as Dv0
(tests/parity.py)."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("name,kw,over", [
    ("c1", {}, {}),
    ("c1", {}, {"pick_chi2": 1}),
    ("c2", {"n_events": 40}, {}),
    ("c2", {"n_events": 20, "mode": "B"}, {"mode": "B"}),
])
def test_dv1_matches_oracle(torch_cuda, weights, name, kw, over):
    from paper_2503_13092_b300 import ds
    cfg = synth.default_config(variant=1, **over)
    b = synth.config_batch(name, **kw)
    g = ds.Downstream(cfg, weights).run(b)
    assert g["stats"]["status"] == 0, g["stats"]
    o = oracle.reconstruct(b, cfg, weights, n_threads=8)
    rep = parity.compare_tracks(b, o, g)
    print(name, over, {k: rep[k] for k in ("n_tracks_oracle", "n_diff", "n_excused")})
    assert rep["n_tracks_oracle"] > 0
    parity.assert_tracks_match(rep)
    parity.assert_vertices_match(parity.compare_vertices(cfg, g))


def test_dv1_recovers_noise_free_truth(torch_cuda, weights):
    from paper_2503_13092_b300 import ds
    b = synth.generate(synth.spec_fixed(3, 40, 0, 160), 41, noise_free=True)
    cfg = synth.default_config(variant=1, pick_chi2=1, nn_threshold=2.0)
    g = ds.Downstream(cfg, weights).run(b)
    t = g["tracks"]
    assert len(t) == len(b["seed_track"])
    assert np.all(b["hit_track"][t["hit"]] == b["seed_track"][t["seed"]][:, None])
