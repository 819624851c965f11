"""Pins of the oracle's Dv1 variant (triplet search in the axial layers,
Algorithm Design section): exhaustive enumeration on tiny events whose only
UTaX hit joins every triplet, noise-free truth recovery (the true UTaX and
UTbX hits are collinear with the magnet point, so every true track comes out
with its four hits), and the bounds that define the variant."""
import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth
from tests import brute
from tests.test_oracle_pins import _tiny_event


@pytest.mark.parametrize("mode", ["nn1", "chi2"])
def test_bruteforce_tiny_events_dv1(mode):
    rng = np.random.default_rng({"nn1": 12, "chi2": 13}[mode])
    w = synth.nn_weights(seed=5, out_bias=-0.5)
    over = dict(variant=1, dv1_w_tri=1e4, dv1_dtx_max=10.0, w2=1e4, dy_tol=1e4)
    if mode == "nn1":
        over["nn_threshold"] = 1.0
    if mode == "chi2":
        over.update(pick_chi2=1, nn_threshold=0.9)
    cfg = synth.default_config(**over)
    n_checked = 0
    for it in range(80):
        ev = _tiny_event(rng, 300 + it)
        if int(np.sum(ev["hit_layer"] == 0)) != 1:
            continue
        cands, best = brute.seed_best(ev, cfg, w, 0)
        oc = oracle.seed_candidates(ev, cfg, w, 0)
        assert oc["n"] == len(cands)
        got = {tuple(h): i for i, h in enumerate(oc["hits"].tolist())}
        for c in cands:
            i = got[tuple(c["hits"])]
            np.testing.assert_allclose(oc["state"][i], c["state"], rtol=1e-9, atol=1e-9)
            assert oc["chi2"][i] == pytest.approx(c["chi2"], rel=1e-8, abs=1e-10)
            np.testing.assert_allclose(oc["phi"][i], c["phi"], rtol=1e-8, atol=1e-9)
        r = oracle.reconstruct(ev, cfg, w)
        if best >= 0:
            assert r["status"][0] == 2 and r["hits"][0].tolist() == cands[best]["hits"]
            n_checked += 1
        else:
            assert r["status"][0] == 0
    assert n_checked >= 8


@pytest.mark.parametrize("mode", ["A"])
def test_noise_free_truth_dv1(mode):
    # mode A only: with the Eq. 4 bending upstream of the kink (mode B) the UT
    # segment of a soft track is not collinear with the magnet point
    b = synth.generate(synth.spec_fixed(1, 40, 0, 160), 41, mode=mode, noise_free=True)
    cfg = synth.default_config(mode=mode, variant=1, pick_chi2=1, nn_threshold=2.0)
    r = oracle.reconstruct(b, cfg, synth.nn_weights())
    st = b["seed_track"]
    for s in range(len(st)):
        assert r["status"][s] == 2, s
        h = r["hits"][s]
        assert np.all(h >= 0) and np.all(b["hit_track"][h] == st[s]), (s, h)


def test_dv1_bounds():
    """The UTbX hit's implied kink must stay below dtx_max, and the UTaX hit
    within w_tri of the magnet-point line; nothing is found outside either."""
    b = synth.generate(synth.spec_fixed(1, 20, 0, 80), 43, noise_free=True)
    w = synth.nn_weights()
    tight = oracle.reconstruct(b, synth.default_config(variant=1, dv1_dtx_max=1e-4, pick_chi2=1, nn_threshold=2.0), w)
    assert np.all(tight["status"] == 0)        # true kinks are far above 1e-4
    narrow = oracle.reconstruct(b, synth.default_config(variant=1, dv1_w_tri=1e-9, pick_chi2=1, nn_threshold=2.0), w)
    wide = oracle.reconstruct(b, synth.default_config(variant=1, pick_chi2=1, nn_threshold=2.0), w)
    assert np.sum(wide["status"] == 2) == len(b["seed_track"])
    assert np.sum(narrow["status"] == 2) <= np.sum(wide["status"] == 2)
