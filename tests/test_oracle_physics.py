"""Pins of the oracle's vertex-level physics (or_vertex_info): tracks built
from two-body decays of a parent of known mass, boosted to the lab, must give
that mass back under the right hypothesis; the parent momentum and transverse
momentum equal the boosted parent's; the impact parameter to the beam line is
zero for a parent pointing at it and the transverse distance for one moving
across it; Eq. 4 bending (mode B) is undone by the slope at the vertex."""
import math

import numpy as np
import pytest

import oracle
from paper_2503_13092_b300 import synth

M_PI, M_P, M_KS, M_LAMBDA = 139.57039, 938.27208, 497.611, 1115.683


def boost(p4, beta):
    """Lorentz boost of four-vector (E, px, py, pz) by velocity vector beta."""
    b2 = float(beta @ beta)
    g = 1.0 / math.sqrt(1.0 - b2)
    bp = float(beta @ p4[1:])
    E = g * (p4[0] + bp)
    p = p4[1:] + ((g - 1.0) * bp / b2 + g * p4[0]) * beta
    return np.concatenate([[E], p])


def decay(M, m1, m2, P_lab, rng):
    """Lab four-momenta of a two-body decay, parent momentum P_lab (3-vector)."""
    ps = math.sqrt((M * M - (m1 + m2) ** 2) * (M * M - (m1 - m2) ** 2)) / (2 * M)
    d = rng.normal(size=3); d /= np.linalg.norm(d)
    q1 = np.concatenate([[math.hypot(ps, m1)], ps * d])
    q2 = np.concatenate([[math.hypot(ps, m2)], -ps * d])
    E = math.sqrt(P_lab @ P_lab + M * M)
    beta = P_lab / E
    return boost(q1, beta), boost(q2, beta)


def track_through(cfg, v, p3, q):
    """Track state at z_ref whose Eq. 4 trajectory passes through vertex v with direction p3."""
    qop = q / np.linalg.norm(p3)
    g = oracle.gamma(cfg, qop)
    u = v[2] - cfg["z_ref"]
    txv, tyv = p3[0] / p3[2], p3[1] / p3[2]
    tx = txv - 2.0 * g * u                    # slope at z_ref
    x = v[0] - tx * u - g * u * u
    y = v[1] - tyv * u
    return np.array([x, y, tx, tyv, qop])


@pytest.mark.parametrize("mode", ["A", "B"])
@pytest.mark.parametrize("parent,m_pos,m_neg,slot", [("KS", M_PI, M_PI, 0), ("L", M_P, M_PI, 1), ("Lbar", M_PI, M_P, 2)])
def test_mass_of_boosted_decays(mode, parent, m_pos, m_neg, slot):
    cfg = synth.default_config(mode=mode)
    M = M_KS if parent == "KS" else M_LAMBDA
    rng = np.random.default_rng(7 + slot)
    for _ in range(20):
        P = np.array([rng.uniform(-800, 800), rng.uniform(-800, 800), rng.uniform(5e3, 4e4)])
        a, b = decay(M, m_pos, m_neg, P, rng)
        if a[3] <= 0 or b[3] <= 0:
            continue
        v = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), rng.uniform(200, 2000)])
        tp = track_through(cfg, v, a[1:], +1.0)
        tn = track_through(cfg, v, b[1:], -1.0)
        for ti, tj in ((tp, tn), (tn, tp)):              # either order of the pair
            info = oracle.vertex_info(cfg, ti, tj, v)
            assert info[slot] == pytest.approx(M, rel=1e-9)
            assert info[3] == pytest.approx(np.linalg.norm(P), rel=1e-9)
            assert info[4] == pytest.approx(math.hypot(P[0], P[1]), rel=1e-9)
            assert info[7] == pytest.approx(np.linalg.norm(a[1:]), rel=1e-12)
            assert info[8] == pytest.approx(np.linalg.norm(b[1:]), rel=1e-12)
            c = float(a[1:] @ b[1:]) / (np.linalg.norm(a[1:]) * np.linalg.norm(b[1:]))
            assert info[6] == pytest.approx(1.0 - c, rel=1e-6, abs=1e-15)


def test_impact_parameter_to_the_beam_line():
    cfg = synth.default_config()
    v = np.array([30.0, -40.0, 1000.0])
    # parent moving radially away from the axis: its line crosses the beam line
    P = np.array([3.0, -4.0, 100.0]) * 100.0
    ti = track_through(cfg, v, 0.5 * P, 1.0)
    tj = track_through(cfg, v, 0.5 * P, -1.0)
    assert oracle.vertex_info(cfg, ti, tj, v)[5] == pytest.approx(0.0, abs=1e-9)
    # parent moving across (transverse direction perpendicular to V_T): ip = |V_T|
    P = np.array([4.0, 3.0, 100.0]) * 100.0
    ti = track_through(cfg, v, 0.6 * P, 1.0)
    tj = track_through(cfg, v, 0.4 * P, -1.0)
    assert oracle.vertex_info(cfg, ti, tj, v)[5] == pytest.approx(50.0, rel=1e-12)


def test_line_scores_are_the_networks_on_the_features():
    import torch
    cfg = synth.default_config()
    rng = np.random.default_rng(3)
    nets = synth.line_weights()
    n = 12
    tracks = dict(x=rng.normal(0, 300, 2 * n), y=rng.normal(0, 300, 2 * n), tx=rng.normal(0, .1, 2 * n),
                  ty=rng.normal(0, .1, 2 * n), qop=np.tile([1e-4, -2e-4], n), chi2=rng.uniform(0, 3, 2 * n),
                  ndof=np.full(2 * n, 2))
    vtx = dict(i=np.arange(0, 2 * n, 2), j=np.arange(1, 2 * n, 2), pos=rng.normal(0, 100, (n, 3)) + [0, 0, 1000],
               doca=rng.uniform(0, 2, n))
    r = oracle.vertex_infos(cfg, tracks, vtx, nets)
    for k, w in enumerate(nets):
        l1 = torch.nn.Linear(16, 32).double(); l3 = torch.nn.Linear(32, 1).double()
        with torch.no_grad():
            l1.weight.copy_(torch.from_numpy(w["w1"].astype(np.float64)).view(32, 16)); l1.bias.zero_()
            l3.weight.copy_(torch.from_numpy(w["w3"].astype(np.float64)).view(1, 32)); l3.bias.fill_(float(w["b3"]))
            z = l3(torch.relu(l1(torch.from_numpy(r["features"])))).squeeze(1)
        assert np.allclose(torch.sigmoid(z).numpy(), r["score"][:, k], rtol=0, atol=1e-12)
    # features restate the info: spot-check the mass inputs
    assert np.allclose(r["features"][:, 7], (r["info"][:, 0] - M_KS) / 100.0)
    assert np.allclose(r["features"][:, 15], 0.5 * (tracks["chi2"][0::2] + tracks["chi2"][1::2]) / 2.0)
