"""Ghost-killer trainer (paper_2503_13092_b300/train.py) on the CPU: backward
pass against central finite differences, one Adam step against its closed
form, the stable BCE against the textbook formula, labels on hand-made
candidates, convergence on a separable toy problem and bit-for-bit
reproducibility."""
import numpy as np
import pytest

from paper_2503_13092_b300 import train


def _numgrad(p, x, y, eps=1e-6):
    g = {}
    for k, v in p.items():
        gk = np.zeros_like(v)
        it = np.nditer(v, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = v[i]
            v[i] = old + eps
            lp = train.bce_loss(train.forward(p, x)[0], y)
            v[i] = old - eps
            lm = train.bce_loss(train.forward(p, x)[0], y)
            v[i] = old
            gk[i] = (lp - lm) / (2 * eps)
        g[k] = gk
    return g


@pytest.mark.parametrize("n_h2", [3, 0])
def test_backward_matches_finite_differences(n_h2):
    rng = np.random.default_rng(1)
    p = train.init_params(5, 4, n_h2, seed=3)
    for k in p:                      # biases away from zero so every ReLU is decided
        p[k] = p[k] + rng.normal(0, 0.3, p[k].shape)
    x = rng.normal(size=(8, 5))
    y = rng.integers(0, 2, 8).astype(float)
    loss, g = train.gradients(p, x, y)
    assert loss == pytest.approx(train.bce_loss(train.forward(p, x)[0], y))
    ng = _numgrad(p, x, y)
    for k in p:
        assert np.allclose(g[k], ng[k], rtol=1e-5, atol=1e-8), k


def test_adam_first_step_closed_form():
    # after one step m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    p = dict(a=np.array([1.0, -2.0, 0.5]))
    g = dict(a=np.array([0.3, -1e-3, 5.0]))
    opt = train.Adam(p, lr=0.01, eps=1e-8)
    opt.step(p, g)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(p["a"], want, rtol=0, atol=1e-15)


def test_bce_matches_textbook_formula():
    z = np.linspace(-8, 8, 33)
    y = (np.arange(33) % 2).astype(float)
    f = 1 / (1 + np.exp(-z))
    ref = -np.mean(y * np.log(f) + (1 - y) * np.log(1 - f))
    assert train.bce_loss(z, y) == pytest.approx(ref, rel=1e-12)


def test_labels():
    batch = dict(seed_track=np.array([7, -1, 9]), hit_track=np.array([7, 7, 7, 7, 9, 3, -1]))
    seed = np.array([0, 0, 0, 1, 2])
    hits = np.array([[0, 1, 2, 3],       # 4 of 4 own hits: real
                     [0, 1, 4, -1],      # 2 of 3: ghost
                     [0, 1, 5, 2],       # 3 of 4: real
                     [0, 1, 2, 3],       # fake seed: ghost
                     [4, 5, 6, -1]])     # 1 of 3: ghost
    assert train.label_candidates(batch, seed, hits).tolist() == [0, 1, 0, 1, 1]


def test_converges_on_separable_toy_and_is_reproducible():
    rng = np.random.default_rng(5)
    n = 4000
    y = rng.integers(0, 2, n).astype(float)
    x = rng.normal(size=(n, 16)) + 2.5 * y[:, None] * np.eye(16)[0]   # one informative input
    x[:, 3] = 4.0                                                      # a constant input
    hist = []
    w = train.train(x, y, epochs=15, batch_size=256, lr=3e-3, seed=2, history=hist)
    assert hist[-1] < 0.5 * hist[0]
    z = train.forward(dict(w1=w["w1"].astype(float), b1=w["b1"].astype(float), w2=w["w2"].astype(float),
                           b2=w["b2"].astype(float), w3=w["w3"].astype(float), b3=np.array([float(w["b3"])])),
                      (x - w["mean"]) * w["scale"])[0]
    acc = np.mean((z > 0) == (y > 0.5))
    assert acc > 0.88        # the two classes overlap: Bayes accuracy ~0.89
    w2 = train.train(x, y, epochs=15, batch_size=256, lr=3e-3, seed=2)
    for k in ("w1", "b1", "w2", "b2", "w3", "mean", "scale"):
        assert np.array_equal(w[k], w2[k])
    assert w["scale"][3] == 1.0
