"""Ghost-killer training (Ghost-Killer Neural Network section).

The paper trains its network on simulated events with the binary
cross-entropy loss (label 1 = ghost, 0 = real track) and the Adam optimiser,
on the candidates the tracking produces in training mode: fixed 100 mm /
10 mm windows and clone killing off, so that the sample is not shaped by the
final selection.  Here the events are the synthetic ones of `synth` (their
generator truth gives the labels), the candidates come from the GPU path in
training mode (`ds_candidates`), and the network is trained on the CPU in
FP64 with plain numpy forward and backward passes, from a fixed seed, so the
result is reproducible bit for bit.

Labels: a candidate is real when its seed is a true track and at least 70 %
of its hits (3 of 3, 3 of 4) belong to that track, the usual matching rule;
every other candidate is a ghost.
"""
from __future__ import annotations

import math

import numpy as np


def label_candidates(batch: dict, seed: np.ndarray, hits: np.ndarray) -> np.ndarray:
    """1.0 for ghosts, 0.0 for real tracks (batch-global seed and hit indices)."""
    st = np.asarray(batch["seed_track"])[seed]
    h = np.asarray(hits)
    ht = np.where(h >= 0, np.asarray(batch["hit_track"])[np.clip(h, 0, None)], -2)
    n_hits = np.sum(h >= 0, axis=1)
    own = np.sum((ht == st[:, None]) & (h >= 0), axis=1)
    real = (st >= 0) & (own >= np.ceil(0.7 * n_hits))
    return (~real).astype(np.float64)


def _xavier(rng, fo, fi):
    a = math.sqrt(6.0 / (fi + fo))
    return rng.uniform(-a, a, (fo, fi))


def init_params(n_in: int, n_h1: int, n_h2: int, seed: int = 0) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    p = dict(w1=_xavier(rng, n_h1, n_in), b1=np.zeros(n_h1))
    if n_h2 > 0:
        p.update(w2=_xavier(rng, n_h2, n_h1), b2=np.zeros(n_h2), w3=_xavier(rng, 1, n_h2)[0])
    else:
        p.update(w3=_xavier(rng, 1, n_h1)[0])
    p["b3"] = np.zeros(1)
    return p


def forward(p: dict, x: np.ndarray):
    """Network output before the sigmoid (z) and the activations for backward."""
    a1 = x @ p["w1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    if "w2" in p:
        a2 = h1 @ p["w2"].T + p["b2"]
        h2 = np.maximum(a2, 0.0)
    else:
        a2 = h2 = None
    last = h2 if h2 is not None else h1
    z = last @ p["w3"] + p["b3"][0]
    return z, (x, a1, h1, a2, h2)


def bce_loss(z: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy of sigmoid(z) against y, written stably in z."""
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def gradients(p: dict, x: np.ndarray, y: np.ndarray):
    """Loss and d loss / d parameter for one minibatch."""
    z, (x, a1, h1, a2, h2) = forward(p, x)
    n = len(y)
    g_z = (1.0 / (1.0 + np.exp(-z)) - y) / n            # d mean-BCE / dz
    g = {}
    last = h2 if h2 is not None else h1
    g["w3"] = last.T @ g_z
    g["b3"] = np.array([g_z.sum()])
    g_last = np.outer(g_z, p["w3"])
    if h2 is not None:
        g_a2 = g_last * (a2 > 0)
        g["w2"] = g_a2.T @ h1
        g["b2"] = g_a2.sum(0)
        g_h1 = g_a2 @ p["w2"]
    else:
        g_h1 = g_last
    g_a1 = g_h1 * (a1 > 0)
    g["w1"] = g_a1.T @ x
    g["b1"] = g_a1.sum(0)
    return bce_loss(z, y), g


class Adam:
    """Adam (Kingma and Ba) with bias correction."""

    def __init__(self, params: dict, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params: dict, grads: dict):
        self.t += 1
        c1, c2 = 1.0 - self.b1 ** self.t, 1.0 - self.b2 ** self.t
        for k in params:
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * grads[k] ** 2
            params[k] -= self.lr * (self.m[k] / c1) / (np.sqrt(self.v[k] / c2) + self.eps)


def normalisation(features: np.ndarray):
    """Per-input mean and 1/std (inputs with no spread get scale 1)."""
    mean = features.mean(0)
    sd = features.std(0)
    return mean, np.where(sd > 0, 1.0 / np.where(sd > 0, sd, 1.0), 1.0)


def train(features: np.ndarray, labels: np.ndarray, n_h1: int = 32, n_h2: int = 32, epochs: int = 20,
          batch_size: int = 1024, lr: float = 3e-3, seed: int = 0, n_in: int | None = None,
          history: list | None = None) -> dict:
    """Train on (features, labels); returns weights in the layout ds_load_nn_weights takes."""
    X = np.asarray(features, np.float64)
    if n_in is not None:
        X = X[:, :n_in]
    y = np.asarray(labels, np.float64)
    mean, scale = normalisation(X)
    Xn = (X - mean) * scale
    p = init_params(X.shape[1], n_h1, n_h2, seed)
    opt = Adam(p, lr=lr)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    for ep in range(epochs):
        order = rng.permutation(len(y))
        tot = 0.0
        for b0 in range(0, len(y), batch_size):
            idx = order[b0:b0 + batch_size]
            loss, g = gradients(p, Xn[idx], y[idx])
            opt.step(p, g)
            tot += loss * len(idx)
        if history is not None:
            history.append(tot / max(len(y), 1))
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    w = dict(n_in=X.shape[1], n_h1=n_h1, n_h2=n_h2, w1=f32(p["w1"]), b1=f32(p["b1"]), w3=f32(p["w3"]),
             b3=np.float32(p["b3"][0]), mean=f32(mean), scale=f32(scale))
    if n_h2 > 0:
        w.update(w2=f32(p["w2"]), b2=f32(p["b2"]))
    else:
        w.update(w2=np.zeros((0, 0), np.float32), b2=np.zeros(0, np.float32))
    return w


def training_set(cfg: dict, batch: dict, weights: dict, device: int = 0) -> tuple:
    """Candidates of `batch` from the GPU path in training mode, with labels."""
    from . import ds
    d = ds.Downstream(cfg, weights, device=device, training=1)
    dev = d.to_device(batch)
    out = d.alloc_tracks(dev["n_events"], dev["n_seeds"])
    d.reconstruct(dev, out)
    c = d.candidates(40 * max(dev["n_seeds"], 1))      # before the counters are cleared
    d.sync()
    d.close()
    # canonical order (seed, then enumeration): the buffer's seed order depends on scheduling
    order = np.argsort(c["seed"], kind="stable")
    for k in ("features", "seed", "hits", "logit"):
        c[k] = c[k][order]
    return c["features"], label_candidates(batch, c["seed"], c["hits"]), c
