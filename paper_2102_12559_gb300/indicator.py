"""Training of the learned refinement indicator (host side, numpy).

The indicator is a 16 -> 32 -> 32 -> 1 MLP with ReLU hidden layers whose logit
decides the lattice of a cell (high-order when the logit is positive).  Its
features are computed on the GPU by ``Solver.indicator_eval`` (16 scaled local
moments and gradients, see include/slbm.h); its labels are the plain
criterion evaluated on states of all-high-order runs, so the plain criterion
is both the target and the reference the indicator's error is measured against.  Inference runs on
the GPU (tensor cores, FP16 weights and inputs, FP32 accumulation).

Training here is written out by hand: forward pass, the logistic loss, its
gradient by back-propagation through the two ReLU layers, and Adam.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 16
N_HID = 32


def init_weights(seed: int = 0) -> dict:
    """He-initialised weights (W1 16x32, W2 32x32 row-major, input first)."""
    rng = np.random.default_rng(seed)
    return {
        "w1": rng.normal(0.0, np.sqrt(2.0 / N_FEAT), (N_FEAT, N_HID)),
        "b1": np.zeros(N_HID),
        "w2": rng.normal(0.0, np.sqrt(2.0 / N_HID), (N_HID, N_HID)),
        "b2": np.zeros(N_HID),
        "w3": rng.normal(0.0, np.sqrt(1.0 / N_HID), N_HID),
        "b3": 0.0,
    }


def forward(w: dict, x: np.ndarray):
    """Logits of the rows of x (m x 16) and the intermediate activations."""
    z1 = x @ w["w1"] + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["w2"] + w["b2"]
    h2 = np.maximum(z2, 0.0)
    logit = h2 @ w["w3"] + w["b3"]
    return logit, (x, z1, h1, z2, h2)


def loss_and_grad(w: dict, x: np.ndarray, y: np.ndarray):
    """Mean logistic loss of labels y (0 / 1) and its gradient."""
    logit, (x, z1, h1, z2, h2) = forward(w, x)
    m = x.shape[0]
    # log(1 + exp(-s z)) with s = 2y - 1, evaluated stably
    s = 2.0 * y - 1.0
    loss = float(np.mean(np.logaddexp(0.0, -s * logit)))
    p = 1.0 / (1.0 + np.exp(-logit))
    dlogit = (p - y) / m
    g = {"w3": h2.T @ dlogit, "b3": float(dlogit.sum())}
    dz2 = np.outer(dlogit, w["w3"]) * (z2 > 0)
    g["w2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["w2"].T) * (z1 > 0)
    g["w1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def train(x: np.ndarray, y: np.ndarray, epochs: int = 30, batch: int = 512, lr: float = 3e-3,
          seed: int = 0, balance: bool = True) -> dict:
    """Adam on mini-batches.  With `balance`, each batch draws the two classes
    equally (the high-order cells are a small minority)."""
    rng = np.random.default_rng(seed)
    w = init_weights(seed)
    mom = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in w.items()}
    vel = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in w.items()}
    b1, b2, eps, t = 0.9, 0.999, 1e-8, 0
    pos, neg = np.flatnonzero(y > 0.5), np.flatnonzero(y <= 0.5)
    steps = max(1, len(y) // batch)
    for _ in range(epochs):
        for _ in range(steps):
            if balance and len(pos) and len(neg):
                idx = np.concatenate([rng.choice(pos, batch // 2), rng.choice(neg, batch // 2)])
            else:
                idx = rng.choice(len(y), batch)
            _, g = loss_and_grad(w, x[idx], y[idx])
            t += 1
            for k in w:
                mom[k] = b1 * mom[k] + (1 - b1) * g[k]
                vel[k] = b2 * vel[k] + (1 - b2) * np.square(g[k])
                mh = mom[k] / (1 - b1 ** t)
                vh = vel[k] / (1 - b2 ** t)
                w[k] = w[k] - lr * mh / (np.sqrt(vh) + eps)
    w["b3"] = float(w["b3"])
    return w


def agreement(w: dict, x: np.ndarray, y: np.ndarray) -> float:
    """Fraction of rows where the indicator's decision equals the label."""
    logit, _ = forward(w, x)
    return float(np.mean((logit > 0) == (y > 0.5)))
