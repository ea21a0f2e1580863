"""Training of the learned refinement indicator.

The indicator is a 16 -> 32 -> 32 -> 1 MLP with ReLU hidden layers whose logit
decides the lattice of a cell (high-order when the logit is positive).  Its
features are computed on the GPU by ``Solver.indicator_eval`` (16 scaled local
moments and gradients, see include/slbm.h).  Its labels are the method's own
per-cell lattice loss (``Solver.lattice_loss``: what the low-order lattice
loses in one step, Sec. III.B-D) above LOSS_THRESHOLD, on states of
all-high-order runs; the plain Mach / Knudsen criteria stay the fallback and
the reference its decisions are compared with.

Two trainers of the same algorithm, fed the same mini-batches
(``draw_batches``): ``train`` on the host in FP64 numpy, written out by hand
(forward pass, the logistic loss, back-propagation through the two ReLU
layers, Adam), the reference; and ``train_gpu``, the library's training
kernel (FP16 operands, FP32 accumulation on the tensor cores, FP32 Adam).
Inference runs on the GPU with the same roundings as the training kernel.
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


LOSS_THRESHOLD = 3e-3  # label: the cell's one-step lattice loss above it
ADAM = (0.9, 0.999, 1e-8)  # beta1, beta2, eps
KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")
SHAPES = {"w1": (N_FEAT, N_HID), "b1": (N_HID,), "w2": (N_HID, N_HID), "b2": (N_HID,),
          "w3": (N_HID,), "b3": ()}


def labels(loss: np.ndarray, threshold: float = LOSS_THRESHOLD) -> np.ndarray:
    """0 / 1 labels of per-cell lattice losses."""
    return (np.asarray(loss) > threshold).astype(np.float64)


def pack(w: dict) -> np.ndarray:
    """The 1633 parameters in the training kernel's order (W1 row-major,
    b1, W2, b2, w3, b3)."""
    return np.concatenate([np.asarray(w[k], dtype=np.float64).ravel() for k in KEYS])


def unpack(v) -> dict:
    out, o = {}, 0
    for k in KEYS:
        n = int(np.prod(SHAPES[k])) if SHAPES[k] else 1
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(SHAPES[k]) if SHAPES[k] \
            else float(v[o])
        o += n
    return out


def draw_batches(y: np.ndarray, epochs: int, batch: int, seed: int = 0,
                 balance: bool = True) -> np.ndarray:
    """(steps, batch) sample indices: epochs x (len(y) // batch) steps.  With
    `balance`, each batch draws the two classes equally (the high-order cells
    are a minority)."""
    rng = np.random.default_rng(seed)
    pos, neg = np.flatnonzero(y > 0.5), np.flatnonzero(y <= 0.5)
    steps = max(1, len(y) // batch)
    out = np.empty((epochs * steps, batch), np.int64)
    for s in range(epochs * steps):
        if balance and len(pos) and len(neg):
            out[s] = np.concatenate([rng.choice(pos, batch // 2), rng.choice(neg, batch // 2)])
        else:
            out[s] = rng.choice(len(y), batch)
    return out


def train_steps(w: dict, x: np.ndarray, y: np.ndarray, idx: np.ndarray, lr: float = 3e-3,
                state=None):
    """Adam on the mini-batches idx (steps, batch), in FP64.  Returns the
    weights, the per-step batch losses (before each update) and the Adam
    state (moments, step count) for a continuation."""
    b1, b2, eps = ADAM
    w = {k: (np.array(v, dtype=np.float64) if k != "b3" else float(v)) for k, v in w.items()}
    if state is None:
        mom = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in w.items()}
        vel = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in w.items()}
        t = 0
    else:
        mom, vel, t = state
    losses = np.empty(len(idx))
    for s, rows in enumerate(idx):
        losses[s], g = loss_and_grad(w, x[rows], y[rows])
        t += 1
        for k in w:
            mom[k] = b1 * mom[k] + (1 - b1) * g[k]
            vel[k] = b2 * vel[k] + (1 - b2) * np.square(g[k])
            mh = mom[k] / (1 - b1 ** t)
            vh = vel[k] / (1 - b2 ** t)
            w[k] = w[k] - lr * mh / (np.sqrt(vh) + eps)
    w["b3"] = float(w["b3"])
    return w, losses, (mom, vel, t)


def train(x: np.ndarray, y: np.ndarray, epochs: int = 30, batch: int = 512, lr: float = 3e-3,
          seed: int = 0, balance: bool = True) -> dict:
    """Host reference trainer: He-initialised weights, Adam on the batches of
    draw_batches."""
    idx = draw_batches(y, epochs, batch, seed, balance)
    return train_steps(init_weights(seed), x, y, idx, lr)[0]


def train_gpu(x: np.ndarray, y: np.ndarray, epochs: int = 30, batch: int = 512,
              lr: float = 3e-3, seed: int = 0, balance: bool = True, w0: dict = None,
              idx: np.ndarray = None):
    """The same training on the GPU (slbm_mlp_train): the same initial
    weights and mini-batches as `train`.  Returns (weights, per-step losses)."""
    from . import slbm
    if idx is None:
        idx = draw_batches(y, epochs, batch, seed, balance)
    params = pack(init_weights(seed) if w0 is None else w0).astype(np.float32)
    adam = np.zeros((2, slbm.MLP_PARAMS), np.float32)
    loss, _ = slbm.slbm_mlp_train(x, y, idx, (lr, *ADAM), 0, params, adam)
    return unpack(params.astype(np.float64)), loss


def agreement(w: dict, x: np.ndarray, y: np.ndarray) -> float:
    """Fraction of rows where the indicator's decision equals the label."""
    logit, _ = forward(w, x)
    return float(np.mean((logit > 0) == (y > 0.5)))
