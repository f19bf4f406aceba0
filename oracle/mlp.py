"""Multilayer perceptron of the learned control variate (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper has no learned component; this restates, plainly, the network the
engine trains on its own prices and sensitivities (an extension of the
method, not a passage of the paper):

* layers l = 1..L with weights W_l (out x in) and biases b_l;
  h_0 = x, z_l = W_l h_{l-1} + b_l, h_l = softplus(z_l) for l < L and the
  output y = z_L (no activation);  softplus(z) = log(1 + e^z).
* loss = (1/B) sum_b sum_j w_j (y_bj - t_bj)^2 over a batch of B samples
  with per-output weights w_j.
* gradients by the chain rule (backpropagation):
  dL/dy = (2/B) w (y - t); for each layer from the top,
  dW_l = dz_l^T h_{l-1}, db_l = column sums of dz_l, dh_{l-1} = dz_l W_l,
  dz_{l-1} = dh_{l-1} * softplus'(z_{l-1}), softplus' = logistic sigmoid.
* Adam (Kingma & Ba, ICLR 2015): m = b1 m + (1 - b1) g,
  v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Samples are rows (batch-major arrays [B, features]), as on the device.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

Params = List[Tuple[np.ndarray, np.ndarray]]


def softplus(z: np.ndarray) -> np.ndarray:
    return np.logaddexp(0.0, z)


def sigmoid(z: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def init(widths: Sequence[int], rng: np.random.Generator) -> Params:
    """Uniform(-1/sqrt(in), 1/sqrt(in)) weights and biases per layer."""
    out = []
    for fin, fout in zip(widths[:-1], widths[1:]):
        a = 1.0 / np.sqrt(fin)
        out.append((rng.uniform(-a, a, (fout, fin)), rng.uniform(-a, a, fout)))
    return out


def forward(params: Params, x: np.ndarray):
    """Network output y [B, out] and the per-layer (h_{l-1}, z_l) pairs."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = softplus(z) if l < len(params) - 1 else z
    return h, cache


def loss(params: Params, x, t, w) -> float:
    y, _ = forward(params, x)
    return float(np.mean(np.sum(np.asarray(w) * (y - t) ** 2, axis=1)))


def backward(params: Params, x, t, w):
    """(loss, [(dW_l, db_l)]) of the weighted mean squared error."""
    y, cache = forward(params, x)
    B = y.shape[0]
    w = np.asarray(w, dtype=np.float64)
    L = float(np.mean(np.sum(w * (y - t) ** 2, axis=1)))
    dz = (2.0 / B) * w * (y - t)
    grads: Params = [None] * len(params)  # type: ignore[list-item]
    for l in range(len(params) - 1, -1, -1):
        h_prev, _ = cache[l]
        W, _ = params[l]
        grads[l] = (dz.T @ h_prev, dz.sum(axis=0))
        if l > 0:
            _, z_prev = cache[l - 1]
            dz = (dz @ W) * sigmoid(z_prev)
    return L, grads


def input_gradient(params: Params, x: np.ndarray, j: int) -> np.ndarray:
    """d y_j / d x for every sample [B, in] (chain rule back to the input)."""
    y, cache = forward(params, x)
    dz = np.zeros_like(y)
    dz[:, j] = 1.0
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dh = dz @ W
        if l > 0:
            _, z_prev = cache[l - 1]
            dz = dh * sigmoid(z_prev)
    return dh


def adam(params: Params, grads: Params, state: dict, lr: float, b1: float = 0.9,
         b2: float = 0.999, eps: float = 1e-8) -> Params:
    """One Adam step; ``state`` holds m, v (lists like params) and the step t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    ms = state.setdefault("m", [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    vs = state.setdefault("v", [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m = b1 * ms[l][k] + (1.0 - b1) * g
            v = b2 * vs[l][k] + (1.0 - b2) * g * g
            ms[l] = (m, ms[l][1]) if k == 0 else (ms[l][0], m)
            vs[l] = (v, vs[l][1]) if k == 0 else (vs[l][0], v)
            mh, vh = m / (1.0 - b1 ** t), v / (1.0 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append((new[0], new[1]))
    return out
