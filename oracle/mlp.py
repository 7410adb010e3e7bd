"""FP64 oracle of the learned early-stop network -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component (its search stops only by Alg. 1's rule).  This module is
the reference for the build's addition: a 16 -> 64 -> 64 -> 1 ReLU network whose logit z
predicts, from the state of a beam search after a hop, whether the top-k result list is
already final; the search stops when z >= logit(threshold).

Parameter vector layout (float, length N_PARAMS), row-major:
    W1 [64, 16] | b1 [64] | W2 [64, 64] | b2 [64] | w3 [64] | b3 [1]
Input normalisation: x_hat = (x - mu) / sigma with per-feature mu, sigma of the training set.
Loss: mean binary cross-entropy with logits,
    l(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)).
Adam: m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
      p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

F, H = 16, 64
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        size = int(np.prod(shape))
        out[name] = p[o:o + size].reshape(shape)
        o += size
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def forward(p, X):
    """Logits z [B] and the activations needed by backward."""
    w = unpack(p)
    X = np.asarray(X, np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["w3"] + w["b3"][0]
    return z, (X, a1, h1, a2, h2)


def bce(z, y) -> float:
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(p, X, y):
    """Mean BCE-with-logits loss and its gradient with respect to the parameter vector."""
    w = unpack(p)
    z, (X, a1, h1, a2, h2) = forward(p, X)
    B = X.shape[0]
    y = np.asarray(y, np.float64)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, w["w3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(0)
    return bce(z, y), pack(g)


def adam(p, m, v, g, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (seeded; used as an input by tests)."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.uniform(-1, 1, (H, F)) * np.sqrt(6 / F), "b1": np.zeros(H),
         "W2": rng.uniform(-1, 1, (H, H)) * np.sqrt(6 / H), "b2": np.zeros(H),
         "w3": rng.uniform(-1, 1, H) * np.sqrt(6 / H), "b3": np.zeros(1)}
    return pack(d)
