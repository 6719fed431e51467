"""ORACLE — test infrastructure only.

The cost model's network in plain numpy FP64: two ReLU hidden layers and a
linear output of one predicted log-time per kernel variant,

    H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),  Y = H2 W3^T + b3,

trained on the masked mean squared error

    loss = sum(mask * (Y - T)^2) / sum(mask)

with Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Backward pass written from the chain rule; pinned by central finite
differences in the tests.  Weight layout matches the library: W1 [H, F],
W2 [H, H], W3 [V, H], row-major.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(F: int, H: int, V: int) -> dict:
    return {"W1": (H, F), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (V, H), "b3": (V,)}


def forward(p: dict, X: np.ndarray):
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss(Y, T, mask) -> float:
    return float(np.sum(mask * (Y - T) ** 2) / np.sum(mask))


def backward(p: dict, cache, Y, T, mask) -> dict:
    X, Z1, H1, Z2, H2 = cache
    dY = 2.0 * mask * (Y - T) / np.sum(mask)
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dH2 = dY @ p["W3"]
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of step t (t starts at 1); state holds m_<name>, v_<name>."""
    for k in PARAM_NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] ** 2
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p
