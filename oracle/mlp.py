"""Reference (float64 numpy) of the planner's cost-model network -- TEST INFRASTRUCTURE ONLY.

The paper's transpiler (Sec. IV.A) is a fixed rule; it notes that better schedules could be
found but gives no method.  The library adds a small regression network that predicts the
kernel time of a candidate blocking section from 16 features of it, and lets the prediction
choose among candidate sections.  The paper has no equations for this part, so the functions
below are the textbook definitions, written out plainly:

* network: x (16) -> h1 = relu(W1 x + b1) (64) -> h2 = relu(W2 h1 + b2) (64) -> y = w3 . h2 + b3;
* loss over a batch of B samples: L = (1/B) sum_i (y_i - t_i)^2;
* gradients by the chain rule (relu'(a) = 1 for a > 0, else 0);
* Adam (Kingma & Ba, 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
  theta <- theta - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps), with b1 = 0.9,
  b2 = 0.999, eps = 1e-8.

Flat parameter layout (float32 on the device, float64 here): W1 (64 x 16, row-major), b1 (64),
W2 (64 x 64, row-major), b2 (64), w3 (64), b3 (1) -- 5313 numbers.

Pins (tests/test_oracle_mlp.py, CPU only): central finite differences of the loss against
every gradient entry on a small random instance; a hand-computed one-hidden-unit case; the
closed form of Adam's first step from zero moments (-lr * g / (|g| + eps)); and the relu
gate (a dead unit contributes nothing)."""
from __future__ import annotations

import numpy as np

N_IN, N_H = 16, 64
SHAPES = (("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("w3", (N_H,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5313
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def unpack(theta: np.ndarray) -> dict:
    """Views of the flat parameter vector by name."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[k:k + size].reshape(shape)
        k += size
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(theta: np.ndarray, X: np.ndarray):
    """Outputs y (B,) and the activations (a1, h1, a2, h2) for inputs X (B, 16)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (a1, h1, a2, h2)


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def gradient(theta: np.ndarray, X: np.ndarray, T: np.ndarray):
    """(dL/dtheta as a flat vector, L) by the chain rule."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    y, (a1, h1, a2, h2) = forward(theta, X)
    dy = 2.0 * (y - T) / B                      # (B,)
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    d2 = np.outer(dy, p["w3"]) * (a2 > 0)       # (B, 64)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)              # (B, 64)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return pack(g), float(np.mean((y - T) ** 2))


def adam_step(theta, m, v, grad, step: int, lr: float):
    """One Adam update; `step` counts from 1.  Returns (theta, m, v)."""
    m = BETA1 * np.asarray(m, dtype=np.float64) + (1.0 - BETA1) * grad
    v = BETA2 * np.asarray(v, dtype=np.float64) + (1.0 - BETA2) * grad * grad
    mhat = m / (1.0 - BETA1 ** step)
    vhat = v / (1.0 - BETA2 ** step)
    theta = np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + EPS)
    return theta, m, v
