"""FP64 CPU oracle of the learned set-to-parameters network.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU legs may import this module; the CUDA library never calls it and shares no
code with it.

The paper has no learned component beyond the CCCP fit itself (Sec. IV-B..D).
This network follows the agreed extension: it reads an instance as a set and
predicts the parameters of the CCCP estimate Sigma_* = c I + U diag(D) U^T,
either to replace the fit or to start it.

  per point i:    x_i = [location / L (2), q_i (d), y_i (1)]
                  h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), h3 = tanh(h2 W3 + b3)
  set code:       z = mean_i h3_i
  log c:          g = tanh(z Wg1 + bg1),   log c = g . wg2 + bg2
  per direction k (features f_k = [log |u_k|, sum_j M_kj^2] of the fit's
                  first stage):
                  e_k = tanh([z, f_k] Wd1 + bd1),   log D_k = e_k . wd2 + bd2
  loss over a batch of B instances:
                  L = (1/B) sum_b [(log c_b - t_b)^2 + (1/K_b) sum_k (log D_bk - T_bk)^2]

Forward and a hand-derived backward, written plainly in float64.  The flat
parameter vector is laid out as W1, b1, W2, b2, W3, b3, Wg1, bg1, wg2, bg2,
Wd1, bd1, wd2, bd2 (matrices row-major, input dimension first).
"""
from __future__ import annotations

import numpy as np


def param_shapes(in_dim: int, hidden: int = 256, dir_hidden: int = 64):
    H, Hd = hidden, dir_hidden
    return [("W1", (in_dim, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
            ("Wg1", (H, H)), ("bg1", (H,)), ("wg2", (H,)), ("bg2", (1,)),
            ("Wd1", (H + 2, Hd)), ("bd1", (Hd,)), ("wd2", (Hd,)), ("bd2", (1,))]


def num_params(in_dim: int, hidden: int = 256, dir_hidden: int = 64) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(in_dim, hidden, dir_hidden)))


def unpack(theta: np.ndarray, in_dim: int, hidden: int = 256, dir_hidden: int = 64) -> dict:
    out, o = {}, 0
    for name, shape in param_shapes(in_dim, hidden, dir_hidden):
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    return out


def pack(parts: dict, in_dim: int, hidden: int = 256, dir_hidden: int = 64) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes(in_dim, hidden, dir_hidden)])


def forward(theta, X, F, in_dim, hidden=256, dir_hidden=64):
    """One instance: X (n x in_dim) point features, F (K x 2) direction
    features.  Returns (log c, log D (K,), cache for backward)."""
    p = unpack(np.asarray(theta, dtype=np.float64), in_dim, hidden, dir_hidden)
    X = np.asarray(X, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    h3 = np.tanh(h2 @ p["W3"] + p["b3"])
    z = h3.mean(axis=0)
    g = np.tanh(z @ p["Wg1"] + p["bg1"])
    logc = float(g @ p["wg2"] + p["bg2"][0])
    V = np.concatenate([np.repeat(z[None, :], F.shape[0], axis=0), F], axis=1)
    e = np.tanh(V @ p["Wd1"] + p["bd1"])
    logD = e @ p["wd2"] + p["bd2"][0]
    cache = dict(X=X, F=F, h1=h1, h2=h2, h3=h3, z=z, g=g, V=V, e=e)
    return logc, logD, cache


def backward(theta, cache, dlogc, dlogD, in_dim, hidden=256, dir_hidden=64):
    """Gradient of sum(dlogc * log c) + sum(dlogD * log D) with respect to the
    flat parameters (the chain rule written out layer by layer)."""
    p = unpack(np.asarray(theta, dtype=np.float64), in_dim, hidden, dir_hidden)
    H = hidden
    gr = {name: np.zeros(shape) for name, shape in param_shapes(in_dim, hidden, dir_hidden)}
    X, h1, h2, h3, z, g, V, e = (cache[k] for k in ("X", "h1", "h2", "h3", "z", "g", "V", "e"))
    dlogD = np.asarray(dlogD, dtype=np.float64)
    n = X.shape[0]
    # log c head
    gr["wg2"] += dlogc * g
    gr["bg2"][0] += dlogc
    dag = dlogc * p["wg2"] * (1.0 - g * g)
    gr["Wg1"] += np.outer(z, dag)
    gr["bg1"] += dag
    dz = p["Wg1"] @ dag
    # direction head
    gr["wd2"] += e.T @ dlogD
    gr["bd2"][0] += dlogD.sum()
    dae = (dlogD[:, None] * p["wd2"][None, :]) * (1.0 - e * e)
    gr["Wd1"] += V.T @ dae
    gr["bd1"] += dae.sum(axis=0)
    dV = dae @ p["Wd1"].T
    dz = dz + dV[:, :H].sum(axis=0)
    # mean pooling and the point MLP
    dh3 = np.repeat((dz / n)[None, :], n, axis=0)
    da3 = dh3 * (1.0 - h3 * h3)
    gr["W3"] += h2.T @ da3
    gr["b3"] += da3.sum(axis=0)
    dh2 = da3 @ p["W3"].T
    da2 = dh2 * (1.0 - h2 * h2)
    gr["W2"] += h1.T @ da2
    gr["b2"] += da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (1.0 - h1 * h1)
    gr["W1"] += X.T @ da1
    gr["b1"] += da1.sum(axis=0)
    return pack(gr, in_dim, hidden, dir_hidden)


def loss_and_grad(theta, batch, in_dim, hidden=256, dir_hidden=64):
    """batch: list of (X, F, target log c, target log D).  Returns (L, dL/dtheta)."""
    B = len(batch)
    L = 0.0
    grad = np.zeros_like(np.asarray(theta, dtype=np.float64))
    for X, F, tc, tD in batch:
        logc, logD, cache = forward(theta, X, F, in_dim, hidden, dir_hidden)
        K = len(tD)
        L += ((logc - tc) ** 2 + np.sum((logD - tD) ** 2) / K) / B
        dlogc = 2.0 * (logc - tc) / B
        dlogD = 2.0 * (logD - np.asarray(tD)) / (K * B)
        grad += backward(theta, cache, dlogc, dlogD, in_dim, hidden, dir_hidden)
    return float(L), grad


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba), bias-corrected; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
