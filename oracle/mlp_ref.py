"""Plain FP64 numpy reference of the source surrogate's network (test infrastructure).

The network: 16 inputs -> 4 hidden layers of 128 SiLU units -> 10 outputs, y = W x + b per
layer (weights stored out x in, as the CUDA library does).  Training loss: masked mean
squared error, L = sum_ij m_ij (yhat_ij - y_ij)^2 / max(1, sum_ij m_ij).

This file is the checker of the library's forward and backward kernels: plain matrix
products and the chain rule written out, pinned against central finite differences in
tests/test_mlp_reference.py.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

LAYERS = (16, 128, 128, 128, 128, 10)


def param_shapes():
    return [((LAYERS[l + 1], LAYERS[l]), (LAYERS[l + 1],)) for l in range(len(LAYERS) - 1)]


def unpack(theta: np.ndarray):
    """Flat parameter vector -> [(W, b), ...] in the library's order (W then b per layer)."""
    out, o = [], 0
    for (wshape, bshape) in param_shapes():
        nw = wshape[0] * wshape[1]
        W = theta[o:o + nw].reshape(wshape)
        o += nw
        b = theta[o:o + bshape[0]]
        o += bshape[0]
        out.append((W, b))
    assert o == theta.size
    return out


def n_params() -> int:
    return sum(w[0] * w[1] + b[0] for w, b in param_shapes())


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X):
    """Returns the output and the per-layer (input, pre-activation) cache."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    layers = unpack(np.asarray(theta, dtype=np.float64))
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = z if l == len(layers) - 1 else silu(z)
    return h, cache


def loss_and_grad(theta, X, Y, M):
    """Masked MSE and its gradient with respect to the flat parameter vector."""
    yhat, cache = forward(theta, X)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(1.0, M.sum())
    r = (yhat - Y) * M
    loss = float((r * (yhat - Y)).sum() / cnt)
    g = 2.0 * r / cnt                       # dL/dyhat
    layers = unpack(np.asarray(theta, dtype=np.float64))
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        h, z = cache[l]
        dz = g if l == len(layers) - 1 else g * dsilu(z)
        grads.append((dz.T @ h, dz.sum(axis=0)))
        g = dz @ W
    grads.reverse()
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat


def init_params(seed: int = 0) -> np.ndarray:
    """He-style uniform initialisation (the library's initialiser is independent)."""
    rng = np.random.default_rng(seed)
    parts = []
    for (o, i), _ in param_shapes():
        lim = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
