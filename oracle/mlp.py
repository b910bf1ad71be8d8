"""FP64 reference of the learned opening criterion's network (test infrastructure).

A 12 -> 64 -> 64 -> 1 multilayer perceptron with ReLU hidden layers and a
linear output that predicts log10 of the relative force error of accepting a
cell (the labels come from oracle.Tree.mlp_samples). Plain numpy, written out
layer by layer, used to check the GPU training kernels' gradients and, with
central finite differences, to check itself.

Parameter vector layout (5057 values), shared with the C forward pass and the
GPU kernels: W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
from __future__ import annotations

import numpy as np

NF, NH = 12, 64
SIZES = (("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + k]).reshape(shape)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SIZES])


def init(seed: int = 0):
    """He-uniform initialisation (ReLU layers), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {"W1": (rng.random((NH, NF)) * 2 - 1) * np.sqrt(6.0 / NF), "b1": np.zeros(NH),
         "W2": (rng.random((NH, NH)) * 2 - 1) * np.sqrt(6.0 / NH), "b2": np.zeros(NH),
         "w3": (rng.random(NH) * 2 - 1) * np.sqrt(3.0 / NH), "b3": np.zeros(1)}
    return pack(p)


def forward(w, X):
    """y [B] and the activations needed by backward."""
    p = unpack(w)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(w, X, t):
    """Mean squared error L = mean((y - t)^2) / 2 and dL/dw (chain rule, layer by layer)."""
    p = unpack(w)
    y, (X, z1, h1, z2, h2) = forward(w, X)
    B = X.shape[0]
    r = y - t
    L = 0.5 * float(np.mean(r * r))
    dy = r / B
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, p["w3"])
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, pack(g)
