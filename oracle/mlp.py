"""FP64 reference of the warm-start network, for checking the GPU kernels.

TEST INFRASTRUCTURE ONLY (same rules as oracle.py: only tests/, the smoke check
and the benchmark's CPU-baseline leg may use it).

The network is the one the library trains and runs: 6 inputs -> three hidden
layers of width 64 with ReLU, relu(z) = max(z, 0) -> 2 outputs, parameters packed
in one vector in the order W1 (64x6, row-major [out][in]), b1, W2 (64x64), b2, W3,
b3, W4 (2x64), b4 (8898 numbers).  The network is not from the paper: it only
proposes the start of the subsystem-I fixed point, whose result does not depend on
it.  Its derivative at z = 0 is taken as 0.
The training loss is the mean over the batch of the squared error summed over
the two outputs.  Gradients are by the chain rule, written out layer by layer;
tests pin them against central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [(64, 6), (64, 64), (64, 64), (2, 64)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unpack(theta: np.ndarray):
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    assert k == theta.size
    return out


def relu(z):
    return np.maximum(z, 0.0)


def relu_grad(z):
    return (z > 0.0).astype(np.float64)


def forward(theta, X):
    """X: (B, 6) -> Y: (B, 2); cache of pre-activations and activations."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    zs, hs = [], [h]
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = relu(z) if li < len(layers) - 1 else z
        hs.append(h)
    return h, (zs, hs)


def loss(theta, X, T):
    Y, _ = forward(theta, X)
    return float(np.mean(np.sum((Y - T) ** 2, axis=1)))


def grad(theta, X, T):
    """d loss / d theta, same packing as theta."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    Y, (zs, hs) = forward(theta, X)
    B = X.shape[0]
    d = 2.0 * (Y - T) / B                       # d loss / d y
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li < len(layers) - 1:
            d = d * relu_grad(zs[li])           # through the activation
        grads[li] = (d.T @ hs[li], d.sum(axis=0))
        d = d @ W                               # to the previous layer's output
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def init(seed: int = 0):
    """He-style initialisation with small output layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (o, i) in enumerate(SIZES):
        s = math.sqrt(2.0 / i) * (0.1 if li == len(SIZES) - 1 else 1.0)
        parts += [rng.normal(0.0, s, o * i), np.zeros(o)]
    return np.concatenate(parts)
