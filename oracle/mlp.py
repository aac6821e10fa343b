"""Oracle of the learned colloid-velocity correction (FP64, numpy).

Test infrastructure; part of the oracle.  The correction is a multilayer
perceptron 27 -> 64 -> 64 -> 3 with SiLU activations,

    h1 = silu(W1 x + b1),  h2 = silu(W2 h1 + b2),  y = W3 h2 + b3,
    silu(z) = z / (1 + e^{-z}),

trained by mean squared error L = (1 / 3B) sum_{b,k} (y_bk - t_bk)^2.  The
input x of a colloid s is its fractional lattice offset R_s - floor(R_s)
(3 numbers) followed by the minimum-image vectors R_j - R_s to its 8
nearest other colloids within R_CUT lattice units, nearest first (equal
distances: lower index first), each divided by FEAT_LENGTH (24 numbers);
absent neighbours are zero vectors.  The neighbour vectors, and the
distances that select and order the neighbours, are float32 (the
network's input precision), each operation rounded once: positions
rounded to float32, d = p_j - p_s, then d - box where d > box/2 and
d + box where d < -box/2, r2 = (dx dx + dy dy) + dz dz, kept where
r2 <= R_CUT^2.

`forward`/`backward` follow these definitions with plain numpy matrix
products.  With `bf16_round=True` they round, as the CUDA kernels do, every
operand of a product to bfloat16 (round to nearest even): the weights, the
input and the activations h1, h2; in the backward pass dL/dy where it
enters the layer-3 weight and bias gradients, and the pre-activation
gradients gz2, gz1 where they enter the weight and bias gradients and
gh1 = gz2 W2 (gh2 = (dL/dy) W3 takes the unrounded dL/dy).  Everything else
stays FP64.
"""
from __future__ import annotations

import numpy as np

DIMS = (27, 64, 64, 3)
FEAT_LENGTH = 4.0  # neighbour vectors are given in units of 4 lattice spacings
N_NEIGH = 8
R_CUT = 8.0        # neighbours farther than this (lattice units) are left out


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed=0):
    """Seeded initial weights (uniform, fan-in scaled), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = {}
    for l, (a, b) in enumerate(zip(DIMS[:-1], DIMS[1:]), start=1):
        lim = np.sqrt(6.0 / a)
        P[f"W{l}"] = rng.uniform(-lim, lim, size=(b, a))
        P[f"b{l}"] = np.zeros(b)
    return P


def forward(P, x, bf16_round=False):
    r = bf16 if bf16_round else (lambda v: np.asarray(v, dtype=np.float64))
    x = r(x)
    z1 = x @ r(P["W1"]).T + P["b1"]
    h1 = r(silu(z1))
    z2 = h1 @ r(P["W2"]).T + P["b2"]
    h2 = r(silu(z2))
    y = h2 @ r(P["W3"]).T + P["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(P, x, t, bf16_round=False):
    y, _ = forward(P, x, bf16_round)
    return float(np.mean((y - t) ** 2))


def backward(P, x, t, bf16_round=False):
    """Gradients of the mean squared error with respect to every parameter."""
    r = bf16 if bf16_round else (lambda v: np.asarray(v, dtype=np.float64))
    y, (xr, z1, h1, z2, h2) = forward(P, x, bf16_round)
    B = x.shape[0]
    gy = 2.0 * (y - t) / (B * y.shape[1])
    gyr = r(gy)
    G = {"W3": gyr.T @ h2, "b3": gyr.sum(0)}
    gh2 = gy @ r(P["W3"])
    gz2 = r(gh2 * dsilu(z2))
    G["W2"] = gz2.T @ h1
    G["b2"] = gz2.sum(0)
    gh1 = gz2 @ r(P["W2"])
    gz1 = r(gh1 * dsilu(z1))
    G["W1"] = gz1.T @ xr
    G["b1"] = gz1.sum(0)
    return G


def features(pos, box):
    """Inputs of every colloid by brute force over all pairs (minimum image,
    float32 neighbour arithmetic as the module docstring states)."""
    pos = np.asarray(pos, dtype=np.float64)
    p = pos.astype(np.float32)
    bf = np.asarray(box, dtype=np.float32)
    half = bf * np.float32(0.5)
    rc2 = np.float32(R_CUT * R_CUT)
    n = len(pos)
    out = np.zeros((n, DIMS[0]))
    out[:, :3] = pos - np.floor(pos)
    for s in range(n):
        d = p - p[s]
        d = np.where(d > half, d - bf, np.where(d < -half, d + bf, d))
        r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        assert r2.dtype == np.float32
        ok = r2 <= rc2
        ok[s] = False
        cand = np.nonzero(ok)[0]
        order = cand[np.argsort(r2[cand], kind="stable")][:N_NEIGH]
        for k, j in enumerate(order):
            out[s, 3 + 3 * k: 6 + 3 * k] = d[j] / np.float32(FEAT_LENGTH)
    return out


def adam(v, g, m, s, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on the flat parameter vector v (returns new v, m, s)."""
    m = b1 * m + (1 - b1) * g
    s = b2 * s + (1 - b2) * g * g
    vh = v - lr * (m / (1 - b1 ** t)) / (np.sqrt(s / (1 - b2 ** t)) + eps)
    return vh, m, s


def flatten(P):
    return np.concatenate([P[k].ravel() for k in param_order()])


def unflatten(v):
    P, o = {}, 0
    for k, shape in zip(param_order(), param_shapes()):
        size = int(np.prod(shape))
        P[k] = np.asarray(v[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return P


def param_order():
    return ["W1", "b1", "W2", "b2", "W3", "b3"]


def param_shapes():
    return [(DIMS[1], DIMS[0]), (DIMS[1],), (DIMS[2], DIMS[1]), (DIMS[2],), (DIMS[3], DIMS[2]), (DIMS[3],)]


__all__ = ["DIMS", "FEAT_LENGTH", "N_NEIGH", "R_CUT", "bf16", "silu", "dsilu", "init_params", "forward", "loss",
           "backward", "features", "adam", "flatten", "unflatten", "param_order", "param_shapes"]
