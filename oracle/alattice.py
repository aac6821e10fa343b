"""Lattice offset parameter a_L of Appendix A (FP64, numpy).

Test infrastructure; part of the oracle.

The interpolated velocity of a regularised Stokeslet on its own position,
with the k = 0 mode removed (Appendix A):

    (1/a_L)_ab = (6 pi / V) sum_{k != 0} |delta^P(k; R)|^2 / k^2 (delta_ab - k_a k_b / k^2)

with k = 2 pi m / n per axis, m in (-n/2, n/2], |k|^2 the continuum
wavenumber squared, and delta^P(k; R) = sum_r delta^P(r - R) e^{-i k.r}
the lattice transform of the spreading stencil.  The stencil is a product
over axes, so delta^P(k; R) is the product of three one-dimensional sums
over the 4 nodes of each axis.  The normalisation 1/V follows from the
Fourier convention v(r) = (1/V) sum_k v(k) e^{ik.r} of the same appendix.
"""
from __future__ import annotations

import math

import numpy as np


def _phi(r):
    s = abs(r)
    if s <= 1:
        return (3 - 2 * s + math.sqrt(1 + 4 * s - 4 * s * s)) / 8
    if s <= 2:
        return (5 - 2 * s - math.sqrt(-7 + 12 * s - 4 * s * s)) / 8
    return 0.0


def _axis_transform(n, X):
    m = np.arange(n)
    m = np.where(m > n // 2, m - n, m)
    k = 2 * np.pi * m / n
    b = math.floor(X) - 1
    d = np.zeros(n, dtype=np.complex128)
    for j in range(b, b + 4):
        d += _phi(j - X) * np.exp(-1j * k * j)
    return k, d


def inv_aL_tensor(n, R):
    """The 3x3 tensor (1/a_L)_ab for a lattice n = (nx, ny, nz) and point R."""
    ks, ds = zip(*[_axis_transform(int(n[a]), float(R[a])) for a in range(3)])
    kx, ky, kz = np.meshgrid(ks[0], ks[1], ks[2], indexing="ij")
    d2 = (np.abs(ds[0])[:, None, None] ** 2 * np.abs(ds[1])[None, :, None] ** 2
          * np.abs(ds[2])[None, None, :] ** 2)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    d2 = d2.copy()
    d2[0, 0, 0] = 0.0
    kk = (kx, ky, kz)
    T = np.zeros((3, 3))
    V = float(n[0]) * n[1] * n[2]
    for a in range(3):
        for b in range(3):
            proj = (1.0 if a == b else 0.0) - kk[a] * kk[b] / k2
            T[a, b] = 6 * np.pi / V * np.sum(d2 / k2 * proj)
    return T


def aL_along(n, R, direction=None):
    """Scalar a_L: 1 / (d . T . d) along a unit direction, or 3 / tr T."""
    T = inv_aL_tensor(n, R)
    if direction is None:
        return 3.0 / np.trace(T)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return 1.0 / float(d @ T @ d)
