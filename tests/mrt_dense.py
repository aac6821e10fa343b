"""Population-space form of the forced MRT update, Eq. (mrtlbe), built as a
dense 19x19 collision matrix.  Used only to pin the oracle's moment-space
collision: it shares nothing with it but the lattice, which it builds itself.

    fbar' = fbar + (1 + L/2)^{-1} [ -L (fbar - f0) + Phi ]

L is built from its eigen-decomposition: with the weighted inner product
<a, b> = sum_i w_i a_i b_i, the mode vectors 1, c_a (conserved, eigenvalue
0), tr Q (bulk, 1/tau_b), the five traceless combinations of Q (shear,
1/tau_s) and the nine remaining orthogonal "ghost" vectors (eigenvalue 2,
i.e. (1 + L/2)^{-1} L = 1: ghosts projected out) span R^19.  With
G = diag(sqrt(w)) and U the orthonormal image of the modes under G,
L = G U Lambda U^T G^{-1}.  f0 and Phi are the second-order Hermite
equilibrium (Eq. eqf) and forcing term of Sec. II, evaluated at the
physical velocity v = (sum fbar c + F/2) / rho, F a force density.
The linear system is solved with numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def d3q19():
    c = [(0, 0, 0)]
    for a in range(3):
        for s in (1, -1):
            v = [0, 0, 0]
            v[a] = s
            c.append(tuple(v))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        for sa, sb in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
            v = [0, 0, 0]
            v[a], v[b] = sa, sb
            c.append(tuple(v))
    c = np.array(c, dtype=np.float64)
    s = (c * c).sum(1)
    w = np.where(s == 0, 1 / 3, np.where(s == 1, 1 / 18, 1 / 36))
    return c, w


def collision_matrix(c, w, tau_s, tau_b, ghost=2.0):
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    G = np.sqrt(w)
    groups = [
        ([np.ones(len(w)), c[:, 0], c[:, 1], c[:, 2]], 0.0),
        ([Q[:, 0, 0] + Q[:, 1, 1] + Q[:, 2, 2]], 1.0 / tau_b),
        ([Q[:, 0, 0] - Q[:, 1, 1], Q[:, 0, 0] + Q[:, 1, 1] - 2 * Q[:, 2, 2],
          Q[:, 0, 1], Q[:, 0, 2], Q[:, 1, 2]], 1.0 / tau_s),
    ]
    cols, lam = [], []
    for vecs, l in groups:
        M = np.stack([G * v for v in vecs], axis=1)
        q, _ = np.linalg.qr(M)
        cols.append(q)
        lam += [l] * q.shape[1]
    U = np.concatenate(cols, axis=1)
    # ghosts: orthonormal complement of the ten hydrodynamic directions
    P = np.eye(len(w)) - U @ U.T
    uu, ss, _ = np.linalg.svd(P)
    ghosts = uu[:, ss > 0.5]
    U = np.concatenate([U, ghosts], axis=1)
    lam += [ghost] * ghosts.shape[1]
    assert U.shape == (len(w), len(w))
    Lam = np.diag(lam)
    return (G[:, None] * (U @ Lam @ U.T)) / G[None, :]


def equilibrium(c, w, rho, v):
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    return w * (rho + rho * (c @ v) / CS2 + rho * np.einsum("iab,a,b->i", Q, v, v) / (2 * CS2 ** 2))


def forcing(c, w, v, F):
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    VF = np.outer(v, F) + np.outer(F, v)
    return w * ((c @ F) / CS2 + np.einsum("iab,ab->i", Q, VF) / (2 * CS2 ** 2))


def mrt_update(df, F, tau_s, tau_b):
    """Post-collision df* = fbar' - w from the dense Eq. (mrtlbe)."""
    c, w = d3q19()
    fbar = w + np.asarray(df, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    rho = fbar.sum()
    v = (fbar @ c + F / 2) / rho
    L = collision_matrix(c, w, tau_s, tau_b)
    rhs = -L @ (fbar - equilibrium(c, w, rho, v)) + forcing(c, w, v, F)
    R = np.linalg.solve(np.eye(len(w)) + L / 2, rhs)
    return (fbar + R) - w


def bgk_update(df, F, tau):
    """Guo-forced single-relaxation-time update, Eq. (bgklbe)."""
    c, w = d3q19()
    fbar = w + np.asarray(df, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    rho = fbar.sum()
    v = (fbar @ c + F / 2) / rho
    out = fbar + (1.0 / (tau + 0.5)) * (-(fbar - equilibrium(c, w, rho, v)) + tau * forcing(c, w, v, F))
    return out - w


def moments(c, df):
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    return df.sum(), df @ c, np.einsum("i,iab->ab", df, Q)


__all__ = ["d3q19", "collision_matrix", "mrt_update", "bgk_update", "moments",
           "equilibrium", "forcing"]
