"""Point-force kinds of Sec. III/IV expanded into monopoles (FP64, numpy).

Test infrastructure; part of the oracle.

  STOKESLET (p, F)        -- one fixed force monopole F at p (Sec. III A).
  STRESSLET (p, f, sep)   -- symmetric collinear force pair (Fig. stresslet):
                             +f at p + (sep/2) f^ and -f at p - (sep/2) f^,
                             dipole strength |f| sep.
  ROTLET    (p, T, arm)   -- four tangential forces in the swastika-like
                             arrangement of Fig. rotlet, in the plane normal
                             to T: with (e1, e2, T^) right-handed,
                             +F e2 at p + (arm/2) e1,  -F e2 at p - (arm/2) e1,
                             -F e1 at p + (arm/2) e2,  +F e1 at p - (arm/2) e2,
                             F = |T| / (2 arm), so the torque is T and the
                             net force is zero.
  COLLOID   (p, F, a)     -- a mobile point colloid of radius a pushed by the
                             external force F (Sec. IV).
e1 is the coordinate axis least aligned with T^ (lowest index on ties),
made orthogonal to T^ and normalised; e2 = T^ x e1.
"""
from __future__ import annotations

import numpy as np

STOKESLET, STRESSLET, ROTLET, COLLOID = 0, 1, 2, 3


def _rotlet_frame(t_hat):
    k = int(np.argmin(np.abs(t_hat)))
    axis = np.zeros(3)
    axis[k] = 1.0
    e1 = axis - np.dot(axis, t_hat) * t_hat
    e1 = e1 / np.linalg.norm(e1)
    e2 = np.cross(t_hat, e1)
    return e1, e2


def expand_points(kind, pos, F, param=None):
    """Return (pos (m,3), f (m,3), mobile (m,), radius (m,)) for n inputs."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 3)
    n = len(pos)
    par = np.zeros(n) if param is None else np.asarray(param, dtype=np.float64).reshape(n)
    P, Fo, M, Rr = [], [], [], []
    for s in range(n):
        p, f = pos[s], F[s]
        if kind == STOKESLET:
            P += [p]; Fo += [f]; M += [0]; Rr += [0.0]
        elif kind == COLLOID:
            P += [p]; Fo += [f]; M += [1]; Rr += [par[s]]
        elif kind == STRESSLET:
            nrm = np.linalg.norm(f)
            d = f / nrm * (par[s] / 2)
            P += [p + d, p - d]; Fo += [f, -f]; M += [0, 0]; Rr += [0.0, 0.0]
        elif kind == ROTLET:
            nrm = np.linalg.norm(f)
            t_hat = f / nrm
            e1, e2 = _rotlet_frame(t_hat)
            h = par[s] / 2
            m = nrm / (2 * par[s])
            P += [p + h * e1, p - h * e1, p + h * e2, p - h * e2]
            Fo += [m * e2, -m * e2, -m * e1, m * e1]
            M += [0] * 4; Rr += [0.0] * 4
        else:
            raise ValueError(f"unknown point kind {kind}")
    if not P:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int32), np.zeros(0)
    return (np.array(P), np.array(Fo), np.array(M, dtype=np.int32), np.array(Rr))


def counter_force(f, n_fluid):
    """Uniform force density that cancels the net point force: -sum f / V_fluid."""
    f = np.asarray(f, dtype=np.float64).reshape(-1, 3)
    if len(f) == 0:
        return np.zeros(3)
    return -f.sum(axis=0) / n_fluid
