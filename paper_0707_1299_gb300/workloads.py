"""Seeded synthetic inputs for the benchmark and parity workloads.

Only inputs live here (lattice sizes, relaxation times, point positions,
forces and parameters drawn from numpy PCG64 generators); none of the
method's arithmetic does.  Both the CUDA path and the oracle take their
inputs from this module.

Point-force kinds: 0 Stokeslet, 1 stresslet, 2 rotlet, 3 colloid.

Workloads (lattice units, rho0 = 1):
  stokeslet_32   -- 32^3, tau_s = tau_b = 1/2 (eta = 1/6, every rate 1),
                    one Stokeslet F = (0, 0, 1e-5) at (16.3, 15.7, 16.45),
                    uniform counter-force, 1000 steps, FP64.
  channel_256    -- 256^3 FP32, four independent lattices, 2000 steps:
                    (i) body-force channel, solid planes z = 0 and 255,
                    g = (1e-6, 0, 0); (ii) a Stokeslet F = (0, 0, 1e-5);
                    (iii) a stresslet with force 5e-5 along z and
                    separation 2 (dipole 1e-4); (iv) a rotlet with torque
                    (0, 0, 1e-4) and arm 2; positions (ii)-(iv) uniform in
                    [L/4, 3L/4)^3 from seed 2.
  colloids_512   -- 512^3, 1e5 colloids uniform in the box (seed 3), force
                    (0, 0, -1e-6), radius a = 0.117 (Table I), counter-force.
  replicas       -- 64 independent periodic boxes, sides uniform in
                    {48, 56, ..., 128} (seed 4), 100-2000 colloids each,
                    force 1e-6, 5000 steps.
Every workload takes a size argument so that the same recipe runs at
sizes a CPU oracle finishes in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STOKESLET, STRESSLET, ROTLET, COLLOID = 0, 1, 2, 3
A_TABLE1 = 0.117  # point-particle radius of Table I


@dataclass
class PointSet:
    kind: int
    pos: np.ndarray            # (n, 3)
    F: np.ndarray              # (n, 3)
    param: np.ndarray | None   # (n,) or None


@dataclass
class Problem:
    name: str
    grid: tuple
    tau_s: float
    tau_b: float
    g: tuple = (0.0, 0.0, 0.0)
    walls: tuple | None = None
    counter: bool = True
    a_L: float = float("inf")
    points: list = field(default_factory=list)
    steps: int = 0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def stokeslet_32(L: int = 32, steps: int = 1000) -> Problem:
    c = L / 32.0
    pos = np.array([[16.3 * c, 15.7 * c, 16.45 * c]]) if L == 32 else \
        np.array([[L / 2 + 0.3, L / 2 - 0.3, L / 2 + 0.45]])
    return Problem("stokeslet_32", (L, L, L), 0.5, 0.5,
                   points=[PointSet(STOKESLET, pos, np.array([[0.0, 0.0, 1e-5]]), None)], steps=steps)


def channel_256(L: int = 256, steps: int = 2000, nx: int | None = None, ny: int | None = None):
    """The four lattices of the wall-bounded channel / multipole workload."""
    nx = L if nx is None else nx
    ny = L if ny is None else ny
    r = rng(2)
    P = r.uniform(L / 4, 3 * L / 4, size=(3, 3))
    P[:, 0] *= nx / L
    P[:, 1] *= ny / L
    grid = (nx, ny, L)
    return [
        Problem("channel", grid, 0.5, 0.5, g=(1e-6, 0.0, 0.0), walls=(0, L - 1), counter=False, steps=steps),
        Problem("stokeslet", grid, 0.5, 0.5, steps=steps,
                points=[PointSet(STOKESLET, P[0:1], np.array([[0.0, 0.0, 1e-5]]), None)]),
        Problem("stresslet", grid, 0.5, 0.5, steps=steps,
                points=[PointSet(STRESSLET, P[1:2], np.array([[0.0, 0.0, 5e-5]]), np.array([2.0]))]),
        Problem("rotlet", grid, 0.5, 0.5, steps=steps,
                points=[PointSet(ROTLET, P[2:3], np.array([[0.0, 0.0, 1e-4]]), np.array([2.0]))]),
    ]


def colloids(L: int = 512, n: int = 100000, seed: int = 3, force: float = 1e-6, steps: int = 1000,
             a_L: float = float("inf")) -> Problem:
    r = rng(seed)
    pos = r.uniform(0, L, size=(n, 3))
    F = np.tile([0.0, 0.0, -force], (n, 1))
    prm = np.full(n, A_TABLE1)
    return Problem(f"colloids_{L}", (L, L, L), 0.5, 0.5, a_L=a_L,
                   points=[PointSet(COLLOID, pos, F, prm)], steps=steps)


def replicas(n: int = 64, seed: int = 4, L_min: int = 48, L_max: int = 128, L_step: int = 8,
             n_min: int = 100, n_max: int = 2000, force: float = 1e-6, steps: int = 5000):
    """Independent periodic sedimentation boxes of seeded uneven sizes: side
    uniform in {L_min, L_min + L_step, ..., L_max}, colloid count uniform in
    [n_min, n_max], colloids uniform in the box with force (0, 0, -force),
    radius a = 0.117, counter-force on."""
    r = rng(seed)
    sides = np.arange(L_min, L_max + 1, L_step)
    out = []
    for k in range(n):
        L = int(r.choice(sides))
        m = int(r.integers(n_min, n_max + 1))
        pos = r.uniform(0, L, size=(m, 3))
        F = np.tile([0.0, 0.0, -force], (m, 1))
        out.append(Problem(f"replica{k}", (L, L, L), 0.5, 0.5,
                           points=[PointSet(COLLOID, pos, F, np.full(m, A_TABLE1))], steps=steps))
    return out


def random_state(grid, seed: int, amp: float = 1e-4) -> np.ndarray:
    """A seeded non-equilibrium initial population deviation df[19][z][y][x]."""
    r = rng(seed)
    return r.normal(0.0, amp, size=(19, grid[2], grid[1], grid[0]))


__all__ = ["Problem", "PointSet", "stokeslet_32", "channel_256", "colloids", "replicas", "random_state", "rng",
           "STOKESLET", "STRESSLET", "ROTLET", "COLLOID", "A_TABLE1"]
