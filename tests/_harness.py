"""Shared helpers of the GPU parity tests: run one workload Problem through
the C ABI (CUDA path) and through the oracle, and compare.

Error measure (spec tolerance): max over sites and components of
|v_gpu - v_ref| divided by max |v_ref| after the stated steps; for colloid
positions, the displacement error divided by the largest displacement.
"""
from __future__ import annotations

import numpy as np

# FP64 / FP32: the spec bars.  The 16-bit storage formats carry the
# stated errors of their rows: df rounded stochastically to half (scaled) or
# bfloat16 each step, arithmetic in float.
TOL = {"f64": 1e-12, "f32": 1e-5, "f16s": 1e-3, "bf16s": 1e-2}


def gpu_lattice(problem, precision):
    from paper_0707_1299_gb300 import lb
    g = lb.Lattice(problem.grid, problem.tau_s, problem.tau_b, precision)
    g.set_body_force(problem.g)
    if problem.walls is not None:
        g.set_walls_z(*problem.walls)
    g.set_counterforce(problem.counter)
    if np.isfinite(problem.a_L):
        g.set_colloid_aL(problem.a_L)
    for ps in problem.points:
        g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    return g


def oracle_lattice(problem, fc=None):
    import oracle
    o = oracle.OracleLB(problem.grid, problem.tau_s, problem.tau_b, g=problem.g, walls=problem.walls,
                        counter=problem.counter, a_L=problem.a_L, fc=fc)
    for ps in problem.points:
        o.add_points(ps.kind, ps.pos, ps.F, ps.param)
    return o


def disp_tol(prec, grid, steps, dmax):
    """Tolerance of a colloid displacement error relative to the largest
    displacement dmax: the format's bar, but not below what FP64 positions
    can resolve -- each step rounds a position to its ulp (the two sides may
    round differently: contracted or separate multiply-add), at most one
    ulp of the box size per step."""
    floor = float(np.spacing(float(max(grid)))) * steps / dmax
    return max(TOL[prec], floor)


def rel_err(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(a - ref).max() / (scale if scale > 0 else 1.0))


def periodic_diff(a, b, n):
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return d - n * np.round(d / n)
