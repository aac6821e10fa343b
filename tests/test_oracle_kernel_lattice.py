"""Pins of the oracle's building blocks against what the paper and the
mathematics fix: the Peskin kernel (Eq. deltadef), the D3Q19 lattice
identities, and the point-force kinds of Sec. III."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_phi():
    rows = []
    for line in open(os.path.join(GOLDEN, "peskin_phi.txt")):
        if line.startswith("#") or not line.strip():
            continue
        r, v = line.split()[:2]
        rows.append((float(r), float(v)))
    return rows


@pytest.mark.parametrize("precision", ["double", "longdouble"])
def test_phi_worked_values(precision):
    # Eq. (deltadef) substituted by hand at the branch points
    for r, v in _golden_phi():
        assert abs(float(oracle.phi([r], precision)[0]) - v) < 1e-16


def test_phi_peskin_conditions():
    # Sec. III: the kernel keeps the delta function's properties on the grid
    # (Peskin's conditions): for every offset X the 4 stencil weights
    # sum to 1, have zero first moment, sum of squares 3/8, and the even and
    # odd nodes each carry 1/2.
    rng = np.random.default_rng(11)
    X = np.concatenate([rng.uniform(0, 1, 400), [0.0, 0.5, 1e-12, 1 - 1e-12]])
    for x in X:
        nodes = np.arange(-1, 3)
        w = oracle.phi(nodes - x)
        assert abs(w.sum() - 1) < 1e-15
        assert abs(((nodes - x) * w).sum()) < 1e-15
        assert abs((w * w).sum() - 3 / 8) < 1e-15
        assert abs(w[nodes % 2 == 0].sum() - 0.5) < 1e-15
        assert abs(w[nodes % 2 == 1].sum() - 0.5) < 1e-15


def test_phi_continuity_and_support():
    e = 1e-9
    for r in (1.0, 2.0):
        a, b = oracle.phi([r - e, r + e])
        assert abs(a - b) < 1e-7
    assert np.all(oracle.phi(np.linspace(2, 5, 11)) == 0)
    r = np.linspace(-2, 2, 401)
    assert np.allclose(oracle.phi(r), oracle.phi(-r), atol=0, rtol=0)


def test_lattice_isotropy_exact():
    # D3Q19 Gauss-Hermite quadrature (Sec. II): weights sum to 1, second
    # moment cs^2 I with cs^2 = 1/3, odd moments vanish, fourth moment
    # cs^4 (dd + dd + dd); checked in exact rationals.
    c, w = oracle.lattice()
    W = [Fraction(float(x)).limit_denominator(1000) for x in w]
    assert sorted(set(W)) == [Fraction(1, 36), Fraction(1, 18), Fraction(1, 3)]
    for i in range(19):
        assert abs(float(W[i]) - w[i]) < 1e-17
    cs2 = Fraction(1, 3)
    assert sum(W) == 1
    d = lambda a, b: 1 if a == b else 0
    for a in range(3):
        assert sum(W[i] * c[i, a] for i in range(19)) == 0
        for b in range(3):
            assert sum(W[i] * c[i, a] * c[i, b] for i in range(19)) == cs2 * d(a, b)
            for g in range(3):
                assert sum(W[i] * c[i, a] * c[i, b] * c[i, g] for i in range(19)) == 0
                for h in range(3):
                    m4 = sum(W[i] * c[i, a] * c[i, b] * c[i, g] * c[i, h] for i in range(19))
                    assert m4 == cs2 * cs2 * (d(a, b) * d(g, h) + d(a, g) * d(b, h) + d(a, h) * d(b, g))
    # the 19 vectors are distinct, come in opposite pairs and have |c|^2 <= 2
    assert len({tuple(v) for v in c}) == 19
    for v in c:
        assert any((c == -v).all(1))
    assert (c * c).sum(1).max() == 2


def test_long_double_lattice_agrees():
    c, w = oracle.lattice()
    cl, wl = oracle.lattice("longdouble")
    assert (c == cl).all()
    assert np.abs(w - wl.astype(np.float64)).max() == 0


def test_stresslet_rotlet_expansion():
    # Sec. III: a stresslet is a collinear force pair, a rotlet four
    # tangential forces; both carry zero net force.  The rotlet's torque
    # and the stresslet's dipole strength are what was asked for.
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = rng.uniform(4, 12, 3)
        f = rng.normal(size=3)
        sep = rng.uniform(0.5, 3)
        P, F, M, _ = oracle.expand_points(oracle.STRESSLET, p, f, [sep])
        assert len(P) == 2 and not M.any()
        assert np.abs(F.sum(0)).max() < 1e-15
        assert abs(np.linalg.norm(P[0] - P[1]) - sep) < 1e-13
        assert np.allclose(np.cross(P[0] - P[1], F[0]), 0, atol=1e-14)  # collinear
        assert np.allclose(P.mean(0), p, atol=1e-14)
        T = rng.normal(size=3)
        arm = rng.uniform(0.5, 3)
        P, F, M, _ = oracle.expand_points(oracle.ROTLET, p, T, [arm])
        assert len(P) == 4
        assert np.abs(F.sum(0)).max() < 1e-15
        torque = np.cross(P - p, F).sum(0)
        assert np.allclose(torque, T, rtol=1e-13, atol=1e-15)
        # forces tangential: perpendicular to both their arm and the torque axis
        assert np.allclose(((P - p) * F).sum(1), 0, atol=1e-14)
        assert np.allclose(F @ T, 0, atol=1e-14)
        # symmetric stresslet part of the four forces vanishes (the reason
        # for using four forces, Sec. III)
        S = np.einsum("sa,sb->ab", P - p, F)
        assert np.allclose(S + S.T, 0, atol=1e-14)
    # rotlet frame about z: e1 = x, e2 = y
    P, F, _, _ = oracle.expand_points(oracle.ROTLET, [0, 0, 0], [0, 0, 1.0], [2.0])
    assert np.allclose(P, [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]])
    assert np.allclose(F, [[0, .25, 0], [0, -.25, 0], [-.25, 0, 0], [.25, 0, 0]])


def test_force_field_spreads_total_force_and_first_moment():
    # Grid representation of point forces (Sec. III): the lattice sum of
    # F equals the point force and its first moment is the force's position
    # (the kernel's zeroth and first moment conditions), also across the
    # periodic boundary.
    n = (12, 10, 9)
    rng = np.random.default_rng(5)
    for R in ([5.3, 4.1, 2.7], [0.2, 9.9, 8.6], [11.95, 0.0, 4.5]):
        f = rng.normal(size=3)
        F = oracle.force_field(n, R, f)
        assert np.allclose(F.sum(axis=(1, 2, 3)), f, rtol=0, atol=1e-15)
        for a, axis in zip(range(3), (3, 2, 1)):
            nodes = np.arange(n[a])
            # minimum-image offset from R in this axis
            off = (nodes - R[a] + n[a] / 2) % n[a] - n[a] / 2
            shape = [1, 1, 1, 1]
            shape[axis] = n[a]
            m1 = (F[0] * off.reshape(shape[1:])).sum()
            assert abs(m1) < 1e-14 * max(1, abs(f[0]))


def test_counter_force_and_walls():
    f = np.array([[0, 0, 1e-5], [1e-6, 0, 0]])
    fc = oracle.counter_force(f, 1000)
    assert np.allclose(fc * 1000 + f.sum(0), 0, atol=1e-20)
    lb = oracle.OracleLB((4, 4, 10), 0.5, 0.5, walls=(0, 9))
    assert lb.n_fluid == 4 * 4 * 8


def test_table1_consistency():
    # Table I: the volume fraction and the Stokes times follow from the
    # other columns (tau_S = rho a^2 / (eta Re), Sec. V).
    vals = {}
    for line in open(os.path.join(GOLDEN, "table1_point_particle.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    phi_v = vals["n_particles"] * 4 / 3 * math.pi * vals["a"] ** 3 / vals["L"] ** 3
    assert abs(phi_v / vals["volume_fraction"] - 1) < 0.02
    ts = vals["rho"] * vals["a"] ** 2 / (vals["eta"] * vals["Re"])
    assert abs(ts - vals["stokes_time"]) < 0.5
    tr = vals["rho"] * vals["a_resolved"] ** 2 / (vals["eta"] * vals["Re"])
    assert abs(tr - vals["stokes_time_resolved"]) < 1
