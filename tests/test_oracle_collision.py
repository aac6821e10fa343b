"""Pins of the oracle's one-site collision (Eq. fiexp with A and B) against
an independent dense population-space build of Eq. (mrtlbe), the
single-relaxation-time Eq. (bgklbe), and the conservation constraints of
Eq. (conservation)."""
import numpy as np
import pytest

import oracle
import mrt_dense as md


def test_dense_lattice_matches_oracle_order():
    c, w = oracle.lattice()
    cd, wd = md.d3q19()
    assert (c == cd).all() and np.allclose(w, wd, rtol=0, atol=1e-17)


@pytest.mark.parametrize("tau_s,tau_b", [(0.5, 0.5), (0.3, 1.0), (2.0, 0.7), (1.0, 1.0), (0.55, 0.5)])
def test_moment_form_equals_dense_mrtlbe(tau_s, tau_b):
    # The moment-space update (ghosts projected out, stress relaxed at
    # 1/(tau + 1/2)) must equal (1 + L/2)^{-1}[-L(f - f0) + Phi] solved
    # densely with the same eigenvalues.  A flipped sign in B, a missing
    # forcing term or a wrong rate all give O(1) relative differences.
    rng = np.random.default_rng(int(tau_s * 100 + tau_b * 10))
    for _ in range(25):
        scale = 10 ** rng.uniform(-7, -2)
        df = rng.normal(0, scale, 19)
        F = rng.normal(0, scale * 0.3, 3)
        ref = md.mrt_update(df, F, tau_s, tau_b)
        got = oracle.collide_site(df, F, tau_s, tau_b)
        # the dense form adds and removes w ~ 1/3, so compare on that scale
        assert np.abs(got - ref).max() < 1e-14 * (1 + 0) + 1e-12 * np.abs(ref).max()


def test_unit_rates_equal_guo_bgk():
    # With every relaxation rate 1 (tau_s = tau_b = 1/2) the moment form is
    # Eq. (bgklbe) at tau = 1/2.
    rng = np.random.default_rng(7)
    for _ in range(25):
        df = rng.normal(0, 1e-3, 19)
        F = rng.normal(0, 1e-4, 3)
        ref = md.bgk_update(df, F, 0.5)
        got = oracle.collide_site(df, F, 0.5, 0.5)
        assert np.abs(got - ref).max() < 1e-15


@pytest.mark.parametrize("tau", [0.3, 1.0, 2.0])
def test_hydrodynamic_moments_equal_bgk(tau):
    # For tau_s = tau_b = tau the MRT and BGK updates differ only in the
    # ghost modes; rho, momentum and stress of the output agree.
    c, _ = md.d3q19()
    rng = np.random.default_rng(int(tau * 10))
    for _ in range(10):
        df = rng.normal(0, 1e-3, 19)
        F = rng.normal(0, 1e-4, 3)
        a = md.moments(c, md.bgk_update(df, F, tau))
        b = md.moments(c, oracle.collide_site(df, F, tau, tau))
        for x, y in zip(a, b):
            assert np.abs(np.asarray(x) - np.asarray(y)).max() < 1e-15


def test_equilibrium_is_fixed_point():
    c, w = md.d3q19()
    rng = np.random.default_rng(9)
    for _ in range(10):
        rho = 1 + rng.normal(0, 1e-3)
        v = rng.normal(0, 1e-3, 3)
        df = md.equilibrium(c, w, rho, v) - w
        for ts, tb in ((0.5, 0.5), (1.3, 0.8)):
            out = oracle.collide_site(df, np.zeros(3), ts, tb)
            # df came from f0 - w with |w| <= 1/3: compare at that rounding scale
            assert np.abs(out - df).max() < 1e-16


def test_mass_and_momentum_per_site():
    # Eq. (conservation): collisions conserve mass; forcing adds F to the
    # momentum of the auxiliary distribution (A = sum fbar c + F).
    c, _ = md.d3q19()
    rng = np.random.default_rng(13)
    for _ in range(25):
        df = rng.normal(0, 1e-4, 19)
        F = rng.normal(0, 1e-5, 3)
        out = oracle.collide_site(df, F, rng.uniform(0.3, 2), rng.uniform(0.3, 2))
        assert abs(out.sum() - df.sum()) < 1e-18
        assert np.abs(out @ c - (df @ c + F)).max() < 1e-18


def test_macro_site_half_force():
    # Eq. (macrovariables2): rho v = sum fbar c + F/2
    c, _ = md.d3q19()
    rng = np.random.default_rng(17)
    df = rng.normal(0, 1e-4, 19)
    F = rng.normal(0, 1e-5, 3)
    rho, v = oracle.macro_site(df, F)
    assert abs(rho - (1 + df.sum())) < 1e-16
    assert np.abs(rho * v - (df @ c + F / 2)).max() < 1e-18


def test_long_double_collision_agrees():
    rng = np.random.default_rng(19)
    df = rng.normal(0, 1e-5, 19)
    F = rng.normal(0, 1e-6, 3)
    a = oracle.collide_site(df, F, 0.7, 0.9)
    b = oracle.collide_site(df.astype(np.longdouble), F.astype(np.longdouble), 0.7, 0.9, "longdouble")
    assert np.abs(a - b.astype(np.float64)).max() < 1e-15 * np.abs(a).max()
