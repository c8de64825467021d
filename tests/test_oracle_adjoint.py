"""Pins of the oracle's discrete adjoint: transposition identities against the forward oracle,
finite differences of the forward map, and the M-similarity S_h^T = M S_h M^{-1}."""
import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, adjoint as AD
from paper_2606_31842_b300 import inputs as I


def _grid(npts=(21, 19), order=4, speed="c5", omega=9.0):
    c2 = None if speed is None else I.speed_squared(speed, npts, 8)
    g = O.Grid(npts, order=order, c2=c2)
    return g, WH.time_grid_for(g, omega)


@pytest.mark.parametrize("npts,order,speed", [((21, 19), 4, "c5"), ((23,), 2, None), ((9, 8, 7), 2, "c5")])
def test_dot_product_test(npts, order, speed):
    """<S x, y> = <x, S^T y> (Euclidean) with S from the forward oracle."""
    g, tg = _grid(npts, order, speed, 7.0)
    x, y = I.random_field(g.shape, 1), I.random_field(g.shape, 2)
    lhs = float(np.sum(WH.apply_S(g, tg, x) * y))
    rhs = float(np.sum(x * AD.apply_St(g, tg, y)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_laplacian_is_symmetric():
    for order in (2, 4):
        g = O.Grid((15, 13), order=order)
        x, y = I.random_field(g.shape, 3), I.random_field(g.shape, 4)
        a, b = float(np.sum(O.laplacian(g, x) * y)), float(np.sum(x * O.laplacian(g, y)))
        assert abs(a - b) < 1e-12 * abs(a)


def test_m_similarity():
    """S^T = M S M^{-1}, M = diag(1/c^2) (the mass-matrix symmetrisation of Sec. 4.1)."""
    g, tg = _grid()
    a = I.random_field(g.shape, 5)
    lhs = AD.apply_St(g, tg, a)
    rhs = WH.apply_S(g, tg, g.c2 * a) / g.c2
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_reverse_sweep_matches_forward_differences():
    """<dPi(v; f, c^2)/dc^2 . d, a> by central differences of the forward oracle equals
    <c2bar, d>; Pi is linear in f, so <Pi(v; f + e) - Pi(v; f), a> = <fbar, e> exactly."""
    g, tg = _grid()
    v, f, a = I.random_field(g.shape, 6), I.random_field(g.shape, 7), I.random_field(g.shape, 8)
    d, e = I.random_field(g.shape, 9), I.random_field(g.shape, 10)
    _, c2b, fb = AD.reverse_sweep(g, tg, WH.wave_states(g, tg, v, f), a)
    eps = 1e-6
    gp = O.Grid(g.npts, order=g.order, c2=g.c2 + eps * d)
    gm = O.Grid(g.npts, order=g.order, c2=g.c2 - eps * d)
    fd = float(np.sum((WH.apply_pi(gp, tg, v, f) - WH.apply_pi(gm, tg, v, f)) * a)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(c2b * d)), rel=1e-7)
    lin = float(np.sum((WH.apply_pi(g, tg, v, f + e) - WH.apply_pi(g, tg, v, f)) * a))
    assert lin == pytest.approx(float(np.sum(fb * e)), rel=1e-10)


def test_full_gradient_matches_finite_differences():
    """dL/dc^2 and dL/df of L = 1/2 ||u - u_obs||^2 (u the WaveHoltz fixed point) against central
    differences of L in seeded random directions."""
    npts, omega = (17, 15), 8.0
    c2 = I.speed_squared("c5", npts, 2024)
    g = O.Grid(npts, order=2, c2=c2)
    tg = WH.time_grid_for(g, omega)
    f = I.gaussian(npts, [0.45, 0.55], 1 / omega, omega ** 2)
    g_obs = O.Grid(npts, order=2, c2=c2 + 0.05 * I.bumps(npts, 2025))
    _, u_obs = AD.misfit(g_obs, tg, f, np.zeros(g.shape))
    L0, u = AD.misfit(g, tg, f, u_obs)
    lam, gc2, gf, _ = AD.adjoint_gradient(g, tg, u, f, u - u_obs)
    rng = np.random.default_rng(0)
    eps = 1e-5
    for _ in range(3):
        d = rng.standard_normal(g.shape)
        Lp, _ = AD.misfit(O.Grid(npts, order=2, c2=c2 + eps * d), tg, f, u_obs)
        Lm, _ = AD.misfit(O.Grid(npts, order=2, c2=c2 - eps * d), tg, f, u_obs)
        assert (Lp - Lm) / (2 * eps) == pytest.approx(float(np.sum(gc2 * d)), rel=1e-5)
        e = rng.standard_normal(g.shape)
        Lp, _ = AD.misfit(g, tg, f + eps * e, u_obs)
        Lm, _ = AD.misfit(g, tg, f - eps * e, u_obs)
        assert (Lp - Lm) / (2 * eps) == pytest.approx(float(np.sum(gf * e)), rel=1e-5)
