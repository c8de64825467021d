"""Pins of the oracle's Pi_h against the discrete Helmholtz problem it must reproduce."""
import math

import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


def test_time_grid_counts():
    """dt0 = 0.5 h (2nd order) / 0.4 h (4th order), Nt = ceil(Tbar/dt0), dt = Tbar/Nt."""
    expect = {"c1": 240, "c2": 129, "c5": 81}
    for name, nt in expect.items():
        w = I.WORKLOADS[name]
        g = O.Grid(w.npts, order=w.order)
        assert WH.time_grid_for(g, w.omega).nt == nt
    tg = WH.time_grid(50.0, 1 / 512)
    assert tg.nt * tg.dt == pytest.approx(2 * math.pi / 50.0, rel=1e-15)


def test_filter_weights_reproduce_resonant_mode():
    """Trapezoid filter over the period: a time-harmonic cos(omega t) passes with weight 1
    (beta(omega) = 1) and a constant with weight -1/2 (beta(0) = -1/2), eq. beta_fun."""
    tg = WH.time_grid(13.0, 1 / 300)
    assert float(np.sum(tg.filter_weights() * tg.forcing_phase())) == pytest.approx(1.0, abs=1e-13)
    assert float(np.sum(tg.filter_weights())) == pytest.approx(-0.5, abs=1e-13)


def test_adjusted_frequency_closed_form():
    tg = WH.time_grid(50.0, 1 / 512, adjust=True)
    assert tg.omega_eff == pytest.approx(50.0, rel=1e-14)
    assert tg.dt <= 0.5 / 512
    assert tg.omega_hat * tg.tbar == pytest.approx(2 * math.pi, rel=1e-14)


def _fixed_point(g, tg, f, maxit=3000):
    return K.devd_solve(g, tg, f, method="cg", tol=1e-14, maxit=maxit).u


CASES = [
    ("1d", (65,), 2, 9.0, None),
    ("2d", (31, 27), 2, 14.0, None),
    ("3d", (11, 10, 9), 2, 8.0, None),
    ("2d-o4", (29, 25), 4, 12.0, None),
    ("2d-o4-varc", (27, 29), 4, 11.0, "c3"),
    ("3d-varc", (9, 10, 11), 2, 6.0, "c5"),
]


@pytest.mark.parametrize("name,npts,order,omega,speed", CASES)
@pytest.mark.parametrize("adjust", [False, True])
def test_fixed_point_equals_direct_helmholtz_solve(name, npts, order, omega, speed, adjust):
    """Sec. 2.1/2.2: the fixed point of Pi_h is the discrete Helmholtz solution (at
    omega_eff unadjusted, at omega with the adjusted frequency)."""
    c2 = None if speed is None else I.speed_squared(speed, npts, 7)
    g = O.Grid(npts, order=order, c2=c2)
    tg = WH.time_grid_for(g, omega, adjust=adjust)
    f = I.gaussian(npts, [0.45, 0.55, 0.5][: len(npts)], 0.2, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, order, c2)
    u = _fixed_point(g, tg, f)
    # both sides carry the conditioning of the near-resonant problem (kappa ~ 1e3): 1e-9
    assert IND.relmax(u, U) < 1e-9
    if adjust:
        assert tg.omega_eff == pytest.approx(omega, rel=1e-13)


def test_pi_is_affine_and_s_is_m_selfadjoint():
    """Pi_h v = S_h v + b (eq. Sh) and <S x, y>_M = <x, S y>_M for c^2 Delta_h."""
    npts = (21, 19)
    g = O.Grid(npts, order=4, c2=I.speed_squared("c3", npts, 3))
    tg = WH.time_grid_for(g, 9.0)
    f = I.random_field(g.shape, 1)
    x, y = I.random_field(g.shape, 2), I.random_field(g.shape, 3)
    b = WH.rhs_b(g, tg, f)
    assert np.abs(WH.apply_pi(g, tg, x, f) - (WH.apply_S(g, tg, x) + b)).max() < 1e-12
    lhs, rhs = g.inner(WH.apply_S(g, tg, x), y), g.inner(x, WH.apply_S(g, tg, y))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_first_step_and_leapfrog_match_time_harmonic_solution():
    """W^n = U cos(omega_hat t^n) exactly when U is the discrete Helmholtz solution at omega_eff."""
    npts = (40,)
    g = O.Grid(npts)
    tg = WH.time_grid_for(g, 7.0)
    f = I.gaussian(npts, [0.3], 0.1, 49.0)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f).reshape(g.shape)
    states = WH.wave_states(g, tg, U, f)
    ph = tg.forcing_phase()
    for n in [0, 1, 2, 17, tg.nt]:
        assert np.abs(states[n] - U * ph[n]).max() < 1e-11 * np.abs(U).max()


def test_stability_limit_is_refused():
    g = O.Grid((33, 33))
    with pytest.raises(ValueError):
        WH.time_grid_for(g, 5.0, cfl=0.8)
