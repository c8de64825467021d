"""Pins of the oracle's conservative operator div_h(c^2 grad_h) (eq. L, second order): it equals
an independently assembled sparse matrix, is symmetric negative definite in the Euclidean inner
product, reduces to kappa Delta_h for constant c^2 = kappa, and the WaveHoltz fixed point with it
is the direct Helmholtz solution."""
import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


def _dense(g):
    return np.stack([O.apply_L(g, e.reshape(g.shape)).ravel() for e in np.eye(g.n)], axis=1)


@pytest.mark.parametrize("npts", [(23,), (11, 9), (7, 6, 5)])
def test_conservative_operator_equals_independent_assembly(npts):
    c2 = I.speed_squared("c3", npts, 2) if len(npts) == 2 else 1.0 + np.random.default_rng(1).random(
        tuple(p - 2 for p in reversed(npts)))
    g = O.Grid(npts, c2=c2, form="conservative")
    D = _dense(g)
    A = IND.conservative_matrix(npts, c2).toarray()
    assert np.allclose(D, A, rtol=1e-13, atol=1e-9)
    assert np.allclose(D, D.T, atol=1e-9 * np.abs(D).max())
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).max() < 0.0
    assert np.allclose(g.weights(), 1.0)


def test_constant_speed_reduces_to_scaled_laplacian():
    npts = (13, 10)
    g = O.Grid(npts, c2=np.full((8, 11), 2.5), form="conservative")
    u = I.random_field(g.shape, 3)
    assert np.allclose(O.apply_L(g, u), 2.5 * O.laplacian(g, u), rtol=1e-13, atol=1e-10)


def test_conservative_fixed_point_is_the_direct_solution():
    npts, omega = (41, 37), 12.0
    c2 = I.speed_squared("c3", npts, 5)
    g = O.Grid(npts, c2=c2, form="conservative")
    tg = WH.time_grid_for(g, omega)
    f = I.gaussian(npts, [0.45, 0.5], 0.08, omega ** 2)
    r = K.devd_solve(g, tg, f, None, None, "cg", 1e-12, 4000)
    assert r.solve.converged
    U = IND.helmholtz_direct_conservative(npts, tg.omega_eff, f, c2)
    assert IND.relmax(r.u, U) < 1e-8
