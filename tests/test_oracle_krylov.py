"""Pins of the oracle's solvers: every accelerator reaches the direct solution, deflation
keeps the solution, DCG variants agree, rates match the theory the paper quotes."""
import math

import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


@pytest.fixture(scope="module")
def c1():
    w = I.WORKLOADS["c1"]
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    f = I.forcing_for(w)
    modes, lam2, bh = SP.select_modes(g, tg, w.nd)
    V = SP.basis(g, modes)
    U = IND.helmholtz_direct(w.npts, tg.omega_eff, f)
    return dict(g=g, tg=tg, f=f, modes=modes, lam2=lam2, bh=bh, V=V, U=U)


def test_c1_mode_set(c1):
    """Deflation set of the 1-D workload (8 sines with beta_h closest to 1)."""
    assert [int(m[0]) for m in c1["modes"]] == [3, 4, 2, 7, 11, 8, 14, 21]


@pytest.mark.parametrize("method", ["cg", "gmres", "fpi"])
@pytest.mark.parametrize("deflate", [False, True])
def test_c1_solvers_reach_direct_solution(c1, method, deflate):
    V = c1["V"] if deflate else None
    lam2 = c1["lam2"] if deflate else None
    tol = 1e-12 if method != "fpi" else 1e-11
    r = K.devd_solve(c1["g"], c1["tg"], c1["f"], V, lam2, method, tol, 3000)
    assert r.solve.converged
    assert IND.relmax(r.u, c1["U"]) < 1e-10


def test_deflated_forcing_orthogonal_and_inflation_is_modal(c1):
    """Algorithm 2: f_d is orthogonal to the deflation set; the inflated components equal
    the modal solution (f, phi_m)/(omega_eff^2 - lambda_m^2)."""
    g, V = c1["g"], c1["V"]
    fd = K.project_out(g, V, c1["f"])
    assert np.abs(V.T @ fd.ravel()).max() < 1e-13 * np.abs(c1["f"]).max()
    coef_direct = V.T @ c1["U"]
    coef_modal = (V.T @ c1["f"].ravel()) / (c1["tg"].omega_eff ** 2 - c1["lam2"])
    assert np.allclose(coef_direct, coef_modal, rtol=1e-9, atol=1e-12)


def test_dcg_exact_and_projected_agree(c1):
    """Sec. 3.1: with true eigenvectors the per-iteration projections of DCG are unnecessary."""
    g, tg = c1["g"], c1["tg"]
    b = WH.rhs_b(g, tg, c1["f"])
    r1 = K.dcg(g, K.Operator(g, tg), b, c1["V"], 1e-12, 200, mu=1.0 - c1["bh"])
    r2 = K.dcg(g, K.Operator(g, tg), b, c1["V"], 1e-12, 200)
    assert IND.relmax(r1.x, c1["U"]) < 1e-10
    assert IND.relmax(r2.x, c1["U"]) < 1e-10
    assert abs(r1.iterations - r2.iterations) <= 1


def test_fpi_rate_matches_acr(c1):
    """eq. WaveHoltzFPIconvergence: FPI error ratio -> max over non-deflated |beta_h|."""
    g, tg = c1["g"], c1["tg"]
    rho = SP.acr(g, tg, c1["modes"])
    r = K.devd_solve(g, tg, c1["f"], c1["V"], c1["lam2"], "fpi", 1e-13, 200)
    h = r.solve.history
    ratio = (h[-3] / h[-13]) ** 0.1
    assert ratio == pytest.approx(rho, rel=0.02)


def test_cg_within_theorem_bound():
    """Theorem 3.1 with kappa from Theorem 3.2: ||x - x_j||_A <= 2 q^j ||x - x_0||_A."""
    npts = (41, 37)
    g = O.Grid(npts)
    tg = WH.time_grid_for(g, 17.0)
    f = I.gaussian(npts, [0.4, 0.6], 1 / 17.0, 289.0)
    nd = 10
    modes, lam2, bh = SP.select_modes(g, tg, nd)
    V = SP.basis(g, modes)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    kap = SP.kappa(g, tg, nd)
    q = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    b = WH.rhs_b(g, tg, f)
    A = K.Operator(g, tg)
    anorm = lambda e: math.sqrt(g.inner(e, A(e)))  # noqa: E731
    x0 = V @ ((V.T @ b.ravel()) / (1.0 - bh))
    e0 = anorm((U - x0).reshape(g.shape))
    for j in [2, 5, 8, 12]:
        r = K.dcg(g, K.Operator(g, tg), b, V, 0.0, j, mu=1.0 - bh)
        ej = anorm((U - r.x.ravel()).reshape(g.shape))
        assert ej <= 2 * q ** j * e0 * (1 + 1e-6) + 1e-12


def test_deflation_reduces_iterations_2d():
    npts = (65, 65)
    g = O.Grid(npts)
    tg = WH.time_grid_for(g, 25.0)
    f = I.gaussian(npts, [0.37, 0.61], 1 / 25.0, 625.0)
    modes, lam2, _ = SP.select_modes(g, tg, 16)
    V = SP.basis(g, modes)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    r0 = K.devd_solve(g, tg, f, None, None, "cg", 1e-10, 2000)
    r1 = K.devd_solve(g, tg, f, V, lam2, "cg", 1e-10, 2000)
    assert r1.solve.iterations < r0.solve.iterations
    assert IND.relmax(r0.u, U) < 1e-7 and IND.relmax(r1.u, U) < 1e-7
    assert IND.relmax(r0.u, r1.u) < 1e-7


def test_gmres_restart_and_redeflation_variable_speed():
    """GMRES(m) on the variable-speed 4th-order problem, with re-deflation of each operator
    output against (approximate) vectors, reaches the direct solution."""
    npts = (25, 23)
    c2 = I.speed_squared("c3", npts, 5)
    g = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(g, 10.0)
    f = I.gaussian(npts, [0.5, 0.5], 0.1, 100.0)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    r = K.devd_solve(g, tg, f, None, None, "gmres", 1e-12, 2000, restart=8)
    assert IND.relmax(r.u, U) < 1e-9


def test_true_residual(c1):
    r = K.devd_solve(c1["g"], c1["tg"], c1["f"], c1["V"], c1["lam2"], "cg", 1e-10, 500)
    assert K.true_residual(c1["g"], c1["tg"], r.u, c1["f"]) < 1e-9
