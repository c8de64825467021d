"""Pins of the oracle's Algorithm 5 (augmented GMRES): the minimal-residual property over the
augmented Krylov space by brute force (dense least squares over an explicitly built basis), the
direct Helmholtz solution, exact eigenvectors needing no Arnoldi step, and GMRES as the p = 0
case."""
import math

import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


class _DenseGrid:
    """Shape and M weights of a made-up problem; the operator is a dense matrix."""

    def __init__(self, shape, w):
        self.shape, self.n = shape, int(np.prod(shape))
        self._w = np.asarray(w, dtype=np.float64).reshape(shape)

    def weights(self):
        return self._w


def _brute_force_cycle(Amat, w, b, x0, W, j):
    """argmin ||b - A x||_M over x in x0 + span(W) + K_j((I-P) A, (I-P) b0), P the M-orthogonal
    projector onto range(A W): the Krylov basis is built from explicit powers and the
    minimisation is a dense weighted least-squares problem (numpy lstsq)."""
    n = b.size
    sq = np.sqrt(w)
    b0 = b - Amat @ x0
    AW = Amat @ W
    # M-orthogonal projector onto range(A W): P = AW (AW^T M AW)^{-1} AW^T M
    G = AW.T @ (w[:, None] * AW)
    P = AW @ np.linalg.solve(G, AW.T * w[None, :]) if W.shape[1] else np.zeros((n, n))
    IP = np.eye(n) - P
    cols = [IP @ b0]
    for _ in range(j - 1):
        cols.append(IP @ (Amat @ cols[-1]))
    Kr = np.linalg.qr(np.array(cols).T)[0] if j else np.zeros((n, 0))
    Z = np.hstack([W, Kr])
    y = np.linalg.lstsq(sq[:, None] * (Amat @ Z), sq * b0, rcond=None)[0]
    x = x0 + Z @ y
    return x, math.sqrt(np.sum(w * (b - Amat @ x) ** 2))


@pytest.mark.parametrize("p,j", [(0, 5), (3, 4), (5, 7), (4, 0)])
def test_agmres_is_minimal_residual_over_augmented_space(p, j):
    rng = np.random.default_rng(10 + p + j)
    shape = (5, 6)
    n = 30
    Amat = np.eye(n) + 0.35 * rng.standard_normal((n, n)) / math.sqrt(n)
    w = rng.uniform(0.5, 2.0, n)
    g = _DenseGrid(shape, w)
    A = lambda v: (Amat @ np.asarray(v).ravel()).reshape(shape)  # noqa: E731
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    W = rng.standard_normal((n, p))
    res = K.agmres(g, A, b, W, 0.0, j, restart=max(j, 1), x0=x0)
    xb, rb = _brute_force_cycle(Amat, w, b, x0, W, j)
    assert res.iterations == j
    assert np.allclose(res.x.ravel(), xb, rtol=1e-9, atol=1e-10)
    r = math.sqrt(np.sum(w * (b - Amat @ res.x.ravel()) ** 2))
    assert r == pytest.approx(rb, rel=1e-9, abs=1e-12)


def test_agmres_restarts_are_cycles_of_the_minimal_residual_step():
    """Restarted after m steps: each cycle is the minimal-residual step from the previous
    iterate (the augmentation is kept over restarts)."""
    rng = np.random.default_rng(3)
    shape, n, p, m, cycles = (4, 6), 24, 3, 4, 3
    Amat = np.eye(n) + 0.5 * rng.standard_normal((n, n)) / math.sqrt(n)
    w = rng.uniform(0.5, 2.0, n)
    g = _DenseGrid(shape, w)
    A = lambda v: (Amat @ np.asarray(v).ravel()).reshape(shape)  # noqa: E731
    b = rng.standard_normal(n)
    W = rng.standard_normal((n, p))
    res = K.agmres(g, A, b, W, 0.0, m * cycles, restart=m)
    x = np.zeros(n)
    for _ in range(cycles):
        x, _ = _brute_force_cycle(Amat, w, b, x, W, m)
    assert res.iterations == m * cycles
    assert np.allclose(res.x.ravel(), x, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("exact_aw", [True, False])
def test_agmres_reaches_direct_solution_2d(exact_aw):
    """2-D WaveHoltz system with the closed-form deflation set as augmentation (A W from the
    modal multipliers or by wave solves): the solution is the sparse direct one."""
    npts, om = (41, 37), 14.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, om)
    f = I.gaussian(npts, [0.4, 0.6], 0.08, om ** 2)
    modes, lam2, _ = SP.select_modes(og, tg, 6)
    V = SP.basis(og, modes)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    r = K.augmented_solve(og, tg, f, V, lam2 if exact_aw else None, tol=1e-12, maxit=3000, restart=30)
    assert r.solve.converged
    assert IND.relmax(r.u, U) < 1e-9
    # augmentation with the modes nearest resonance shortens the iteration
    r0 = K.augmented_solve(og, tg, f, None, None, tol=1e-12, maxit=3000, restart=30)
    assert r.solve.iterations < r0.solve.iterations / 4


def test_agmres_variable_speed_approximate_vectors():
    """Variable speed, 4th order, augmentation by perturbed (inexact) vectors: the method stays a
    minimal-residual solver over a larger space and reaches the direct solution."""
    npts, om = (33, 29), 14.0
    c2 = I.speed_squared("c3", npts, 5)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, om)
    f = I.gaussian(npts, [0.45, 0.5], 0.1, om ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    rng = np.random.default_rng(2)
    W = rng.standard_normal((og.n, 5))
    r = K.augmented_solve(og, tg, f, W, None, tol=1e-12, maxit=4000, restart=40)
    assert r.solve.converged
    assert IND.relmax(r.u, U) < 1e-8


def test_agmres_exact_eigenvectors_b_in_span():
    """b in span(W) with exact eigenvectors: A W spans b, the least-squares solve over span(W)
    is exact and no Arnoldi step is needed: x = W diag(1/mu) W^T M b."""
    npts, om = (23, 19), 10.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, om)
    modes, lam2, bh = SP.select_modes(og, tg, 4)
    V = SP.basis(og, modes)
    c = np.array([1.0, -2.0, 0.5, 3.0])
    b = (V @ c).reshape(og.shape)
    AW = V * (1.0 - bh)[None, :]
    res = K.agmres(og, K.Operator(og, tg), b, V, 1e-13, 50, restart=10, AW=AW)
    assert res.iterations == 0 or res.converged
    x_modal = V @ (c / (1.0 - bh))
    assert np.allclose(res.x.ravel(), x_modal, rtol=1e-12, atol=1e-14)
