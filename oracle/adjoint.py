"""Discrete adjoint of the WaveHoltz solve (oracle; test infrastructure only).

The solution u is the fixed point u = Pi_h(u; f, c^2) (Sec. 2.1-2.2).  For a misfit
L = 1/2 ||u - u_obs||^2 (Euclidean), differentiating the fixed point gives
(I - S_h) du = dPi/dtheta dtheta, so with lambda solving (I - S_h)^T lambda = g, g = u - u_obs,
    dL/dtheta = lambda^T dPi_h(u; f, c^2)/dtheta,   theta in {f, c^2}.
Both S_h^T and lambda^T dPi/dtheta are the reverse (transposed) sweep of one wave solve: the
forward recurrence of eq. discreteWaveExplicit with the trapezoid filter of eq. quadrature,
transposed step by step:
    forward   W^1 = W^0 + dt^2/2 (c^2 Delta W^0 - f)
              W^{n+1} = 2 W^n - W^{n-1} + dt^2 (c^2 Delta W^n - f cos(w t^n))
              out = sum_n w_n W^n
    reverse   Wb^n += w_n ab (all n); then for n = Nt-1 .. 1:
              Wb^n += 2 Wb^{n+1} + dt^2 Delta^T (c^2 Wb^{n+1});  Wb^{n-1} -= Wb^{n+1}
              c2b += dt^2 (Delta W^n) Wb^{n+1};  fb -= dt^2 cos(w t^n) Wb^{n+1}
              and for the first step: Wb^0 += Wb^1 + dt^2/2 Delta^T (c^2 Wb^1),
              c2b += dt^2/2 (Delta W^0) Wb^1, fb -= dt^2/2 Wb^1.
Delta_h is symmetric (2nd order; 4th order with the odd-reflection closure), so Delta^T = Delta.
The time grid (dt, Nt) is held fixed: it is a discrete parameter of the scheme, not a function
of c^2 being differentiated.
"""
from __future__ import annotations

import math

import numpy as np

from .operators import Grid, laplacian
from .waveholtz import TimeGrid, wave_states, apply_pi
from . import krylov as K


def _nonconservative_only(grid: Grid):
    if getattr(grid, "form", "nonconservative") != "nonconservative" and grid.c2 is not None:
        raise ValueError("the adjoint here differentiates the non-conservative operator c^2 Delta_h")


def reverse_sweep(grid: Grid, tg: TimeGrid, states, abar):
    """Transpose of one wave solve at the forward states W^0..W^Nt: returns (vbar, c2bar, fbar)
    for the adjoint seed abar of the filtered output."""
    _nonconservative_only(grid)
    dt2 = tg.dt * tg.dt
    w = tg.filter_weights()
    ph = tg.forcing_phase()
    nt = tg.nt
    c2 = np.ones(grid.shape) if grid.c2 is None else grid.c2
    abar = np.asarray(abar, dtype=np.float64).reshape(grid.shape)
    Wb = [w[n] * abar for n in range(nt + 1)]
    c2b = np.zeros(grid.shape)
    fb = np.zeros(grid.shape)
    for n in range(nt - 1, 0, -1):
        nxt = Wb[n + 1]
        Wb[n] = Wb[n] + 2.0 * nxt + dt2 * laplacian(grid, c2 * nxt)
        Wb[n - 1] = Wb[n - 1] - nxt
        c2b += dt2 * laplacian(grid, states[n]) * nxt
        fb -= dt2 * ph[n] * nxt
    one = Wb[1]
    Wb[0] = Wb[0] + one + 0.5 * dt2 * laplacian(grid, c2 * one)
    c2b += 0.5 * dt2 * laplacian(grid, states[0]) * one
    fb -= 0.5 * dt2 * ph[0] * one
    return Wb[0], c2b, fb


def apply_St(grid: Grid, tg: TimeGrid, a):
    """S_h^T a (reverse sweep with f = 0; the forward states do not enter vbar)."""
    _nonconservative_only(grid)
    dt2 = tg.dt * tg.dt
    w = tg.filter_weights()
    c2 = np.ones(grid.shape) if grid.c2 is None else grid.c2
    a = np.asarray(a, dtype=np.float64).reshape(grid.shape)
    Wb = [w[n] * a for n in range(tg.nt + 1)]
    for n in range(tg.nt - 1, 0, -1):
        nxt = Wb[n + 1]
        Wb[n] = Wb[n] + 2.0 * nxt + dt2 * laplacian(grid, c2 * nxt)
        Wb[n - 1] = Wb[n - 1] - nxt
    return Wb[0] + Wb[1] + 0.5 * dt2 * laplacian(grid, c2 * Wb[1])


class _EuclideanGrid:
    """View of a grid with Euclidean inner products (the adjoint system is solved in them)."""

    def __init__(self, grid):
        self.shape, self.n = grid.shape, grid.n

    def weights(self):
        return np.ones(self.shape)

    def inner(self, u, v):
        return float(np.sum(u * v))

    def norm(self, u):
        return math.sqrt(self.inner(u, u))


def adjoint_gradient(grid: Grid, tg: TimeGrid, u, f, g, tol=1e-12, maxit=5000, restart=60):
    """lambda = (I - S_h)^{-T} g by GMRES with the reverse-sweep operator, then
    (dL/dc^2, dL/df) = lambda^T dPi_h(u; f)/d(c^2, f).  Returns (lambda, grad_c2, grad_f, its)."""
    eg = _EuclideanGrid(grid)
    op = lambda x: np.asarray(x).reshape(grid.shape) - apply_St(grid, tg, x)  # noqa: E731
    res = K.gmres(eg, op, np.asarray(g, dtype=np.float64).reshape(grid.shape), tol, maxit, restart)
    lam = res.x.reshape(grid.shape)
    states = wave_states(grid, tg, u, f)
    _, c2b, fb = reverse_sweep(grid, tg, states, lam)
    return lam, c2b, fb, res.iterations


def misfit(grid: Grid, tg: TimeGrid, f, u_obs, tol=1e-13, maxit=5000):
    """L = 1/2 ||u - u_obs||^2 with u the fixed point (undeflated CG, tight tolerance)."""
    r = K.devd_solve(grid, tg, f, method="cg", tol=tol, maxit=maxit)
    d = r.u - np.asarray(u_obs).reshape(grid.shape)
    return 0.5 * float(np.sum(d * d)), r.u


def pi_output(grid: Grid, tg: TimeGrid, v, f):
    return apply_pi(grid, tg, v, f)
