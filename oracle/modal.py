"""DEVD-CG of the constant-speed box in the sine eigenbasis (oracle; test infrastructure only).

For c = 1 on the box the closed-form sine vectors (Sec. 4.3) are a complete orthonormal
eigenbasis of L_h, hence of S_h and A = I - S_h (spectral.py).  In that basis A is the
diagonal matrix diag(mu_k), mu_k = 1 - beta_h(lambda_k), and the forced wave solve
b = Pi_h(0; f) multiplies the k-th coefficient of f by the forced transfer value
gamma_h(lambda_k) of the filtered leapfrog started from rest.  CG is invariant under an
orthogonal change of basis, so CG on diag(mu) x^ = b^ produces the sine coefficients of the
iterates of `krylov.devd_solve(..., method="cg")` (Algorithm 2 with CG): the same residual
norms and, up to rounding, the same iteration count, at O(N) work per iteration instead of
one wave solve.  The benchmark uses it for the oracle's own iteration counts on grids where
running the time-domain oracle to convergence takes hours.

* sine_coefficients   u -> u^ (orthonormal type-I sine transform along every axis, i.e.
                      W^T u for the full closed-form basis W of spectral.basis).
* forced_transfer     gamma_h(lambda): Pi_h(0; phi) = gamma_h phi for an eigenvector phi,
                      from the scalar leapfrog of eq. discreteWaveExplicit with the forcing
                      -phi cos(omega_hat t^n) and the trapezoid filter of eq. quadrature.
* devd_cg             Algorithm 2 with CG (stopping rule of krylov.cg) for one or several
                      forcings at once, in sine coefficients.

Pinned (tests/test_oracle_modal.py) against the time-domain oracle it restates: coefficients
= W^T u with the explicit basis matrix, Pi_h(0; phi) = gamma_h phi, and iteration counts,
residual histories and solutions equal to krylov.devd_solve on small grids.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

from .operators import Grid
from .waveholtz import TimeGrid
from . import spectral as SP


def _mode_array(grid: Grid, values: np.ndarray) -> np.ndarray:
    """Values given per row of spectral.all_modes (x index outermost) laid out on the interior
    array shape (z, y, x): entry [k_z - 1, k_y - 1, k_x - 1]."""
    per_dir = [n - 2 for n in grid.npts]            # x, y, z counts
    return np.asarray(values).reshape(per_dir).transpose(tuple(reversed(range(grid.dim))))


def sine_coefficients(grid: Grid, u: np.ndarray) -> np.ndarray:
    """Coefficients of u (interior array, or a stack of them along a leading axis) in the
    orthonormal sine basis: entry [k_z-1, k_y-1, k_x-1] = <u, phi_(k_x, k_y, k_z)>."""
    u = np.asarray(u, dtype=np.float64)
    axes = tuple(range(u.ndim - grid.dim, u.ndim))
    return scipy.fft.dstn(u, type=1, axes=axes, norm="ortho")


def from_sine_coefficients(grid: Grid, c: np.ndarray) -> np.ndarray:
    """Inverse of sine_coefficients (the orthonormal type-I transform is its own inverse)."""
    c = np.asarray(c, dtype=np.float64)
    axes = tuple(range(c.ndim - grid.dim, c.ndim))
    return scipy.fft.idstn(c, type=1, axes=axes, norm="ortho")


def forced_transfer(lam2: np.ndarray, tg: TimeGrid) -> np.ndarray:
    """gamma_h(lambda) with Pi_h(0; phi) = gamma_h(lambda) phi for L_h phi = -lambda^2 phi:
    the leapfrog w^{n+1} = 2 w^n - w^{n-1} + dt^2 (-lambda^2 w^n - cos(omega_hat t^n)) from
    w^0 = 0 with the Taylor first step w^1 = -dt^2/2 cos(omega_hat t^0), filtered by the
    trapezoid weights (eq. discreteWaveExplicit, eq. quadrature)."""
    lam2 = np.asarray(lam2, dtype=np.float64)
    dt2 = tg.dt * tg.dt
    phase = tg.forcing_phase()
    weight = tg.filter_weights()
    w_prev = np.zeros_like(lam2)
    w_cur = np.full_like(lam2, -0.5 * dt2 * phase[0])
    acc = weight[1] * w_cur
    for n in range(1, tg.nt):
        w_next = 2.0 * w_cur - w_prev + dt2 * (-lam2 * w_cur - phase[n])
        acc = acc + weight[n + 1] * w_next
        w_prev, w_cur = w_cur, w_next
    return acc


class ModalSystem:
    """The diagonal form of the box's WaveHoltz system for one (grid, time grid): per mode
    lambda^2, mu = 1 - beta_h, gamma_h, and the deflation mask of the nd modes Algorithm 2
    removes (spectral.deflation_order)."""

    def __init__(self, grid: Grid, tg: TimeGrid, nd: int):
        if grid.c2 is not None:
            raise ValueError("the sine basis diagonalises the constant-speed operator only")
        modes = SP.all_modes(grid)
        lam2 = SP.mode_lambda2(grid, modes)
        bh = SP.beta_h(lam2, tg)
        defl = np.zeros(len(modes), dtype=bool)
        defl[SP.deflation_order(grid, modes, bh)[:nd]] = True
        self.grid, self.tg, self.nd = grid, tg, nd
        self.lam2 = _mode_array(grid, lam2)
        self.mu = _mode_array(grid, 1.0 - bh)
        self.gamma = _mode_array(grid, forced_transfer(lam2, tg))
        self.deflated = _mode_array(grid, defl)


def devd_cg(system: ModalSystem, f: np.ndarray, tol: float, maxit: int):
    """Algorithm 2 with CG for the forcings f (one interior array, or a stack along axis 0),
    in sine coefficients: f_d = f with the deflated coefficients removed, b = gamma_h f_d,
    CG on diag(mu) x = b stopped as krylov.cg stops (||r|| <= tol ||b||, checked after each
    iteration), inflation u_m = f_m / (omega_eff^2 - lambda_m^2) on the deflated modes.
    Returns (iterations[S], converged[S], u[S, ...]) with u the solutions on the grid."""
    g = system.grid
    f = np.asarray(f, dtype=np.float64)
    single = f.ndim == g.dim
    F = sine_coefficients(g, f[None] if single else f)
    S = F.shape[0]
    keep = ~system.deflated
    fd = np.where(keep, F, 0.0)
    b = (system.gamma * fd).reshape(S, -1)
    mu = system.mu.ravel()
    x = np.zeros_like(b)
    its = np.zeros(S, dtype=np.int64)
    done = np.zeros(S, dtype=bool)
    for s in range(S):   # krylov.cg from x_0 = 0 on diag(mu) x = b_s
        r = b[s].copy()
        p = r.copy()
        q = np.empty_like(r)
        rr = float(r @ r)
        bnorm = math.sqrt(rr)
        done[s] = math.sqrt(rr) <= tol * bnorm
        for k in range(maxit):
            if done[s]:
                break
            np.multiply(mu, p, out=q)
            alpha = rr / float(p @ q)
            x[s] += alpha * p
            r -= alpha * q
            rr_new = float(r @ r)
            its[s] = k + 1
            if math.sqrt(rr_new) <= tol * bnorm:
                done[s] = True
                break
            p *= rr_new / rr
            p += r
            rr = rr_new
    om2 = system.tg.omega_eff ** 2
    u_hat = np.where(keep, x.reshape(F.shape), F / (om2 - system.lam2))
    u = from_sine_coefficients(g, u_hat)
    if single:
        return int(its[0]), bool(done[0]), u[0]
    return its, done, u
