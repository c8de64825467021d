"""Filter transfer functions, closed-form eigenpairs and the deflation set (oracle; test
infrastructure only).

* Continuous filter transfer, Sec. 2.3 eq. beta_fun:
    beta(lambda; omega) = sinc(omega + lambda) + sinc(omega - lambda) - sinc(lambda)/2,
  reading sinc(x) = sin(x Tbar)/(x Tbar), sinc(0) = 1 (the paper does not define sinc; this
  reading reproduces its gap constant C_beta, eq. betaGap).
* Discrete transfer: for an eigenvector phi with L_h phi = -lambda^2 phi and f = 0 the
  leapfrog of eq. discreteWaveExplicit gives W^n = cos(n theta) phi with
  cos(theta) = 1 - dt^2 lambda^2 / 2, so eq. quadrature gives
    Pi_h phi = beta_h(lambda) phi,  beta_h = sum_n w_n cos(n theta),
  w_n the trapezoid filter weights.  beta_h -> beta as dt -> 0.
* Closed-form eigenvectors on the box (Sec. 4.3): tensor products of the 1-D vectors
  z_{k,i} = d_k sin(pi k i/(n-1)), i = 1..n-2, d_k = sqrt(2/(n-1)) so that z_k^T z_l = delta;
  2nd order: lambda_k^2 = (2 - 2 cos(theta_k))/h^2, 4th order (odd-reflection closure):
  lambda_k^2 = (30 - 32 cos(theta_k) + 2 cos(2 theta_k))/(12 h^2), theta_k = pi k/(n-1).
  Valid for constant speed c = 1.
* Deflation set (Sec. 2.3): deflate the eigenvectors with eigenvalues closest to omega,
  i.e. the smallest eigenvalues mu = 1 - beta_h of A.  Reading: order all modes by
  |1 - beta_h(lambda)|, ties (degenerate tensor-product modes) broken by the mode tuple
  (k_x, k_y, k_z) in lexicographic order; multi-D lambda^2 is summed over directions in
  ascending order of the per-direction values so that permuted tuples tie exactly.
"""
from __future__ import annotations

import numpy as np

from .operators import Grid
from .waveholtz import TimeGrid


def sinc_T(x, tbar):
    x = np.asarray(x, dtype=np.float64)
    xt = x * tbar
    out = np.ones_like(xt)
    nz = xt != 0.0
    out[nz] = np.sin(xt[nz]) / xt[nz]
    return out


def beta(lam, omega, tbar):
    """Continuous filter transfer beta(lambda; omega) (eq. beta_fun)."""
    lam = np.asarray(lam, dtype=np.float64)
    return sinc_T(omega + lam, tbar) + sinc_T(omega - lam, tbar) - 0.5 * sinc_T(lam, tbar)


def beta_h(lam2, tg: TimeGrid):
    """Discrete filter transfer of Pi_h on an eigenvector with eigenvalue lambda^2."""
    lam2 = np.asarray(lam2, dtype=np.float64)
    x = 1.0 - 0.5 * tg.dt * tg.dt * lam2
    if np.any(np.abs(x) > 1.0):
        raise ValueError("eigenvalue outside the leapfrog stability range")
    theta = np.arccos(x)
    w = tg.filter_weights()
    out = np.zeros_like(lam2)
    for n in range(tg.nt + 1):
        out = out + w[n] * np.cos(n * theta)
    return out


def eig1d(n: int, h: float, order: int):
    """1-D Dirichlet sine vectors and eigenvalues lambda_k^2, k = 1..n-2 (n nodes)."""
    N = n - 2
    k = np.arange(1, N + 1, dtype=np.float64)
    theta = np.pi * k / (n - 1)
    if order == 2:
        lam2 = (2.0 - 2.0 * np.cos(theta)) / (h * h)
    else:
        lam2 = (30.0 - 32.0 * np.cos(theta) + 2.0 * np.cos(2.0 * theta)) / (12.0 * h * h)
    return lam2


def eigvec1d(n: int, k: int) -> np.ndarray:
    i = np.arange(1, n - 1, dtype=np.float64)
    return np.sqrt(2.0 / (n - 1)) * np.sin(np.pi * k * i / (n - 1))


def mode_lambda2(grid: Grid, modes: np.ndarray) -> np.ndarray:
    """lambda^2 of tensor-product modes, modes[:, m] = k along direction m (1-based)."""
    modes = np.atleast_2d(modes)
    parts = []
    for m in range(grid.dim):
        l1 = eig1d(grid.npts[m], grid.h[m], grid.order)
        parts.append(l1[modes[:, m] - 1])
    parts = np.sort(np.stack(parts, axis=1), axis=1)
    lam2 = np.zeros(modes.shape[0])
    for m in range(grid.dim):
        lam2 = lam2 + parts[:, m]
    return lam2


def all_modes(grid: Grid) -> np.ndarray:
    axes = [np.arange(1, n - 1) for n in grid.npts]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def select_modes(grid: Grid, tg: TimeGrid, nd: int):
    """The nd modes with the smallest |1 - beta_h| (ties: lexicographic mode tuple).
    Returns (modes[nd, dim], lambda2[nd], beta_h[nd])."""
    if grid.c2 is not None:
        raise ValueError("closed-form eigenpairs need constant speed")
    modes = all_modes(grid)
    lam2 = mode_lambda2(grid, modes)
    bh = beta_h(lam2, tg)
    order = deflation_order(grid, modes, bh)[:nd]
    return modes[order], lam2[order], bh[order]


def deflation_order(grid: Grid, modes: np.ndarray, bh: np.ndarray) -> np.ndarray:
    """Indices of `modes` sorted by |1 - beta_h| ascending, ties by the mode tuple
    (k_x, k_y, k_z) in lexicographic order (the reading of Sec. 2.3 used by select_modes)."""
    key = np.abs(1.0 - bh)
    keys = [modes[:, m] for m in reversed(range(grid.dim))] + [key]
    return np.lexsort(keys)


def mode_vector(grid: Grid, mode) -> np.ndarray:
    """Tensor-product eigenvector for one mode tuple, on the interior array shape."""
    vec = np.ones(())
    for m in reversed(range(grid.dim)):  # build (z, y, x) outer product
        vec = np.multiply.outer(vec, eigvec1d(grid.npts[m], int(mode[m])))
    return vec.reshape(grid.shape)


def basis(grid: Grid, modes) -> np.ndarray:
    """Deflation matrix W, shape (N, nd), columns the mode vectors flattened (x fastest)."""
    return np.stack([mode_vector(grid, md).ravel() for md in modes], axis=1)


def acr(grid: Grid, tg: TimeGrid, deflated_modes=None) -> float:
    """Asymptotic convergence rate of the FPI (eq. WaveHoltzFPIconvergence): max |beta_h|
    over the modes not in the deflation set."""
    modes = all_modes(grid)
    bh = beta_h(mode_lambda2(grid, modes), tg)
    keep = np.ones(len(modes), dtype=bool)
    if deflated_modes is not None and len(deflated_modes):
        dm = {tuple(int(x) for x in m) for m in deflated_modes}
        keep = np.array([tuple(int(x) for x in m) not in dm for m in modes])
    return float(np.max(np.abs(bh[keep])))


def kappa(grid: Grid, tg: TimeGrid, nd: int = 0) -> float:
    """Condition number of A (nd = 0) or of the eigenvector-deflated operator (Theorem 3.2:
    mu_max / mu_{nd+1}, mu = 1 - beta_h sorted ascending)."""
    modes = all_modes(grid)
    mu = np.sort(1.0 - beta_h(mode_lambda2(grid, modes), tg))
    return float(mu[-1] / mu[nd])
