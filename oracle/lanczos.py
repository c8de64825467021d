"""Krylov eigen-solve on the WaveHoltz operator (oracle; test infrastructure only).

EigenWave idea (Sec. 4.1, "computed using EigenWave"): eigenvectors of L_h are eigenvectors
of S_h with eigenvalue beta_h(lambda), and the ones wanted for deflation (lambda nearest the
frequency) sit at the top of the spectrum of S_h (beta_h near 1).  A Krylov method on S_h --
one wave solve per matrix-vector product -- therefore finds them as its extremal Ritz pairs.

This oracle runs the plain Lanczos three-term recurrence in the M inner product (S_h is
M-self-adjoint, see operators.py), with full re-orthogonalisation of every new vector against
all previous ones (classical Gram-Schmidt applied twice), for `m` steps from a given start
vector; the Ritz pairs of the m x m tridiagonal matrix are computed with numpy's symmetric
eigen-solver; the nd Ritz vectors with the largest Ritz values are returned, with
lambda^2 = -<y, L_h y>_M / <y, y>_M (Rayleigh quotient) and the residual ||L_h y + lambda^2 y||_M.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .operators import Grid, apply_L
from .waveholtz import TimeGrid, apply_S


@dataclass
class LanczosResult:
    V: np.ndarray          # (N, nd) Ritz vectors, M-orthonormal
    theta: np.ndarray      # Ritz values (approximations of beta_h), descending
    lambda2: np.ndarray    # Rayleigh quotients of -L_h
    resid: np.ndarray      # ||L_h y + lambda^2 y||_M / lambda^2
    T: np.ndarray          # the tridiagonal matrix
    steps: int


def lanczos(grid: Grid, tg: TimeGrid, m: int, nd: int, v0: np.ndarray) -> LanczosResult:
    w = grid.weights().ravel()
    ip = lambda a, b: float(np.sum(w * a * b))  # noqa: E731
    N = grid.n
    Q = np.zeros((N, m))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    q = np.asarray(v0, dtype=np.float64).ravel()
    q = q / np.sqrt(ip(q, q))
    k = 0
    for j in range(m):
        Q[:, j] = q
        z = apply_S(grid, tg, q.reshape(grid.shape)).ravel()
        alpha[j] = ip(q, z)
        for _ in range(2):  # full re-orthogonalisation, classical Gram-Schmidt twice
            h = Q[:, : j + 1].T @ (w * z)
            z = z - Q[:, : j + 1] @ h
        k = j + 1
        b = np.sqrt(ip(z, z))
        if j + 1 < m:
            beta[j] = b
            if b == 0.0:
                break
            q = z / b
    T = np.diag(alpha[:k]) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    theta, S = np.linalg.eigh(T)
    order = np.argsort(-theta)[:nd]
    Y = Q[:, :k] @ S[:, order]
    lam2 = np.zeros(len(order))
    res = np.zeros(len(order))
    for i in range(len(order)):
        y = Y[:, i]
        Ly = apply_L(grid, y.reshape(grid.shape)).ravel()
        lam2[i] = -ip(y, Ly) / ip(y, y)
        r = Ly + lam2[i] * y
        res[i] = np.sqrt(ip(r, r)) / lam2[i]
    return LanczosResult(Y, theta[order], lam2, res, T, k)


@dataclass
class ThickResult(LanczosResult):
    restarts: int = 0
    wave_solves: int = 0
    converged: int = 0


def lanczos_thick(grid: Grid, tg: TimeGrid, nd: int, m: int, v0: np.ndarray, max_restarts: int = 50,
                  tol: float = 1e-10, keep: int | None = None) -> ThickResult:
    """Thick-restart Lanczos (Wu and Simon, 2000) on S_h in the M inner product, for the nd largest
    eigenpairs with a basis of at most m vectors.  Every step re-orthogonalises against the whole
    basis (classical Gram-Schmidt twice), so the projected matrix H = Q^T M S_h Q is filled from the
    Gram-Schmidt coefficients.  When the basis is full: Ritz pairs of H (numpy eigh); the residual
    of Ritz pair i is |b s_{m,i}| (b the norm of the last, unnormalised vector); if the nd largest
    are below tol -- or the restarts are used up -- stop, else keep the `keep` largest Ritz vectors
    and the last vector as the new basis (H = diag(theta) bordered by b s_{m,i}) and continue."""
    w = grid.weights().ravel()
    ip = lambda a, b: float(np.sum(w * a * b))  # noqa: E731
    N = grid.n
    keep = min(m - 2, nd + max(nd // 2, 8)) if keep is None else keep
    if not (nd <= keep < m - 1):
        raise ValueError("need nd <= keep < m - 1")
    Q = np.zeros((N, m))
    H = np.zeros((m, m))
    q = np.asarray(v0, dtype=np.float64).ravel()
    Q[:, 0] = q / np.sqrt(ip(q, q))
    j0, nws, restarts = 0, 0, 0
    while True:
        b, qn = 0.0, None
        for j in range(j0, m):
            z = apply_S(grid, tg, Q[:, j].reshape(grid.shape)).ravel()
            nws += 1
            hsum = np.zeros(j + 1)
            for _ in range(2):
                h = Q[:, : j + 1].T @ (w * z)
                z = z - Q[:, : j + 1] @ h
                hsum += h
            H[: j + 1, j] = hsum
            H[j, : j + 1] = hsum
            b = np.sqrt(ip(z, z))
            if j + 1 < m:
                H[j + 1, j] = H[j, j + 1] = b
                Q[:, j + 1] = z / b
            else:
                qn = z / b
        theta, S = np.linalg.eigh(H)
        order = np.argsort(-theta)
        est = np.abs(b * S[m - 1, order[:nd]])
        conv = int(np.sum(est <= tol))
        if conv == nd or restarts == max_restarts:
            break
        restarts += 1
        Y = Q @ S[:, order[:keep]]
        Q[:, :keep] = Y
        Q[:, keep] = qn
        Q[:, keep + 1:] = 0.0
        H[:] = 0.0
        H[:keep, :keep] = np.diag(theta[order[:keep]])
        H[:keep, keep] = H[keep, :keep] = b * S[m - 1, order[:keep]]
        j0 = keep
    Y = Q @ S[:, order[:nd]]
    lam2 = np.zeros(nd)
    res = np.zeros(nd)
    for i in range(nd):
        y = Y[:, i]
        Ly = apply_L(grid, y.reshape(grid.shape)).ravel()
        lam2[i] = -ip(y, Ly) / ip(y, y)
        r = Ly + lam2[i] * y
        res[i] = np.sqrt(ip(r, r)) / lam2[i]
    return ThickResult(Y, theta[order[:nd]], lam2, res, H, m, restarts, nws, conv)
