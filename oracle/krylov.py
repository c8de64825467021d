"""Iterative solvers of the WaveHoltz fixed-point system (oracle; test infrastructure only).

All inner products are <u, v>_M = sum u v / c^2 (the Euclidean one for c = 1), in which
A = I - S_h is self-adjoint (see operators.py).

* fpi          Algorithm 1 (fixed-point iteration v <- Pi_h v).
* cg           conjugate gradients on A x = b (Sec. 3: CG-accelerated WaveHoltz).
* dcg          Algorithm 4 (deflated CG of Saad et al.), with the typos of the listing
               corrected: r2 = r_0^T r_0 and r_{k+1} = r_k - alpha_k q_k.
* gmres        restarted GMRES(m) with classical Gram-Schmidt applied twice and Givens
               rotations (the unaugmented base of Algorithm 5).
* agmres       Algorithm 5 (augmented GMRES of Baglama and Reichel with Givens rotations):
               the search space is span(W) + the Krylov space of A started from the part of
               b_0 outside range(A W); restarted after m Arnoldi steps, keeping the QR factors
               of A W.
* abicgstab    Algorithm 6 (augmented / recycled BiCGStab of Amritkar et al.), with the listing's
               typos corrected: eta_1 = Q^T r and r <- r - Q eta_1 at the start, p = r in the
               first iteration (i = 1), alpha = rho / <r~, v>.
* augmented_solve  A u = b (b = Pi_h(0; f), undeflated forcing) by agmres or abicgstab with the
               basis W.
* devd_solve   Algorithm 2 (direct eigenvector deflation): deflate the forcing, solve with
               FPI / CG / GMRES, optionally re-deflate each operator output, inflate.

Stopping rule (reading): ||r_k||_M <= tol ||b||_M on the system actually iterated on
(b = Pi_h(0; f_d) for DEVD; the deflated start residual r_0 for DCG, as in Algorithm 4).
Each result reports `wave_solves`, the number of applications of Pi_h.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .operators import Grid
from .waveholtz import TimeGrid, apply_pi, apply_A


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    wave_solves: int
    converged: bool
    history: list = field(default_factory=list)


class Operator:
    """A = I - S_h with a counter of wave solves and optional re-deflation of outputs."""

    def __init__(self, grid: Grid, tg: TimeGrid, V=None, redeflate=False):
        self.grid, self.tg, self.V, self.redeflate = grid, tg, V, redeflate
        self.count = 0

    def __call__(self, v):
        self.count += 1
        out = apply_A(self.grid, self.tg, v)
        if self.redeflate and self.V is not None:
            out = project_out(self.grid, self.V, out)
        return out


def project_coeffs(grid: Grid, V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """V^T M r (the deflation projections (r, phi_m)_Omega of Algorithm 2)."""
    w = grid.weights().ravel()
    return V.T @ (w * np.asarray(r).ravel())


def project_out(grid: Grid, V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """r - V (V^T M r)  (Algorithm 2, deflate forcing / iterate)."""
    r = np.asarray(r).reshape(grid.shape)
    return r - (V @ project_coeffs(grid, V, r)).reshape(grid.shape)


def fpi(grid, tg, f, tol, maxit, x0=None, V=None, redeflate=False):
    """Algorithm 1: v^{k+1} = Pi_h v^k; converged when ||Pi_h v - v||_M <= tol ||Pi_h 0||_M."""
    v = np.zeros(grid.shape) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(grid.shape).copy()
    b = apply_pi(grid, tg, np.zeros(grid.shape), f)
    bnorm = grid.norm(b)
    count = 1
    hist = []
    for k in range(maxit):
        nv = apply_pi(grid, tg, v, f)
        count += 1
        if redeflate and V is not None:
            nv = project_out(grid, V, nv)
        res = grid.norm(nv - v) / bnorm
        hist.append(res)
        v = nv
        if res <= tol:
            return SolveResult(v, k + 1, count, True, hist)
    return SolveResult(v, maxit, count, False, hist)


def cg(grid, A, b, tol, maxit, x0=None):
    """Conjugate gradients on A x = b in the M inner product."""
    x = np.zeros(grid.shape) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(grid.shape).copy()
    r = b - A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = grid.inner(r, r)
    bnorm = grid.norm(b)
    hist = [math.sqrt(rr) / bnorm]
    if hist[-1] <= tol:
        return SolveResult(x, 0, 0, True, hist)
    for k in range(maxit):
        q = A(p)
        pq = grid.inner(p, q)
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = grid.inner(r, r)
        hist.append(math.sqrt(rr_new) / bnorm)
        if hist[-1] <= tol:
            return SolveResult(x, k + 1, 0, True, hist)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return SolveResult(x, maxit, 0, False, hist)


def dcg(grid, A, b, W, tol, maxit, mu=None, AW=None):
    """Algorithm 4 (deflated CG).  With exact eigenvectors pass mu = diag(W^T A W)
    (= 1 - beta_h(lambda_m)): then x_0 and r_0 need no wave solve and the per-iteration
    A-orthogonalisation of the search direction against W (the eta / mu update) is skipped,
    as the paper allows for true eigenvectors.  Otherwise pass AW = A W (or nothing: it is
    then formed with nd wave solves) and the projections are applied."""
    wts = grid.weights().ravel()
    shape = grid.shape
    exact = mu is not None
    if exact:
        WtAW_inv = lambda y: y / mu  # noqa: E731
    else:
        if AW is None:
            AW = np.stack([A(W[:, m].reshape(shape)).ravel() for m in range(W.shape[1])], axis=1)
        WtAW = W.T @ (wts[:, None] * AW)
        WtAW_inv = lambda y: np.linalg.solve(WtAW, y)  # noqa: E731
    bf = np.asarray(b).ravel()
    # x_{-1} = 0, r_{-1} = b
    r_m1 = bf.copy()
    x = W @ WtAW_inv(W.T @ (wts * r_m1))
    if exact:
        r = r_m1 - W @ (mu * WtAW_inv(W.T @ (wts * r_m1)))   # A W = W diag(mu)
        p = r.copy()                                           # W^T M r_0 = 0
    else:
        r = bf - A(x.reshape(shape)).ravel()
        eta = AW.T @ (wts * r)                                 # W^T A r_0 (A self-adjoint in M)
        p = r - W @ WtAW_inv(eta)
    r2 = float(np.sum(wts * r * r))
    r0 = r2
    hist = [1.0]
    k = 0
    while r2 / r0 > tol * tol and k < maxit:
        q = A(p.reshape(shape)).ravel()
        alpha = r2 / float(np.sum(wts * p * q))
        x = x + alpha * p
        r = r - alpha * q
        r2_old = r2
        r2 = float(np.sum(wts * r * r))
        beta_k = r2 / r2_old
        if exact:
            p = beta_k * p + r
        else:
            eta = AW.T @ (wts * r)
            p = beta_k * p + r - W @ WtAW_inv(eta)
        k += 1
        hist.append(math.sqrt(r2 / r0))
    return SolveResult(x.reshape(shape), k, 0, r2 / r0 <= tol * tol, hist)


def gmres(grid, A, b, tol, maxit, restart=30, x0=None):
    """Restarted GMRES(m); Arnoldi with classical Gram-Schmidt applied twice; the least-
    squares problem is reduced with Givens rotations and solved by back substitution.
    `maxit` bounds the number of Arnoldi steps (operator applications in the cycles)."""
    shape = grid.shape
    wts = grid.weights().ravel()
    ip = lambda u, v: float(np.sum(wts * u * v))  # noqa: E731
    bf = np.asarray(b, dtype=np.float64).ravel()
    x = np.zeros(bf.size) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    bnorm = math.sqrt(ip(bf, bf))
    r = bf.copy() if x0 is None else bf - A(x.reshape(shape)).ravel()
    its = 0
    hist = []
    while True:
        beta0 = math.sqrt(ip(r, r))
        hist.append(beta0 / bnorm)
        if beta0 / bnorm <= tol or its >= maxit:
            return SolveResult(x.reshape(shape), its, 0, beta0 / bnorm <= tol, hist)
        m = restart
        basis = [r / beta0]
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta0
        k = 0
        for j in range(m):
            w = A(basis[j].reshape(shape)).ravel()
            its += 1
            for _ in range(2):  # classical Gram-Schmidt, applied twice
                h = np.array([ip(vi, w) for vi in basis])
                w = w - sum(hi * vi for hi, vi in zip(h, basis))
                H[: j + 1, j] += h
            H[j + 1, j] = math.sqrt(ip(w, w))
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                basis.append(w / H[j + 1, j])
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[k]) / bnorm <= tol or its >= maxit or breakdown:
                break
        y = np.zeros(k)
        for i in reversed(range(k)):
            y[i] = (g[i] - H[i, i + 1: k] @ y[i + 1:]) / H[i, i]
        x = x + sum(yi * vi for yi, vi in zip(y, basis))
        if abs(g[k]) / bnorm <= tol:
            hist.append(abs(g[k]) / bnorm)
            return SolveResult(x.reshape(shape), its, 0, True, hist)
        r = bf - A(x.reshape(shape)).ravel()


def agmres(grid, A, b, W, tol, maxit, restart=30, x0=None, AW=None):
    """Algorithm 5, restarted after `restart` Arnoldi steps.  W: n x p augmentation vectors
    (columns); AW: A W if known (A W = W diag(mu) for exact eigenvectors), else formed with p
    applications of A.  Per cycle, in the notation of Algorithm 5 (inner products <.,.>_M):
        b_0 = b - A x_0
        A W = V_{1:p} H_{1:p,1:p}              thin QR (classical Gram-Schmidt, twice)
        v_{p+1} = (I - V_p V_p^T M) b_0 / ||.||
        g_k = <v_k, b_0>,  k = 1 .. p+1
        Arnoldi from v_{p+1}: v_{k+1} = A v_k made orthogonal to v_1 .. v_k (twice), h_{k+1,k}
        Givens rotations on columns k > p (the first p columns are already triangular)
        |g_{k+1}| = residual norm;  stop when |g_{k+1}| <= tol ||b||
        H_{1:k,1:k} y = g_{1:k};  x = x_0 + [W | V_{p+1:k}] y
    The QR factors of A W are computed once and kept over restarts.  `maxit` bounds the Arnoldi
    steps.  SolveResult.wave_solves counts the applications of A made here."""
    shape = grid.shape
    wts = grid.weights().ravel()
    ip = lambda u, v: float(np.sum(wts * u * v))  # noqa: E731
    bf = np.asarray(b, dtype=np.float64).ravel()
    W = np.zeros((bf.size, 0)) if W is None else np.asarray(W, dtype=np.float64).reshape(bf.size, -1)
    p = W.shape[1]
    m = restart
    nA = 0
    if AW is None:
        AW = np.zeros_like(W)
        for j in range(p):
            AW[:, j] = A(W[:, j].reshape(shape)).ravel()
            nA += 1
    else:
        AW = np.asarray(AW, dtype=np.float64).reshape(bf.size, p)
    # A W = V_{1:p} H_{1:p,1:p}
    Vp = []
    Hp = np.zeros((p, p))
    for j in range(p):
        w = AW[:, j].copy()
        for _ in range(2):
            h = np.array([ip(vi, w) for vi in Vp])
            if len(Vp):
                w = w - sum(hi * vi for hi, vi in zip(h, Vp))
                Hp[:j, j] += h
        Hp[j, j] = math.sqrt(ip(w, w))
        Vp.append(w / Hp[j, j])
    x = np.zeros(bf.size) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    bnorm = math.sqrt(ip(bf, bf))
    b0 = bf.copy()
    if x0 is not None:
        b0 = bf - A(x.reshape(shape)).ravel()
        nA += 1
    its = 0
    hist = []
    cycle = 0
    while True:
        beta0 = math.sqrt(ip(b0, b0))
        hist.append(beta0 / bnorm)
        # (the first cycle always runs: with maxit = 0 it is the least-squares fit over span(W))
        if beta0 / bnorm <= tol or (cycle > 0 and its >= maxit):
            return SolveResult(x.reshape(shape), its, nA, beta0 / bnorm <= tol, hist)
        cycle += 1
        v = b0.copy()
        for _ in range(2):
            v = v - sum(ip(vi, v) * vi for vi in Vp) if p else v
        vn = math.sqrt(ip(v, v))
        V = list(Vp) + [v / vn if vn > 0.0 else v]
        H = np.zeros((p + m + 1, p + m))
        H[:p, :p] = Hp
        g = np.zeros(p + m + 1)
        for k in range(p + 1):
            g[k] = ip(V[k], b0)
        cs, sn = np.zeros(p + m), np.zeros(p + m)
        k = p
        breakdown = False
        # |g_{p+1}| = ||(I - V_p V_p^T M) b_0|| is already the residual of the least-squares fit
        # over span(W) alone: no Arnoldi step when that meets tol
        steps = range(p, p + min(m, maxit - its)) if abs(g[p]) / bnorm > tol else range(0)
        for j in steps:
            w = A(V[j].reshape(shape)).ravel()
            nA += 1
            its += 1
            for _ in range(2):
                h = np.array([ip(vi, w) for vi in V])
                w = w - sum(hi * vi for hi, vi in zip(h, V))
                H[: j + 1, j] += h
            H[j + 1, j] = math.sqrt(ip(w, w))
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V.append(w / H[j + 1, j])
            for i in range(p, j):   # previous rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[k]) / bnorm <= tol or its >= maxit or breakdown:
                break
        y = np.zeros(k)
        for i in reversed(range(k)):
            y[i] = (g[i] - H[i, i + 1: k] @ y[i + 1:]) / H[i, i]
        x = x + W @ y[:p] + sum((y[i] * V[i] for i in range(p, k)), np.zeros(bf.size))
        if abs(g[k]) / bnorm <= tol or breakdown or its >= maxit:
            hist.append(abs(g[k]) / bnorm)
            return SolveResult(x.reshape(shape), its, nA, abs(g[k]) / bnorm <= tol, hist)
        b0 = bf - A(x.reshape(shape)).ravel()   # restart
        nA += 1


def _thin_qr(ip, AW):
    """A W = Q R with M-orthonormal Q (classical Gram-Schmidt, twice) and upper-triangular R."""
    p = AW.shape[1]
    Q = []
    R = np.zeros((p, p))
    for j in range(p):
        w = AW[:, j].copy()
        for _ in range(2):
            if Q:
                h = np.array([ip(q, w) for q in Q])
                w = w - sum(hi * q for hi, q in zip(h, Q))
                R[:j, j] += h
        R[j, j] = math.sqrt(ip(w, w))
        Q.append(w / R[j, j])
    return (np.array(Q).T if p else np.zeros((AW.shape[0], 0))), R


def abicgstab(grid, A, b, W, tol, maxit, x0=None, AW=None):
    """Algorithm 6 (inner products <.,.>_M).  `maxit` bounds the iterations (two applications of
    A each).  In the notation of Algorithm 6:
        r = b - A x,  r~ = r
        A W = Q R;  eta_1 = Q^T r;  r <- r - Q eta_1;  xi = -eta_1
        loop: rho = <r~, r>;  p = r (first) or r + beta (p - omega v), beta = (rho/rho_old)(alpha/omega)
              v = A p;  eta_1 = Q^T v;  v <- v - Q eta_1;  alpha = rho / <r~, v>;  s = r - alpha v
              ||s|| <= tol ||b||: x += alpha p, r = s, xi += alpha eta_1, stop
              t = A s;  eta_2 = Q^T t;  t <- t - Q eta_2;  omega = <t, s> / <t, t>
              xi += alpha eta_1 + omega eta_2;  x += alpha p + omega s;  r = s - omega t
              ||r|| <= tol ||b||: stop
        x <- x - W R^{-1} xi
    The tracked r is the residual of the final x (the W correction removes its range(A W) part)."""
    shape = grid.shape
    wts = grid.weights().ravel()
    ip = lambda u, v: float(np.sum(wts * u * v))  # noqa: E731
    bf = np.asarray(b, dtype=np.float64).ravel()
    W = np.zeros((bf.size, 0)) if W is None else np.asarray(W, dtype=np.float64).reshape(bf.size, -1)
    p_ = W.shape[1]
    nA = 0
    if AW is None:
        AW = np.zeros_like(W)
        for j in range(p_):
            AW[:, j] = A(W[:, j].reshape(shape)).ravel()
            nA += 1
    Q, R = _thin_qr(ip, np.asarray(AW, dtype=np.float64).reshape(bf.size, p_))
    QtM = lambda v: Q.T @ (wts * v)  # noqa: E731
    x = np.zeros(bf.size) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    r = bf.copy()
    if x0 is not None:
        r = bf - A(x.reshape(shape)).ravel()
        nA += 1
    rt = r.copy()
    eta1 = QtM(r)
    r = r - Q @ eta1
    xi = -eta1
    bnorm = math.sqrt(ip(bf, bf))
    hist = [math.sqrt(ip(r, r)) / bnorm]
    converged = hist[0] <= tol
    its = 0
    rho_old = alpha = omega = 1.0
    pv = np.zeros(bf.size)
    v = np.zeros(bf.size)
    while not converged and its < maxit:
        its += 1
        rho = ip(rt, r)
        if rho == 0.0:
            break
        if its == 1:
            pv = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            pv = r + beta * (pv - omega * v)
        v = A(pv.reshape(shape)).ravel()
        nA += 1
        eta1 = QtM(v)
        v = v - Q @ eta1
        alpha = rho / ip(rt, v)
        s = r - alpha * v
        if math.sqrt(ip(s, s)) <= tol * bnorm:
            x = x + alpha * pv
            r = s
            xi = xi + alpha * eta1
            converged = True
            hist.append(math.sqrt(ip(r, r)) / bnorm)
            break
        t = A(s.reshape(shape)).ravel()
        nA += 1
        eta2 = QtM(t)
        t = t - Q @ eta2
        omega = ip(t, s) / ip(t, t)
        xi = xi + alpha * eta1 + omega * eta2
        x = x + alpha * pv + omega * s
        r = s - omega * t
        hist.append(math.sqrt(ip(r, r)) / bnorm)
        converged = hist[-1] <= tol
        rho_old = rho
    if p_:
        x = x - W @ np.linalg.solve(R, xi)
    return SolveResult(x.reshape(shape), its, nA, converged, hist)


def augmented_solve(grid: Grid, tg: TimeGrid, f, W, lam2=None, tol=1e-10, maxit=1000, restart=30, x0=None,
                    method="agmres"):
    """A u = b with b = Pi_h(0; f) (the forcing is not deflated) by Algorithm 5 (agmres) or
    Algorithm 6 (abicgstab) augmented with the columns of W.  With lam2 (W exact eigenvectors)
    A W = W diag(1 - beta_h(lambda)) costs no wave solve; without, A W takes one wave solve per
    column."""
    from .spectral import beta_h
    f = np.asarray(f, dtype=np.float64).reshape(grid.shape)
    A = Operator(grid, tg)
    b = apply_pi(grid, tg, np.zeros(grid.shape), f)
    AW = None
    if lam2 is not None and W is not None:
        AW = np.asarray(W) * (1.0 - beta_h(np.asarray(lam2), tg))[None, :]
    if method == "agmres":
        res = agmres(grid, A, b, W, tol, maxit, restart, x0, AW)
    elif method == "abicgstab":
        res = abicgstab(grid, A, b, W, tol, maxit, x0, AW)
    else:
        raise ValueError(method)
    return DevdResult(res.x, res, A.count + 1, np.zeros(0), b)


@dataclass
class DevdResult:
    u: np.ndarray
    solve: SolveResult
    wave_solves: int
    coeffs: np.ndarray
    b: np.ndarray


def devd_solve(grid: Grid, tg: TimeGrid, f, V=None, lam2=None, method="cg", tol=1e-10,
               maxit=1000, restart=30, redeflate=False, x0=None):
    """Algorithm 2 with an accelerator: f_d = f - V V^T M f; solve A x = Pi_h(0; f_d);
    u = x + V diag(1/(omega_eff^2 - lambda_m^2)) V^T M f.  V = None solves undeflated."""
    f = np.asarray(f, dtype=np.float64).reshape(grid.shape)
    if V is not None:
        coeffs = project_coeffs(grid, V, f)
        fd = f - (V @ coeffs).reshape(grid.shape)
    else:
        coeffs = np.zeros(0)
        fd = f
    A = Operator(grid, tg, V, redeflate)
    b = apply_pi(grid, tg, np.zeros(grid.shape), fd)
    if method == "cg":
        res = cg(grid, A, b, tol, maxit, x0)
    elif method == "gmres":
        res = gmres(grid, A, b, tol, maxit, restart, x0)
    elif method == "fpi":
        res = fpi(grid, tg, fd, tol, maxit, x0, V, redeflate)
        A.count = res.wave_solves - 1
    else:
        raise ValueError(method)
    u = res.x.copy()
    if V is not None:
        om2 = tg.omega_eff ** 2
        u = u + (V @ (coeffs / (om2 - lam2))).reshape(grid.shape)
    return DevdResult(u, res, A.count + 1, coeffs, b)


def true_residual(grid: Grid, tg: TimeGrid, u, f) -> float:
    """||Pi_h(u; f) - u||_M / ||Pi_h(0; f)||_M = ||b - A u|| / ||b|| of the undeflated system."""
    b = apply_pi(grid, tg, np.zeros(grid.shape), f)
    return grid.norm(apply_pi(grid, tg, u, f) - np.asarray(u).reshape(grid.shape)) / grid.norm(b)
