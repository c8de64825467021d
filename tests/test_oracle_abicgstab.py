"""Pins of the oracle's Algorithm 6 (augmented BiCGStab): without augmentation it is scipy's
BiCGStab iterate for iterate; with augmentation it is BiCGStab on the projected system
(I - Q Q^T) A y = (I - Q Q^T) r_0 (scipy, dense, Q from numpy's QR of A W) followed by the W
correction; the M inner product is BiCGStab on the similarity transform M^{1/2} A M^{-1/2}; and the
method reaches the direct Helmholtz solution."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


class _DenseGrid:
    def __init__(self, shape, w):
        self.shape = shape
        self._w = np.asarray(w, dtype=np.float64).reshape(shape)

    def weights(self):
        return self._w


def _problem(seed, n=30):
    rng = np.random.default_rng(seed)
    Amat = np.eye(n) + 0.4 * rng.standard_normal((n, n)) / math.sqrt(n)
    return rng, Amat, rng.standard_normal(n)


@pytest.mark.parametrize("k", [1, 2, 5, 8])
def test_abicgstab_without_augmentation_is_scipy_bicgstab(k):
    rng, Amat, b = _problem(k)
    shape = (5, 6)
    A = lambda v: (Amat @ np.asarray(v).ravel()).reshape(shape)  # noqa: E731
    res = K.abicgstab(_DenseGrid(shape, np.ones(30)), A, b, None, 0.0, k)
    xs, info = spl.bicgstab(Amat, b, rtol=0.0, atol=0.0, maxiter=k)
    assert res.iterations == k
    assert np.allclose(res.x.ravel(), xs, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p,k", [(3, 4), (5, 7)])
def test_abicgstab_is_bicgstab_on_the_projected_system(p, k):
    rng, Amat, b = _problem(20 + p)
    shape = (5, 6)
    A = lambda v: (Amat @ np.asarray(v).ravel()).reshape(shape)  # noqa: E731
    W = rng.standard_normal((30, p))
    x0 = rng.standard_normal(30)
    res = K.abicgstab(_DenseGrid(shape, np.ones(30)), A, b, W, 0.0, k, x0=x0)
    Q, _ = np.linalg.qr(Amat @ W)
    P = np.eye(30) - Q @ Q.T
    r0 = b - Amat @ x0
    y, _ = spl.bicgstab(P @ Amat, P @ r0, rtol=0.0, atol=0.0, maxiter=k)
    # the W correction removes the range(A W) part of the residual: A W c = Q Q^T (r0 - A y)
    c = np.linalg.lstsq(Amat @ W, Q @ (Q.T @ (r0 - Amat @ y)), rcond=None)[0]
    x_expected = x0 + y + W @ c
    assert np.allclose(res.x.ravel(), x_expected, rtol=1e-10, atol=1e-11)
    # the tracked residual is the true one of the returned iterate
    r_true = b - Amat @ res.x.ravel()
    assert np.allclose(Q.T @ r_true, 0.0, atol=1e-11)
    assert math.sqrt(r_true @ r_true) / math.sqrt(b @ b) == pytest.approx(res.history[-1], rel=1e-8)


def test_abicgstab_m_inner_product_is_a_similarity_transform():
    """BiCGStab in <u, v>_M on A equals Euclidean BiCGStab on S A S^{-1} (S = M^{1/2}) with the
    iterates mapped by S."""
    rng, Amat, b = _problem(7)
    shape = (5, 6)
    w = rng.uniform(0.5, 2.0, 30)
    S = np.sqrt(w)
    A = lambda v: (Amat @ np.asarray(v).ravel()).reshape(shape)  # noqa: E731
    k = 6
    res = K.abicgstab(_DenseGrid(shape, w), A, b, None, 0.0, k)
    Ahat = (S[:, None] * Amat) / S[None, :]
    xs, _ = spl.bicgstab(Ahat, S * b, rtol=0.0, atol=0.0, maxiter=k)
    assert np.allclose(S * res.x.ravel(), xs, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("basis", ["none", "exact", "general"])
def test_abicgstab_reaches_direct_solution(basis):
    npts, om = (41, 37), 14.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, om)
    f = I.gaussian(npts, [0.4, 0.6], 0.08, om ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    W = lam2 = None
    if basis != "none":
        modes, lam2, _ = SP.select_modes(og, tg, 6)
        W = SP.basis(og, modes)
        if basis == "general":
            W = W + 0.1 * np.random.default_rng(3).standard_normal(W.shape) / math.sqrt(og.n)
            lam2 = None
    r = K.augmented_solve(og, tg, f, W, lam2, tol=1e-11, maxit=3000, method="abicgstab")
    assert r.solve.converged
    assert IND.relmax(r.u, U) < 1e-8


def test_abicgstab_exact_eigenvectors_b_in_span():
    npts, om = (23, 19), 10.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, om)
    modes, lam2, bh = SP.select_modes(og, tg, 4)
    V = SP.basis(og, modes)
    c = np.array([1.0, -2.0, 0.5, 3.0])
    b = (V @ c).reshape(og.shape)
    res = K.abicgstab(og, K.Operator(og, tg), b, V, 1e-13, 50, AW=V * (1.0 - bh)[None, :])
    assert res.iterations == 0 and res.converged
    assert np.allclose(res.x.ravel(), V @ (c / (1.0 - bh)), rtol=1e-12, atol=1e-14)
