"""Pins of the oracle's SVD compression of deflation vectors: closed-form sine vectors are rank 1,
the truncation rank is the smallest meeting the Frobenius tolerance (checked by explicit
reconstruction), compressed projections and expansions equal dense ones with the reconstructed
vectors, and the deflated solve takes the same iterations with compressed vectors (Sec. 4.3)."""
import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K, compression as C
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


def test_sine_tensor_vectors_are_rank_one():
    og = O.Grid((41, 33))
    tg = WH.time_grid_for(og, 14.0)
    modes, _, _ = SP.select_modes(og, tg, 10)
    comp = C.compress_basis(og, SP.basis(og, modes), 1e-10)
    assert all(c.rank == 1 for c in comp)
    assert all(abs(c.s[0] - 1.0) < 1e-13 for c in comp)   # unit vectors
    ny, nx = og.shape
    assert C.compression_ratio(og, comp) == pytest.approx((nx + ny + 1) / (nx * ny))


@pytest.mark.parametrize("tau", [1e-2, 1e-4, 1e-7])
def test_truncation_rank_is_minimal(tau):
    rng = np.random.default_rng(5)
    ny, nx = 37, 29
    # decaying spectrum: singular values 10^(-k/2)
    A = np.linalg.qr(rng.standard_normal((ny, ny)))[0][:, :nx]
    B = np.linalg.qr(rng.standard_normal((nx, nx)))[0]
    s = 10.0 ** (-0.5 * np.arange(nx))
    Q = (A * s) @ B.T
    c = C.truncated_svd(Q, tau)
    err = np.linalg.norm(Q - c.U @ np.diag(c.s) @ c.V.T)
    assert err < tau and err == pytest.approx(c.error, rel=1e-6, abs=1e-15)
    if c.rank > 0:   # one vector fewer misses the tolerance
        r = c.rank - 1
        err1 = np.linalg.norm(Q - c.U[:, :r] @ np.diag(c.s[:r]) @ c.V[:, :r].T)
        assert err1 >= tau


def test_compressed_contractions_equal_dense_ones():
    npts = (33, 27)
    c2 = I.speed_squared("c3", npts, 3)
    og = O.Grid(npts, order=4, c2=c2)
    rng = np.random.default_rng(1)
    W = rng.standard_normal((og.n, 4)) @ np.diag([1, 0.5, 0.2, 0.1])
    comp = C.compress_basis(og, W, 1e-3)
    D = np.stack([C.dense(og, c) for c in comp], axis=1)
    r = rng.standard_normal(og.n)
    y = rng.standard_normal(4)
    wts = og.weights().ravel()
    assert np.allclose(C.project(og, comp, r), D.T @ (wts * r), rtol=1e-12, atol=1e-12)
    assert np.allclose(C.expand(og, comp, y), D @ y, rtol=1e-12, atol=1e-12)


def test_compressed_exact_eigenvectors_keep_the_iterations():
    """Degenerate pairs of sine modes mixed into rank-2 exact eigenvectors: compressed to
    tau = 1e-8 they stay exact, and DEVD-CG (Algorithm 2) takes the same iterations to the same
    solution as with the full vectors (Sec. 4.3 reports identical iteration counts)."""
    npts, omega = (45, 45), 20.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    modes, lam2, _ = SP.select_modes(og, tg, 12)
    V = SP.basis(og, modes)
    # rotate each degenerate pair (k,l), (l,k) by 45 degrees: still eigenvectors, rank 2
    Vr, key = V.copy(), {tuple(m): j for j, m in enumerate(modes.tolist())}
    for j, m in enumerate(modes.tolist()):
        t = key.get((m[1], m[0]))
        if t is not None and t > j:
            a, b = V[:, j].copy(), V[:, t].copy()
            Vr[:, j], Vr[:, t] = (a + b) / np.sqrt(2), (a - b) / np.sqrt(2)
    comp = C.compress_basis(og, Vr, 1e-8)
    assert max(c.rank for c in comp) == 2
    Vc = np.stack([C.dense(og, c) for c in comp], axis=1)
    f = I.gaussian(npts, [0.4, 0.55], 1.0 / omega, omega ** 2)
    full = K.devd_solve(og, tg, f, Vr, lam2, "cg", 1e-10, 2000)
    comp_s = K.devd_solve(og, tg, f, Vc, lam2, "cg", 1e-10, 2000)
    assert comp_s.solve.iterations == full.solve.iterations
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    assert IND.relmax(comp_s.u, U) < 1e-8
