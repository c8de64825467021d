"""Pins of the oracle's Krylov eigen-solve on S_h against a dense symmetric eigen-solve."""
import numpy as np
import scipy.sparse as sp

from oracle import operators as O, waveholtz as WH, spectral as SP, lanczos as LZ
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


def _dense_pairs(npts, order, c2):
    """Eigenpairs of -c^2 Delta_h via the symmetric similar matrix diag(c) (-Delta_h) diag(c)."""
    L = IND.laplacian_matrix(npts, order)
    c = np.sqrt(np.asarray(c2).ravel())
    Ssym = (sp.diags(c) @ (-L) @ sp.diags(c)).toarray()
    Ssym = 0.5 * (Ssym + Ssym.T)
    lam2, Z = np.linalg.eigh(Ssym)
    return lam2, (Z.T / c).T   # eigenvectors of -c^2 Delta_h (columns)


def test_full_krylov_recovers_top_of_spectrum():
    npts = (17, 15)
    c2 = I.speed_squared("c3", npts, 4)
    g = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(g, 14.0)
    nd = 10
    res = LZ.lanczos(g, tg, g.n, nd, I.random_field(g.shape, 1))
    lam2_all, _ = _dense_pairs(npts, 4, c2)
    beta_all = SP.beta_h(lam2_all, tg)
    top = np.sort(lam2_all[np.argsort(-beta_all)[:nd]])
    assert np.allclose(np.sort(res.lambda2), top, rtol=1e-9)
    assert res.resid.max() < 1e-8
    # Ritz values are the beta_h of the Ritz vectors' eigenvalues
    assert np.allclose(res.theta, SP.beta_h(res.lambda2, tg), atol=1e-10)
    # M-orthonormal
    W = res.V
    assert np.abs(W.T @ (g.weights().ravel()[:, None] * W) - np.eye(nd)).max() < 1e-10


def test_partial_krylov_converges_for_constant_speed():
    npts = (41, 41)
    g = O.Grid(npts)
    tg = WH.time_grid_for(g, 20.0)
    nd = 12
    res = LZ.lanczos(g, tg, 120, nd, I.random_field(g.shape, 2))
    modes, lam2, _ = SP.select_modes(g, tg, nd)
    # the converged Ritz vectors lie in the span of the closed-form modes with the same eigenvalues
    good = res.resid < 1e-6
    assert good.sum() >= nd - 2
    allm = SP.all_modes(g)
    all_l2 = SP.mode_lambda2(g, allm)
    for y, l2 in zip(res.V.T[good], res.lambda2[good]):
        close = np.abs(all_l2 - l2) < 1e-7 * l2
        Z = SP.basis(g, allm[close])
        assert np.linalg.norm(y - Z @ (Z.T @ y)) < 1e-5


def test_thick_restart_recovers_top_of_spectrum_with_a_small_basis():
    """Thick-restart Lanczos with a basis of 3 nd + 4 vectors, restarted, reaches the same top
    eigenpairs as the dense eigen-solve of the independent matrix."""
    npts = (19, 17)
    c2 = I.speed_squared("c3", npts, 4)
    g = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(g, 14.0)
    nd = 8
    res = LZ.lanczos_thick(g, tg, nd, 3 * nd + 4, I.random_field(g.shape, 1), max_restarts=400, tol=1e-11)
    assert res.converged == nd
    assert res.restarts > 0 and res.wave_solves < g.n   # restarted, and cheaper than a full space
    lam2_all, _ = _dense_pairs(npts, 4, c2)
    beta_all = SP.beta_h(lam2_all, tg)
    top = np.sort(lam2_all[np.argsort(-beta_all)[:nd]])
    assert np.allclose(np.sort(res.lambda2), top, rtol=1e-9)
    assert res.resid.max() < 1e-8
    W = res.V
    assert np.abs(W.T @ (g.weights().ravel()[:, None] * W) - np.eye(nd)).max() < 1e-10
