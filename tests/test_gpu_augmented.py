"""Augmented Krylov methods on the device against the oracle's: Algorithm 5 (AGMRES) and
Algorithm 6 (ABICGSTAB), fixed-iteration iterates (exact eigenvectors, general vectors, variable
speed, 1-D/2-D/3-D, restarts), the unaugmented cases, convergence to the direct solution and the
FP32-stepping form inside FP64 residual correction with a device Lanczos basis."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _m_orthonormal(og, nd, seed):
    rng = np.random.default_rng(seed)
    w = og.weights().ravel()
    W = rng.standard_normal((og.n, nd))
    for j in range(nd):
        for _ in range(2):
            for i in range(j):
                W[:, j] -= np.sum(w * W[:, i] * W[:, j]) * W[:, i]
        W[:, j] /= np.sqrt(np.sum(w * W[:, j] ** 2))
    return W


@pytest.mark.parametrize("npts,omega,nd,k,m", [((41, 37), 14.0, 6, 12, 5), ((201,), 10.5, 8, 9, 30),
                                               ((13, 11, 12), 8.0, 5, 7, 3)])
def test_agmres_exact_basis_fixed_iterations(npts, omega, nd, k, m):
    """Closed-form eigenvectors (A W = W diag(1 - beta_h)), k Arnoldi steps in cycles of m, FP64:
    the iterate equals the oracle's."""
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.42, 0.57, 0.5][: len(npts)], 0.1, omega ** 2)
    modes, lam2, _ = SP.select_modes(og, tg, nd)
    ref = K.augmented_solve(og, tg, f, SP.basis(og, modes), lam2, tol=0.0, maxit=k, restart=m)
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    prm = whv.make_params(omega, method="agmres", tol=0.0, maxit=k, restart=m)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == k == ref.solve.iterations
    assert IND.relmax(u.cpu().numpy(), ref.u) < 1e-11


@pytest.mark.parametrize("npts,order,speed", [((37, 33), 4, "c3"), ((29, 31), 2, "c3")])
def test_agmres_general_basis_fixed_iterations(npts, order, speed):
    """Vectors that are not eigenvectors (A W by wave solves), variable speed, M inner products."""
    c2 = I.speed_squared(speed, npts, 8)
    og = O.Grid(npts, order=order, c2=c2)
    omega = 14.0
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.45, 0.55], 0.1, omega ** 2)
    nd, k, m = 5, 10, 4
    W = _m_orthonormal(og, nd, 11)
    ref = K.augmented_solve(og, tg, f, W, None, tol=0.0, maxit=k, restart=m)
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="agmres", tol=0.0, maxit=k, restart=m)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_USER, V=dev(W.T), lambda2=np.linspace(1, 2, nd))
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == k
    assert IND.relmax(u.cpu().numpy(), ref.u) < 1e-11


def test_agmres_without_basis_is_gmres():
    npts, omega = (33, 29), 12.0
    f = I.gaussian(npts, [0.5, 0.4], 0.1, omega ** 2)
    out = []
    for method in ("gmres", "agmres"):
        g = whv.Grid(npts, precision=whv.WHV_FP64)
        prm = whv.make_params(omega, method=method, tol=0.0, maxit=11, restart=4)
        out.append(g.whv_solve(prm, dev(f))[0].cpu().numpy())
    assert IND.relmax(out[1], out[0]) < 1e-12


def test_agmres_converges_to_direct_solution():
    npts, omega = (65, 57), 24.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.4, 0.6], 0.05, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    its = {}
    for nd in (0, 16):
        g = whv.Grid(npts, precision=whv.WHV_FP64)
        prm = whv.make_params(omega, method="agmres", tol=1e-11, maxit=4000, restart=30, true_residual=True)
        if nd:
            g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        u, info = g.whv_solve(prm, dev(f))
        assert info["status"] == "OK"
        assert info["true_rel_residual"] < 2e-11
        assert IND.relmax(u.cpu().numpy(), U) < 1e-8
        its[nd] = info["iterations"]
    assert its[16] < its[0] / 2


def test_agmres_lanczos_basis_fp32_with_fp64_correction():
    """The variable-speed 4th-order problem with a device Lanczos basis (approximate eigenvectors)
    as augmentation, FP32 stepping inside FP64 residual correction, to 1e-9."""
    npts, omega = (161, 161), 30.0
    c2 = I.speed_squared("c3", npts, 1234)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.37, 0.58], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    # restart 60: with these approximate vectors (Ritz residuals 1e-2 .. 1) GMRES(30) stagnates
    # in the correction solves (thousands of iterations), GMRES(60) does not
    prm = whv.make_params(omega, method="agmres", tol=1e-9, maxit=6000, restart=60, true_residual=True,
                          refine_fp64=True)
    g.whv_set_deflation_basis(prm, 24, whv.WHV_BASIS_LANCZOS)
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK", info
    assert info["true_rel_residual"] < 2e-9
    assert IND.relmax(u.cpu().numpy(), U) < 1e-6


@pytest.mark.parametrize("npts,omega,nd,k", [((41, 37), 14.0, 6, 7), ((13, 11, 12), 8.0, 5, 5), ((201,), 10.5, 0, 6)])
def test_abicgstab_exact_basis_fixed_iterations(npts, omega, nd, k):
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.42, 0.57, 0.5][: len(npts)], 0.1, omega ** 2)
    W = lam2 = None
    if nd:
        modes, lam2, _ = SP.select_modes(og, tg, nd)
        W = SP.basis(og, modes)
    ref = K.augmented_solve(og, tg, f, W, lam2, tol=0.0, maxit=k, method="abicgstab")
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    prm = whv.make_params(omega, method="abicgstab", tol=0.0, maxit=k)
    if nd:
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == k == ref.solve.iterations
    assert IND.relmax(u.cpu().numpy(), ref.u) < 1e-11


def test_abicgstab_general_basis_variable_speed_fixed_iterations():
    npts, order = (37, 33), 4
    c2 = I.speed_squared("c3", npts, 8)
    og = O.Grid(npts, order=order, c2=c2)
    omega = 14.0
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.45, 0.55], 0.1, omega ** 2)
    nd, k = 5, 6
    W = _m_orthonormal(og, nd, 12)
    ref = K.augmented_solve(og, tg, f, W, None, tol=0.0, maxit=k, method="abicgstab")
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="abicgstab", tol=0.0, maxit=k)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_USER, V=dev(W.T), lambda2=np.linspace(1, 2, nd))
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == k
    assert IND.relmax(u.cpu().numpy(), ref.u) < 1e-11


def test_abicgstab_fp32_with_fp64_correction_reaches_direct_solution():
    npts, omega = (97, 89), 20.0
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.4, 0.6], 0.05, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f)
    g = whv.Grid(npts, precision=whv.WHV_FP32_STEP)
    prm = whv.make_params(omega, method="abicgstab", tol=1e-10, maxit=4000, true_residual=True, refine_fp64=True)
    g.whv_set_deflation_basis(prm, 12, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK", info
    assert info["true_rel_residual"] < 2e-10
    assert IND.relmax(u.cpu().numpy(), U) < 1e-7
