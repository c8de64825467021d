"""Device eigen-solve (Lanczos on S_h) vs the oracle's, and the deflated variable-speed solve it
feeds (GMRES with re-deflation, FP32 stepping in FP64 residual correction)."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, lanczos as LZ, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


@pytest.mark.parametrize("npts,order,speed,omega,m,nd", [((33, 29), 4, "c3", 14.0, 60, 8),
                                                         ((41, 37), 2, "c3", 18.0, 80, 12),
                                                         ((13, 11, 9), 2, "c5", 9.0, 50, 6)])
def test_lanczos_matches_oracle(npts, order, speed, omega, m, nd):
    c2 = I.speed_squared(speed, npts, 5)
    og = O.Grid(npts, order=order, c2=c2)
    tg = WH.time_grid_for(og, omega)
    v0 = I.random_field(og.shape, 3)
    ref = LZ.lanczos(og, tg, m, nd, v0)
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega)
    theta, resid = g.whv_lanczos(prm, nd, m, dev(v0))
    got = g.whv_get_basis(want_vectors=True)
    assert np.allclose(theta, ref.theta, atol=1e-9)
    conv = ref.resid < 1e-6
    assert conv.sum() >= nd // 2
    assert np.allclose(np.array(got["lambda2"])[conv], ref.lambda2[conv], rtol=1e-9)
    assert np.allclose(np.array(resid)[conv], ref.resid[conv], atol=1e-7)
    # converged Ritz vectors agree up to sign (M inner product)
    w = og.weights().ravel()
    V = got["V"].cpu().numpy()
    for j in np.flatnonzero(conv):
        ip = float(np.sum(w * V[j] * ref.V[:, j]))
        assert abs(abs(ip) - 1.0) < 1e-6


def test_lanczos_deflated_dcg_variable_speed():
    """A variable-speed 4th-order problem shaped like the 1025^2 workload at 161^2: device Lanczos
    basis (BASIS_LANCZOS mode: approximate eigenvectors), Algorithm 4 with the per-iteration
    A-orthogonalisation (the augmented path for inexact vectors), FP32 stepping inside FP64
    residual correction, to 1e-6: the solution matches the direct solve and deflation cuts CG
    iterations."""
    npts, omega = (161, 161), 30.0
    c2 = I.speed_squared("c3", npts, 1234)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.37, 0.58], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    prm0 = whv.make_params(omega, method="cg", tol=1e-6, maxit=6000, true_residual=True, refine_fp64=True)
    g0 = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g0.whv_set_speed(dev(c2))
    u0, info0 = g0.whv_solve(prm0, dev(f))
    prm = whv.make_params(omega, method="dcg", tol=1e-6, maxit=6000, true_residual=True, refine_fp64=True)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    g.whv_set_deflation_basis(prm, 24, whv.WHV_BASIS_LANCZOS)
    u, info = g.whv_solve(prm, dev(f))
    assert info0["status"] == "OK" and info["status"] == "OK", (info0, info)
    assert info["true_rel_residual"] < 2e-6
    # the residual bound times the condition number of this problem bounds the error
    assert IND.relmax(u.cpu().numpy(), U) < 1e-4
    assert IND.relmax(u.cpu().numpy(), u0.cpu().numpy()) < 1e-4
    assert info["iterations"] < info0["iterations"]


@pytest.mark.parametrize("npts,order,speed", [((201,), 2, None), ((37, 33), 4, "c3")])
def test_dcg_general_basis_fixed_iterations(npts, order, speed):
    """Algorithm 4 with a basis that is not made of eigenvectors (random M-orthonormal vectors):
    the per-iteration projections are on; FP64 iterates agree with the oracle's after k steps."""
    c2 = None if speed is None else I.speed_squared(speed, npts, 6)
    og = O.Grid(npts, order=order, c2=c2)
    omega = 10.5 if len(npts) == 1 else 14.0
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.45, 0.55][: len(npts)], 0.1, omega ** 2)
    nd = 6
    rng = np.random.default_rng(4)
    w = og.weights().ravel()
    W = rng.standard_normal((og.n, nd))
    # M-orthonormalise (Gram-Schmidt in <.,.>_M)
    for j in range(nd):
        for i in range(j):
            W[:, j] -= np.sum(w * W[:, i] * W[:, j]) * W[:, i]
        W[:, j] /= np.sqrt(np.sum(w * W[:, j] ** 2))
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    if c2 is not None:
        g.whv_set_speed(dev(c2))
    k = 7
    prm = whv.make_params(omega, method="dcg", tol=0.0, maxit=k)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_USER, V=dev(W.T), lambda2=np.linspace(1, 2, nd))
    u, info = g.whv_solve(prm, dev(f))
    ref = K.dcg(og, K.Operator(og, tg), WH.rhs_b(og, tg, f), W, 0.0, k)
    assert info["iterations"] == k
    assert IND.relmax(u.cpu().numpy(), ref.x) < 1e-11


def test_thick_restart_lanczos_matches_the_dense_spectrum():
    """Thick-restart Lanczos on the device (basis of 3 nd + 4 vectors, restarted) converges to the
    top eigenpairs the oracle's restarted Lanczos and the dense eigen-solve give."""
    npts, nd = (19, 17), 8
    c2 = I.speed_squared("c3", npts, 4)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, 14.0)
    v0 = I.random_field(og.shape, 1)
    ref = LZ.lanczos_thick(og, tg, nd, 3 * nd + 4, v0, max_restarts=400, tol=1e-11)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(14.0)
    theta, resid, st = g.whv_lanczos_restarted(prm, nd, 3 * nd + 4, max_restarts=400, tol=1e-11, v0=dev(v0))
    assert st["converged"] == nd and st["restarts"] > 0
    assert np.allclose(theta, ref.theta, atol=1e-9)
    got = g.whv_get_basis(want_vectors=True)
    assert np.allclose(np.array(got["lambda2"]), ref.lambda2, rtol=1e-8)
    assert max(resid) < 1e-7


def test_thick_restart_basis_deflates_a_solve():
    """A larger variable-speed grid: 32 vectors from a 100-vector restarted basis deflate DCG
    (Algorithm 4) to the direct solution with fewer iterations than undeflated CG."""
    npts, omega = (129, 121), 24.0
    c2 = I.speed_squared("c3", npts, 7)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.42, 0.57], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="dcg", tol=1e-9, maxit=5000, true_residual=True)
    _, _, st = g.whv_lanczos_restarted(prm, 32, 100, max_restarts=60, tol=1e-8)
    assert st["converged"] >= 24
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK"
    assert IND.relmax(u.cpu().numpy(), U) < 1e-6
    g0 = whv.Grid(npts, order=4, precision=whv.WHV_FP64)
    g0.whv_set_speed(dev(c2))
    _, i0 = g0.whv_solve(whv.make_params(omega, method="cg", tol=1e-9, maxit=5000), dev(f))
    assert info["iterations"] < i0["iterations"]


@pytest.mark.parametrize("method", ["gmres", "cg"])
def test_devd_with_lanczos_basis_in_fp64_correction(method):
    """Algorithm 2 (DEVD) with Lanczos vectors and FP32 stepping inside the FP64 correction: the
    residual's components on the basis are solved by the Galerkin step (W^T M A W)^{-1} W^T M r
    before each inner solve, so the re-deflated inner iteration sees a consistent system; GMRES(m)
    and CG reach the direct solution with far fewer operator applications than the undeflated
    solve."""
    npts, omega = (129, 121), 24.0
    c2 = I.speed_squared("c3", npts, 7)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.42, 0.57], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method=method, tol=1e-8, maxit=5000, restart=30, refine_fp64=True,
                          true_residual=True)
    g.whv_lanczos(prm, 32, 300, None, True)           # FP64-stepped Lanczos, re-deflation on
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK", info
    assert info["true_rel_residual"] <= 1e-8
    assert IND.relmax(u.cpu().numpy(), U) < 1e-6
    g0 = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g0.whv_set_speed(dev(c2))
    _, i0 = g0.whv_solve(whv.make_params(omega, method=method, tol=1e-8, maxit=5000, restart=30, refine_fp64=True),
                         dev(f))
    assert info["iterations"] < i0["iterations"]
