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


def test_lanczos_deflated_gmres_variable_speed():
    """A variable-speed 4th-order problem shaped like the 1025^2 workload at 161^2: Lanczos basis
    (BASIS_LANCZOS mode), DEVD + GMRES(30) with re-deflation, FP32 stepping inside FP64 residual
    correction, to 1e-6; the solution matches the direct solve and deflation cuts iterations."""
    npts, omega = (161, 161), 30.0
    c2 = I.speed_squared("c3", npts, 1234)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.37, 0.58], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    prm = whv.make_params(omega, method="gmres", restart=30, tol=1e-6, maxit=4000, true_residual=True,
                          refine_fp64=True)
    g0 = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g0.whv_set_speed(dev(c2))
    u0, info0 = g0.whv_solve(prm, dev(f))
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    g.whv_set_deflation_basis(prm, 24, whv.WHV_BASIS_LANCZOS)
    u, info = g.whv_solve(prm, dev(f))
    assert info0["status"] == "OK" and info["status"] == "OK"
    assert info["true_rel_residual"] < 2e-6
    assert IND.relmax(u.cpu().numpy(), U) < 1e-5
    assert info["iterations"] < info0["iterations"]
