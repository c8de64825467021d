"""SVD-compressed deflation vectors on the device (Sec. 4.3) against the oracle's compression:
ranks, compressed vectors, contractions, and deflated solves with the compressed basis."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K, compression as C
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def test_closed_form_basis_compresses_to_rank_one_and_solves_identically():
    npts, omega, nd = (129, 121), 30.0, 24
    og = O.Grid(npts)
    f = I.gaussian(npts, [0.4, 0.6], 1.0 / omega, omega ** 2)
    prm = whv.make_params(omega, method="cg", tol=1e-10, maxit=3000)
    out = {}
    for compress in (False, True):
        g = whv.Grid(npts, precision=whv.WHV_FP64)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        r = dev(I.random_field(og.shape, 4))
        c0 = torch.zeros(nd, dtype=torch.float64, device="cuda")
        g.whv_project(r, c0)
        if compress:
            ranks = g.whv_compress_basis(1e-9)
            assert ranks == [1] * nd
            c1 = torch.zeros_like(c0)
            g.whv_project(r, c1)
            assert float((c1 - c0).abs().max()) < 1e-12 * float(c0.abs().max())
        u, info = g.whv_solve(prm, dev(f))
        out[compress] = (u.cpu().numpy(), info["iterations"])
    assert out[True][1] == out[False][1]
    assert IND.relmax(out[True][0], out[False][0]) < 1e-11


def test_lanczos_vectors_compress_like_the_oracle():
    """Variable-speed 4th-order grid, device Lanczos vectors: the compression ranks match the
    oracle's exact truncated SVD of the same vectors (within one at the threshold), every
    compressed vector is within tau of the dense one, and the projections agree."""
    npts, omega, nd, tau = (97, 89), 20.0, 12, 1e-4
    c2 = I.speed_squared("c3", npts, 1234)
    og = O.Grid(npts, order=4, c2=c2)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="dcg", tol=1e-9, maxit=3000)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_LANCZOS)
    Vd = g.whv_get_basis(want_vectors=True)["V"].cpu().numpy()          # nd x N
    ref = C.compress_basis(og, Vd.T, tau)
    ranks = g.whv_compress_basis(tau)
    for r_gpu, c in zip(ranks, ref):
        assert abs(r_gpu - c.rank) <= 1
    Vc = g.whv_get_basis(want_vectors=True)["V"].cpu().numpy()
    for m in range(nd):
        assert np.linalg.norm(Vc[m] - Vd[m]) < tau
    r = I.random_field(og.shape, 9)
    coef = torch.zeros(nd, dtype=torch.float64, device="cuda")
    g.whv_project(dev(r), coef)
    expect = Vc @ (og.weights().ravel() * r.ravel())
    assert np.allclose(coef.cpu().numpy(), expect, rtol=1e-10, atol=1e-12)


def test_compressed_exact_rank_two_vectors_keep_the_iterations():
    """Rotated degenerate pairs of sine modes (exact eigenvectors of rank 2) as a user basis:
    compressed they stay exact, and DEVD-CG takes the same iterations as the oracle's dense solve."""
    npts, omega, nd = (45, 45), 20.0, 12
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    modes, lam2, _ = SP.select_modes(og, tg, nd)
    V = SP.basis(og, modes)
    Vr, key = V.copy(), {tuple(m): j for j, m in enumerate(modes.tolist())}
    for j, m in enumerate(modes.tolist()):
        t = key.get((m[1], m[0]))
        if t is not None and t > j:
            a, b = V[:, j].copy(), V[:, t].copy()
            Vr[:, j], Vr[:, t] = (a + b) / np.sqrt(2), (a - b) / np.sqrt(2)
    f = I.gaussian(npts, [0.4, 0.55], 1.0 / omega, omega ** 2)
    ref = K.devd_solve(og, tg, f, Vr, lam2, "cg", 1e-10, 2000)
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    prm = whv.make_params(omega, method="cg", tol=1e-10, maxit=2000)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_USER, V=dev(Vr.T), lambda2=lam2, flags=whv.WHV_BASIS_EXACT)
    ranks = g.whv_compress_basis(1e-8)
    assert max(ranks) == 2
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == ref.solve.iterations
    assert IND.relmax(u.cpu().numpy(), ref.u) < 1e-9


def test_compressed_lanczos_basis_fp32_solve_reaches_direct_solution():
    npts, omega = (161, 161), 30.0
    c2 = I.speed_squared("c3", npts, 1234)
    og = O.Grid(npts, order=4, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.37, 0.58], 1 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    g = whv.Grid(npts, order=4, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="dcg", tol=1e-8, maxit=6000, true_residual=True, refine_fp64=True)
    g.whv_set_deflation_basis(prm, 24, whv.WHV_BASIS_LANCZOS)
    # eigenvectors of a variable-speed operator are not low-rank (at this tolerance they keep
    # nearly all 159 singular vectors); the compressed basis is an approximate one for Algorithm 4
    ranks = g.whv_compress_basis(1e-6)
    assert 1 <= min(ranks) and max(ranks) <= 159
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK", info
    assert info["true_rel_residual"] < 2e-8
    assert IND.relmax(u.cpu().numpy(), U) < 1e-5


def test_compress_refuses_non_2d_and_missing_basis():
    g = whv.Grid((33, 31, 29))
    with pytest.raises(whv.WhvError):
        g.whv_compress_basis(1e-6)
    g2 = whv.Grid((33, 31))
    with pytest.raises(whv.WhvError):
        g2.whv_compress_basis(1e-6)
