"""The conservative operator div_h(c^2 grad_h) on the device against the oracle's: wave solves,
fixed-iteration CG (Euclidean inner products), a converged FP32-stepping solve against the
independent direct solve, the device Lanczos on it, and the refusals."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, krylov as K, lanczos as LZ
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _speed(npts, seed):
    if len(npts) == 2:
        return I.speed_squared("c3", npts, seed)
    rng = np.random.default_rng(seed)
    return 1.0 + rng.random(tuple(p - 2 for p in reversed(npts)))


def _grid(npts, c2, precision=None):
    g = whv.Grid(npts, precision=whv.WHV_FP64 if precision is None else precision)
    g.whv_set_speed_form(dev(c2), whv.WHV_SPEED_CONSERVATIVE)
    return g


@pytest.mark.parametrize("npts,omega", [((151,), 9.0), ((47, 39), 14.0), ((17, 15, 13), 7.0)])
@pytest.mark.parametrize("forcing", [False, True])
def test_conservative_pi_fp64(npts, omega, forcing):
    c2 = _speed(npts, 3)
    og = O.Grid(npts, c2=c2, form="conservative")
    tg = WH.time_grid_for(og, omega)
    v = I.random_field(og.shape, 5)
    f = I.gaussian(npts, [0.4, 0.55, 0.5][: len(npts)], 0.1, omega ** 2) if forcing else None
    g = _grid(npts, c2)
    out = g.whv_apply_pi(whv.make_params(omega), dev(v), None if f is None else dev(f))
    ref = WH.apply_pi(og, tg, v, f)
    assert IND.relmax(out.cpu().numpy(), ref) < 1e-12


def test_conservative_pi_fp32_within_bound():
    npts, omega = (65, 57), 16.0
    c2 = _speed(npts, 4)
    og = O.Grid(npts, c2=c2, form="conservative")
    v = I.random_field(og.shape, 6)
    g = _grid(npts, c2, whv.WHV_FP32_STEP)
    out = g.whv_apply_pi(whv.make_params(omega), dev(v)).cpu().numpy()
    ref = WH.apply_pi(og, WH.time_grid_for(og, omega), v)
    assert np.abs(out - ref.ravel()).max() <= 2e-5 * max(np.abs(v).max(), np.abs(ref).max())


@pytest.mark.parametrize("npts", [(47, 39), (13, 12, 11)])
def test_conservative_cg_fixed_iterations(npts):
    c2 = _speed(npts, 7)
    og = O.Grid(npts, c2=c2, form="conservative")
    omega = 12.0 if len(npts) == 2 else 6.0
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.45, 0.5, 0.5][: len(npts)], 0.1, omega ** 2)
    k = 7
    g = _grid(npts, c2)
    u, info = g.whv_solve(whv.make_params(omega, method="cg", tol=0.0, maxit=k), dev(f))
    ref = K.devd_solve(og, tg, f, None, None, "cg", 0.0, k).u
    assert info["iterations"] == k
    assert IND.relmax(u.cpu().numpy(), ref) < 1e-12


def test_conservative_fp32_solve_reaches_direct_solution():
    npts, omega = (97, 89), 18.0
    c2 = _speed(npts, 8)
    og = O.Grid(npts, c2=c2, form="conservative")
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.4, 0.6], 1.0 / omega, omega ** 2)
    U = IND.helmholtz_direct_conservative(npts, tg.omega_eff, f, c2)
    g = _grid(npts, c2, whv.WHV_FP32_STEP)
    u, info = g.whv_solve(whv.make_params(omega, method="cg", tol=1e-10, maxit=6000, true_residual=True,
                                          refine_fp64=True), dev(f))
    assert info["status"] == "OK"
    assert info["true_rel_residual"] < 2e-10
    assert IND.relmax(u.cpu().numpy(), U) < 1e-7


def test_conservative_lanczos_matches_oracle():
    npts, omega, m, nd = (33, 29), 14.0, 60, 8
    c2 = _speed(npts, 5)
    og = O.Grid(npts, c2=c2, form="conservative")
    tg = WH.time_grid_for(og, omega)
    v0 = I.random_field(og.shape, 3)
    ref = LZ.lanczos(og, tg, m, nd, v0)
    g = _grid(npts, c2)
    theta, resid = g.whv_lanczos(whv.make_params(omega), nd, m, dev(v0))
    assert np.allclose(theta, ref.theta, atol=1e-9)
    conv = ref.resid < 1e-6
    got = g.whv_get_basis()
    assert np.allclose(np.array(got["lambda2"])[conv], ref.lambda2[conv], rtol=1e-9)


def test_conservative_refusals():
    npts = (33, 29)
    c2 = _speed(npts, 5)
    g4 = whv.Grid(npts, order=4)
    with pytest.raises(whv.WhvError):
        g4.whv_set_speed_form(dev(c2), whv.WHV_SPEED_CONSERVATIVE)
    g = _grid(npts, c2)
    prm = whv.make_params(10.0, method="cg", tol=1e-6)
    f = dev(np.ones(g.N))
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g], [prm], [f])
    u = torch.zeros_like(f)
    with pytest.raises(whv.WhvError):
        g.whv_solve_adjoint(prm, f, u, u)
