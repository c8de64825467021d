"""The reverse (transposed) sweep on its own (whv_apply_pi_vjp) against the oracle's
adjoint.reverse_sweep for fixed forward data v, f and seed abar -- FP64 to 1e-12, the FP32 sweep
within its rounding bound -- and the whole FP32-stepping adjoint (FP32 solves of u and lambda and
an FP32 sweep, no FP64 correction) against the oracle's adjoint and central differences to 1e-4."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, adjoint as AD
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


CASES = [((33, 29), 2, 10.0, 16), ((41, 37), 4, 12.0, 5), ((13, 11, 12), 2, 6.0, 3), ((15, 13, 14), 4, 7.0, 7)]


def _case(npts, order, omega):
    c2 = I.speed_squared("c5", npts, 2024)
    og = O.Grid(npts, order=order, c2=c2)
    tg = WH.time_grid_for(og, omega)
    v = I.random_field(og.shape, 11)
    f = I.gaussian(npts, [0.45, 0.55, 0.5][: len(npts)], 1 / omega, omega ** 2)
    abar = I.random_field(og.shape, 12)
    ref = AD.reverse_sweep(og, tg, WH.wave_states(og, tg, v, f), abar)
    return c2, v, f, abar, ref


@pytest.mark.parametrize("npts,order,omega,K", CASES)
def test_reverse_sweep_fp64_matches_oracle(npts, order, omega, K):
    """Fixed v, f, abar: vbar = S_h^T abar, c2bar and fbar equal the oracle's reverse sweep to 1e-12."""
    c2, v, f, abar, (vb_ref, c2b_ref, fb_ref) = _case(npts, order, omega)
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    vb, c2b, fb = g.whv_apply_pi_vjp(whv.make_params(omega), dev(v), dev(f), dev(abar), checkpoint_every=K)
    assert IND.relmax(vb.cpu().numpy(), vb_ref) < 1e-12
    assert IND.relmax(c2b.cpu().numpy(), c2b_ref) < 1e-12
    assert IND.relmax(fb.cpu().numpy(), fb_ref) < 1e-12
    g.close()


@pytest.mark.parametrize("npts,order,omega,K", CASES)
def test_reverse_sweep_fp32(npts, order, omega, K):
    """The FP32 sweep (FP32 states and adjoint states, FP64 gradient sums) stays within 1e-4 of the
    FP64 oracle; with WHV_REFINE_FP64 the FP32 grid sweeps in FP64 and meets 1e-12."""
    c2, v, f, abar, (vb_ref, c2b_ref, fb_ref) = _case(npts, order, omega)
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(dev(c2))
    vb, c2b, fb = g.whv_apply_pi_vjp(whv.make_params(omega), dev(v), dev(f), dev(abar), checkpoint_every=K)
    errs = [IND.relmax(x.cpu().numpy(), r) for x, r in ((vb, vb_ref), (c2b, c2b_ref), (fb, fb_ref))]
    assert max(errs) < 1e-4, errs
    vb, c2b, fb = g.whv_apply_pi_vjp(whv.make_params(omega, refine_fp64=True), dev(v), dev(f), dev(abar),
                                     checkpoint_every=K)
    assert IND.relmax(vb.cpu().numpy(), vb_ref) < 1e-12
    assert IND.relmax(c2b.cpu().numpy(), c2b_ref) < 1e-12
    assert IND.relmax(fb.cpu().numpy(), fb_ref) < 1e-12
    g.close()


def _misfit64(npts, c2, f, u_obs, omega):
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    g.whv_set_speed(c2)
    u, info = g.whv_solve(whv.make_params(omega, method="cg", tol=1e-12, maxit=5000), f)
    assert info["status"] == "OK", info
    d = u - u_obs
    g.close()
    return 0.5 * float(torch.dot(d, d))


def test_fp32_stepping_adjoint_without_correction():
    """FP32 grid, no WHV_REFINE_FP64: u and lambda by FP32-stepping CG, gradients by the FP32 sweep.
    dL/dc^2 and dL/df agree with the oracle's FP64 adjoint at the same u, and with central
    differences of L (FP64 solves) in 8 seeded directions, to 1e-4 relative."""
    npts, omega = (129, 121), 12.0
    c2 = I.speed_squared("c5", npts, 2024)
    f = I.gaussian(npts, [0.4, 0.55], 0.1, 100.0)
    c2d, fd = dev(c2), dev(f)
    u_obs = dev(I.random_field(I.interior_shape(npts), 4)) * 1e-3
    g = whv.Grid(npts, precision=whv.WHV_FP32_STEP)
    g.whv_set_speed(c2d)
    prm = whv.make_params(omega, method="cg", tol=1e-7, maxit=5000)
    u, info = g.whv_solve(prm, fd)
    assert info["status"] == "OK", info
    z, gc2, gf, ainfo = g.whv_solve_adjoint(prm, fd, u, u - u_obs, checkpoint_every=16)
    assert ainfo["status"] == "OK", ainfo
    og = O.Grid(npts, c2=c2)
    tg = WH.time_grid_for(og, omega)
    uh = u.cpu().numpy().reshape(og.shape)
    _, gc2_ref, gf_ref, _ = AD.adjoint_gradient(og, tg, uh, f, uh - u_obs.cpu().numpy().reshape(og.shape), tol=1e-12)
    assert IND.relmax(gc2.cpu().numpy(), gc2_ref) < 1e-4
    assert IND.relmax(gf.cpu().numpy(), gf_ref) < 1e-4
    gen = torch.Generator(device="cpu").manual_seed(0)
    for k in range(8):
        d = torch.randn(g.N, generator=gen, dtype=torch.float64).cuda()
        if k % 2 == 0:
            eps = 1e-4 / d.abs().max().item()
            fdv = (_misfit64(npts, c2d + eps * d, fd, u_obs, omega) - _misfit64(npts, c2d - eps * d, fd, u_obs, omega)) / (2 * eps)
            an = float(torch.dot(gc2, d))
        else:
            eps = 1e-4 * fd.abs().max().item() / d.abs().max().item()
            fdv = (_misfit64(npts, c2d, fd + eps * d, u_obs, omega) - _misfit64(npts, c2d, fd - eps * d, u_obs, omega)) / (2 * eps)
            an = float(torch.dot(gf, d))
        assert fdv == pytest.approx(an, rel=1e-4), (k, fdv, an)
    g.close()
