"""The device adjoint (whv_solve_adjoint) against the oracle's discrete adjoint, its checkpointing,
and central finite differences of the misfit on the 128^3 variable-speed workload."""
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


@pytest.mark.parametrize("npts,order,omega,K", [((17, 15), 2, 8.0, 16), ((21, 19), 4, 9.0, 5), ((9, 8, 7), 2, 6.0, 3)])
def test_adjoint_matches_oracle(npts, order, omega, K):
    c2 = I.speed_squared("c5", npts, 2024)
    og = O.Grid(npts, order=order, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.45, 0.55, 0.5][: len(npts)], 1 / omega, omega ** 2)
    u_obs = I.random_field(og.shape, 3)
    g = whv.Grid(npts, order=order, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="cg", tol=1e-13, maxit=5000)
    u, info = g.whv_solve(prm, dev(f))
    assert info["status"] == "OK"
    uh = u.cpu().numpy().reshape(og.shape)
    lam_ref, gc2_ref, gf_ref, _ = AD.adjoint_gradient(og, tg, uh, f, uh - u_obs, tol=1e-13)
    z, gc2, gf, ainfo = g.whv_solve_adjoint(prm, dev(f), u, u - dev(u_obs), checkpoint_every=K)
    assert ainfo["status"] == "OK"
    assert IND.relmax(z.cpu().numpy(), lam_ref) < 1e-9
    assert IND.relmax(gc2.cpu().numpy(), gc2_ref) < 1e-9
    assert IND.relmax(gf.cpu().numpy(), gf_ref) < 1e-9


def test_checkpoint_interval_does_not_change_gradients():
    npts, omega = (33, 31), 12.0
    c2 = I.speed_squared("c5", npts, 2024)
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    g.whv_set_speed(dev(c2))
    prm = whv.make_params(omega, method="cg", tol=1e-12, maxit=3000)
    f = dev(I.gaussian(npts, [0.5, 0.4], 1 / omega, omega ** 2))
    u, _ = g.whv_solve(prm, f)
    dL = dev(I.random_field(g.shape, 5))
    res = [g.whv_solve_adjoint(prm, f, u, dL, checkpoint_every=K) for K in (1, 4, 16, 1000)]
    for z, gc2, gf, _ in res[1:]:
        assert torch.allclose(z, res[0][0], rtol=0, atol=1e-13 * res[0][0].abs().max().item())
        assert torch.allclose(gc2, res[0][1], rtol=0, atol=1e-12 * res[0][1].abs().max().item())
        assert torch.allclose(gf, res[0][2], rtol=0, atol=1e-12 * res[0][2].abs().max().item())


def _misfit(npts, c2, f, u_obs, prm, prec):
    g = whv.Grid(npts, precision=prec)
    g.whv_set_speed(c2)
    u, info = g.whv_solve(prm, f)
    assert info["status"] == "OK", info
    d = u - u_obs
    return 0.5 * float(torch.dot(d, d)), u, g, info


@pytest.mark.parametrize("prec", [whv.WHV_FP64, whv.WHV_FP32_STEP])
def test_adjoint_gradient_finite_differences_128cube(prec):
    """The 3-D adjoint grid: 128^3 nodes, c^2 = 1 + 0.3 bumps, u_obs from a perturbed c^2,
    checkpoints every 16 steps; dL/dc^2 and dL/df against central differences of L in 20 seeded
    random directions (FP32 stepping: FP64 residual correction and FP64 reverse sweep, relative 1e-4;
    FP64 stepping: 1e-5, the central-difference truncation at this step).  The frequency is
    6: at 40 this variable-speed cube is within ~1e-4 (relative) of an eigenvalue, so the
    undeflated solve needs far more than thousands of iterations; at 6 the filter interval has
    ~300 steps, so the checkpointing runs through 19 segments."""
    w = I.WORKLOADS["c5adj"]
    npts = w.npts
    omega = 6.0
    c2 = dev(I.speed_squared("c5", npts, 2024))
    c2_obs = c2 + 0.05 * dev(I.bumps(npts, 2025))
    f = dev(I.gaussian(npts, [0.4, 0.55, 0.5], 0.1, 100.0))
    refine = prec == whv.WHV_FP32_STEP
    prm = whv.make_params(omega, method="cg", tol=1e-11, maxit=5000, refine_fp64=refine)
    _, u_obs, _, _ = _misfit(npts, c2_obs, f, torch.zeros_like(f), prm, prec)
    L0, u, g, info = _misfit(npts, c2, f, u_obs, prm, prec)
    nt0 = info["nt"]
    z, gc2, gf, ainfo = g.whv_solve_adjoint(prm, f, u, u - u_obs, checkpoint_every=16)
    assert ainfo["status"] == "OK"
    gen = torch.Generator(device="cpu").manual_seed(0)
    tol = 1e-4 if refine else 1e-5
    for k in range(20):
        d = torch.randn(g.N, generator=gen, dtype=torch.float64).cuda()
        eps = 1e-4 / d.abs().max().item()
        if k % 2 == 0:   # c^2 direction
            Lp, _, _, ip = _misfit(npts, c2 + eps * d, f, u_obs, prm, prec)
            Lm, _, _, im = _misfit(npts, c2 - eps * d, f, u_obs, prm, prec)
            assert ip["nt"] == nt0 and im["nt"] == nt0
            an = float(torch.dot(gc2, d))
        else:            # f direction
            fs = f.abs().max().item()
            Lp, _, _, _ = _misfit(npts, c2, f + eps * fs * d, u_obs, prm, prec)
            Lm, _, _, _ = _misfit(npts, c2, f - eps * fs * d, u_obs, prm, prec)
            eps = eps * fs
            an = float(torch.dot(gf, d))
        fd = (Lp - Lm) / (2 * eps)
        assert fd == pytest.approx(an, rel=tol), (k, fd, an)


def test_autograd_function():
    npts, omega = (41, 37), 10.0
    c2 = dev(I.speed_squared("c5", npts, 7)).requires_grad_(True)
    f = dev(I.gaussian(npts, [0.5, 0.5], 1 / omega, omega ** 2)).requires_grad_(True)
    u_obs = dev(I.random_field(I.interior_shape(npts), 1))
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    prm = whv.make_params(omega, method="cg", tol=1e-12, maxit=3000)
    u = whv.WaveHoltzSolve.apply(f, c2, g, prm)
    L = 0.5 * ((u - u_obs) ** 2).sum()
    L.backward()
    d = dev(I.random_field(I.interior_shape(npts), 2))
    eps = 1e-6
    with torch.no_grad():
        Lp = 0.5 * ((whv.WaveHoltzSolve.apply(f, c2 + eps * d, g, prm) - u_obs) ** 2).sum()
        Lm = 0.5 * ((whv.WaveHoltzSolve.apply(f, c2 - eps * d, g, prm) - u_obs) ** 2).sum()
    assert float((Lp - Lm) / (2 * eps)) == pytest.approx(float(torch.dot(c2.grad, d)), rel=1e-6)
    assert f.grad is not None and torch.isfinite(f.grad).all()
