"""Batched solves (one persistent launch per CG iteration for all problems) against the oracle."""
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


def _problems(sizes, omegas, sources, nd, dim=2):
    probs = []
    for n in sizes:
        for om in omegas:
            for s in range(sources):
                npts = tuple([n] * dim)
                c = I.source_centers(n + s, 1, dim)[0]
                f = I.gaussian(npts, c, 2.0 / (n - 1) * 3, om ** 2)
                probs.append((npts, om, f, nd))
    return probs


@pytest.mark.parametrize("dim", [2, 3])
def test_batched_fixed_iterations_match_oracle(dim):
    """Uneven grids and frequencies, DEVD with closed-form bases, FP64: after k iterations every
    problem's iterate equals the oracle's DEVD-CG iterate."""
    sizes = (33, 47, 29) if dim == 2 else (13, 11)
    omegas = (9.0, 14.0) if dim == 2 else (6.0, 8.0)
    probs = _problems(sizes, omegas, 1, 5, dim)
    stream = torch.cuda.Stream()   # batched grids share one stream
    grids, params, fs = [], [], []
    k = 6
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
        prm = whv.make_params(om, method="cg", tol=0.0, maxit=k)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (npts, om, f, nd), u, info in zip(probs, us, infos):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        modes, lam2, _ = SP.select_modes(og, tg, nd)
        ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, k).u
        assert info["iterations"] == k
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-12


def test_batched_fp32_converges_like_single_solves():
    """FP32 stepping, 12 problems (3 sizes x 2 frequencies x 2 sources) to 1e-6; each solution
    matches the FP64 oracle's converged one within the FP32 operator-error bound."""
    probs = _problems((65, 97, 129), (12.0, 18.0), 2, 8)
    stream = torch.cuda.Stream()
    grids, params, fs = [], [], []
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP32_STEP, stream=stream)
        prm = whv.make_params(om, method="cg", tol=1e-6, maxit=2000)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    its = [i["iterations"] for i in infos]
    assert all(i["status"] == "OK" for i in infos), infos
    assert len(set(its)) > 1        # problems stop independently
    for (npts, om, f, nd), u in zip(probs, us):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        U = IND.helmholtz_direct(npts, tg.omega_eff, f)
        assert IND.relmax(u.cpu().numpy(), U) < 1e-4


def test_batched_rejects_mixed_grids():
    s = torch.cuda.Stream()
    g1 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    g2 = whv.Grid((33, 33), precision=whv.WHV_FP64, stream=s)
    prm = whv.make_params(8.0, method="cg", tol=1e-6)
    f = dev(np.ones(g1.N))
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g2], [prm, prm], [f, f])
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g1], [prm, prm], [f, f])


@pytest.mark.parametrize("k", [1, 3, 8, 16])
def test_batched_blocked_sweeps_fp64(k):
    """2-D batched wave solves with k steps per sweep, on problems whose Nt is not a multiple of k
    (and one with Nt < 16): fixed-iteration DEVD-CG iterates equal the oracle's."""
    spec = [(33, 9.0), (47, 14.0), (17, 40.0), (29, 11.0)]
    stream = torch.cuda.Stream()
    grids, params, fs, probs = [], [], [], []
    it = 5
    for n, om in spec:
        npts = (n, n)
        f = I.gaussian(npts, I.source_centers(n, 1, 2)[0], 0.12, om ** 2)
        g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
        prm = whv.make_params(om, method="cg", tol=0.0, maxit=it)
        g.whv_set_deflation_basis(prm, 4, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f)); probs.append((npts, om, f))
    grids[0].whv_set_steps_per_sweep(k)   # the batch takes its sweep length from the first grid
    us, infos = whv.whv_solve_batched(grids, params, fs)
    nts = []
    for (npts, om, f), u, info in zip(probs, us, infos):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        nts.append(tg.nt)
        modes, lam2, _ = SP.select_modes(og, tg, 4)
        ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, it).u
        assert info["iterations"] == it and info["nt"] == tg.nt
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-12
    assert min(nts) < 16 and any(nt % k for nt in nts) or k == 1


def test_batched_variable_speed_order4_fixed_iterations():
    """Variable speed (c^2 Delta_h, M = diag(1/c^2) inner products) with the 9-point-wide
    4th-order stencil, no basis, FP64: batched CG iterates equal the oracle's."""
    spec = [((33, 29), 14.0, 5), ((41, 37), 18.0, 6), ((25, 31), 10.0, 7)]
    stream = torch.cuda.Stream()
    grids, params, fs, refs = [], [], [], []
    it = 6
    for npts, om, seed in spec:
        c2 = I.speed_squared("c3", npts, seed)
        f = I.gaussian(npts, [0.4, 0.55], 0.1, om ** 2)
        g = whv.Grid(npts, order=4, precision=whv.WHV_FP64, stream=stream)
        g.whv_set_speed(dev(c2))
        grids.append(g); params.append(whv.make_params(om, method="cg", tol=0.0, maxit=it)); fs.append(dev(f))
        og = O.Grid(npts, order=4, c2=c2)
        tg = WH.time_grid_for(og, om)
        refs.append(K.devd_solve(og, tg, f, None, None, "cg", 0.0, it).u)
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for u, ref, info in zip(us, refs, infos):
        assert info["iterations"] == it
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_batched_fp32_with_fp64_correction(dim):
    """FP32 stepping inside FP64 residual correction: every problem's FP64 residual of the full
    system meets tol (recomputed here on separate FP64 grids), and the solutions match the
    oracle's converged ones within the residual bound times the conditioning."""
    if dim == 2:
        probs = _problems((65, 97, 129), (12.0, 18.0), 2, 8)
    else:
        probs = _problems((17, 13), (7.0, 9.0), 1, 6, dim=3)
    tol = 1e-10
    stream = torch.cuda.Stream()
    grids, params, fs = [], [], []
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP32_STEP, stream=stream)
        prm = whv.make_params(om, method="cg", tol=tol, maxit=3000, refine_fp64=True)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    assert all(i["status"] == "OK" for i in infos), infos
    assert max(i["outer_iterations"] for i in infos) >= 2
    for (npts, om, f, nd), u, info, prm in zip(probs, us, infos, params):
        assert 0 <= info["true_rel_residual"] <= tol
        # b in the stepping precision, then one FP64 wave solve per residual r = Pi_h(u; f) - u
        assert info["wave_solves_fp64"] == info["outer_iterations"]
        g64 = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
        r = g64.whv_apply_pi(prm, u, dev(f))
        b = g64.whv_apply_pi(prm, torch.zeros_like(u), dev(f))
        assert float((r - u).norm() / b.norm()) <= 1.01 * tol
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        U = IND.helmholtz_direct(npts, tg.omega_eff, f)
        assert IND.relmax(u.cpu().numpy(), U) < 1e-7


def test_batched_refine_flag_must_agree():
    s = torch.cuda.Stream()
    g1 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    g2 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    p1 = whv.make_params(8.0, method="cg", tol=1e-6, refine_fp64=True)
    p2 = whv.make_params(8.0, method="cg", tol=1e-6)
    f = dev(np.ones(g1.N))
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g2], [p1, p2], [f, f])


def test_batched_host_driven_loop_matches_device_loop():
    """check_every > 1 runs the batched CG iteration as a graph launched by the host (convergence
    tested every check_every iterations): same iterates and iteration counts as the device loop."""
    probs = _problems((33, 47), (9.0, 14.0), 1, 5)
    out = {}
    for ce in (1, 3):
        stream = torch.cuda.Stream()
        grids, params, fs = [], [], []
        for npts, om, f, nd in probs:
            g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
            prm = whv.make_params(om, method="cg", tol=1e-9, maxit=500, check_every=ce)
            g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
            grids.append(g); params.append(prm); fs.append(dev(f))
        us, infos = whv.whv_solve_batched(grids, params, fs)
        assert all(i["status"] == "OK" for i in infos)
        out[ce] = ([u.cpu().numpy() for u in us], [i["iterations"] for i in infos])
    assert out[1][1] == out[3][1]
    for a, b in zip(out[1][0], out[3][0]):
        assert IND.relmax(a, b) < 1e-13


def test_batched_autotuner_picks_a_valid_k_and_keeps_results():
    probs = _problems((65, 97), (12.0, 18.0), 1, 6)
    stream = torch.cuda.Stream()
    grids, params, fs = [], [], []
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
        prm = whv.make_params(om, method="cg", tol=0.0, maxit=5)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    k = whv.whv_autotune_batched(grids, params)
    assert k in (2, 4, 6, 8, 10, 12) and grids[0].whv_get_steps_per_sweep() == k
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (npts, om, f, nd), u in zip(probs, us):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        modes, lam2, _ = SP.select_modes(og, tg, nd)
        ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, 5).u
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("k", [3, 8, 16])
def test_batched_fp32_sweeps_match_single_grid_fp32(k):
    """FP32 stepping without correction, fixed iterations: the batched four-cell sweeps (Taylor
    start inside the first sweep, ragged last sweeps, regions inside and across the boundary) give
    the single-grid FP32 iterates up to the rounding of the start step, and the FP64 oracle's
    within the FP32 operator error."""
    spec = [((33, 33), 9.0), ((97, 97), 14.0), ((150, 131), 21.0), ((70, 45), 30.0)]
    stream = torch.cuda.Stream()
    it = 4
    grids, params, fs, singles = [], [], [], []
    for npts, om in spec:
        f = I.gaussian(npts, I.source_centers(npts[0], 1, 2)[0], 0.1, om ** 2)
        prm = whv.make_params(om, method="cg", tol=0.0, maxit=it)
        g = whv.Grid(npts, precision=whv.WHV_FP32_STEP, stream=stream)
        g.whv_set_deflation_basis(prm, 4, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
        s1 = whv.Grid(npts, precision=whv.WHV_FP32_STEP)
        s1.whv_set_steps_per_sweep(1)
        s1.whv_set_deflation_basis(prm, 4, whv.WHV_BASIS_CLOSED_FORM)
        singles.append((s1.whv_solve(prm, dev(f))[0].cpu().numpy(), npts, om, f))
    grids[0].whv_set_steps_per_sweep(k)
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for u, info, (u1, npts, om, f) in zip(us, infos, singles):
        assert info["iterations"] == it
        assert IND.relmax(u.cpu().numpy(), u1) < 2e-5
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        modes, lam2, _ = SP.select_modes(og, tg, 4)
        ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, it).u
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("df", [False, True])
def test_batched_refine_with_double_float_residuals(df):
    """FP32 stepping inside FP64 residual correction with the b and residual wave solves in FP64 or
    in double-float pairs (2-D, c = 1): every problem's true FP64 residual meets 1e-9 and its
    solution is the direct one; problems of uneven size and frequency stop independently."""
    probs = _problems((65, 97, 150), (12.0, 18.0), 1, 8)
    stream = torch.cuda.Stream()
    grids, params, fs = [], [], []
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP32_STEP, stream=stream)
        prm = whv.make_params(om, method="cg", tol=1e-9, maxit=4000, refine_fp64=True, residual_df64=df)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    assert all(i["status"] == "OK" for i in infos), infos
    for (npts, om, f, nd), u, info in zip(probs, us, infos):
        assert info["true_rel_residual"] < 1e-9
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        assert IND.relmax(u.cpu().numpy(), IND.helmholtz_direct(npts, tg.omega_eff, f)) < 1e-6
        # the residual recomputed with an FP64 wave solve of the FP64 grid
        g64 = whv.Grid(npts, precision=whv.WHV_FP64)
        prm64 = whv.make_params(om)
        ff = dev(f)
        r = g64.whv_apply_pi(prm64, u, ff)
        b = g64.whv_apply_pi(prm64, torch.zeros_like(ff), ff)
        assert float((r - u).norm() / b.norm()) < 2e-9


def test_batched_residual_precision_must_agree():
    s = torch.cuda.Stream()
    g1 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    g2 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    p1 = whv.make_params(8.0, method="cg", tol=1e-6, refine_fp64=True, residual_df64=True)
    p2 = whv.make_params(8.0, method="cg", tol=1e-6, refine_fp64=True, residual_df64=False)
    f = dev(np.ones(g1.N))
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g2], [p1, p2], [f, f])
