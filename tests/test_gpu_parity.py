"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 stepping 1e-12 relative max-norm (the target of the FP64 path); FP32 stepping
is compared with a bound derived from FP32 rounding: each of the Nt <= 400 steps rounds the state
at u = 6e-8 relative and the leapfrog carries the errors forward without damping, so the
wave-solve output is off by at most ~Nt u |W| ~ 2e-5 max|W| (measured ~5e-6 in a float32
emulation); the solution of a deflated solve adds the condition number kappa_D (<= ~40 here)
times the operator error ~2e-7, which the 1e-5 solution bound covers.
"""
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


def host(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    return IND.relmax(a, b)


def make(npts, order=2, speed=None, precision=whv.WHV_FP64, seed=7):
    c2 = None if speed is None else I.speed_squared(speed, npts, seed)
    g = whv.Grid(npts, order=order, precision=precision)
    if c2 is not None:
        g.whv_set_speed(dev(c2))
    return g, O.Grid(npts, order=order, c2=c2), c2


PI_CASES = [
    ((201,), 2, None, 10.5),          # 1-D workload size
    ((70,), 4, None, 9.0),
    ((70, 45), 2, None, 14.0),        # ragged against 32 x 8 blocks
    ((37, 61), 4, "c3", 11.0),        # variable speed, 4th order
    ((37, 20, 11), 2, None, 8.0),     # 3-D, ragged
    ((19, 23, 17), 2, "c5", 7.0),     # 3-D variable speed
    ((14, 13, 12), 4, None, 5.0),
    ((12, 10, 40), 2, None, 6.0),     # 3-D, several z chunks with a ragged last one
    ((17, 13, 45), 2, "c5", 9.0),
    ((3,), 2, None, 1.0),             # a single interior node
    ((3, 3), 2, None, 1.0),
    ((4, 5), 4, None, 2.0),
]


@pytest.mark.parametrize("npts,order,speed,omega", PI_CASES)
@pytest.mark.parametrize("forcing", [False, True])
@pytest.mark.parametrize("adjust", [False, True])
@pytest.mark.parametrize("per_step", [False, True])
def test_apply_pi_fp64(npts, order, speed, omega, forcing, adjust, per_step):
    """per_step: one kernel per time step (otherwise grids of <= 4096 unknowns run the whole
    wave solve in one CTA)."""
    g, og, _ = make(npts, order, speed)
    if per_step:
        g.whv_set_steps_per_sweep(1)
    prm = whv.make_params(omega, adjust_omega=adjust)
    tg = WH.time_grid_for(og, omega, adjust=adjust)
    assert g.whv_time_grid(prm)["nt"] == tg.nt
    v = I.random_field(og.shape, 1)
    f = I.random_field(og.shape, 2) if forcing else None
    out = g.whv_apply_pi(prm, dev(v), None if f is None else dev(f))
    ref = WH.apply_pi(og, tg, v, f)
    assert relmax(host(out), ref) < 1e-12


@pytest.mark.parametrize("npts,order,speed,omega", PI_CASES[:9])
@pytest.mark.parametrize("per_step", [False, True])
def test_apply_pi_fp32(npts, order, speed, omega, per_step):
    g, og, _ = make(npts, order, speed, precision=whv.WHV_FP32_STEP)
    if per_step:
        g.whv_set_steps_per_sweep(1)
    prm = whv.make_params(omega)
    tg = WH.time_grid_for(og, omega)
    v = I.random_field(og.shape, 3)
    f = I.random_field(og.shape, 4)
    out = host(g.whv_apply_pi(prm, dev(v), dev(f)))
    ref = WH.apply_pi(og, tg, v, f)
    scale = max(np.abs(v).max(), np.abs(ref).max())
    assert np.abs(out - ref.ravel()).max() <= 2e-5 * scale


def test_apply_pi_in_place():
    g, og, _ = make((40, 33))
    prm = whv.make_params(9.0)
    v = I.random_field(og.shape, 5)
    t = dev(v)
    g.whv_apply_pi(prm, t, None, t)
    assert relmax(host(t), WH.apply_pi(og, WH.time_grid_for(og, 9.0), v)) < 1e-12


@pytest.mark.parametrize("npts,omega,nd", [((201,), 10.5, 8), ((37, 29), 20.0, 24), ((13, 12, 11), 9.0, 17),
                                           ((129, 129), 25.0, 40)])
def test_closed_form_basis_matches_oracle(npts, omega, nd):
    g, og, _ = make(npts)
    prm = whv.make_params(omega)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    got = g.whv_get_basis(want_vectors=True)
    tg = WH.time_grid_for(og, omega)
    modes, lam2, _ = SP.select_modes(og, tg, nd)
    assert [list(map(int, m)) for m in modes] == got["modes"]          # integer decision: exact
    assert np.allclose(got["lambda2"], lam2, rtol=1e-13, atol=0)
    W = SP.basis(og, modes)
    assert np.abs(host(got["V"]).T - W).max() < 1e-13


@pytest.mark.parametrize("npts,speed,nd", [((201,), None, 8), ((70, 45), "c3", 33), ((21, 19, 17), "c5", 64)])
def test_project_expand_dot(npts, speed, nd):
    g, og, c2 = make(npts, speed=speed)
    rng = np.random.default_rng(9)
    Wm = np.linalg.qr(rng.standard_normal((og.n, nd)))[0]
    lam2 = np.linspace(1.0, 50.0, nd)
    prm = whv.make_params(3.0)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_USER, V=dev(Wm.T), lambda2=lam2)
    r = I.random_field(og.shape, 10)
    coef = torch.zeros(nd, dtype=torch.float64, device="cuda")
    g.whv_project(dev(r), coef)
    assert relmax(host(coef), K.project_coeffs(og, Wm, r)) < 1e-12
    y = rng.standard_normal(nd)
    out = dev(r)
    g.whv_expand(dev(y), -0.75, out)
    assert relmax(host(out), r.ravel() - 0.75 * Wm @ y) < 1e-12
    x2 = I.random_field(og.shape, 11)
    assert g.whv_dot(dev(r), dev(x2)) == pytest.approx(og.inner(r, x2), rel=1e-12)


# --------------------------------------------------------------------------- solves
def oracle_fixed(og, tg, f, method, k, V=None, lam2=None, mu=None, restart=30):
    if method == "dcg":
        A = K.Operator(og, tg)
        b = WH.rhs_b(og, tg, f)
        return K.dcg(og, A, b, V, 0.0, k, mu=mu).x
    return K.devd_solve(og, tg, f, V, lam2, method, 0.0, k, restart=restart).u


@pytest.mark.parametrize("method,k,restart", [("cg", 6, 30), ("dcg", 6, 30), ("gmres", 7, 30), ("gmres", 11, 4),
                                              ("fpi", 5, 30)])
@pytest.mark.parametrize("deflate", [False, True])
def test_solve_fixed_iterations_1d(method, k, restart, deflate):
    """Same seeded input, same iteration count: the FP64 iterates agree to 1e-12."""
    if method == "dcg" and not deflate:
        pytest.skip("DCG needs a basis")
    w = I.WORKLOADS["c1"]
    g, og, _ = make(w.npts)
    tg = WH.time_grid_for(og, w.omega)
    f = I.forcing_for(w)
    prm = whv.make_params(w.omega, method=method, tol=0.0, maxit=k, restart=restart)
    V = lam2 = mu = None
    if deflate:
        g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
        modes, lam2, bh = SP.select_modes(og, tg, w.nd)
        V, mu = SP.basis(og, modes), 1.0 - bh
    u, info = g.whv_solve(prm, dev(f))
    assert info["iterations"] == k
    ref = oracle_fixed(og, tg, f, method, k, V, lam2, mu, restart)
    assert relmax(host(u), ref) < 1e-12


def test_c1_converged_matches_direct_solve():
    w = I.WORKLOADS["c1"]
    g, og, _ = make(w.npts)
    prm = whv.make_params(w.omega, method="cg", tol=w.tol, maxit=500, true_residual=True)
    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
    f = I.forcing_for(w)
    u, info = g.whv_solve(prm, dev(f))
    tg = WH.time_grid_for(og, w.omega)
    U = IND.helmholtz_direct(w.npts, tg.omega_eff, f)
    assert info["status"] == "OK" and info["true_rel_residual"] < 10 * w.tol
    assert relmax(host(u), U) < 1e-8


@pytest.mark.parametrize("npts,order,speed,method", [((129, 129), 2, None, "cg"), ((65, 57), 4, "c3", "cg"),
                                                     ((65, 57), 4, "c3", "gmres"), ((21, 19, 17), 2, None, "cg")])
def test_solve_fixed_iterations_2d_3d(npts, order, speed, method):
    g, og, _ = make(npts, order, speed)
    omega = 20.0 if len(npts) == 2 else 9.0
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.41, 0.57, 0.5][: len(npts)], 1 / omega, omega ** 2)
    prm = whv.make_params(omega, method=method, tol=0.0, maxit=9, restart=5)
    u, info = g.whv_solve(prm, dev(f))
    ref = K.devd_solve(og, tg, f, None, None, method, 0.0, 9, restart=5).u
    assert relmax(host(u), ref) < 1e-12


def test_c2_full_size_fixed_iterations_fp64():
    """The 513^2 workload in the benchmark's configuration (64 closed-form vectors, DEVD-CG)."""
    w = I.WORKLOADS["c2"]
    g, og, _ = make(w.npts)
    tg = WH.time_grid_for(og, w.omega)
    f = I.forcing_for(w)
    k = 6
    prm = whv.make_params(w.omega, method="cg", tol=0.0, maxit=k)
    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
    modes, lam2, _ = SP.select_modes(og, tg, w.nd)
    assert [list(map(int, m)) for m in modes] == g.whv_get_basis()["modes"]
    u, _ = g.whv_solve(prm, dev(f))
    ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, k).u
    assert relmax(host(u), ref) < 1e-12


@pytest.mark.parametrize("n", [129, 513])
@pytest.mark.parametrize("method", ["cg", "dcg"])
def test_c2_fp32_stepping_with_fp64_correction(n, method):
    """FP32 stepping + FP64 Krylov inside FP64 residual correction: the FP64 true residual meets
    1e-6 and the solution is within 1e-5 of the FP64 oracle's converged solution."""
    w = I.scaled(I.WORKLOADS["c2"], n) if n != 513 else I.WORKLOADS["c2"]
    g, og, _ = make(w.npts, precision=whv.WHV_FP32_STEP)
    tg = WH.time_grid_for(og, w.omega)
    f = I.forcing_for(w)
    nd = w.nd if n == 513 else 16
    prm = whv.make_params(w.omega, method=method, tol=1e-6, maxit=2000, true_residual=True, refine_fp64=True)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    modes, lam2, _ = SP.select_modes(og, tg, nd)
    ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 1e-11, 3000).u
    assert info["status"] == "OK" and info["outer_iterations"] >= 1
    assert info["true_rel_residual"] < 2e-6
    assert relmax(host(u), ref) < 1e-5


def test_c2_fp32_stepping_without_correction():
    """Plain FP32-stepping CG stops on its recursive residual; its solution error against the
    FP64 oracle is reported by the benchmark and bounded here at the operator-error level."""
    w = I.WORKLOADS["c2"]
    g, og, _ = make(w.npts, precision=whv.WHV_FP32_STEP)
    tg = WH.time_grid_for(og, w.omega)
    f = I.forcing_for(w)
    prm = whv.make_params(w.omega, method="cg", tol=1e-6, maxit=2000)
    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    modes, lam2, _ = SP.select_modes(og, tg, w.nd)
    ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 1e-11, 3000).u
    assert info["status"] == "OK"
    assert relmax(host(u), ref) < 1e-4


def test_fp32_correction_variable_speed_deep_residual():
    """FP32 stepping reaches an FP64 residual of 1e-9 on a kappa ~ 1e3 variable-speed 4th-order
    problem through the FP64 residual correction (CG inner solves)."""
    npts = (129, 121)
    g, og, c2 = make(npts, order=4, speed="c3", precision=whv.WHV_FP32_STEP)
    tg = WH.time_grid_for(og, 25.0)
    f = I.gaussian(npts, [0.45, 0.55], 1 / 25.0, 625.0)
    prm = whv.make_params(25.0, method="cg", tol=1e-9, maxit=6000, true_residual=True, refine_fp64=True)
    u, info = g.whv_solve(prm, dev(f))
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, 4, c2)
    assert info["status"] == "OK" and info["true_rel_residual"] < 2e-9, info
    assert info["outer_iterations"] >= 2
    assert relmax(host(u), U) < 1e-6


def test_fp32_correction_devd_gmres():
    """DEVD + GMRES(30) on the FP32-stepping grid inside the FP64 residual correction."""
    w = I.scaled(I.WORKLOADS["c2"], 257)
    g, og, _ = make(w.npts, precision=whv.WHV_FP32_STEP)
    tg = WH.time_grid_for(og, w.omega)
    f = I.forcing_for(w)
    prm = whv.make_params(w.omega, method="gmres", restart=30, tol=1e-8, maxit=4000, true_residual=True,
                          refine_fp64=True)
    g.whv_set_deflation_basis(prm, 32, whv.WHV_BASIS_CLOSED_FORM)
    u, info = g.whv_solve(prm, dev(f))
    U = IND.helmholtz_direct(w.npts, tg.omega_eff, f)
    assert info["status"] == "OK" and info["true_rel_residual"] < 2e-8, info
    assert relmax(host(u), U) < 1e-6


# --------------------------------------------------------------------------- errors
def test_invalid_inputs_are_refused():
    g, og, _ = make((33, 33))
    with pytest.raises(whv.WhvError) as e:
        g.whv_time_grid(whv.make_params(5.0, cfl=0.9))            # above the stability limit
    assert e.value.status == whv.WHV_ERR_INVALID
    with pytest.raises(whv.WhvError):
        g.whv_set_deflation_basis(whv.make_params(5.0), 5000, whv.WHV_BASIS_CLOSED_FORM)  # nd > N
    with pytest.raises(whv.WhvError):
        g.whv_solve(whv.make_params(5.0, method="dcg"), dev(np.ones(og.shape)))         # no basis
    g.whv_set_deflation_basis(whv.make_params(5.0), 4, whv.WHV_BASIS_CLOSED_FORM)
    with pytest.raises(whv.WhvError):
        g.whv_solve(whv.make_params(6.0), dev(np.ones(og.shape)))                        # other omega
    gv, _, _ = make((33, 33), speed="c3")
    with pytest.raises(whv.WhvError):
        gv.whv_set_deflation_basis(whv.make_params(5.0), 4, whv.WHV_BASIS_CLOSED_FORM)   # c != 1
    with pytest.raises(whv.WhvError):
        gv.whv_set_speed(dev(-np.ones(og.shape)))                                          # c^2 <= 0


def test_nan_forcing_reports_breakdown():
    g, og, _ = make((33, 33))
    f = np.ones(og.shape)
    f[3, 4] = np.nan
    with pytest.raises(whv.WhvError) as e:
        g.whv_solve(whv.make_params(5.0), dev(f))
    assert e.value.status == whv.WHV_ERR_BREAKDOWN


def test_not_converged_returns_iterate():
    g, og, _ = make((65, 65))
    f = I.gaussian((65, 65), [0.5, 0.5], 0.05, 400.0)
    u, info = g.whv_solve(whv.make_params(20.0, tol=1e-14, maxit=3), dev(f))
    assert info["status"] == "NOT_CONVERGED" and info["iterations"] == 3
    assert torch.isfinite(u).all()


def test_user_stream_ordering():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = whv.Grid((50, 40), stream=s)
        og = O.Grid((50, 40))
        v = I.random_field(og.shape, 12)
        t = dev(v)
        out = g.whv_apply_pi(whv.make_params(8.0), t)
    s.synchronize()
    assert relmax(host(out), WH.apply_pi(og, WH.time_grid_for(og, 8.0), v)) < 1e-12


# --------------------------------------------------------------------------- blocked sweeps
BLK_CASES = [((70, 45), 2, None, 14.0), ((37, 61), 4, "c3", 11.0), ((101, 99), 2, "c3", 20.0),
             ((6, 40), 4, None, 5.0), ((3, 3), 2, None, 1.0), ((130, 67), 4, None, 17.0)]


@pytest.mark.parametrize("npts,order,speed,omega", BLK_CASES)
@pytest.mark.parametrize("k", [1, 2, 5, 8, 16])
def test_blocked_sweeps_fp64(npts, order, speed, omega, k):
    """The temporally blocked 2-D kernel (k steps per launch) gives the single-step result, forced
    and unforced, with the operator epilogue."""
    g, og, _ = make(npts, order, speed)
    g.whv_set_steps_per_sweep(k)
    assert g.whv_get_steps_per_sweep() == k
    prm = whv.make_params(omega)
    tg = WH.time_grid_for(og, omega)
    v = I.random_field(og.shape, 21)
    out = g.whv_apply_pi(prm, dev(v))
    assert relmax(host(out), WH.apply_pi(og, tg, v)) < 1e-12
    # operator epilogue inside a solve (A p and p^T A p on the last sweep)
    f = I.gaussian(npts, [0.45, 0.5], 0.1, omega ** 2)
    prm2 = whv.make_params(omega, method="cg", tol=0.0, maxit=4)
    u, _ = g.whv_solve(prm2, dev(f))
    ref = K.devd_solve(og, tg, f, None, None, "cg", 0.0, 4).u
    assert relmax(host(u), ref) < 1e-12


@pytest.mark.parametrize("npts,order,speed,omega", BLK_CASES[:4])
@pytest.mark.parametrize("k", [3, 8, 16])
def test_blocked_sweeps_fp32(npts, order, speed, omega, k):
    g, og, _ = make(npts, order, speed, precision=whv.WHV_FP32_STEP)
    g.whv_set_steps_per_sweep(k)
    prm = whv.make_params(omega)
    v = I.random_field(og.shape, 22)
    out = host(g.whv_apply_pi(prm, dev(v)))
    ref = WH.apply_pi(og, WH.time_grid_for(og, omega), v)
    assert np.abs(out - ref.ravel()).max() <= 2e-5 * max(np.abs(v).max(), np.abs(ref).max())


@pytest.mark.parametrize("npts,omega,order,speed", [
    ((200, 150), 21.0, 2, None), ((70, 45), 14.0, 2, None), ((130, 67), 17.0, 2, None), ((66, 66), 9.0, 2, None),
    ((200, 150), 21.0, 4, "c3"), ((101, 99), 20.0, 4, "c3"), ((130, 67), 17.0, 4, None), ((180, 140), 19.0, 2, "c3")])
def test_blocked_fp32_four_cell_sweeps_equal_single_steps_bitwise(npts, omega, order, speed):
    """FP32: the four-cells-per-thread sweeps (5-point with c = 1; c^2 Delta_h and the 4th-order
    stencil with its odd-reflection closure; regions inside the domain and crossing its boundary,
    odd and even k, a ragged last sweep) perform the single-step kernel's operations in its order,
    so Pi_h v is bitwise the k = 1 result."""
    g, og, _ = make(npts, order, speed, precision=whv.WHV_FP32_STEP)
    prm = whv.make_params(omega)
    v = dev(I.random_field(og.shape, 24))
    g.whv_set_steps_per_sweep(1)
    ref = host(g.whv_apply_pi(prm, v))
    for k in ((2, 3, 5, 8, 11, 16) if order == 2 else (2, 3, 5, 8, 11, 12)):
        g.whv_set_steps_per_sweep(k)
        out = host(g.whv_apply_pi(prm, v))
        assert np.array_equal(out, ref), (k, np.abs(out - ref).max())


@pytest.mark.parametrize("npts,omega", [((37, 20, 11), 8.0), ((12, 10, 40), 6.0), ((70, 33, 45), 9.0),
                                         ((70, 33, 45), 9.7), ((5, 6, 4), 3.0), ((40, 75, 21), 7.0),
                                         ((131, 70, 30), 9.0)])
def test_two_step_3d_equals_single_steps_bitwise(npts, omega):
    """3-D FP32, c = 1: two leapfrog steps per launch (64 x 32 tiles with a one-node ring, several
    tiles in x and y, odd and even row lengths, CTA ranges of (tile, plane) pairs that start and
    end inside a tile's planes, an odd number of steps handled by one single step first) perform
    the single-step kernel's operations in its order: Pi_h v is bitwise the k = 1 result, and the
    operator epilogue inside fixed-iteration CG agrees to rounding of the reductions."""
    g, og, _ = make(npts, 2, None, precision=whv.WHV_FP32_STEP)
    prm = whv.make_params(omega)
    tg = WH.time_grid_for(og, omega)
    v = dev(I.random_field(og.shape, 25))
    g.whv_set_steps_per_sweep(1)
    ref = host(g.whv_apply_pi(prm, v))
    f = dev(I.gaussian(npts, [0.4, 0.5, 0.55], 0.15, omega ** 2))
    prm2 = whv.make_params(omega, method="cg", tol=0.0, maxit=4)
    u1 = host(g.whv_solve(prm2, f)[0])
    g.whv_set_steps_per_sweep(2)
    out = host(g.whv_apply_pi(prm, v))
    assert np.array_equal(out, ref), (tg.nt, np.abs(out - ref).max())
    u2 = host(g.whv_solve(prm2, f)[0])
    assert relmax(u2, u1) < 1e-9


def test_autotune_picks_valid_k_and_keeps_results():
    g, og, _ = make((257, 257), precision=whv.WHV_FP32_STEP)
    prm = whv.make_params(30.0, method="cg", tol=1e-6, maxit=500)
    k = g.whv_autotune(prm)
    assert k in (1, 2, 4, 6, 8, 10, 12, 16) and g.whv_get_steps_per_sweep() == k
    v = I.random_field(og.shape, 23)
    out = host(g.whv_apply_pi(prm, dev(v)))
    ref = WH.apply_pi(og, WH.time_grid_for(og, 30.0), v)
    assert np.abs(out - ref.ravel()).max() <= 2e-5 * max(np.abs(v).max(), np.abs(ref).max())


def test_batched_barrier_failure_is_reported_and_recovers():
    """The failure path of the grid barriers without a GPU fault: the host raises the barrier error
    flag of a batched solve (whv_inject_barrier_error on one of its grids), every CTA of the first
    batched wave solve leaves at its first grid barrier, the call reports WHV_ERR_TIMEOUT; the next
    batched solve on the same grids is exact again (FP64 and FP32 stepping)."""
    npts, omega = (70, 45), 14.0
    og = O.Grid(npts)
    f = I.gaussian(npts, [0.45, 0.5], 0.1, omega ** 2)
    ref = K.devd_solve(og, WH.time_grid_for(og, omega), f, None, None, "cg", 0.0, 4).u
    for prec, tol in ((whv.WHV_FP64, 1e-12), (whv.WHV_FP32_STEP, 1e-4)):
        stream = torch.cuda.Stream()
        grids = [whv.Grid(npts, precision=prec, stream=stream) for _ in range(2)]
        prm = whv.make_params(omega, method="cg", tol=0.0, maxit=4)
        grids[1].whv_inject_barrier_error()
        with pytest.raises(whv.WhvError) as ei:
            whv.whv_solve_batched(grids, [prm, prm], [dev(f), dev(f)])
        assert "barrier" in str(ei.value)
        us, _ = whv.whv_solve_batched(grids, [prm, prm], [dev(f), dev(f)])
        for u in us:
            assert relmax(host(u), ref) < tol
        grids[0].whv_inject_barrier_error()
        with pytest.raises(whv.WhvError):
            whv.whv_apply_pi_batched(grids, [prm, prm], [dev(f), dev(f)], None)


@pytest.mark.parametrize("npts,speed,omega,order", [
    ((129, 121), None, 24.0, 2), ((97, 89), "c3", 18.0, 2), ((21, 19, 17), None, 8.0, 2),
    ((129, 121), None, 24.0, 4), ((97, 89), "c3", 18.0, 4), ((17, 15, 14), None, 7.0, 4),
    ((41, 37), None, 12.0, 2)])
def test_residual_correction_in_double_float(npts, speed, omega, order):
    """FP32 stepping with the residual wave solves in double-float arithmetic (pairs of FP32),
    second- and fourth-order stencils (the latter with its odd-reflection closure): the
    FP64-checked true residual meets tol = 1e-9 and the solution is the direct one; the result
    agrees with the FP64-residual form."""
    c2 = None if speed is None else I.speed_squared(speed, npts, 3)
    og = O.Grid(npts, order=order, c2=c2)
    tg = WH.time_grid_for(og, omega)
    f = I.gaussian(npts, [0.4, 0.6, 0.5][: len(npts)], 1.0 / omega, omega ** 2)
    U = IND.helmholtz_direct(npts, tg.omega_eff, f, order, c2)
    out = {}
    for df in (True, False):
        g = whv.Grid(npts, order=order, precision=whv.WHV_FP32_STEP)
        if c2 is not None:
            g.whv_set_speed(dev(c2))
        prm = whv.make_params(omega, method="cg", tol=1e-9, maxit=6000, true_residual=True, refine_fp64=True,
                              residual_df64=df)
        if c2 is None:
            g.whv_set_deflation_basis(prm, 12, whv.WHV_BASIS_CLOSED_FORM)
        u, info = g.whv_solve(prm, dev(f))
        assert info["status"] == "OK", info
        assert info["true_rel_residual"] < 2e-9
        assert relmax(host(u), U) < 1e-6
        out[df] = host(u)
    assert relmax(out[True], out[False]) < 1e-7


def test_solve_many_equals_single_solves():
    """Several right-hand sides on one grid: each column equals its own whv_solve, and the
    direct solution."""
    npts, omega, nd = (129, 121), 24.0, 16
    og = O.Grid(npts)
    tg = WH.time_grid_for(og, omega)
    fs = [I.gaussian(npts, I.source_centers(40 + j, 1, 2)[0], 1.0 / omega, omega ** 2) for j in range(4)]
    F = torch.stack([dev(f) for f in fs])
    g = whv.Grid(npts, precision=whv.WHV_FP64)
    prm = whv.make_params(omega, method="cg", tol=1e-10, maxit=3000)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    U, infos = g.whv_solve_many(prm, F)
    assert all(i["status"] == "OK" for i in infos)
    for j, f in enumerate(fs):
        u1, _ = g.whv_solve(prm, dev(f))
        assert relmax(host(U[j]), host(u1)) < 1e-14
        assert relmax(host(U[j]), IND.helmholtz_direct(npts, tg.omega_eff, f)) < 1e-7
