"""Pins of the oracle's spectral pieces against textbook facts and the paper's closed forms."""
import json
import math
import os

import numpy as np
import pytest

from oracle import operators as O, spectral as SP, waveholtz as WH
from tests import _independent as IND

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("npts,order", [((17,), 2), ((13, 11), 2), ((7, 6, 5), 2), ((15, 12), 4), ((19,), 4)])
def test_closed_form_eigenvalues_match_dense_eigh(npts, order):
    """Sec. 4.3 sine tensor products: oracle lambda^2 == eigh of the independent matrix."""
    g = O.Grid(npts, order=order)
    L = IND.laplacian_matrix(npts, order).toarray()
    ev = np.sort(np.linalg.eigvalsh(-0.5 * (L + L.T)))
    lam2 = np.sort(SP.mode_lambda2(g, SP.all_modes(g)))
    assert np.allclose(lam2, ev, rtol=1e-11, atol=1e-9 * ev.max())


@pytest.mark.parametrize("npts,order", [((21,), 2), ((11, 9), 2), ((6, 7, 5), 2), ((13, 10), 4)])
def test_mode_vectors_are_eigenvectors_of_oracle_operator(npts, order):
    """L_h phi = -lambda^2 phi with the textbook sine vectors (built independently)."""
    g = O.Grid(npts, order=order)
    rng = np.random.default_rng(0)
    for _ in range(4):
        mode = [int(rng.integers(1, n - 1)) for n in npts]
        vec = np.ones(())
        for m in reversed(range(len(npts))):
            vec = np.multiply.outer(vec, IND.sine_vector(npts[m], mode[m]))
        vec = vec.reshape(g.shape)
        lam2 = SP.mode_lambda2(g, np.array([mode]))[0]
        assert np.abs(O.apply_L(g, vec) + lam2 * vec).max() < 1e-9 * lam2
        assert np.allclose(SP.mode_vector(g, mode), vec, atol=1e-14)


def test_basis_orthonormal():
    g = O.Grid((23, 17))
    tg = WH.time_grid_for(g, 15.0)
    modes, _, _ = SP.select_modes(g, tg, 12)
    W = SP.basis(g, modes)
    assert np.abs(W.T @ W - np.eye(12)).max() < 1e-13


def test_beta_special_values_and_bound():
    """eq. beta_fun: beta(omega) = 1, beta(0) = -1/2, beta >= -1/2 (Sec. 2.3, Sec. 3.1)."""
    for om, Np in [(10.5, 1), (50.0, 1), (7.0, 2), (60.0, 3)]:
        tbar = Np * 2 * math.pi / om
        assert SP.beta(om, om, tbar) == pytest.approx(GOLD["beta_at_omega"]["value"], abs=1e-14)
        assert SP.beta(0.0, om, tbar) == pytest.approx(GOLD["beta_at_zero"]["value"], abs=1e-14)
        lam = np.linspace(0, 20 * om, 200001)
        assert SP.beta(lam, om, tbar).min() >= GOLD["beta_lower_bound"]["value"] - 1e-12
        assert (1.0 - SP.beta(lam, om, tbar)).max() <= GOLD["mu_upper_bound"]["value"] + 1e-12


def test_beta_integral_definition():
    """eq. beta_fun first line: (2/T) int_0^T (cos wt - 1/4) cos(lambda t) dt by quadrature."""
    from scipy.integrate import quad
    om, tbar = 9.0, 2 * math.pi / 9.0
    for lam in [0.0, 3.3, 8.2, 9.0, 12.7, 31.0]:
        val = quad(lambda t: (math.cos(om * t) - 0.25) * math.cos(lam * t), 0, tbar, limit=200)[0] * 2 / tbar
        assert SP.beta(lam, om, tbar) == pytest.approx(val, abs=1e-12)


@pytest.mark.parametrize("Np", [1, 2])
def test_gap_law(Np):
    """eq. betaGap: beta = 1 - C_beta z^2 + O(z^3), C_beta = 2/3 Np^2 pi^2 - 1/4."""
    om = 20.0
    tbar = Np * 2 * math.pi / om
    Cb = GOLD["gap_constant"][f"Np{Np}"]
    assert Cb == pytest.approx(2.0 / 3.0 * Np * Np * math.pi ** 2 - 0.25, rel=1e-14)
    for z in [1e-3, -1e-3, 2e-3]:
        est = (1.0 - SP.beta(om * (1 + z), om, tbar)) / z ** 2
        assert est == pytest.approx(Cb, rel=5e-3)


def test_beta_h_converges_to_beta_second_order():
    """beta_h (the exact transfer of the discrete scheme) -> beta as dt -> 0, error O(dt^2)."""
    om = 10.0
    lam = np.array([2.0, 7.5, 9.7, 10.0, 13.0, 25.0])
    errs = []
    for nt in [100, 200, 400, 800]:
        tbar = 2 * math.pi / om
        tg = WH.TimeGrid(om, om, 1, nt, tbar / nt, tbar)
        errs.append(np.abs(SP.beta_h(lam ** 2, tg) - SP.beta(lam, om, tbar)).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(rates) > 1.8, (errs, rates)


@pytest.mark.parametrize("npts,order,omega", [((41,), 2, 10.5), ((21, 17), 2, 14.0), ((9, 8, 7), 2, 7.0), ((19, 15), 4, 11.0)])
def test_pi_on_eigenvector_is_multiplication_by_beta_h(npts, order, omega):
    g = O.Grid(npts, order=order)
    tg = WH.time_grid_for(g, omega)
    modes, lam2, bh = SP.select_modes(g, tg, 5)
    for md, b in zip(modes, bh):
        phi = SP.mode_vector(g, md)
        assert np.abs(WH.apply_pi(g, tg, phi) - b * phi).max() < 1e-12


def test_selected_modes_minimise_distance_to_one():
    """Deflation set (Sec. 2.3): no excluded mode is closer to beta_h = 1 than a selected one."""
    g = O.Grid((19, 23))
    tg = WH.time_grid_for(g, 16.0)
    nd = 9
    modes, lam2, bh = SP.select_modes(g, tg, nd)
    allm = SP.all_modes(g)
    allb = SP.beta_h(SP.mode_lambda2(g, allm), tg)
    chosen = {tuple(m) for m in modes}
    worst_in = max(abs(1 - b) for b in bh)
    best_out = min(abs(1 - b) for m, b in zip(allm, allb) if tuple(m) not in chosen)
    assert worst_in <= best_out
    assert len(chosen) == nd


def test_deflation_lowers_fpi_rate_and_condition():
    """ACR (eq. WaveHoltzFPIconvergence) and kappa (Theorem 3.2) drop when the modes nearest
    resonance are deflated."""
    g = O.Grid((201,))
    tg = WH.time_grid_for(g, 10.5)
    modes, _, _ = SP.select_modes(g, tg, 8)
    assert SP.acr(g, tg, modes) < SP.acr(g, tg) < 1.0
    assert SP.kappa(g, tg, 8) < SP.kappa(g, tg, 0)


def test_kappa_example_rate():
    """Sec. 3.1: kappa_D = 3 gives the Theorem 3.1 rate ~0.27."""
    k = GOLD["kappa_example"]["kappa_D"]
    rate = (math.sqrt(k) - 1) / (math.sqrt(k) + 1)
    assert rate == pytest.approx(GOLD["kappa_example"]["rate"], abs=GOLD["kappa_example"]["rate_tol"])


def test_break_even_model():
    """Sec. 4.1 cost model: deflated 20 N_f + 150 beats standard 125 N_f from N_f = 2."""
    b = GOLD["break_even"]
    nf = next(n for n in range(1, 100) if b["deflated_per_rhs"] * n + b["eigen_setup"] < b["standard_per_rhs"] * n)
    assert nf == b["break_even_nf"]


def test_nd_proportional_to_omega_squared_keeps_the_rate_bounded():
    """Sec. 4.4 (Weyl + gap law): with N_D = floor(omega^2/10) deflated modes the asymptotic
    convergence rate of the deflated iteration stays bounded away from 1 as omega grows on the unit
    square, while N_D = floor(3 omega/2) lets it drift towards 1."""
    og = O.Grid((129, 129))
    modes = SP.all_modes(og)
    lam2 = SP.mode_lambda2(og, modes)
    quad, lin = {}, {}
    for om in (10, 15, 20, 25, 30):
        tg = WH.time_grid_for(og, float(om))
        bh = SP.beta_h(lam2, tg)
        order = np.lexsort((np.arange(len(bh)), np.abs(1.0 - bh)))

        def acr(nd):
            rest = np.ones(len(bh), bool)
            rest[order[:nd]] = False
            return float(np.abs(bh[rest]).max())
        quad[om], lin[om] = acr(om * om // 10), acr(3 * om // 2)
    assert max(quad.values()) < 0.5
    assert quad[30] - quad[15] < 0.1
    assert lin[30] > 0.8 and lin[30] - lin[15] > 0.3
