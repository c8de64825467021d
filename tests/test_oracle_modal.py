"""Pins of oracle/modal.py (DEVD-CG of the constant-speed box in its sine eigenbasis) against
the time-domain oracle it restates and against independent constructions: the sine transform
is W^T u with the explicit basis matrix, Pi_h(0; phi) = gamma_h phi on eigenvectors, and the
iteration counts and solutions of Algorithm 2 with CG agree with krylov.devd_solve and with
the sparse direct Helmholtz solve."""
import numpy as np
import pytest

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K, modal as MD
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND


@pytest.mark.parametrize("npts", [(9, 7), (6, 8, 7)])
def test_sine_coefficients_are_the_basis_projection(npts):
    g = O.Grid(npts)
    u = I.random_field(g.shape, 3)
    W = SP.basis(g, SP.all_modes(g))                       # every mode, x index outermost
    c = MD.sine_coefficients(g, u)
    ref = W.T @ u.ravel()
    assert np.abs(MD._mode_array(g, ref) - c).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(MD.from_sine_coefficients(g, c) - u).max() < 1e-13 * np.abs(u).max()


def test_sine_coefficients_of_textbook_sines():
    """A product of textbook sines has one nonzero coefficient, at its mode (independent of
    spectral.py)."""
    npts = (13, 10)
    g = O.Grid(npts)
    u = np.outer(IND.sine_vector(10, 3), IND.sine_vector(13, 5))   # (y, x): k_y = 3, k_x = 5
    c = MD.sine_coefficients(g, u)
    assert abs(abs(c[2, 4]) - 1.0) < 1e-13
    c[2, 4] = 0.0
    assert np.abs(c).max() < 1e-13


@pytest.mark.parametrize("mode", [(1, 1), (3, 2), (7, 9)])
def test_forced_transfer_on_eigenvectors(mode):
    g = O.Grid((17, 13))
    tg = WH.time_grid_for(g, 20.0)
    phi = SP.mode_vector(g, mode)
    out = WH.apply_pi(g, tg, np.zeros(g.shape), phi)      # b = Pi_h(0; phi)
    gam = MD.forced_transfer(SP.mode_lambda2(g, np.array([mode])), tg)[0]
    assert np.abs(out - gam * phi).max() < 1e-13 * max(1.0, abs(gam))


@pytest.mark.parametrize("n,omega,nd", [(33, 30.0, 8), (41, 20.0, 12)])
def test_devd_cg_matches_time_domain_oracle(n, omega, nd):
    w = I.scaled(I.WORKLOADS[f"c4_257_{int(omega)}"], n)
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    F = np.stack([I.forcing_for(w, s) for s in range(3)])
    ms = MD.ModalSystem(g, tg, nd)
    modes, lam2, _ = SP.select_modes(g, tg, nd)
    V = SP.basis(g, modes)
    for tol in (1e-6, 1e-12):
        its, conv, U = MD.devd_cg(ms, F, tol, 2000)
        for s in range(3):
            r = K.devd_solve(g, tg, F[s], V, lam2, "cg", tol, 2000)
            assert conv[s] and r.solve.converged
            assert abs(int(its[s]) - r.solve.iterations) <= 1      # rounding at the threshold
            assert IND.relmax(U[s], r.u) < (1e-11 if tol < 1e-9 else 1e-5)
    # converged solutions are the discrete Helmholtz solution at omega_eff (independent LU)
    for s in range(3):
        Ud = IND.helmholtz_direct(w.npts, tg.omega_eff, F[s])
        assert IND.relmax(U[s], Ud) < 1e-10


def test_deflated_modes_are_the_selected_set():
    g = O.Grid((21, 19))
    tg = WH.time_grid_for(g, 25.0)
    ms = MD.ModalSystem(g, tg, 10)
    modes, _, _ = SP.select_modes(g, tg, 10)
    got = sorted((int(kx) + 1, int(ky) + 1) for ky, kx in zip(*np.nonzero(ms.deflated)))
    assert got == sorted((int(m[0]), int(m[1])) for m in modes)
