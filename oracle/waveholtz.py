"""The WaveHoltz operator Pi_h of the oracle (test infrastructure only).

Sec. 2.1 eq. waveHoltzFilter: Pi v = (2/Tbar) int_0^Tbar (cos(omega t) - 1/4) w(t; v) dt
with w the solution of the wave IBVP eq. waveEquation, w_tt = L w - f cos(omega t),
w(0) = v, w_t(0) = 0.  Discretely (Sec. 2.2):
  * eq. discreteWaveExplicit: D+t D-t W^n = L_h W^n - f cos(omega t^n), W^0 = V,
    D0t W^0 = 0, i.e. W^{n+1} = 2 W^n - W^{n-1} + dt^2 (L_h W^n - f cos(omega t^n)) with
    the first step W^1 = W^0 + dt^2/2 (L_h W^0 - f) (D0t W^0 = 0 gives W^{-1} = W^1);
  * eq. quadrature: Pi_h V = (2/Tbar) sum_{n=0}^{Nt} eta_n (cos(omega t^n) - 1/4) W^n dt,
    eta_0 = eta_Nt = 1/2, eta_n = 1 otherwise;
  * eq. Sh / WaveHoltzMatrixEquation: Pi_h V = S_h V + b, b = Pi_h 0, A = I - S_h.

Readings (the paper is silent on these):
  * Time step: dt0 = cfl h_min / c_max with cfl = 0.5 (2nd order) or 0.4 (4th order);
    Tbar = Np 2 pi / omega; Nt = ceil(Tbar / dt0); dt = Tbar / Nt ("dt adjusted so that
    T/dt is an integer").
  * Removal of the time-discretisation error (Sec. 2.2, last paragraph): with
    `adjust=True` the cos / filter frequency is replaced by omega_hat such that
    (2/dt) sin(omega_hat dt/2) = omega; with Nt fixed this gives dt = 2 sin(pi Np/Nt)/omega,
    omega_hat = 2 pi Np / (Nt dt), Tbar = Nt dt, and Nt is the smallest integer with
    dt <= dt0.  Without adjustment the fixed point solves the discrete Helmholtz problem
    at omega_eff = (2/dt) sin(omega dt / 2) instead of omega.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .operators import Grid, apply_L, spectral_radius_bound


@dataclass
class TimeGrid:
    omega: float        # requested frequency
    omega_hat: float    # frequency used in cos(.) and in the filter
    periods: int
    nt: int
    dt: float
    tbar: float

    @property
    def omega_eff(self) -> float:
        """Frequency whose discrete Helmholtz problem the fixed point solves."""
        return 2.0 / self.dt * math.sin(self.omega_hat * self.dt / 2.0)

    def forcing_phase(self) -> np.ndarray:
        """cos(omega_hat t^n), n = 0..Nt."""
        n = np.arange(self.nt + 1, dtype=np.float64)
        return np.cos(self.omega_hat * n * self.dt)

    def filter_weights(self) -> np.ndarray:
        """(2/Tbar) eta_n (cos(omega_hat t^n) - 1/4) dt, n = 0..Nt (eq. quadrature)."""
        eta = np.ones(self.nt + 1)
        eta[0] = eta[-1] = 0.5
        return (2.0 / self.tbar) * eta * (self.forcing_phase() - 0.25) * self.dt


def default_cfl(order: int) -> float:
    return 0.5 if order == 2 else 0.4


def time_grid(omega: float, h_min: float, c_max: float = 1.0, order: int = 2,
              periods: int = 1, adjust: bool = False, cfl: float | None = None) -> TimeGrid:
    cfl = default_cfl(order) if cfl is None else cfl
    dt0 = cfl * h_min / c_max
    if not adjust:
        tbar = periods * 2.0 * math.pi / omega
        nt = int(math.ceil(tbar / dt0))
        dt = tbar / nt
        return TimeGrid(omega, omega, periods, nt, dt, tbar)
    nt = 2 * periods + 1
    while 2.0 * math.sin(math.pi * periods / nt) / omega > dt0:
        nt += 1
    dt = 2.0 * math.sin(math.pi * periods / nt) / omega
    omega_hat = 2.0 * math.pi * periods / (nt * dt)
    return TimeGrid(omega, omega_hat, periods, nt, dt, nt * dt)


def time_grid_for(grid: Grid, omega: float, periods: int = 1, adjust: bool = False,
                  cfl: float | None = None) -> TimeGrid:
    tg = time_grid(omega, min(grid.h), grid.c_max, grid.order, periods, adjust, cfl)
    # explicit leapfrog is stable iff dt^2 lambda_max^2 / 4 <= 1
    if tg.dt ** 2 * spectral_radius_bound(grid) / 4.0 > 1.0:
        raise ValueError("time step above the stability limit")
    return tg


def apply_pi(grid: Grid, tg: TimeGrid, v: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    """Pi_h V: leapfrog over one filter interval from (V, 0) with forcing f, trapezoid-
    filtered (eq. discreteWaveExplicit + eq. quadrature).  f = None means f = 0."""
    dt2 = tg.dt * tg.dt
    phase = tg.forcing_phase()
    weight = tg.filter_weights()
    w0 = np.asarray(v, dtype=np.float64).reshape(grid.shape).copy()
    force = (lambda n: 0.0) if f is None else (lambda n: np.asarray(f).reshape(grid.shape) * phase[n])  # noqa: E731
    # first step from D0t W^0 = 0
    w1 = w0 + 0.5 * dt2 * (apply_L(grid, w0) - force(0))
    acc = weight[0] * w0 + weight[1] * w1
    w_prev, w_cur = w0, w1
    for n in range(1, tg.nt):
        w_next = 2.0 * w_cur - w_prev + dt2 * (apply_L(grid, w_cur) - force(n))
        acc = acc + weight[n + 1] * w_next
        w_prev, w_cur = w_cur, w_next
    return acc


def wave_states(grid: Grid, tg: TimeGrid, v: np.ndarray, f: np.ndarray | None = None):
    """All states W^0..W^Nt of the leapfrog (for tests of the adjoint and of steps)."""
    dt2 = tg.dt * tg.dt
    phase = tg.forcing_phase()
    w0 = np.asarray(v, dtype=np.float64).reshape(grid.shape).copy()
    force = (lambda n: 0.0) if f is None else (lambda n: np.asarray(f).reshape(grid.shape) * phase[n])  # noqa: E731
    states = [w0, w0 + 0.5 * dt2 * (apply_L(grid, w0) - force(0))]
    for n in range(1, tg.nt):
        states.append(2.0 * states[-1] - states[-2] + dt2 * (apply_L(grid, states[-1]) - force(n)))
    return states


def apply_S(grid: Grid, tg: TimeGrid, v: np.ndarray) -> np.ndarray:
    """S_h v = Pi_h v - Pi_h 0; with f = 0 this is Pi_h v itself (Sec. 2.1)."""
    return apply_pi(grid, tg, v, None)


def rhs_b(grid: Grid, tg: TimeGrid, f: np.ndarray) -> np.ndarray:
    """b = Pi_h 0 (eq. WaveHoltzDiscreteFPI)."""
    return apply_pi(grid, tg, np.zeros(grid.shape), f)


def apply_A(grid: Grid, tg: TimeGrid, v: np.ndarray) -> np.ndarray:
    """A v = (I - S_h) v (eq. WaveHoltzMatrixEquation)."""
    v = np.asarray(v, dtype=np.float64).reshape(grid.shape)
    return v - apply_S(grid, tg, v)
