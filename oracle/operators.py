"""Grid and difference operator L_{p,h} of the oracle (test infrastructure only).

Sec. 2.2, eq. discreteHelmholtz: L_{p,h} is a p-th order accurate difference
approximation of L = div(c^2 grad) (eq. L) on a structured grid with Dirichlet boundary
nodes.  Readings used here:
  * Grid functions live on interior nodes j_m = 1..n_m-2; the boundary nodes hold 0.
  * Variable speed uses the non-conservative form L_h = c^2(x) Delta_h (the squared
    speed multiplies the discrete Laplacian).  It is self-adjoint in the inner product
    <u, v>_M = sum_j u_j v_j / c_j^2, the diagonal-mass-matrix symmetrisation of Sec. 4.1
    with M = diag(1/c^2); for c = 1 this is the Euclidean inner product.
  * The conservative form L_h = div_h(c^2 grad_h) (order 2 only, `form="conservative"`):
    per direction (c^2_{j+1/2} (u_{j+1} - u_j) - c^2_{j-1/2} (u_j - u_{j-1})) / h^2 with the
    face values c^2_{j+1/2} = (c^2_j + c^2_{j+1}) / 2 and, on the two boundary faces, the value
    of the adjacent interior node (reading: c^2 is given on the interior nodes only).  It is
    self-adjoint in the Euclidean inner product (M = I).
  * 4th order (p = 4): the centred five-point formula per direction, with the value at the
    ghost node outside the Dirichlet boundary taken as the odd reflection of the first
    interior value (u_{-1} = -u_1).  The paper leaves the near-boundary closure to
    "compatibility conditions" (Sec. 2.2); odd reflection keeps the sine vectors exact
    eigenvectors.
"""
from __future__ import annotations

import numpy as np


class Grid:
    """Structured box grid: `npts` nodes per direction (x first), boundary included."""

    def __init__(self, npts, lo=None, hi=None, order=2, c2=None, form="nonconservative"):
        self.dim = len(npts)
        self.npts = tuple(int(n) for n in npts)
        self.lo = [0.0] * self.dim if lo is None else [float(a) for a in lo]
        self.hi = [1.0] * self.dim if hi is None else [float(b) for b in hi]
        self.h = [(b - a) / (n - 1) for n, a, b in zip(self.npts, self.lo, self.hi)]
        if order not in (2, 4):
            raise ValueError("order must be 2 or 4")
        self.order = order
        # array axes are (z, y, x): axis for direction m is dim-1-m
        self.shape = tuple(n - 2 for n in reversed(self.npts))
        self.c2 = None if c2 is None else np.asarray(c2, dtype=np.float64).reshape(self.shape)
        if form not in ("nonconservative", "conservative"):
            raise ValueError(form)
        if form == "conservative" and order != 2:
            raise ValueError("the conservative form is second order")
        self.form = form

    @property
    def n(self):
        return int(np.prod(self.shape))

    @property
    def c_max(self):
        return 1.0 if self.c2 is None else float(np.sqrt(self.c2.max()))

    def weights(self):
        """Diagonal of M: 1/c^2 (ones for c = 1 and for the conservative form)."""
        if self.c2 is None or self.form == "conservative":
            return np.ones(self.shape)
        return 1.0 / self.c2

    def inner(self, u, v):
        """<u, v>_M = sum u v / c^2."""
        return float(np.sum(u * v * self.weights()))

    def norm(self, u):
        return float(np.sqrt(self.inner(u, u)))


def _second_difference(u, axis, h):
    """(u_{j+1} - 2 u_j + u_{j-1}) / h^2 with zero Dirichlet values beyond the interior."""
    pad = [(0, 0)] * u.ndim
    pad[axis] = (1, 1)
    up = np.pad(u, pad)  # zeros at the two boundary nodes
    n = u.shape[axis]
    sl = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(u.ndim))  # noqa: E731
    return (up[sl(2, n + 2)] - 2.0 * up[sl(1, n + 1)] + up[sl(0, n)]) / (h * h)


def _fourth_order_second_difference(u, axis, h):
    """(-u_{j+2} + 16 u_{j+1} - 30 u_j + 16 u_{j-1} - u_{j-2}) / (12 h^2), Dirichlet node 0,
    ghost node by odd reflection u_{-1} = -u_1 (and at the far end likewise)."""
    n = u.shape[axis]
    take = lambda i: np.take(u, [i], axis=axis)  # noqa: E731
    zero = np.zeros_like(take(0))
    full = np.concatenate([-take(0), zero, u, zero, -take(n - 1)], axis=axis)
    sl = lambda a: tuple(slice(a, a + n) if k == axis else slice(None) for k in range(u.ndim))  # noqa: E731
    # interior node j sits at index j+1 of `full` (index 0 = ghost, 1 = boundary node)
    c = 2
    return (-full[sl(c + 2)] + 16.0 * full[sl(c + 1)] - 30.0 * full[sl(c)]
            + 16.0 * full[sl(c - 1)] - full[sl(c - 2)]) / (12.0 * h * h)


def laplacian(grid: Grid, u: np.ndarray) -> np.ndarray:
    """Delta_{p,h} u: sum over directions of the p-th order second difference."""
    u = np.asarray(u, dtype=np.float64).reshape(grid.shape)
    out = np.zeros(grid.shape)
    for m in range(grid.dim):
        axis = grid.dim - 1 - m
        if grid.order == 2:
            out += _second_difference(u, axis, grid.h[m])
        else:
            out += _fourth_order_second_difference(u, axis, grid.h[m])
    return out


def _conservative_difference(u, c2, axis, h):
    """(c^2_{j+1/2} (u_{j+1} - u_j) - c^2_{j-1/2} (u_j - u_{j-1})) / h^2 along `axis`, u = 0 at
    the boundary nodes, interior faces by the mean of their two nodes, boundary faces by the
    adjacent interior node."""
    n = u.shape[axis]
    sl = lambda a, b: tuple(slice(a, b) if k == axis else slice(None) for k in range(u.ndim))  # noqa: E731
    pad = [(0, 0)] * u.ndim
    pad[axis] = (1, 1)
    up = np.pad(u, pad)
    # faces j - 1/2 for j = 0 .. n (n + 1 of them)
    faces = np.concatenate([c2[sl(0, 1)], 0.5 * (c2[sl(0, n - 1)] + c2[sl(1, n)]), c2[sl(n - 1, n)]], axis=axis)
    flux = faces * (up[sl(1, n + 2)] - up[sl(0, n + 1)])   # c^2_{j-1/2} (u_j - u_{j-1}), j = 0 .. n
    return (flux[sl(1, n + 1)] - flux[sl(0, n)]) / (h * h)


def apply_L(grid: Grid, u: np.ndarray) -> np.ndarray:
    """L_{p,h} u = c^2 Delta_{p,h} u (eq. discreteHelmholtz with L = c^2 Delta), or the
    conservative div_h(c^2 grad_h) u."""
    if grid.c2 is not None and grid.form == "conservative":
        u = np.asarray(u, dtype=np.float64).reshape(grid.shape)
        out = np.zeros(grid.shape)
        for m in range(grid.dim):
            out += _conservative_difference(u, grid.c2, grid.dim - 1 - m, grid.h[m])
        return out
    lap = laplacian(grid, u)
    return lap if grid.c2 is None else grid.c2 * lap


def spectral_radius_bound(grid: Grid) -> float:
    """Upper bound of the largest eigenvalue lambda^2 of -L_{p,h} (Fourier symbol maxima:
    4/h^2 per direction for p = 2, 16/(3 h^2) for p = 4), times max c^2."""
    per = 4.0 if grid.order == 2 else 16.0 / 3.0
    s = sum(per / (h * h) for h in grid.h)
    return s * grid.c_max ** 2
