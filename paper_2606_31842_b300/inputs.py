"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates data*: grid-point coordinates, Gaussian sources, smooth
wave-speed fields and random vectors, plus the table of workload parameters.  It holds
none of the WaveHoltz arithmetic (no difference operator, no time stepping, no filter,
no eigenpairs, no Krylov step), so the CPU oracle and the CUDA path can both draw their
inputs from it without sharing any of the method.

Array convention used everywhere: a grid function lives on the *interior* nodes only
(boundary nodes carry the homogeneous Dirichlet value 0), stored C-contiguous with x the
fastest axis, i.e. shape (Nx,), (Ny, Nx) or (Nz, Ny, Nx) with N_m = npts_m - 2.

Source shape: the Gaussian a_g exp(-b_g^2 |x - x0|^2) of the paper's forcing
(Sec. 5, eq. gaussianSource) with a_g = omega^2 and b_g = omega unless a workload says
otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "interior_coords", "gaussian", "source_centers", "bumps",
    "speed_squared", "random_field", "interior_shape", "forcing_for",
]


def interior_shape(npts) -> tuple:
    """Shape of the interior array for `npts` nodes per direction (x first in `npts`)."""
    return tuple(int(n) - 2 for n in reversed(list(npts)))


def interior_coords(npts, lo=None, hi=None):
    """1-D coordinate arrays of the interior nodes, x_i = lo + i h, i = 1..n-2."""
    dim = len(npts)
    lo = [0.0] * dim if lo is None else list(lo)
    hi = [1.0] * dim if hi is None else list(hi)
    out = []
    for n, a, b in zip(npts, lo, hi):
        h = (b - a) / (n - 1)
        out.append(a + h * np.arange(1, n - 1, dtype=np.float64))
    return out


def _mesh(npts, lo, hi):
    xs = interior_coords(npts, lo, hi)
    # reversed so that the last axis is x
    grids = np.meshgrid(*reversed(xs), indexing="ij")
    return list(reversed(grids))  # [X, Y, Z] each of the interior shape


def gaussian(npts, center, width, amplitude=1.0, lo=None, hi=None) -> np.ndarray:
    """amplitude * exp(-(|x - center| / width)^2) on the interior nodes (float64)."""
    comps = _mesh(npts, lo, hi)
    r2 = np.zeros(comps[0].shape)
    for X, c in zip(comps, center):
        r2 += (X - c) ** 2
    return amplitude * np.exp(-r2 / (width * width))


def source_centers(seed: int, count: int, dim: int, margin: float = 0.1) -> np.ndarray:
    """`count` source centres drawn uniformly from [margin, 1 - margin]^dim."""
    rng = np.random.default_rng(seed)
    return rng.uniform(margin, 1.0 - margin, size=(count, dim))


def bumps(npts, seed: int, count: int = 16, width: float = 0.05, lo=None, hi=None) -> np.ndarray:
    """Sum of `count` unit Gaussian bumps of the given width at seeded centres,
    min-max normalised to [0, 1] over the interior nodes."""
    dim = len(npts)
    centers = source_centers(seed, count, dim)
    s = np.zeros(interior_shape(npts))
    for c in centers:
        s += gaussian(npts, c, width, 1.0, lo, hi)
    smin, smax = s.min(), s.max()
    return (s - smin) / (smax - smin)


def speed_squared(kind: str, npts, seed: int) -> np.ndarray:
    """Squared wave speed c^2 on the interior nodes.

    kind = "c3":  c = 1 + 0.4 * bumps  (16 bumps of width 0.05), returned squared;
    kind = "c5":  c^2 = 1 + 0.3 * bumps.
    """
    b = bumps(npts, seed)
    if kind == "c3":
        return (1.0 + 0.4 * b) ** 2
    if kind == "c5":
        return 1.0 + 0.3 * b
    raise ValueError(kind)


def random_field(shape, seed: int) -> np.ndarray:
    """Standard-normal float64 array of the given shape."""
    return np.random.default_rng(seed).standard_normal(shape)


@dataclass(frozen=True)
class Workload:
    """Parameters of one synthetic workload shaped like the paper's problems."""
    name: str
    dim: int
    npts: tuple            # nodes per direction including both boundary nodes (x first)
    omega: float
    nd: int                # deflation vectors
    tol: float
    order: int = 2
    periods: int = 1
    source_width: float = 0.0   # 0 => width 1/omega (b_g = omega)
    source_amp: float = 0.0     # 0 => amplitude omega^2
    seed: int = 0
    speed: str = ""             # "" => c = 1
    speed_seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return interior_shape(self.npts)

    @property
    def n_unknowns(self):
        return int(np.prod(self.shape))


def forcing_for(w: Workload, source: int = 0) -> np.ndarray:
    """Forcing f of workload `w`; `source` picks one of its seeded centres."""
    if w.name.startswith("c1"):
        # 1-D workload: f(x) = exp(-((x - 0.5)/0.05)^2), amplitude 1
        return gaussian(w.npts, [0.5], 0.05, 1.0)
    width = w.source_width if w.source_width > 0 else 1.0 / w.omega
    amp = w.source_amp if w.source_amp > 0 else w.omega ** 2
    centers = source_centers(w.seed + source, 1, w.dim)
    return gaussian(w.npts, centers[0], width, amp)


def _sq(n, dim=2):
    return tuple([n] * dim)


WORKLOADS = {
    # 1-D, 201 nodes, omega = 10.5, 8 deflated sines, CG to 1e-10, FP64
    "c1": Workload("c1", 1, (201,), 10.5, 8, 1e-10),
    # 2-D 513^2 square, omega = 50, Gaussian of width 0.02 (= 1/omega), 64 sin*sin vectors
    "c2": Workload("c2", 2, _sq(513), 50.0, 64, 1e-8, source_width=0.02),
    # 2-D 1025^2, 4th order, variable speed c = 1 + 0.4 bumps, omega = 60, 128 Lanczos vectors
    "c3": Workload("c3", 2, _sq(1025), 60.0, 128, 1e-6, order=4, speed="c3", speed_seed=1234),
    # 3-D 256^3 cube, omega = 40, 32 closed-form vectors
    "c5": Workload("c5", 3, _sq(256, 3), 40.0, 32, 1e-6),
    # adjoint grid of the 3-D workload: 128^3, c^2 = 1 + 0.3 bumps
    "c5adj": Workload("c5adj", 3, _sq(128, 3), 40.0, 32, 1e-6, speed="c5", speed_seed=2024),
}

# batched workload: 4 uneven squares x 16 point sources x 4 frequencies, width 2h
C4_SIZES = (257, 513, 769, 1025)
C4_OMEGAS = (20.0, 30.0, 40.0, 50.0)
C4_SOURCES = 16
for _n in C4_SIZES:
    for _om in C4_OMEGAS:
        WORKLOADS[f"c4_{_n}_{int(_om)}"] = Workload(
            f"c4_{_n}_{int(_om)}", 2, _sq(_n), _om, 32, 1e-6,
            source_width=2.0 / (_n - 1), seed=_n)


def scaled(w: Workload, n: int) -> Workload:
    """The same workload on a smaller grid of n nodes per direction (for quick tests)."""
    from dataclasses import replace
    return replace(w, name=f"{w.name}@{n}", npts=tuple([n] * w.dim))


def h_of(npts, lo=None, hi=None):
    dim = len(npts)
    lo = [0.0] * dim if lo is None else lo
    hi = [1.0] * dim if hi is None else hi
    return [(b - a) / (n - 1) for n, a, b in zip(npts, lo, hi)]


if __name__ == "__main__":  # pragma: no cover
    for k, w in WORKLOADS.items():
        print(k, w.shape, w.n_unknowns, math.tau / w.omega)
