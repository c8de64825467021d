"""SVD compression of the deflation vectors (Sec. 4.3, experiment with compressed eigenvectors).

Oracle -- test infrastructure only; nothing in the product path imports it.

A 2-D grid function phi is an ny x nx matrix Q (row y, column x, the interior array with x
fastest).  With its singular value decomposition Q = sum_k u_k s_k v_k^T (s_1 >= s_2 >= ...),
the truncated form keeps the smallest r for which the Frobenius norm of the discarded part is
below the tolerance:  ||Q - sum_{k<=r} u_k s_k v_k^T||_F^2 = sum_{k>r} s_k^2 < tau^2  (reading:
the paper calls r "the largest value" for which this holds, but the inequality holds for every r
above the smallest one; the smallest is the compression).  Storage r (nx + ny + 1) instead of
nx ny.  The deflation contractions with compressed vectors are
    <phi_m, R>_M = sum_k s_k u_k^T (M o R) v_k          (projection W^T M r)
    W y = sum_m y_m sum_k s_k u_k v_k^T                   (expansion)
Library primitive: numpy.linalg.svd.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .operators import Grid


@dataclass
class Compressed:
    U: np.ndarray      # ny x r
    s: np.ndarray      # r
    V: np.ndarray      # nx x r
    rank: int
    error: float       # ||Q - U diag(s) V^T||_F


def truncated_svd(Q: np.ndarray, tau: float) -> Compressed:
    """Smallest-rank truncated SVD of Q with Frobenius error < tau."""
    U, s, Vt = np.linalg.svd(np.asarray(Q, dtype=np.float64), full_matrices=False)
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])   # tail[r] = sum_{k>=r} s_k^2
    r = int(np.argmax(tail < tau * tau))
    return Compressed(U[:, :r], s[:r], Vt[:r].T, r, float(np.sqrt(tail[r])))


def compress_basis(grid: Grid, W: np.ndarray, tau: float) -> list[Compressed]:
    """Compress every column of W (N x nd, x fastest) as an ny x nx matrix."""
    if grid.dim != 2:
        raise ValueError("SVD compression needs a 2-D grid")
    return [truncated_svd(W[:, m].reshape(grid.shape), tau) for m in range(W.shape[1])]


def dense(grid: Grid, c: Compressed) -> np.ndarray:
    """The compressed vector written out (N, x fastest)."""
    return (c.U @ np.diag(c.s) @ c.V.T).ravel()


def project(grid: Grid, comp: list[Compressed], r: np.ndarray) -> np.ndarray:
    """coef_m = <phi_m, r>_M with the compressed phi_m: sum_k s_k u_k^T (M o R) v_k."""
    R = (grid.weights() * np.asarray(r).reshape(grid.shape))
    out = np.zeros(len(comp))
    for m, c in enumerate(comp):
        out[m] = sum(c.s[k] * (c.U[:, k] @ R @ c.V[:, k]) for k in range(c.rank))
    return out


def expand(grid: Grid, comp: list[Compressed], y: np.ndarray) -> np.ndarray:
    """sum_m y_m phi_m with the compressed phi_m (N, x fastest)."""
    out = np.zeros(grid.shape)
    for m, c in enumerate(comp):
        out += y[m] * (c.U @ np.diag(c.s) @ c.V.T)
    return out.ravel()


def compression_ratio(grid: Grid, comp: list[Compressed]) -> float:
    ny, nx = grid.shape
    return sum(c.rank * (nx + ny + 1) for c in comp) / (len(comp) * nx * ny)
