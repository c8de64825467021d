"""Independent textbook constructions used to pin the oracle (no oracle code here).

The sparse matrices are built from the 1-D second-difference matrices with Kronecker
products, the standard construction of the Dirichlet Laplacian on a tensor grid; the
direct Helmholtz solve is scipy's sparse LU.  Nothing here calls `oracle/`.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def second_difference_1d(n, h, order=2):
    """1-D Dirichlet second-difference matrix on the n-2 interior nodes."""
    N = n - 2
    if order == 2:
        return (sp.diags([np.ones(N - 1), -2 * np.ones(N), np.ones(N - 1)], [-1, 0, 1]) / h ** 2).tocsr()
    T = sp.diags([-np.ones(N - 2), 16 * np.ones(N - 1), -30 * np.ones(N), 16 * np.ones(N - 1),
                  -np.ones(N - 2)], [-2, -1, 0, 1, 2]).tolil()
    # ghost node outside the boundary = -(first interior value): -u_{-1} = +u_1 enters row 1
    T[0, 0] += 1.0
    T[N - 1, N - 1] += 1.0
    return (T.tocsr() / (12.0 * h * h)).tocsr()


def laplacian_matrix(npts, order=2, lo=None, hi=None):
    """Sparse Delta_h on the interior of a box grid, unknowns ordered x fastest."""
    dim = len(npts)
    lo = [0.0] * dim if lo is None else lo
    hi = [1.0] * dim if hi is None else hi
    L = None
    for m in range(dim):
        h = (hi[m] - lo[m]) / (npts[m] - 1)
        factors = [sp.identity(npts[k] - 2, format="csr") for k in reversed(range(dim))]
        factors[dim - 1 - m] = second_difference_1d(npts[m], h, order)
        M = factors[0]
        for F in factors[1:]:
            M = sp.kron(M, F, format="csr")
        L = M if L is None else L + M
    return L.tocsr()


def helmholtz_direct(npts, omega, f, order=2, c2=None):
    """Solve (c^2 Delta_h + omega^2) U = f by sparse LU."""
    L = laplacian_matrix(npts, order)
    if c2 is not None:
        L = sp.diags(np.asarray(c2).ravel()) @ L
    A = (L + omega ** 2 * sp.identity(L.shape[0])).tocsc()
    return spl.spsolve(A, np.asarray(f).ravel())


def sine_vector(n, k):
    """Textbook Dirichlet sine vector sin(k pi x_i), x_i = i/(n-1), i = 1..n-2, unit 2-norm."""
    i = np.arange(1, n - 1)
    v = np.sin(np.pi * k * i / (n - 1))
    return v / np.linalg.norm(v)


def relmax(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def conservative_matrix(npts, c2, lo=None, hi=None):
    """Sparse div_h(c^2 grad_h) on the interior (second order), assembled entry by entry: for
    every interior node and direction, the faces to the two neighbours carry the mean of the two
    nodes' c^2 (the adjacent interior value on a face to a boundary node); unknowns x fastest."""
    dim = len(npts)
    lo = [0.0] * dim if lo is None else lo
    hi = [1.0] * dim if hi is None else hi
    n = [p - 2 for p in npts]
    N = int(np.prod(n))
    c2 = np.asarray(c2, dtype=np.float64).ravel()
    stride = [int(np.prod(n[:m])) for m in range(dim)]
    rows, cols, vals = [], [], []
    for idx in range(N):
        coord = [(idx // stride[m]) % n[m] for m in range(dim)]
        for m in range(dim):
            h2 = ((hi[m] - lo[m]) / (npts[m] - 1)) ** 2
            for s in (-1, 1):
                j = coord[m] + s
                if 0 <= j < n[m]:
                    nb = idx + s * stride[m]
                    face = 0.5 * (c2[idx] + c2[nb])
                    rows.append(idx); cols.append(nb); vals.append(face / h2)
                else:
                    face = c2[idx]
                rows.append(idx); cols.append(idx); vals.append(-face / h2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def helmholtz_direct_conservative(npts, omega, f, c2):
    """Solve (div_h(c^2 grad_h) + omega^2) U = f by sparse LU."""
    A = (conservative_matrix(npts, c2) + omega ** 2 * sp.identity(int(np.prod([p - 2 for p in npts])))).tocsc()
    return spl.spsolve(A, np.asarray(f).ravel())
