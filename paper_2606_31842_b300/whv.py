"""Thin Python binding of the C ABI in include/whv.h (argument marshalling only).

Every function has the name of the C entry point it wraps and forwards raw device pointers of
contiguous float64 CUDA tensors; all arithmetic runs in the library's CUDA kernels.  There is
no CPU fallback: importing this module fails loudly when libwhv.so is missing, and every call
checks the returned status.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libwhv.so")

WHV_OK, WHV_ERR_INVALID, WHV_ERR_CUDA, WHV_ERR_OOM, WHV_ERR_NOT_CONVERGED, WHV_ERR_BREAKDOWN, WHV_ERR_TIMEOUT = range(7)
WHV_FP64, WHV_FP32_STEP = 0, 1
WHV_FPI, WHV_CG, WHV_DCG, WHV_GMRES, WHV_AGMRES, WHV_ABICGSTAB = 0, 1, 2, 3, 4, 5
WHV_BASIS_NONE, WHV_BASIS_USER, WHV_BASIS_CLOSED_FORM, WHV_BASIS_LANCZOS = 0, 1, 2, 3
WHV_BASIS_EXACT, WHV_BASIS_REDEFLATE = 1, 2
WHV_TRUE_RESIDUAL, WHV_REFINE_FP64, WHV_RESIDUAL_DF64 = 1, 2, 4
WHV_SPEED_NONCONSERVATIVE, WHV_SPEED_CONSERVATIVE = 0, 1
STATUS_NAMES = ["OK", "INVALID", "CUDA", "OOM", "NOT_CONVERGED", "BREAKDOWN", "TIMEOUT"]
METHODS = {"fpi": WHV_FPI, "cg": WHV_CG, "dcg": WHV_DCG, "gmres": WHV_GMRES, "agmres": WHV_AGMRES,
           "abicgstab": WHV_ABICGSTAB}


class whv_params(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("periods", ctypes.c_int), ("adjust_omega", ctypes.c_int),
                ("cfl", ctypes.c_double), ("method", ctypes.c_int), ("restart", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("check_every", ctypes.c_int),
                ("flags", ctypes.c_int), ("inner_tol", ctypes.c_double)]


class whv_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("wave_solves", ctypes.c_int), ("nt", ctypes.c_int),
                ("dt", ctypes.c_double), ("omega_hat", ctypes.c_double), ("omega_eff", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("outer_iterations", ctypes.c_int),
                ("wave_solves_fp64", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class WhvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libwhv.so not built ({_LIB_PATH}); run python -m paper_2606_31842_b300.build")
    lib = ctypes.CDLL(_LIB_PATH)
    P, D, I, L = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    sig = {
        "whv_create_grid": [I, ctypes.POINTER(L), ctypes.POINTER(D), ctypes.POINTER(D), I, I, P, ctypes.POINTER(P)],
        "whv_destroy_grid": [P],
        "whv_set_speed": [P, P],
        "whv_time_grid": [P, ctypes.POINTER(whv_params), ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)],
        "whv_set_deflation_basis": [P, ctypes.POINTER(whv_params), I, P, ctypes.POINTER(D), I, I],
        "whv_get_basis": [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), P],
        "whv_apply_pi": [P, ctypes.POINTER(whv_params), P, P, P],
        "whv_solve": [P, ctypes.POINTER(whv_params), P, I, P, ctypes.POINTER(whv_info)],
        "whv_project": [P, P, P],
        "whv_expand": [P, P, D, P],
        "whv_dot": [P, P, P, ctypes.POINTER(D)],
        "whv_set_steps_per_sweep": [P, I],
        "whv_get_steps_per_sweep": [P, ctypes.POINTER(I)],
        "whv_autotune": [P, ctypes.POINTER(whv_params), ctypes.POINTER(I)],
        "whv_project_noalloc": [L, I, P, P, P, P, P],
        "whv_lanczos": [P, ctypes.POINTER(whv_params), I, I, P, I, I, ctypes.POINTER(D), ctypes.POINTER(D)],
        "whv_solve_adjoint": [P, ctypes.POINTER(whv_params), P, P, P, P, P, P, I, ctypes.POINTER(whv_info)],
        "whv_inject_barrier_error": [P],
        "whv_compress_basis": [P, D, ctypes.POINTER(I)],
        "whv_set_speed_form": [P, P, I],
        "whv_solve_many": [P, ctypes.POINTER(whv_params), I, L, P, I, P, ctypes.POINTER(whv_info)],
        "whv_autotune_batched": [I, ctypes.POINTER(P), ctypes.POINTER(whv_params), ctypes.POINTER(I)],
        "whv_lanczos_restarted": [P, ctypes.POINTER(whv_params), I, I, I, I, D, P, I, I, ctypes.POINTER(D),
                                  ctypes.POINTER(D), ctypes.POINTER(I)],
        "whv_solve_batched": [I, ctypes.POINTER(P), ctypes.POINTER(whv_params), ctypes.POINTER(P),
                              ctypes.POINTER(P), ctypes.POINTER(whv_info)],
        "whv_apply_pi_batched": [I, ctypes.POINTER(P), ctypes.POINTER(whv_params), ctypes.POINTER(P),
                                 ctypes.POINTER(P), ctypes.POINTER(P)],
        "whv_share_basis": [P, P],
        "whv_apply_pi_vjp": [P, ctypes.POINTER(whv_params), P, P, P, P, P, P, I],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.whv_num_unknowns.argtypes = [P]
    lib.whv_num_unknowns.restype = L
    lib.whv_last_error.argtypes = [P]
    lib.whv_last_error.restype = ctypes.c_char_p
    lib.whv_kernel_launches.argtypes = []
    lib.whv_kernel_launches.restype = L
    lib.whv_version.argtypes = []
    lib.whv_version.restype = ctypes.c_char_p
    return lib


lib = _load()

# every symbol include/whv.h declares (checked by the CPU tests)
EXPORTED = ["whv_create_grid", "whv_destroy_grid", "whv_set_speed", "whv_time_grid",
            "whv_set_deflation_basis", "whv_get_basis", "whv_apply_pi", "whv_solve", "whv_project",
            "whv_expand", "whv_dot", "whv_num_unknowns", "whv_last_error", "whv_version",
            "whv_kernel_launches", "whv_set_steps_per_sweep", "whv_get_steps_per_sweep", "whv_autotune",
            "whv_project_noalloc", "whv_lanczos", "whv_solve_adjoint", "whv_solve_batched",
            "whv_inject_barrier_error", "whv_compress_basis", "whv_lanczos_restarted", "whv_set_speed_form",
            "whv_solve_many", "whv_autotune_batched", "whv_apply_pi_batched", "whv_share_basis",
            "whv_apply_pi_vjp"]


def _check(status, handle=None, allow=()):
    if status != WHV_OK and status not in allow:
        raise WhvError(status, lib.whv_last_error(handle).decode())
    return status


def _ptr(t, numel=None):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def make_params(omega, periods=1, adjust_omega=False, cfl=0.0, method="cg", restart=30, tol=1e-8,
                maxit=1000, check_every=1, true_residual=False, refine_fp64=False, inner_tol=0.0,
                residual_df64=False) -> whv_params:
    m = METHODS[method] if isinstance(method, str) else int(method)
    flags = ((WHV_TRUE_RESIDUAL if true_residual else 0) | (WHV_REFINE_FP64 if refine_fp64 else 0)
             | (WHV_RESIDUAL_DF64 if residual_df64 else 0))
    return whv_params(float(omega), int(periods), int(bool(adjust_omega)), float(cfl), m, int(restart),
                      float(tol), int(maxit), int(check_every), flags, float(inner_tol))


def whv_version() -> str:
    return lib.whv_version().decode()


def whv_project_noalloc(W, r, coef, w=None, stream=None):
    """Allocation-free W^T M r: W is (nd, n) row-major (= n x nd column-major), r and w have n
    entries, coef has nd; all float64 CUDA tensors owned by the caller (see include/whv.h)."""
    nd, n = W.shape
    s = (torch.cuda.current_stream() if stream is None else stream).cuda_stream
    _check(lib.whv_project_noalloc(n, nd, _ptr(W), _ptr(r, n), _ptr(w, n) if w is not None else None,
                                   _ptr(coef, nd), ctypes.c_void_p(s)))
    return coef


def whv_solve_batched(grids, params, fs, us=None, raise_not_converged=False):
    """Batched solve (see include/whv.h): lists of Grid objects, whv_params and forcing tensors."""
    n = len(grids)
    if us is None:
        us = [torch.zeros(g.N, dtype=torch.float64, device="cuda") for g in grids]
    G = (ctypes.c_void_p * n)(*[g.handle for g in grids])
    Pm = (whv_params * n)(*params)
    F = (ctypes.c_void_p * n)(*[_ptr(f, g.N) for f, g in zip(fs, grids)])
    U = (ctypes.c_void_p * n)(*[_ptr(u, g.N) for u, g in zip(us, grids)])
    infos = (whv_info * n)()
    allow = () if raise_not_converged else (WHV_ERR_NOT_CONVERGED,)
    grids[0]._pre()
    st = _check(lib.whv_solve_batched(n, G, Pm, F, U, infos), grids[0].handle, allow)
    grids[0]._post()
    return us, [dict(i.as_dict(), status=STATUS_NAMES[st]) for i in infos]


def whv_apply_pi_batched(grids, params, vs=None, fs=None, outs=None):
    """Batched wave solve out_p = Pi_h(v_p; f_p) in one persistent launch (see include/whv.h);
    vs / fs are lists of tensors or None entries (or None for all zero)."""
    n = len(grids)
    if outs is None:
        outs = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in grids]
    G = (ctypes.c_void_p * n)(*[g.handle for g in grids])
    Pm = (whv_params * n)(*params)
    Vp = None if vs is None else (ctypes.c_void_p * n)(*[_ptr(v, g.N) for v, g in zip(vs, grids)])
    Fp = None if fs is None else (ctypes.c_void_p * n)(*[_ptr(f, g.N) for f, g in zip(fs, grids)])
    O = (ctypes.c_void_p * n)(*[_ptr(o, g.N) for o, g in zip(outs, grids)])
    grids[0]._pre()
    _check(lib.whv_apply_pi_batched(n, G, Pm, Vp, Fp, O), grids[0].handle)
    grids[0]._post()
    return outs


def whv_autotune_batched(grids, params):
    """Batched steps-per-sweep autotuner (see include/whv.h); returns the chosen k."""
    n = len(grids)
    G = (ctypes.c_void_p * n)(*[g.handle for g in grids])
    Pm = (whv_params * n)(*params)
    k = ctypes.c_int()
    grids[0]._pre()
    _check(lib.whv_autotune_batched(n, G, Pm, ctypes.byref(k)), grids[0].handle)
    return k.value


def whv_kernel_launches() -> int:
    return int(lib.whv_kernel_launches())


class Grid:
    """Owns one whv_grid.  `npts` are nodes per direction including boundary nodes (x first)."""

    def __init__(self, npts, lo=None, hi=None, order=2, precision=WHV_FP64, stream=None):
        dim = len(npts)
        n3 = (ctypes.c_int64 * 3)(*(list(npts) + [3] * (3 - dim)))
        lo3 = (ctypes.c_double * 3)(*((list(lo) if lo else [0.0] * dim) + [0.0] * (3 - dim)))
        hi3 = (ctypes.c_double * 3)(*((list(hi) if hi else [1.0] * dim) + [1.0] * (3 - dim)))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.whv_create_grid(dim, n3, lo3, hi3, order, precision, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self.handle = h
        self.dim, self.npts, self.order, self.precision = dim, tuple(npts), order, precision
        self.shape = tuple(int(n) - 2 for n in reversed(list(npts)))
        self.N = int(lib.whv_num_unknowns(h))

    # Stream ordering: the library works on self.stream.  Before a call the grid's stream waits for
    # the caller's current stream (inputs written there are complete); after an asynchronous call the
    # caller's stream waits for the grid's (outputs are complete before torch reads them).
    def _pre(self):
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _post(self):
        cur = torch.cuda.current_stream()
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def close(self):
        if getattr(self, "handle", None):
            lib.whv_destroy_grid(self.handle)
            self.handle = None

    __del__ = close

    def whv_set_speed(self, c2):
        self._pre()
        _check(lib.whv_set_speed(self.handle, _ptr(c2, self.N)), self.handle)

    def whv_solve_many(self, params, F, U=None, use_guess=False, raise_not_converged=False):
        """F: (nrhs, N) float64 CUDA tensor (row j = right-hand side j); returns (U, infos)."""
        nrhs = F.shape[0]
        if U is None:
            U = torch.zeros_like(F)
        infos = (whv_info * max(nrhs, 1))()
        self._pre()
        allow = () if raise_not_converged else (WHV_ERR_NOT_CONVERGED,)
        st = _check(lib.whv_solve_many(self.handle, ctypes.byref(params), int(nrhs), int(F.stride(0)), _ptr(F),
                                       int(bool(use_guess)), _ptr(U), infos), self.handle, allow)
        self._post()
        return U, [dict(infos[j].as_dict(), status=STATUS_NAMES[st]) for j in range(nrhs)]

    def whv_set_speed_form(self, c2, form):
        self._pre()
        _check(lib.whv_set_speed_form(self.handle, _ptr(c2, self.N), int(form)), self.handle)

    def whv_time_grid(self, params):
        nt, dt, oh, oe = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib.whv_time_grid(self.handle, ctypes.byref(params), ctypes.byref(nt), ctypes.byref(dt),
                                 ctypes.byref(oh), ctypes.byref(oe)), self.handle)
        return {"nt": nt.value, "dt": dt.value, "omega_hat": oh.value, "omega_eff": oe.value}

    def whv_set_deflation_basis(self, params, nd, mode, V=None, lambda2=None, flags=0):
        self._pre()
        lam = None
        if lambda2 is not None:
            lam = (ctypes.c_double * nd)(*[float(x) for x in lambda2])
        _check(lib.whv_set_deflation_basis(self.handle, ctypes.byref(params), int(nd),
                                           _ptr(V, None if V is None else self.N * nd), lam, int(mode), int(flags)),
               self.handle)

    def whv_share_basis(self, src):
        """Use src's deflation basis (no copy; see include/whv.h)."""
        self._pre()
        _check(lib.whv_share_basis(self.handle, src.handle), self.handle)

    def whv_get_basis(self, want_vectors=False):
        nd = ctypes.c_int()
        _check(lib.whv_get_basis(self.handle, ctypes.byref(nd), None, None, None), self.handle)
        n = nd.value
        if n == 0:
            return {"nd": 0}
        modes = (ctypes.c_int * (n * self.dim))()
        lam = (ctypes.c_double * n)()
        V = torch.empty(n * self.N, dtype=torch.float64, device="cuda") if want_vectors else None
        _check(lib.whv_get_basis(self.handle, ctypes.byref(nd), modes, lam, _ptr(V)), self.handle)
        return {"nd": n, "modes": [list(modes[i * self.dim:(i + 1) * self.dim]) for i in range(n)],
                "lambda2": list(lam), "V": None if V is None else V.view(n, self.N)}

    def whv_apply_pi(self, params, v, f=None, out=None):
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        self._pre()
        _check(lib.whv_apply_pi(self.handle, ctypes.byref(params), _ptr(v, self.N), _ptr(f, self.N), _ptr(out, self.N)),
               self.handle)
        self._post()
        return out

    def whv_solve(self, params, f, u=None, use_guess=False, raise_not_converged=False):
        if u is None:
            u = torch.zeros(self.N, dtype=torch.float64, device="cuda")
        info = whv_info()
        allow = () if raise_not_converged else (WHV_ERR_NOT_CONVERGED,)
        self._pre()
        st = _check(lib.whv_solve(self.handle, ctypes.byref(params), _ptr(f, self.N), int(bool(use_guess)),
                                  _ptr(u, self.N), ctypes.byref(info)), self.handle, allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[st]
        return u, d

    def whv_set_steps_per_sweep(self, k):
        _check(lib.whv_set_steps_per_sweep(self.handle, int(k)), self.handle)

    def whv_get_steps_per_sweep(self):
        k = ctypes.c_int()
        _check(lib.whv_get_steps_per_sweep(self.handle, ctypes.byref(k)), self.handle)
        return k.value

    def whv_lanczos_restarted(self, params, nd, m, max_restarts=50, tol=1e-9, v0=None, fp64_stepping=True,
                              flags=0, keep=0):
        """Thick-restart Lanczos; returns (theta, resid, {restarts, wave_solves, converged})."""
        self._pre()
        theta = (ctypes.c_double * nd)()
        resid = (ctypes.c_double * nd)()
        st = (ctypes.c_int * 3)()
        _check(lib.whv_lanczos_restarted(self.handle, ctypes.byref(params), int(nd), int(m), int(keep),
                                         int(max_restarts), float(tol), _ptr(v0, self.N), int(bool(fp64_stepping)),
                                         int(flags), theta, resid, st), self.handle)
        return list(theta), list(resid), {"restarts": st[0], "wave_solves": st[1], "converged": st[2]}

    def whv_compress_basis(self, tau):
        """SVD-compress the basis (2-D); returns the rank of every vector."""
        self._pre()
        nd = self.whv_get_basis()["nd"]
        ranks = (ctypes.c_int * max(nd, 1))()
        _check(lib.whv_compress_basis(self.handle, float(tau), ranks), self.handle)
        return [ranks[i] for i in range(nd)]

    def whv_inject_barrier_error(self):
        _check(lib.whv_inject_barrier_error(self.handle), self.handle)

    def whv_autotune(self, params):
        k = ctypes.c_int()
        _check(lib.whv_autotune(self.handle, ctypes.byref(params), ctypes.byref(k)), self.handle)
        return k.value

    def whv_lanczos(self, params, nd, m, v0=None, fp64_stepping=True, flags=WHV_BASIS_REDEFLATE):
        self._pre()
        theta = (ctypes.c_double * nd)()
        resid = (ctypes.c_double * nd)()
        _check(lib.whv_lanczos(self.handle, ctypes.byref(params), int(nd), int(m), _ptr(v0, self.N),
                               int(bool(fp64_stepping)), int(flags), theta, resid), self.handle)
        return list(theta), list(resid)

    def whv_solve_adjoint(self, params, f, u, dLdu, want_c2=True, want_f=True, checkpoint_every=16,
                          raise_not_converged=False):
        z = torch.empty(self.N, dtype=torch.float64, device="cuda")
        gc2 = torch.empty_like(z) if want_c2 else None
        gf = torch.empty_like(z) if want_f else None
        info = whv_info()
        allow = () if raise_not_converged else (WHV_ERR_NOT_CONVERGED,)
        self._pre()
        st = _check(lib.whv_solve_adjoint(self.handle, ctypes.byref(params), _ptr(f, self.N), _ptr(u, self.N),
                                          _ptr(dLdu, self.N), _ptr(z, self.N), _ptr(gc2), _ptr(gf),
                                          int(checkpoint_every), ctypes.byref(info)), self.handle, allow)
        d = info.as_dict()
        d["status"] = STATUS_NAMES[st]
        return z, gc2, gf, d

    def whv_apply_pi_vjp(self, params, v, f, abar, want_v=True, want_c2=True, want_f=True, checkpoint_every=16):
        """(vbar, c2bar, fbar) = the VJP of Pi_h(v; f, c^2) for the seed abar (see include/whv.h)."""
        self._pre()
        mk = lambda want: torch.empty(self.N, dtype=torch.float64, device="cuda") if want else None  # noqa: E731
        vb, cb, fb = mk(want_v), mk(want_c2), mk(want_f)
        _check(lib.whv_apply_pi_vjp(self.handle, ctypes.byref(params), _ptr(v, self.N), _ptr(f, self.N),
                                    _ptr(abar, self.N), _ptr(vb, self.N), _ptr(cb, self.N), _ptr(fb, self.N),
                                    int(checkpoint_every)), self.handle)
        self._post()
        return vb, cb, fb

    def whv_project(self, r, coef):
        self._pre()
        _check(lib.whv_project(self.handle, _ptr(r, self.N), _ptr(coef)), self.handle)
        self._post()
        return coef

    def whv_expand(self, y, alpha, out):
        self._pre()
        _check(lib.whv_expand(self.handle, _ptr(y), float(alpha), _ptr(out, self.N)), self.handle)
        self._post()
        return out

    def whv_dot(self, x, y):
        self._pre()
        out = ctypes.c_double()
        _check(lib.whv_dot(self.handle, _ptr(x, self.N), _ptr(y, self.N), ctypes.byref(out)), self.handle)
        return out.value


class WaveHoltzSolve(torch.autograd.Function):
    """u = WaveHoltz fixed point for forcing f and squared speed c2 on `grid` (whv_set_speed +
    whv_solve); backward runs whv_solve_adjoint and returns dL/df and dL/dc2."""

    @staticmethod
    def forward(ctx, f, c2, grid, params, checkpoint_every=16):
        grid.whv_set_speed(c2.detach().contiguous())
        u, info = grid.whv_solve(params, f.detach().contiguous(), raise_not_converged=True)
        ctx.grid, ctx.params, ctx.K = grid, params, checkpoint_every
        ctx.save_for_backward(f, c2, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        f, c2, u = ctx.saved_tensors
        g = ctx.grid
        g.whv_set_speed(c2.detach().contiguous())
        _, gc2, gf, _ = g.whv_solve_adjoint(ctx.params, f.detach().contiguous(), u.contiguous(),
                                            grad_u.contiguous(), want_c2=ctx.needs_input_grad[1],
                                            want_f=ctx.needs_input_grad[0], checkpoint_every=ctx.K,
                                            raise_not_converged=True)
        return gf, gc2, None, None, None
