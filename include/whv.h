/*
 * whv.h -- C ABI of the B300 WaveHoltz library (eigenvector-deflated WaveHoltz).
 *
 * The library solves the discrete Helmholtz problem  L_h U + omega^2 U = f  with homogeneous
 * Dirichlet boundary nodes (Sec. 2.1 eq. helmholtzBVP, Sec. 2.2 eq. discreteHelmholtz) as the
 * fixed point of the WaveHoltz map Pi_h (eq. waveHoltzFilter, eq. quadrature), i.e. the linear
 * system A u = (I - S_h) u = b, b = Pi_h 0 (eq. WaveHoltzMatrixEquation), accelerated by
 * Krylov methods and eigenvector deflation (Algorithm 2, Algorithm 4).
 *
 * Conventions shared by every entry point
 *  - A grid function lives on the INTERIOR nodes only, in FP64, contiguous with x fastest:
 *    element (i, j, k) is at i + nx*(j + ny*k), nx = npts[0]-2, ny = npts[1]-2, nz = npts[2]-2.
 *    Boundary nodes are not stored (their value is 0).
 *  - Pointers named *_dev are DEVICE pointers owned by the caller; they must stay valid until the
 *    call's work on the grid's stream has completed.  Pointers named *_host are host memory.
 *  - All work is ordered on the CUDA stream given to whv_create_grid.  Calls that return
 *    host values (whv_solve's info, whv_dot, whv_get_basis) synchronise that stream.
 *  - Every call returns a whv_status and never aborts; on failure whv_last_error(grid) holds a
 *    one-line reason.  A grid is not thread-safe: one host thread at a time per grid.
 *  - L_h = c^2(x) Delta_{p,h}: the squared speed multiplies the p-th order (p = 2 or 4) discrete
 *    Laplacian (reading of eq. L for variable speed).  Inner products and norms are weighted by
 *    M = diag(1/c^2), in which A is self-adjoint (the diagonal mass-matrix symmetrisation of
 *    Sec. 4.1); for c = 1 they are Euclidean.
 */
#ifndef WHV_H
#define WHV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct whv_grid_s* whv_grid;

typedef enum {
  WHV_OK = 0,
  WHV_ERR_INVALID = 1,        /* bad argument, size, or state (e.g. dt above the stability limit) */
  WHV_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  WHV_ERR_OOM = 3,            /* device allocation failed */
  WHV_ERR_NOT_CONVERGED = 4,  /* maxit reached; the best iterate is returned */
  WHV_ERR_BREAKDOWN = 5,      /* non-finite or non-positive Krylov scalar (NaN/Inf input, indefinite A) */
  WHV_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up */
} whv_status;

/* precision of the wave stepping (the Krylov / deflation arithmetic is always FP64) */
enum { WHV_FP64 = 0, WHV_FP32_STEP = 1 };

/* accelerators */
enum {
  WHV_FPI = 0,    /* Algorithm 1, fixed-point iteration                              */
  WHV_CG = 1,     /* conjugate gradients on A u = b                                   */
  WHV_DCG = 2,    /* Algorithm 4, deflated CG (needs a basis)                         */
  WHV_GMRES = 3,  /* restarted GMRES(m), classical Gram-Schmidt applied twice         */
  WHV_AGMRES = 4, /* Algorithm 5, augmented GMRES(m): the grid's basis W augments the
                     Krylov space (A W = V_p H_p by a thin QR kept with the basis; for a
                     WHV_BASIS_EXACT basis A W = W diag(1 - beta_h), else one wave solve per
                     column); the forcing is not deflated; no basis = GMRES(m)              */
  WHV_ABICGSTAB = 5 /* Algorithm 6, augmented BiCGStab: BiCGStab on the system projected
                     away from range(A W) (same QR as AGMRES), x -= W R^{-1} xi at the end;
                     two wave solves per iteration; no basis = BiCGStab                    */
};

/* form of the variable-speed operator (whv_set_speed_form) */
enum {
  WHV_SPEED_NONCONSERVATIVE = 0,  /* L_h = c^2 Delta_h (any order), inner products <u,v>_M, M = 1/c^2 */
  WHV_SPEED_CONSERVATIVE = 1      /* L_h = div_h(c^2 grad_h) (eq. L, second order), Euclidean      */
};

/* origin of the deflation basis (whv_set_deflation_basis) */
enum {
  WHV_BASIS_NONE = 0,         /* remove the basis                                          */
  WHV_BASIS_USER = 1,         /* copy caller vectors V_dev and eigenvalues lambda2_host    */
  WHV_BASIS_CLOSED_FORM = 2,  /* sine tensor products of the box (Sec. 4.3), c = 1 only     */
  WHV_BASIS_LANCZOS = 3       /* computed on the device by a Krylov eigen-solve on S_h     */
};
/* basis flags */
enum {
  WHV_BASIS_EXACT = 1,        /* columns are true eigenvectors: A W = W diag(1 - beta_h)  */
  WHV_BASIS_REDEFLATE = 2     /* project every operator output onto span(V)^perp (Algorithm 2, deflate iterate) */
};
/* whv_params.flags */
enum {
  WHV_TRUE_RESIDUAL = 1,      /* at exit compute ||Pi_h(u;f) - u|| / ||Pi_h(0;f)|| (2 extra wave solves,
                                 in FP64 when the grid steps in FP64 or WHV_REFINE_FP64 is set)       */
  WHV_REFINE_FP64 = 2,        /* iterative refinement on the full system b = Pi_h(0; f): the residual
                                 r = b - A x is formed with FP64 wave solves; each correction is the
                                 modal solve of r's deflated components (W diag(1/mu) W^T M r) plus a
                                 Krylov solve of the rest in the grid's stepping precision (the first
                                 to relative tolerance inner_tol, later ones to half the remaining
                                 gap to tol); repeated until the FP64 residual meets tol.
                                 Lets FP32 stepping reach FP64 residuals and corrects approximate
                                 (Lanczos) eigenvectors.  Needs a Krylov method (DCG, AGMRES and
                                 ABICGSTAB use the basis themselves: no modal step); allocates 3 (FP64
                                 grids) or 8 (FP32 grids) more N-vectors of FP64 on first use.       */
  WHV_RESIDUAL_DF64 = 4       /* with WHV_REFINE_FP64 on grids with the operator c^2 Delta_h (order 2
                                 or 4; batched solves: 2-D, order 2, c = 1, else FP64): the b and
                                 residual wave solves of the correction run in double-float
                                 arithmetic -- each value a pair of FP32 numbers, ~48-bit significand,
                                 error-free two-sum / two-product on the FP32 pipes -- instead of FP64
                                 (B300's FP64 rate is 1/64 of FP32).  Enough for tolerances down to
                                 ~1e-10 relative; WHV_TRUE_RESIDUAL still checks in FP64.          */
};

typedef struct {
  double omega;       /* frequency omega > 0                                                       */
  int periods;        /* filter interval Tbar = periods * 2 pi / omega (N_p >= 1)                 */
  int adjust_omega;   /* 1: use omega_hat with (2/dt) sin(omega_hat dt/2) = omega so that the
                         fixed point solves the Helmholtz problem at omega exactly (Sec. 2.2);
                         0: dt = Tbar/ceil(Tbar/dt0) and the fixed point is at omega_eff        */
  double cfl;         /* dt0 = cfl * h_min / c_max; <= 0 selects 0.5 (order 2) or 0.4 (order 4)  */
  int method;         /* WHV_FPI | WHV_CG | WHV_DCG | WHV_GMRES | WHV_AGMRES | WHV_ABICGSTAB      */
  int restart;        /* (A)GMRES restart length m (Arnoldi steps per cycle); <= 0 selects 30     */
  double tol;         /* stop when ||r||_M <= tol ||b||_M of the iterated system                  */
  int maxit;          /* maximum operator applications in the iteration                          */
  int check_every;    /* test convergence every k iterations (CG/FPI); <= 0 selects 1             */
  int flags;          /* WHV_TRUE_RESIDUAL | WHV_REFINE_FP64 | WHV_RESIDUAL_DF64                  */
  double inner_tol;   /* WHV_REFINE_FP64: relative tolerance of the first correction solve (later
                         ones aim at half the remaining gap to tol, at most 10 times tighter);
                         <= 0: 1e-3 */
} whv_params;

typedef struct {
  int iterations;            /* accelerator iterations                                          */
  int wave_solves;           /* applications of Pi_h, including b and the true residual         */
  int nt;                    /* time steps per wave solve                                       */
  double dt, omega_hat, omega_eff;
  double rel_residual;       /* last recursive relative residual of the iterated system         */
  double true_rel_residual;  /* WHV_TRUE_RESIDUAL result, else -1                               */
  double seconds;            /* host wall time of the call                                      */
  int outer_iterations;      /* WHV_REFINE_FP64 corrections (0 otherwise)                        */
  int wave_solves_fp64;      /* wave solves stepped in FP64 (all of them on an FP64 grid)        */
} whv_info;

/* Create a box grid [lo, hi] (per direction, x first) with npts nodes per direction including
 * both boundary nodes (npts >= 3; npts >= 4 for order 4), dim = 1, 2 or 3 (entries beyond dim are
 * ignored), order = 2 or 4 (centred Cartesian stencils, Sec. 2.2; order 4 closes at the boundary
 * by odd reflection of the first interior value), precision = WHV_FP64 or WHV_FP32_STEP.
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Allocates the grid's own
 * device scratch (stepping buffers, Krylov vectors); the grid owns it until whv_destroy_grid. */
whv_status whv_create_grid(int dim, const int64_t npts[3], const double lo[3], const double hi[3],
                           int order, int precision, void* cuda_stream, whv_grid* out);
whv_status whv_destroy_grid(whv_grid grid);

/* Squared wave speed c^2 on the interior nodes (copied; the caller may free its buffer after
 * the call completes on the stream).  c2_dev = NULL restores c = 1.  Any existing deflation basis
 * is dropped.  Requires c^2 > 0 (checked). */
whv_status whv_set_speed(whv_grid grid, const double* c2_dev);

/* Squared speed with the operator form: WHV_SPEED_NONCONSERVATIVE is whv_set_speed;
 * WHV_SPEED_CONSERVATIVE (second-order grids) makes L_h = div_h(c^2 grad_h) u (eq. L): per axis
 * (c^2_{j+1/2} (u_{j+1} - u_j) - c^2_{j-1/2} (u_j - u_{j-1})) / h^2, face values the mean of the
 * two nodes' c^2 (the adjacent interior value on the faces to the boundary nodes).  This operator
 * is symmetric in the Euclidean inner product, which all Krylov and deflation products then use.
 * Its wave solves run one step per launch (the blocked and single-CTA kernels are bypassed); whv_solve_batched and whv_solve_adjoint refuse such grids.  Extra device memory:
 * dim N doubles + dim N floats of face values. */
whv_status whv_set_speed_form(whv_grid grid, const double* c2_dev, int form);

/* Time grid the given parameters select (reading of Sec. 2.2): nt steps of dt over Tbar,
 * cos/filter frequency omega_hat, fixed-point frequency omega_eff.  Host outputs, any may be NULL.
 * Returns WHV_ERR_INVALID if dt is above the explicit leapfrog stability limit. */
whv_status whv_time_grid(whv_grid grid, const whv_params* p, int* nt, double* dt,
                         double* omega_hat, double* omega_eff);

/* Set the deflation basis W (N x nd, column-major, M-orthonormal) used by whv_solve for DEVD
 * (Algorithm 2 with FPI/CG/GMRES) and DCG (Algorithm 4), for the frequency and time grid of `p`.
 *  - WHV_BASIS_USER: V_dev (N*nd doubles) and lambda2_host (nd eigenvalues lambda^2 of -L_h)
 *    are copied.
 *  - WHV_BASIS_CLOSED_FORM: V_dev/lambda2_host ignored (may be NULL); the nd tensor-product sine
 *    modes with the smallest |1 - beta_h(lambda)| (ties: mode tuple (kx,ky,kz) ascending) are
 *    generated on the device (Sec. 2.3 choice of the deflation set; Sec. 4.3 eigenvectors).
 *    Requires c = 1.  Implies WHV_BASIS_EXACT.
 *  - WHV_BASIS_LANCZOS: eigenpairs computed on the device by whv_lanczos with m = min(N, 1024,
 *    max(4 nd, nd + 40)) steps, FP64 stepping, V_dev = the start vector (N doubles) or NULL for
 *    the built-in one; implies WHV_BASIS_REDEFLATE, never WHV_BASIS_EXACT.
 *  - WHV_BASIS_NONE: drop the basis.
 * flags: WHV_BASIS_EXACT, WHV_BASIS_REDEFLATE. */
whv_status whv_set_deflation_basis(whv_grid grid, const whv_params* p, int nd, const double* V_dev,
                                   const double* lambda2_host, int mode, int flags);

/* Device eigen-solve for the deflation basis (EigenWave idea, Sec. 4.1: a Krylov method on the
 * WaveHoltz operator finds the eigenvectors of L_h whose beta_h is nearest 1 as its extremal Ritz
 * pairs).  Runs m Lanczos steps on S_h (one f = 0 wave solve each, FP64 stepping if
 * fp64_stepping else the grid's precision) in the M inner product from v0_dev (N doubles, device;
 * NULL: a built-in SplitMix64 pseudo-random vector), with full FP64 re-orthogonalisation
 * (classical Gram-Schmidt twice), takes the nd largest Ritz values of the tridiagonal matrix, forms
 * the Ritz vectors on the device and computes lambda^2 = -<y, L_h y>_M / <y, y>_M in FP64.  The
 * vectors (M-orthonormal) become the grid's deflation basis for p's frequency and time grid, mode
 * WHV_BASIS_LANCZOS with `flags` (WHV_BASIS_EXACT is removed: they are approximate; pass
 * WHV_BASIS_REDEFLATE to re-deflate operator outputs, Algorithm 2).  theta_host / resid_host
 * (nd doubles each, may be NULL) receive the Ritz values (descending) and ||L_h y + lambda^2 y||_M /
 * lambda^2.  Needs 1 <= nd <= m <= min(N, 1024); temporary device memory m N doubles.  Exactly
 * degenerate eigenvalues (square grids with c = 1) yield one vector per eigenspace: use the closed
 * form there. */
whv_status whv_lanczos(whv_grid grid, const whv_params* p, int nd, int m, const double* v0_dev,
                       int fp64_stepping, int flags, double* theta_host, double* resid_host);

/* Thick-restart Lanczos (Wu and Simon 2000) for the same basis when nd is large: the Krylov basis
 * holds at most m vectors; when it is full, the Ritz pairs of the projected matrix (filled from the
 * FP64 re-orthogonalisation coefficients, dense symmetric eigen-solve on the host by Householder
 * reduction, bisection and inverse iteration) are tested -- the residual of pair i is |b s_{m,i}|,
 * b the norm of the next, unnormalised Lanczos vector -- and unless the nd largest are below tol
 * (on the scale of S_h's eigenvalues, which lie in (-1, 1]) the `keep` largest Ritz vectors and the
 * residual vector restart the basis (keep <= 0: nd + max(nd/2, 8), capped at m - 2).  At most
 * max_restarts restarts.  The nd Ritz vectors become the grid's WHV_BASIS_LANCZOS basis as with
 * whv_lanczos; stats_host (3 ints, may be NULL) receives {restarts, wave solves, converged pairs}.
 * Needs 1 <= nd <= keep <= m - 2, m <= min(N, 1024), tol > 0; temporary device memory
 * (m + keep + nd) N doubles. */
whv_status whv_lanczos_restarted(whv_grid grid, const whv_params* p, int nd, int m, int keep, int max_restarts,
                                 double tol, const double* v0_dev, int fp64_stepping, int flags,
                                 double* theta_host, double* resid_host, int* stats_host);

/* Share src's deflation basis with dst (no copy of the vectors): the many-right-hand-side use of
 * one eigenvector set (Sec. 4.1: the set-up is paid once and amortised over all forcings).  dst
 * takes src's vectors, eigenvalues, mode tuples, flags and the frequency / time grid they were
 * built for; the vector storage is reference-counted and freed with the last grid that uses it,
 * so either grid may be destroyed or get a new basis later.  Both grids must have the same box,
 * node counts, order and speed: both c = 1, or both the same c^2 (compared bit for bit on the
 * device; the basis is M-orthonormal for that c^2); conservative-form grids cannot share.  src
 * needs a dense basis (not SVD-compressed).  What a grid derives from its basis for Algorithm 4
 * (A W) or Algorithm 5 (the QR of A W) stays per grid.  whv_solve_batched contracts the
 * problems that share one basis together: each deflation projection W^T M [r_1 ... r_k] and
 * expansion [u_1 ... u_k] += W Y reads W once.  Allocates nd doubles of scratch in dst;
 * synchronises both grids' streams. */
whv_status whv_share_basis(whv_grid dst, whv_grid src);

/* Read back the basis: nd (host), the mode tuples (host int[nd*dim], closed form only; else
 * zeros), lambda^2 (host double[nd]) and the vectors (device double[N*nd]); any output may be NULL. */
whv_status whv_get_basis(whv_grid grid, int* nd, int* modes_host, double* lambda2_host, double* V_dev);

/* out = Pi_h(v; f): one wave solve (eq. discreteWaveExplicit from W^0 = v, D0t W^0 = 0, forcing
 * -f cos(omega_hat t)) filtered by the trapezoid rule (eq. quadrature).  f_dev = NULL means f = 0,
 * i.e. out = S_h v.  v_dev and out_dev may alias. */
whv_status whv_apply_pi(whv_grid grid, const whv_params* p, const double* v_dev, const double* f_dev,
                        double* out_dev);

/* Solve A u = b for forcing f (b = Pi_h(0; f)) with p->method.  With a basis set and method
 * FPI / CG / GMRES this is DEVD (Algorithm 2): f_d = f - W W^T M f, solve with b = Pi_h(0; f_d),
 * inflate u += W diag(1/(omega_eff^2 - lambda^2)) W^T M f.  With WHV_DCG it is Algorithm 4 on
 * b = Pi_h(0; f).  With WHV_REFINE_FP64 on an FP32-stepping grid the iteration is wrapped in
 * FP64 residual correction (see the flag), and rel_residual is the FP64 one.  use_guess = 1: u_dev holds the initial guess x0 on entry (DEVD projects it
 * onto span(W)^perp first); use_guess = 0: x0 = 0 and u_dev is only written.  On exit u_dev holds
 * the solution.  info (host, may be NULL) receives counts and residuals.
 * Returns WHV_ERR_NOT_CONVERGED (solution still written) if maxit is reached. */
whv_status whv_solve(whv_grid grid, const whv_params* p, const double* f_dev, int use_guess,
                     double* u_dev, whv_info* info);

/* Steps per sweep k of the temporally blocked 2-D stencil kernel: each launch advances k leapfrog
 * steps of the f = 0 wave solves in shared memory (halo of width k r).  k = 1 launches one kernel
 * per time step, k = 0 restores the default (8 for FP32 stepping, 1 for FP64), 0 <= k <= 16.  2-D
 * grids block k steps; 3-D second-order constant-speed FP32 grids take any k >= 2 as two steps per
 * launch (z-marching, W^{n+1} staged plane by plane); other grids step once per launch.  With the
 * default (k = 0) grids of at
 * most 4096 unknowns run each whole wave solve in a single CTA (state in shared memory, one
 * barrier per step); an explicit k turns that off.  Other values: WHV_ERR_INVALID.
 * whv_get_steps_per_sweep returns the value in effect (0 on the small grids above). */
whv_status whv_set_steps_per_sweep(whv_grid grid, int k);
whv_status whv_get_steps_per_sweep(whv_grid grid, int* k);

/* Autotuner: times f = 0 wave solves of p's time grid for each candidate steps-per-sweep value
 * (1, 2, 4, 6, 8, 10, 12, 16 on 2-D grids, 1 and 2 on 3-D constant-speed FP32 grids; small
 * grids keep the single-CTA solve, *best = 0) with CUDA events on the grid's stream and
 * keeps the fastest; *best (host, may be NULL) receives it.  Overwrites the grid's internal work vectors,
 * synchronises the stream.  Must not be called while the grid's stream is being captured. */
whv_status whv_autotune(whv_grid grid, const whv_params* p, int* best);

/* Several right-hand sides on one grid (the multi-right-hand-side use that amortises the
 * eigenvector set-up, Sec. 4.1): column j of F_dev (N doubles at F_dev + j ld, device) is solved
 * into U_dev + j ld exactly as whv_solve(grid, p, ., use_guess, ., infos + j) would; the basis and
 * everything built from it (A W, QR factors, captured graphs, the device CG loop) is reused.
 * With DEVD on a dense basis (FPI / CG / GMRES; no WHV_REFINE_FP64, no WHV_TRUE_RESIDUAL,
 * use_guess = 0, nrhs > 1) the deflation of Algorithm 2 is done for all columns at once: the
 * projection W^T M F, the deflated forcings F - W C (written into U_dev, whose columns then
 * receive the solutions in place) and the inflation each read W once for all columns; temporary
 * device memory nd (nrhs + 1) + ceil(N / 512) nd nrhs doubles.  Results equal the column-by-column
 * solves up to rounding.  infos (host, nrhs entries) may be NULL.  ld >= N; F_dev and U_dev must not
 * overlap.  Returns WHV_ERR_NOT_CONVERGED if a column missed its tolerance (all columns are still
 * solved), any other error at once. */
whv_status whv_solve_many(whv_grid grid, const whv_params* p, int nrhs, int64_t ld, const double* F_dev,
                          int use_guess, double* U_dev, whv_info* infos);

/* Adjoint of the solve (differentiation path): gradients of L = 1/2 ||u - u_obs||^2 with respect
 * to the forcing and the squared speed.  u_dev is the fixed point of Pi_h(.; f_dev) that whv_solve
 * returned for the same p, f_dev the forcing used (NULL = 0), dLdu_dev = dL/du (e.g. u - u_obs).
 *  - z_dev (out): lambda solving (I - S_h)^T lambda = dL/du, by the M-similarity
 *    S_h^T = M S_h M^{-1} (M = diag(1/c^2), Sec. 4.1): (I - S_h) y = c^2 dL/du is solved with
 *    p->method (CG, DCG or GMRES; the grid's basis deflates as in whv_solve; WHV_REFINE_FP64 gives
 *    FP64 residual correction), lambda = y / c^2.
 *  - grad_c2_dev (out, nullable): dL/dc^2 = lambda^T dPi_h(u; f, c^2)/dc^2;
 *    grad_f_dev (out, nullable): dL/df = lambda^T dPi_h/df.  Both by one reverse sweep of the
 *    wave solve from u (leapfrog transposed step by step, filter weights as source, FP64
 *    accumulation), with the forward states checkpointed every `checkpoint_every` steps (<= 0: 16)
 *    and recomputed per segment; temporary device memory (2 ceil(Nt/K) + K + 5) N elements.  The
 *    sweep steps in the grid's precision, or in FP64 when p->flags has WHV_REFINE_FP64.
 * The time grid (dt, Nt) is held fixed.  All device buffers N doubles, caller-owned. */
whv_status whv_solve_adjoint(whv_grid grid, const whv_params* p, const double* f_dev, const double* u_dev,
                             const double* dLdu_dev, double* z_dev, double* grad_c2_dev,
                             double* grad_f_dev, int checkpoint_every, whv_info* info);

/* Vector-Jacobian product of out = Pi_h(v; f, c^2) -- the reverse (transposed) sweep of one wave
 * solve on its own, the building block of whv_solve_adjoint (eq. discreteWaveExplicit and
 * eq. quadrature transposed step by step).  For the seed abar_dev (N doubles):
 *  - vbar_dev  (out, nullable) = S_h^T abar, by S_h^T = M S_h M^{-1} (M = diag(1/c^2)): one forward
 *    wave solve of c^2 abar, divided by c^2;
 *  - c2bar_dev (out, nullable) = abar^T dPi_h(v; f, c^2)/dc^2 and fbar_dev (out, nullable) =
 *    abar^T dPi_h/df: the leapfrog run backwards from the filter weights times abar, with the
 *    forward states from v checkpointed every checkpoint_every (<= 0: 16) steps and recomputed
 *    per segment; temporary device memory (2 ceil(Nt/K) + K + 5) N elements.
 * Steps in the grid's precision, or in FP64 when p->flags has WHV_REFINE_FP64 (FP32 grids; the
 * gradient sums are FP64 either way).  f_dev NULL = 0.  vbar_dev must not alias v_dev or abar_dev.
 * The time grid (dt, Nt) is held fixed.  Synchronises the grid's stream. */
whv_status whv_apply_pi_vjp(whv_grid grid, const whv_params* p, const double* v_dev, const double* f_dev,
                            const double* abar_dev, double* vbar_dev, double* c2bar_dev, double* fbar_dev,
                            int checkpoint_every);

/* Batched solve of nprob (<= 1024) independent problems (right-hand sides, frequencies, grids of uneven
 * size): problem p is grids[p] with params[p] and forcing f_dev[p] (N_p doubles, device), its
 * solution goes to u_dev[p].  Every problem needs its own grid object; all grids share one
 * stream, precision, dimension (2 or 3), order and speed kind (all c = 1 or all variable).
 * Method WHV_CG only; a grid's basis, if set, must be exact eigenvectors for params[p] (DEVD,
 * Algorithm 2).  All problems iterate together: each batched wave solve (b, or q = A p of every
 * active problem) is ONE persistent cooperative kernel launch -- 2-D grids advance k leapfrog
 * steps per sweep in shared-memory tiles (k = the first grid's whv_set_steps_per_sweep value, else
 * 8 in FP32 / 4 in FP64, halved for order 4), 3-D grids one step per sweep, with a grid barrier
 * between sweeps.  The CG loop is one CUDA graph with a conditional WHILE node that runs until
 * every problem has converged or hit its maxit.
 * WHV_REFINE_FP64 in params[].flags (all problems or none) adds FP64 residual correction: b and
 * r = b - A u of the full system come from FP64 batched wave solves, the deflated components of r
 * are solved modally and the rest by the batched CG loop (first pass to params[p].inner_tol, default
 * 1e-3; later passes to half the remaining gap to tol),
 * repeated until each problem's FP64 residual ||b - A u|| / ||b|| <= tol (reported in
 * true_rel_residual).  Without it infos report the recursive residual of the deflated system and
 * true_rel_residual = -1.  Temporary device memory: the descriptor tables (a few KB); with
 * WHV_REFINE_FP64 an FP32 grid also gets its FP64 buffer set (8 N doubles, kept by the grid).
 * The grid barrier waits a bounded time: if it gives up the call returns WHV_ERR_TIMEOUT.
 * infos (host, nprob entries, may be NULL) receive per-problem counts and residuals.  Returns
 * WHV_ERR_NOT_CONVERGED if any problem missed its tolerance (all solutions still written),
 * WHV_ERR_BREAKDOWN if a problem's CG broke down. */
whv_status whv_solve_batched(int nprob, const whv_grid* grids, const whv_params* params,
                             const double* const* f_dev, double* const* u_dev, whv_info* infos);

/* Batched wave solve: out_dev[p] = Pi_h(v_dev[p]; f_dev[p]) (whv_apply_pi for every problem) in ONE
 * persistent cooperative launch -- the batched wave solve each iteration of whv_solve_batched
 * runs (2-D: k leapfrog steps per sweep in shared-memory tiles, k as in whv_solve_batched; 3-D:
 * one step per sweep; grid barriers between sweeps).  Same restrictions on the grids as
 * whv_solve_batched; v_dev / f_dev may be NULL (all zero), as may any of their entries; out_dev
 * entries are N_p doubles each and must not alias v_dev / f_dev entries.  Uses the grids'
 * stepping buffers; temporary device memory: the descriptor tables (a few KB).  Synchronises the
 * shared stream; WHV_ERR_TIMEOUT if a grid barrier gave up. */
whv_status whv_apply_pi_batched(int nprob, const whv_grid* grids, const whv_params* params,
                                const double* const* v_dev, const double* const* f_dev, double* const* out_dev);

/* Autotuner of the batched steps per sweep (2-D grids): times one persistent batched f = 0 wave
 * solve of all nprob problems for k = 2, 4, 6, 8, 10, 12 (CUDA events on the shared stream, after a
 * warm-up launch) and stores the fastest in grids[0] (as whv_set_steps_per_sweep), which
 * whv_solve_batched reads; *best (may be NULL) receives it.  3-D batches step once per sweep
 * (*best = 1).  Uses the grids' scratch buffers; the same restrictions on the grids as
 * whv_solve_batched.  Must not be called while the stream is being captured. */
whv_status whv_autotune_batched(int nprob, const whv_grid* grids, const whv_params* params, int* best);

/* Deflation contractions and reductions on the grid's basis / weights (building blocks of the
 * solve, exposed for testing and for callers composing their own iterations):
 *   whv_project:  coeff_dev[m] = (W^T M r)_m, m < nd                 (Algorithm 2, (r, phi_m))
 *   whv_expand:   out_dev     = out_dev + alpha * W y_dev            (Algorithm 2, inflate)
 *   whv_dot:      *out_host   = <x, y>_M                             (Krylov inner product) */
whv_status whv_project(whv_grid grid, const double* r_dev, double* coeff_dev);
whv_status whv_expand(whv_grid grid, const double* y_dev, double alpha, double* out_dev);
whv_status whv_dot(whv_grid grid, const double* x_dev, const double* y_dev, double* out_host);

/* Allocation-free variant of whv_project, for callers that cannot allocate device memory: code
 * whose device memory is owned by a host framework's pool or arena, real-time or embedded loops
 * that forbid allocation after start-up, and callers working under a stream capture or a
 * latency budget where cudaMalloc (which may synchronise the device) is not allowed.  It needs
 * no grid (creating one allocates) and calls no cudaMalloc / cudaFree or allocating library.
 * The paper has no counterpart: this is a deployment variant of the deflation projection.
 *   coef_dev[m] = sum_i W_dev[i + m n] w_i r_dev[i],  m < nd   (w_dev NULL => w = 1)
 * W_dev (n x nd, column-major), r_dev, w_dev (n) and coef_dev (nd) are caller-owned device
 * buffers; the work is ordered on cuda_stream (a cudaStream_t, NULL = legacy default stream).
 * Scratch: the per-block partial sums go to a static 2 MiB device array (262144 doubles) that
 * every GPU loading the library holds until the process exits.  Limits: 1 <= nd <= 1024 and
 * ceil(n / 2048) * nd <= 262144 (e.g. n = 261121 with nd = 1024, n = 16.7M with nd = 32);
 * larger problems get WHV_ERR_INVALID.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current: make that first call before
 * any stream capture.  All calls share the one array: calls whose kernels overlap on the GPU
 * (other streams, other host threads) race and return wrong sums; serialise them.  Errors are
 * reported through whv_last_error(NULL). */
whv_status whv_project_noalloc(int64_t n, int nd, const double* W_dev, const double* r_dev,
                               const double* w_dev, double* coef_dev, void* cuda_stream);

/* SVD compression of the deflation basis (Sec. 4.3, experiment with compressed eigenvectors);
 * 2-D grids.  Each basis vector, an ny x nx matrix (row y, column x), is replaced by its
 * smallest-rank truncated SVD with Frobenius error < tau (singular values from a randomized range
 * finder with power iterations; tau should be >= 1e-7 times the vector norm, the resolution of
 * that finder), and the dense basis is freed: storage sum_m r_m (nx + ny + 1) doubles instead of
 * nd nx ny.  From then on every use of the basis (DEVD deflation / inflation, DCG, AGMRES,
 * ABICGSTAB, the FP64 residual correction, whv_project / whv_expand, batched solves) runs on the
 * compressed vectors: the projection W^T M r is T = (M o r) V followed by per-vector sums of
 * s_k u_k . T_k, the expansion a GEMM U diag(c) V^T (FP64 kernels of this library);
 * whv_get_basis writes the compressed vectors out dense.  ranks_host (nd ints, may be NULL)
 * receives r_m.  Ranks are capped at 256 (beyond about half the shorter side of the grid the
 * factors take more memory than the vector): a vector that needs more at this tolerance makes
 * the call return WHV_ERR_INVALID and leave the basis dense (grids whose shorter side is <= 256
 * keep up to full rank).  Needs a dense basis (WHV_ERR_INVALID otherwise, or if every rank is 0). */
whv_status whv_compress_basis(whv_grid grid, double tau, int* ranks_host);

/* Test hook for the failure path of the grid barriers of the batched persistent kernels (no
 * counterpart in the paper): marks the grid so that the next whv_solve_batched,
 * whv_apply_pi_batched or whv_autotune_batched call that includes it starts with the batch's
 * barrier error flag raised.  Every CTA of its first batched wave solve then leaves at its first
 * grid barrier exactly as after a barrier wait that gave up; the call returns WHV_ERR_TIMEOUT
 * (outputs unspecified) and the mark is cleared, so the next batched call runs normally.  No GPU
 * wait is made to run out.  Single-grid calls ignore the mark (their kernels have no grid
 * barrier). */
whv_status whv_inject_barrier_error(whv_grid grid);

/* Number of interior unknowns N of the grid (0 for NULL). */
int64_t whv_num_unknowns(whv_grid grid);

/* Last error message of `grid` (or of the calling thread's last failed create when grid is NULL).
 * The string is owned by the library and valid until the next call on the grid. */
const char* whv_last_error(whv_grid grid);

/* Number of CUDA kernels this library has launched in the process so far (a kernel replayed
 * inside one of the library's CUDA graphs counts once per replay).  Diagnostic counter. */
int64_t whv_kernel_launches(void);

/* Library version string. */
const char* whv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WHV_H */
