// whv_solve: the accelerated WaveHoltz iteration on A u = (I - S_h) u = b.
//
//  * DEVD (Algorithm 2): f_d = f - W W^T M f; iterate on b = Pi_h(0; f_d); inflate
//    u += W diag(1/(omega_eff^2 - lambda^2)) W^T M f.  Optional re-deflation of each operator
//    output for approximate eigenvectors.
//  * CG: every iteration is one wave solve q = A p whose last step also reduces p^T M q,
//    then the fused update kernel (x, r, r^T M r, beta) and the direction update; all scalars
//    stay on the device, the host reads them only to test convergence.
//  * DCG (Algorithm 4) with exact eigenvectors: W^T A W = diag(mu), mu = 1 - beta_h, so the
//    deflated start x_0 = W diag(1/mu) W^T r_{-1}, r_0 = r_{-1} - W W^T M r_{-1} costs no wave
//    solve and the per-iteration projections drop out.
//  * GMRES(m): Arnoldi with classical Gram-Schmidt applied twice on the device (the deflation
//    contraction kernels on the Krylov basis), Givens rotations and the triangular solve on the
//    host (m <= 30 scalars per step).
//  * AGMRES (Algorithm 5): GMRES(m) whose least-squares space is augmented by the basis W; the
//    thin QR A W = V_p H_p (classical Gram-Schmidt twice, M inner products) is built once per
//    basis, each cycle projects range(A W) out of the residual, runs the Arnoldi steps
//    orthogonally to [V_p | V_{p+1..}] and solves the triangular system over [W | V_{p+1..k}].
//  * ABICGSTAB (Algorithm 6): BiCGStab on the system projected away from range(A W) (same QR
//    factors as AGMRES), two wave solves per iteration, scalars on the host; the W components
//    are restored at the end, x -= W R^{-1} xi.
//  * FPI (Algorithm 1).
//  * FP64 residual correction (WHV_REFINE_FP64): the outer loop forms the residual r = b - A x of
//    the full system with FP64 wave solves; the correction is the modal solve of its deflated
//    components plus an inner Krylov solve (grid's stepping, FP64 reductions) of the rest to a
//    loose relative tolerance -- iterative refinement, so the FP64 residual reaches tol although
//    one FP32-stepped application of A is only accurate to ~1e-6, and approximate (Lanczos)
//    eigenvectors are corrected instead of leaving their error in the inflated solution.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "whv_internal.cuh"

namespace whv {

struct SolveCtx {
  whv_grid g;
  const TimeGridH& tg;
  bool redefl;
  int ws = 0;      // wave solves in the grid's precision
  int ws64 = 0;    // FP64 (or double-float) wave solves of the residual correction
  int res_prec = WHV_FP64;   // precision of those: WHV_FP64 or kPrecDF64 (WHV_RESIDUAL_DF64)
};

// out = out - W (W^T M out)
static whv_status deflate_vec(whv_grid g, double* vec) {
  TRY(basis_project(g, vec, g->small));
  return basis_expand(g, g->small, -1.0, vec);
}

// q = A v (+ re-deflation) in the grid's stepping precision; scal[S_PQ] = <v, q>_M
static whv_status apply_A(SolveCtx& c, const double* v, double* q) {
  whv_grid g = c.g;
  TRY(wave_solve(g, c.tg, v, nullptr, q, 1));
  c.ws++;
  if (c.redefl) {
    TRY(deflate_vec(g, q));
    TRY(dot_async(g, v, q, S_PQ));
  }
  return WHV_OK;
}

// WHV_LOG=1 in the environment prints the residual history of every solve to stderr
static bool log_on() {
  static const bool on = [] { const char* e = getenv("WHV_LOG"); return e && e[0] == '1'; }();
  return on;
}

// ------------------------------------------------------------------ general deflation (Algorithm 4)
// out = Einv in  (nd x nd row-major, one block)
__global__ void k_small_matvec(const double* __restrict__ Einv, const double* __restrict__ in, int nd,
                               double* __restrict__ out) {
  __shared__ double sin_[kMaxND];
  for (int j = threadIdx.x; j < nd; j += blockDim.x) sin_[j] = in[j];
  __syncthreads();
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nd; ++j) s = fma(Einv[(int64_t)i * nd + j], sin_[j], s);
    out[i] = s;
  }
}

static whv_status small_matvec(whv_grid g, const double* Einv, const double* in, int nd, double* out) {
  k_small_matvec<<<1, 1024, 0, g->stream>>>(Einv, in, nd, out);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

// Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix (host, n <= 1024)
static bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[(size_t)r * n + c]) > fabs(a[(size_t)piv * n + c])) piv = r;
    if (!(fabs(a[(size_t)piv * n + c]) > 0.0)) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    const double d = 1.0 / a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) { a[(size_t)c * n + k] *= d; inv[(size_t)c * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// A W (nd wave solves of the grid's stepping) and (W^T M A W)^{-1} for Algorithm 4 with a basis
// that is not made of exact eigenvectors
static whv_status prepare_general_dcg(struct SolveCtx& c);
static whv_status dcg_project_direction(whv_grid g);

// ------------------------------------------------------------------ device-resident CG loop
// One CUDA graph with a conditional WHILE node: the body is one CG iteration (the wave solve
// q = A p with its p^T M q epilogue, optional re-deflation, the fused x/r update with r^T M r,
// the direction update) followed by a one-thread kernel that counts the iteration and sets the
// loop condition from r^T M r, the breakdown flag and the iteration limit.  An inner CG solve
// is then one graph launch and one host synchronisation.
__global__ void k_cg_check(cudaGraphConditionalHandle h, double* scal) {
  const double it = scal[S_ITER] + 1.0;
  scal[S_ITER] = it;
  const bool go = scal[S_FLAG] == 0.0 && scal[S_RR] > scal[S_STOP] && it < scal[S_MAXIT];
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

struct CgLoop {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double omega = 0, cfl = 0;
  int periods = 0, adjust = 0, nt = 0, kblock = 0;
  bool redefl = false, general = false;
  const void* V = nullptr;     // identity of the basis storage the graph was built with
  int nd = 0;
  int64_t body_launches = 0;
};

void free_cgloop(whv_grid g) {
  if (!g->cgloop) return;
  cudaStreamSynchronize(g->stream);
  if (g->cgloop->exec) cudaGraphExecDestroy(g->cgloop->exec);
  if (g->cgloop->graph) cudaGraphDestroy(g->cgloop->graph);
  delete g->cgloop;
  g->cgloop = nullptr;
}

static int64_t launches_now() { return whv_kernel_launches(); }

// build (or reuse) the loop graph for the current time grid / basis; general: Algorithm 4 with
// the per-iteration A-orthogonalisation against a general basis
static whv_status cg_loop_graph(SolveCtx& c, bool general, CgLoop** out) {
  whv_grid g = c.g;
  const Basis& B = g->basis;
  CgLoop* L = g->cgloop;
  const bool usesV = c.redefl || general;
  if (L && L->omega == c.tg.omega && L->cfl == c.tg.cfl && L->periods == c.tg.periods &&
      L->adjust == c.tg.adjust && L->nt == c.tg.nt && L->kblock == g->kblock && L->redefl == c.redefl &&
      L->general == general && L->V == (usesV ? basis_key(B) : nullptr) && L->nd == (usesV ? B.nd : 0)) {
    *out = L;
    return WHV_OK;
  }
  free_cgloop(g);
  L = new CgLoop();
  g->cgloop = L;
  L->omega = c.tg.omega; L->cfl = c.tg.cfl; L->periods = c.tg.periods; L->adjust = c.tg.adjust;
  L->nt = c.tg.nt; L->kblock = g->kblock; L->redefl = c.redefl; L->general = general;
  L->V = usesV ? basis_key(B) : nullptr; L->nd = usesV ? B.nd : 0;
  WHV_CUDA(g, cudaGraphCreate(&L->graph, 0));
  cudaGraphConditionalHandle h;
  WHV_CUDA(g, cudaGraphConditionalHandleCreate(&h, L->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  WHV_CUDA(g, cudaGraphAddNode(&node, L->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const int64_t l0 = launches_now();
  const int ws0 = c.ws;
  WHV_CUDA(g, cudaStreamBeginCaptureToGraph(g->stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
  whv_status s = apply_A(c, g->p, g->q);
  if (s == WHV_OK) s = cg_update(g);
  if (s == WHV_OK) s = cg_direction(g);
  if (s == WHV_OK && general) s = dcg_project_direction(g);
  if (s == WHV_OK) {
    k_cg_check<<<1, 1, 0, g->stream>>>(h, g->scal);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) s = fail(g, WHV_ERR_CUDA, "k_cg_check launch");
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &captured);
  c.ws = ws0;   // the capture did not run anything
  L->body_launches = launches_now() - l0;
  count_launches(-L->body_launches);
  if (s != WHV_OK) { free_cgloop(g); return s; }
  if (e != cudaSuccess) { free_cgloop(g); return cuda_fail(g, e, "cudaStreamEndCapture (CG loop body)"); }
  e = cudaGraphInstantiate(&L->exec, L->graph, 0);
  if (e != cudaSuccess) { free_cgloop(g); return cuda_fail(g, e, "cudaGraphInstantiate (CG loop)"); }
  *out = L;
  return WHV_OK;
}

static whv_status prepare_general_dcg(SolveCtx& c) {
  whv_grid g = c.g;
  Basis& B = g->basis;
  if (B.AW && B.Einv) return WHV_OK;
  const int64_t N = g->N;
  const int nd = B.nd;
  if (!B.AW) WHV_CUDA(g, cudaMalloc(&B.AW, (size_t)nd * N * sizeof(double)));
  for (int m = 0; m < nd; ++m) {
    // through fixed buffers so that every column replays one cached wave-solve graph
    TRY(basis_column(g, m, g->p));
    TRY(wave_solve(g, c.tg, g->p, nullptr, g->q, 1));   // not t: it may hold the right-hand side
    c.ws++;
    WHV_CUDA(g, cudaMemcpyAsync(B.AW + (size_t)m * N, g->q, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  }
  // E = W^T M (A W), symmetrised (A is M-self-adjoint; FP32 stepping breaks it at rounding level)
  std::vector<double> E((size_t)nd * nd), col(nd);
  for (int m = 0; m < nd; ++m) {
    TRY(basis_project(g, B.AW + (size_t)m * N, g->small));
    TRY(to_host(g, col.data(), g->small, nd));
    for (int i = 0; i < nd; ++i) E[(size_t)i * nd + m] = col[i];
  }
  for (int i = 0; i < nd; ++i)
    for (int j = i + 1; j < nd; ++j) {
      const double a = 0.5 * (E[(size_t)i * nd + j] + E[(size_t)j * nd + i]);
      E[(size_t)i * nd + j] = E[(size_t)j * nd + i] = a;
    }
  if (!invert(E, nd)) return fail(g, WHV_ERR_BREAKDOWN, "W^T M A W is singular (dependent deflation vectors)");
  if (!B.Einv) WHV_CUDA(g, cudaMalloc(&B.Einv, (size_t)nd * nd * sizeof(double)));
  WHV_CUDA(g, cudaMemcpyAsync(B.Einv, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

// p = p - W Einv (AW)^T M r  (the A-orthogonalisation of Algorithm 4 with a general basis)
static whv_status dcg_project_direction(whv_grid g) {
  const Basis& B = g->basis;
  TRY(project(g, B.AW, B.nd, g->r, g->small));
  TRY(small_matvec(g, B.Einv, g->small, B.nd, g->small2));
  return basis_expand(g, g->small2, -1.0, g->p);
}

// Algorithm 5 set-up: A W = QAW Raw, kept with the basis.  A W = W diag(mu) for exact
// eigenvectors, the general-DCG A W if already formed, else one wave solve per column.
static whv_status prepare_agmres(SolveCtx& c) {
  whv_grid g = c.g;
  Basis& B = g->basis;
  if (B.QAW) return WHV_OK;
  const int64_t N = g->N;
  const int nd = B.nd;
  WHV_CUDA(g, cudaMalloc(&B.QAW, (size_t)nd * N * sizeof(double)));
  std::vector<double> R((size_t)nd * nd, 0.0), h(nd);
  for (int j = 0; j < nd; ++j) {
    double* q = B.QAW + (size_t)j * N;
    if (B.flags & WHV_BASIS_EXACT) {
      TRY(basis_column(g, j, q));
      TRY(axpby(g, N, B.mu[j], q, 0.0, q));
    } else if (B.AW) {
      TRY(copy_dev(g, q, B.AW + (size_t)j * N, N));
    } else {
      // through p -> q (the A p buffers: every column replays one cached wave-solve graph; t may
      // hold the right-hand side, which the restarts read again)
      TRY(basis_column(g, j, g->p));
      TRY(wave_solve(g, c.tg, g->p, nullptr, g->q, 1));
      c.ws++;
      TRY(copy_dev(g, q, g->q, N));
    }
    for (int pass = 0; pass < 2 && j > 0; ++pass) {   // classical Gram-Schmidt, twice
      TRY(project(g, B.QAW, j, q, g->small));
      TRY(expand(g, B.QAW, j, g->small, -1.0, q));
      TRY(to_host(g, h.data(), g->small, j));
      for (int i = 0; i < j; ++i) R[(size_t)j * nd + i] += h[i];
    }
    TRY(dot_async(g, q, q, S_TMP));
    TRY(fetch_scalars(g));
    const double rn = sqrt(g->scal_host[S_TMP]);
    if (!(rn > 0.0) || !isfinite(rn)) {
      cudaFree(B.QAW);
      B.QAW = nullptr;
      return fail(g, WHV_ERR_BREAKDOWN, "A W is rank deficient (dependent augmentation vectors)");
    }
    R[(size_t)j * nd + j] = rn;
    TRY(axpby(g, N, 1.0 / rn, q, 0.0, q));
  }
  B.Raw = R;
  return WHV_OK;
}

// Algorithms 5 and 6 use the basis inside the iteration (augmentation): no forcing deflation,
// no modal correction, no re-deflation
static bool augmented(int method) { return method == WHV_AGMRES || method == WHV_ABICGSTAB; }

struct InnerResult {
  int iters = 0;
  bool converged = false, breakdown = false;
  double rel = 1.0;
};

// Krylov solve of A x = b (b: device, FP64, ||b||_M^2 = bb) into g->x, in the grid's stepping
// precision.  use_x0: g->x holds the initial guess, else x0 = 0.  fpi_force: forcing of the
// FPI map (FPI iterates x <- Pi_h(x; f) and does not use b except for its norm).
static whv_status inner_solve(SolveCtx& c, int method, const whv_params* p, const double* b,
                              double bb, bool use_x0, double tol, int maxit,
                              const double* fpi_force, InnerResult* res) {
  whv_grid g = c.g;
  const int64_t N = g->N;
  const Basis& B = g->basis;
  const int check = p->check_every > 0 ? p->check_every : 1;
  InnerResult R;
  if (use_x0) {
    TRY(apply_A(c, g->x, g->q));
    TRY(copy_dev(g, g->r, b, N));
    TRY(axpby(g, N, -1.0, g->q, 1.0, g->r));
  } else {
    WHV_CUDA(g, cudaMemsetAsync(g->x, 0, N * sizeof(double), g->stream));
    TRY(copy_dev(g, g->r, b, N));
  }
  if (bb == 0.0) {
    R.converged = true;
    R.rel = 0.0;
    *res = R;
    return WHV_OK;
  }
  if (method == WHV_CG || method == WHV_DCG) {
    double rr0 = bb;
    const bool general = method == WHV_DCG && !(B.flags & WHV_BASIS_EXACT);
    if (general) {
      // Algorithm 4 with a general basis: x_0 = x_{-1} + W E^{-1} W^T M r_{-1},
      // r_0 = r_{-1} - (A W) E^{-1} W^T M r_{-1},  p_0 = r_0 - W E^{-1} (A W)^T M r_0
      TRY(prepare_general_dcg(c));
      TRY(basis_project(g, g->r, g->small));
      TRY(small_matvec(g, B.Einv, g->small, B.nd, g->small2));
      TRY(basis_expand(g, g->small2, 1.0, g->x));
      TRY(expand(g, B.AW, B.nd, g->small2, -1.0, g->r));
    } else if (method == WHV_DCG) {
      // x_0 = x_{-1} + W diag(1/mu) W^T M r_{-1};  r_0 = r_{-1} - W W^T M r_{-1}  (A W = W diag(mu))
      std::vector<double> cf(B.nd), y(B.nd);
      TRY(basis_project(g, g->r, g->small));
      TRY(to_host(g, cf.data(), g->small, B.nd));
      for (int m = 0; m < B.nd; ++m) y[m] = cf[m] / B.mu[m];
      TRY(to_dev(g, g->small, y.data(), B.nd));
      TRY(basis_expand(g, g->small, 1.0, g->x));
      TRY(to_dev(g, g->small, cf.data(), B.nd));
      TRY(basis_expand(g, g->small, -1.0, g->r));
    }
    TRY(copy_dev(g, g->p, g->r, N));
    if (general) TRY(dcg_project_direction(g));
    TRY(dot_async(g, g->r, g->r, S_RR));
    WHV_CUDA(g, cudaMemsetAsync(g->scal + S_FLAG, 0, sizeof(double), g->stream));
    TRY(fetch_scalars(g));
    const double rrs = g->scal_host[S_RR];
    if (method == WHV_DCG) rr0 = rrs;  // Algorithm 4: relative to the deflated start residual
    R.rel = rr0 > 0.0 ? sqrt(rrs / rr0) : 0.0;
    if (R.rel <= tol) R.converged = true;
    if (!R.converged && maxit > 0 && p->check_every <= 1) {
      // device-resident loop: one graph launch runs the iterations until convergence
      CgLoop* L = nullptr;
      TRY(cg_loop_graph(c, general, &L));
      const double init[3] = {0.0, tol * tol * rr0, (double)maxit};
      TRY(to_dev(g, g->scal + S_ITER, init, 3));
      WHV_CUDA(g, cudaGraphLaunch(L->exec, g->stream));
      TRY(fetch_scalars(g));
      R.iters = (int)g->scal_host[S_ITER];
      c.ws += R.iters;
      count_launches(L->body_launches * R.iters);
      if (g->scal_host[S_FLAG] != 0.0) R.breakdown = true;
      R.rel = sqrt(g->scal_host[S_RR] / rr0);
      if (R.rel <= tol) R.converged = true;
    }
    while (!R.converged && !R.breakdown && R.iters < maxit) {
      TRY(apply_A(c, g->p, g->q));
      TRY(cg_update(g));
      TRY(cg_direction(g));
      if (general) TRY(dcg_project_direction(g));
      ++R.iters;
      if (R.iters % check == 0 || R.iters == maxit) {
        TRY(fetch_scalars(g));
        if (g->scal_host[S_FLAG] != 0.0) { R.breakdown = true; break; }
        R.rel = sqrt(g->scal_host[S_RR] / rr0);
        if (R.rel <= tol) R.converged = true;
      }
    }
  } else if (method == WHV_GMRES) {
    const int m = p->restart > 0 ? p->restart : 30;
    if (m + 1 > kMaxND) return fail(g, WHV_ERR_INVALID, "GMRES restart too large");
    if (g->krylov_cols < m + 1) {
      if (g->krylov) cudaFree(g->krylov);
      g->krylov = nullptr;
      g->krylov_cols = 0;
      WHV_CUDA(g, cudaMalloc(&g->krylov, (size_t)(m + 1) * N * sizeof(double)));
      g->krylov_cols = m + 1;
    }
    double* K = g->krylov;
    const double bnorm = sqrt(bb);
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), h1(m + 1), h2(m + 1), y(m);
    auto Hc = [&](int i, int j) -> double& { return H[(size_t)j * (m + 1) + i]; };
    while (true) {
      TRY(dot_async(g, g->r, g->r, S_TMP));
      TRY(fetch_scalars(g));
      const double beta0 = sqrt(g->scal_host[S_TMP]);
      if (log_on()) fprintf(stderr, "[whv] GMRES cycle start: rel %.3e after %d iterations\n", beta0 / bnorm, R.iters);
      if (!isfinite(beta0)) { R.breakdown = true; break; }
      R.rel = beta0 / bnorm;
      if (R.rel <= tol) { R.converged = true; break; }
      if (R.iters >= maxit) break;
      TRY(axpby(g, N, 1.0 / beta0, g->r, 0.0, K));
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = beta0;
      int k = 0;
      bool lucky = false;
      for (int j = 0; j < m; ++j) {
        double* w = K + (size_t)(j + 1) * N;
        TRY(apply_A(c, K + (size_t)j * N, w));
        ++R.iters;
        // classical Gram-Schmidt, twice
        TRY(project(g, K, j + 1, w, g->small));
        TRY(expand(g, K, j + 1, g->small, -1.0, w));
        TRY(to_host(g, h1.data(), g->small, j + 1));
        TRY(project(g, K, j + 1, w, g->small));
        TRY(expand(g, K, j + 1, g->small, -1.0, w));
        TRY(to_host(g, h2.data(), g->small, j + 1));
        for (int i = 0; i <= j; ++i) Hc(i, j) = h1[i] + h2[i];
        TRY(dot_async(g, w, w, S_TMP));
        TRY(fetch_scalars(g));
        const double hn = sqrt(g->scal_host[S_TMP]);
        if (!isfinite(hn)) {
          if (log_on()) fprintf(stderr, "[whv] GMRES: non-finite Arnoldi norm at step %d\n", j);
          R.breakdown = true;
          break;
        }
        Hc(j + 1, j) = hn;
        lucky = !(hn > 0.0);
        if (!lucky) TRY(axpby(g, N, 1.0 / hn, w, 0.0, w));
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
          Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
          Hc(i, j) = t;
        }
        const double den = hypot(Hc(j, j), Hc(j + 1, j));
        if (!(den > 0.0)) {
          if (log_on()) fprintf(stderr, "[whv] GMRES: zero Givens denominator at step %d (H_jj %.3e)\n", j, Hc(j, j));
          R.breakdown = true;
          break;
        }
        cs[j] = Hc(j, j) / den;
        sn[j] = Hc(j + 1, j) / den;
        Hc(j, j) = den;
        Hc(j + 1, j) = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        k = j + 1;
        R.rel = fabs(gv[k]) / bnorm;
        if (R.rel <= tol || R.iters >= maxit || lucky) break;
      }
      if (R.breakdown && k == 0) break;
      for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= Hc(i, l) * y[l];
        y[i] = s / Hc(i, i);
      }
      TRY(to_dev(g, g->small, y.data(), k));
      TRY(expand(g, K, k, g->small, 1.0, g->x));
      if (R.breakdown) break;
      if (R.rel <= tol || lucky) { R.converged = true; break; }
      // restart: r = b - A x
      TRY(apply_A(c, g->x, g->q));
      TRY(copy_dev(g, g->r, b, N));
      TRY(axpby(g, N, -1.0, g->q, 1.0, g->r));
    }
  } else if (method == WHV_AGMRES) {
    // Algorithm 5 with restarts; augmentation W = the grid's basis (pd columns, may be 0)
    const int m = p->restart > 0 ? p->restart : 30;
    const int pd = B.nd;
    if (m + 1 > kMaxND) return fail(g, WHV_ERR_INVALID, "AGMRES restart too large");
    if (pd > 0) TRY(prepare_agmres(c));
    if (g->krylov_cols < m + 1) {
      if (g->krylov) cudaFree(g->krylov);
      g->krylov = nullptr;
      g->krylov_cols = 0;
      WHV_CUDA(g, cudaMalloc(&g->krylov, (size_t)(m + 1) * N * sizeof(double)));
      g->krylov_cols = m + 1;
    }
    double* K = g->krylov;   // v_{p+1} .. v_{p+m+1}
    const double bnorm = sqrt(bb);
    const int D = pd + m;
    std::vector<double> H((size_t)(D + 1) * D), cs(D), sn(D), gv(D + 1), y(D), hp(std::max(pd, 1)), hk(m + 1);
    auto Hc = [&](int i, int j) -> double& { return H[(size_t)j * (D + 1) + i]; };
    int cycle = 0;
    while (true) {
      TRY(dot_async(g, g->r, g->r, S_TMP));
      TRY(fetch_scalars(g));
      const double beta0 = sqrt(g->scal_host[S_TMP]);
      if (log_on()) fprintf(stderr, "[whv] AGMRES cycle start: rel %.3e after %d iterations\n", beta0 / bnorm, R.iters);
      if (!isfinite(beta0)) { R.breakdown = true; break; }
      R.rel = beta0 / bnorm;
      if (R.rel <= tol) { R.converged = true; break; }
      if (cycle > 0 && R.iters >= maxit) break;   // the first cycle runs even for maxit = 0
      ++cycle;
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(gv.begin(), gv.end(), 0.0);
      // v_{p+1} = (I - V_p V_p^T M) b_0 / ||.||;  g_k = <v_k, b_0>, k <= p + 1
      TRY(copy_dev(g, K, g->r, N));
      if (pd > 0) {
        TRY(project(g, B.QAW, pd, K, g->small));
        TRY(to_host(g, hp.data(), g->small, pd));
        TRY(expand(g, B.QAW, pd, g->small, -1.0, K));
        TRY(project(g, B.QAW, pd, K, g->small));
        TRY(expand(g, B.QAW, pd, g->small, -1.0, K));
        for (int i = 0; i < pd; ++i) gv[i] = hp[i];
        for (int j = 0; j < pd; ++j)
          for (int i = 0; i <= j; ++i) Hc(i, j) = B.Raw[(size_t)j * pd + i];
      }
      TRY(dot_async(g, K, K, S_TMP));
      TRY(fetch_scalars(g));
      const double vn = sqrt(g->scal_host[S_TMP]);
      if (vn > 0.0) TRY(axpby(g, N, 1.0 / vn, K, 0.0, K));
      TRY(dot_async(g, K, g->r, S_TMP));
      TRY(fetch_scalars(g));
      gv[pd] = g->scal_host[S_TMP];
      int k = pd;
      bool lucky = false;
      // |g_{p+1}| is the residual of the fit over span(W) alone: no Arnoldi step if it meets tol
      const int nsteps = fabs(gv[pd]) / bnorm > tol ? std::min(m, maxit - R.iters) : 0;
      for (int j = 0; j < nsteps; ++j) {
        const int jj = pd + j;
        double* w = K + (size_t)(j + 1) * N;
        TRY(apply_A(c, K + (size_t)j * N, w));
        ++R.iters;
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt against [V_p | v_{p+1..}], twice
          if (pd > 0) TRY(project(g, B.QAW, pd, w, g->small));
          TRY(project(g, K, j + 1, w, g->small2));
          if (pd > 0) TRY(expand(g, B.QAW, pd, g->small, -1.0, w));
          TRY(expand(g, K, j + 1, g->small2, -1.0, w));
          if (pd > 0) {
            TRY(to_host(g, hp.data(), g->small, pd));
            for (int i = 0; i < pd; ++i) Hc(i, jj) += hp[i];
          }
          TRY(to_host(g, hk.data(), g->small2, j + 1));
          for (int i = 0; i <= j; ++i) Hc(pd + i, jj) += hk[i];
        }
        TRY(dot_async(g, w, w, S_TMP));
        TRY(fetch_scalars(g));
        const double hn = sqrt(g->scal_host[S_TMP]);
        if (!isfinite(hn)) { R.breakdown = true; break; }
        Hc(jj + 1, jj) = hn;
        lucky = !(hn > 0.0);
        if (!lucky) TRY(axpby(g, N, 1.0 / hn, w, 0.0, w));
        for (int i = pd; i < jj; ++i) {   // previous rotations (the first p columns are triangular)
          const double t = cs[i] * Hc(i, jj) + sn[i] * Hc(i + 1, jj);
          Hc(i + 1, jj) = -sn[i] * Hc(i, jj) + cs[i] * Hc(i + 1, jj);
          Hc(i, jj) = t;
        }
        const double den = hypot(Hc(jj, jj), Hc(jj + 1, jj));
        if (!(den > 0.0)) { R.breakdown = true; break; }
        cs[jj] = Hc(jj, jj) / den;
        sn[jj] = Hc(jj + 1, jj) / den;
        Hc(jj, jj) = den;
        Hc(jj + 1, jj) = 0.0;
        gv[jj + 1] = -sn[jj] * gv[jj];
        gv[jj] = cs[jj] * gv[jj];
        k = jj + 1;
        if (fabs(gv[k]) / bnorm <= tol || R.iters >= maxit || lucky) break;
      }
      if (R.breakdown && k == pd && nsteps > 0) break;
      // H_{1:k,1:k} y = g_{1:k};  x += [W | v_{p+1..k}] y
      for (int i = k - 1; i >= 0; --i) {
        double sacc = gv[i];
        for (int l = i + 1; l < k; ++l) sacc -= Hc(i, l) * y[l];
        y[i] = sacc / Hc(i, i);
      }
      if (pd > 0) {
        TRY(to_dev(g, g->small, y.data(), pd));
        TRY(basis_expand(g, g->small, 1.0, g->x));
      }
      if (k > pd) {
        TRY(to_dev(g, g->small, y.data() + pd, k - pd));
        TRY(expand(g, K, k - pd, g->small, 1.0, g->x));
      }
      R.rel = fabs(gv[k]) / bnorm;
      if (R.breakdown) break;
      if (R.rel <= tol || lucky) { R.converged = true; break; }
      if (R.iters >= maxit) break;
      // restart: b_0 = b - A x
      TRY(apply_A(c, g->x, g->q));
      TRY(copy_dev(g, g->r, b, N));
      TRY(axpby(g, N, -1.0, g->q, 1.0, g->r));
    }
  } else if (method == WHV_ABICGSTAB) {
    // Algorithm 6 (typos corrected: eta_1 = Q^T M r; p = r at i = 1; alpha = rho / <r~, v>)
    const int pd = B.nd;
    if (pd > 0) TRY(prepare_agmres(c));   // A W = Q R
    if (g->krylov_cols < 4) {
      if (g->krylov) cudaFree(g->krylov);
      g->krylov = nullptr;
      g->krylov_cols = 0;
      WHV_CUDA(g, cudaMalloc(&g->krylov, (size_t)4 * N * sizeof(double)));
      g->krylov_cols = 4;
    }
    double* rt = g->krylov;              // shadow residual r~
    double* v = g->krylov + N;
    double* sv = g->krylov + 2 * N;
    double* tv = g->krylov + 3 * N;
    const double bnorm = sqrt(bb);
    std::vector<double> xi(std::max(pd, 1), 0.0), e1(std::max(pd, 1), 0.0), e2(std::max(pd, 1), 0.0);
    auto dot = [&](const double* a, const double* b2, double* out) -> whv_status {
      TRY(dot_async(g, a, b2, S_TMP));
      TRY(fetch_scalars(g));
      *out = g->scal_host[S_TMP];
      return WHV_OK;
    };
    // u <- u - Q (Q^T M u), coefficients to eta (host)
    auto project_Q = [&](double* u, double* eta) -> whv_status {
      TRY(project(g, B.QAW, pd, u, g->small));
      TRY(to_host(g, eta, g->small, pd));
      return expand(g, B.QAW, pd, g->small, -1.0, u);
    };
    TRY(copy_dev(g, rt, g->r, N));
    if (pd > 0) {
      TRY(project_Q(g->r, e1.data()));
      for (int i = 0; i < pd; ++i) xi[i] = -e1[i];
    }
    double rr;
    TRY(dot(g->r, g->r, &rr));
    R.rel = sqrt(rr) / bnorm;
    if (!isfinite(R.rel)) R.breakdown = true;
    else if (R.rel <= tol) R.converged = true;
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (!R.converged && !R.breakdown && R.iters < maxit) {
      ++R.iters;
      double rho;
      TRY(dot(rt, g->r, &rho));
      if (!(rho != 0.0) || !isfinite(rho)) { R.breakdown = true; break; }
      if (R.iters == 1) {
        TRY(copy_dev(g, g->p, g->r, N));
      } else {
        const double beta = (rho / rho_old) * (alpha / omega);
        TRY(axpby(g, N, -omega, v, 1.0, g->p));     // p - omega v
        TRY(axpby(g, N, 1.0, g->r, beta, g->p));    // r + beta (p - omega v)
      }
      TRY(apply_A(c, g->p, v));
      if (pd > 0) TRY(project_Q(v, e1.data()));
      double rtv;
      TRY(dot(rt, v, &rtv));
      alpha = rho / rtv;
      if (!isfinite(alpha)) { R.breakdown = true; break; }
      TRY(copy_dev(g, sv, g->r, N));
      TRY(axpby(g, N, -alpha, v, 1.0, sv));
      double ss;
      TRY(dot(sv, sv, &ss));
      if (sqrt(ss) <= tol * bnorm) {
        TRY(axpby(g, N, alpha, g->p, 1.0, g->x));
        TRY(copy_dev(g, g->r, sv, N));
        for (int i = 0; i < pd; ++i) xi[i] += alpha * e1[i];
        R.rel = sqrt(ss) / bnorm;
        R.converged = true;
        break;
      }
      TRY(apply_A(c, sv, tv));
      if (pd > 0) TRY(project_Q(tv, e2.data()));
      double ts, tt;
      TRY(dot(tv, sv, &ts));
      TRY(dot(tv, tv, &tt));
      omega = ts / tt;
      if (!isfinite(omega) || omega == 0.0) { R.breakdown = true; break; }
      for (int i = 0; i < pd; ++i) xi[i] += alpha * e1[i] + omega * e2[i];
      TRY(axpby(g, N, alpha, g->p, 1.0, g->x));
      TRY(axpby(g, N, omega, sv, 1.0, g->x));
      TRY(copy_dev(g, g->r, sv, N));
      TRY(axpby(g, N, -omega, tv, 1.0, g->r));
      TRY(dot(g->r, g->r, &rr));
      R.rel = sqrt(rr) / bnorm;
      if (!isfinite(R.rel)) { R.breakdown = true; break; }
      if (R.rel <= tol) R.converged = true;
      rho_old = rho;
      if (log_on() && R.iters % 10 == 0) fprintf(stderr, "[whv] ABICGSTAB %d: rel %.3e\n", R.iters, R.rel);
    }
    if (pd > 0) {   // x <- x - W R^{-1} xi  (R upper triangular)
      std::vector<double> y(pd);
      for (int i = pd - 1; i >= 0; --i) {
        double acc = xi[i];
        for (int l = i + 1; l < pd; ++l) acc -= B.Raw[(size_t)l * pd + i] * y[l];
        y[i] = acc / B.Raw[(size_t)i * pd + i];
      }
      TRY(to_dev(g, g->small, y.data(), pd));
      TRY(basis_expand(g, g->small, -1.0, g->x));
    }
  } else {  // FPI, Algorithm 1: x <- Pi_h(x; f_d)
    const double bnorm = sqrt(bb);
    while (R.iters < maxit) {
      TRY(wave_solve(g, c.tg, g->x, fpi_force, g->q, 0));
      c.ws++;
      if (c.redefl) TRY(deflate_vec(g, g->q));
      TRY(copy_dev(g, g->r, g->q, N));
      TRY(axpby(g, N, -1.0, g->x, 1.0, g->r));
      TRY(copy_dev(g, g->x, g->q, N));
      ++R.iters;
      if (R.iters % check == 0 || R.iters == maxit) {
        TRY(dot_async(g, g->r, g->r, S_TMP));
        TRY(fetch_scalars(g));
        R.rel = sqrt(g->scal_host[S_TMP]) / bnorm;
        if (!isfinite(R.rel)) { R.breakdown = true; break; }
        if (R.rel <= tol) { R.converged = true; break; }
      }
    }
  }
  *res = R;
  return WHV_OK;
}

// Solve A x = b for a given FP64 right-hand side b (||b||_M^2 = bb) into g->xo by correction
// passes: r = b - A x (FP64 wave solves when fp64_res, else the grid's stepping; with a forcing
// f_res, r = Pi_h(x; f_res) - x, the same residual for b = Pi_h(0; f_res) by one forced wave
// solve, so that b is needed only as the first pass's right-hand side), then
// x += W diag(1/mu) W^T M r (deflated components; with a basis set and a method other than DCG)
// + the inner Krylov solution of the rest.  With fp64_res the passes repeat until the residual
// meets p->tol (iterative refinement); without it one pass is made (x0 = 0: exact DEVD for
// exact eigenvectors).  use_x0: g->xo holds the initial guess.
static whv_status outer_solve(SolveCtx& c, int method, const whv_params* p, const double* b, double bb,
                              bool fp64_res, bool use_x0, InnerResult* res, int* n_outer,
                              const double* f_res = nullptr) {
  whv_grid g = c.g;
  const int64_t N = g->N;
  const Basis& B = g->basis;
  // Deflated components of the residual before each inner solve (Algorithm 2 solves them
  // directly, the accelerator iterates on the rest):
  //  - exact eigenvectors: the modal solve x += W diag(1/mu) c, r -= W c, c = W^T M r;
  //  - approximate ones (Lanczos), with the FP64 correction: the Galerkin solve on span(W),
  //    y = (W^T M A W)^{-1} W^T M r, x += W y, r -= (A W) y (A W formed once, as for Algorithm 4
  //    with a general basis), after which W^T M r = 0: the residual is consistent with the
  //    re-deflated operator the inner iteration applies, and the outer FP64 passes correct what
  //    the stepping precision and the inexact vectors leave.  (W diag(1/mu) W^T M is not a
  //    Galerkin solve for approximate vectors and the passes can diverge.)
  // DCG and the augmented methods use the basis inside the iteration instead.
  const bool devd = B.nd > 0 && method != WHV_DCG && !augmented(method);
  const bool defl = devd && (B.flags & WHV_BASIS_EXACT);
  const bool gal = devd && !(B.flags & WHV_BASIS_EXACT) && fp64_res;
  if (gal) TRY(prepare_general_dcg(c));
  const double inner_tol = fp64_res ? (p->inner_tol > 0.0 ? p->inner_tol : 1e-3) : p->tol;
  if (!use_x0) WHV_CUDA(g, cudaMemsetAsync(g->xo, 0, N * sizeof(double), g->stream));
  bool have_x = use_x0;
  int its = 0, outer = 0;
  InnerResult R;
  R.rel = 1.0;
  std::vector<double> cf(defl ? B.nd : 0), y(defl ? B.nd : 0);
  while (true) {
    if (have_x) {
      if (fp64_res) {
        TRY(wave_solve(g, c.tg, g->xo, f_res, g->q, 1, c.res_prec));
        c.ws64++;
      } else {
        TRY(wave_solve(g, c.tg, g->xo, f_res, g->q, 1));
        c.ws++;
      }
      if (f_res) {   // q = x - Pi_h(x; f) = -r
        TRY(axpby(g, N, -1.0, g->q, 0.0, g->ro));
      } else {
        TRY(copy_dev(g, g->ro, b, N));
        TRY(axpby(g, N, -1.0, g->q, 1.0, g->ro));
      }
    } else {
      TRY(copy_dev(g, g->ro, b, N));
    }
    TRY(dot_async(g, g->ro, g->ro, S_TMP2));
    TRY(fetch_scalars(g));
    R.rel = bb > 0.0 ? sqrt(g->scal_host[S_TMP2] / bb) : 0.0;
    if (log_on()) fprintf(stderr, "[whv] outer %d: residual %.3e (inner iterations so far %d)\n", outer, R.rel, its);
    if (!isfinite(R.rel)) { R.breakdown = true; break; }
    if (R.rel <= p->tol) { R.converged = true; break; }
    if (its >= p->maxit || outer >= 50 || (!fp64_res && outer >= 1)) break;
    if (defl) {
      // deflated components: x += W diag(1/mu) c, r -= W c, c = W^T M r
      TRY(basis_project(g, g->ro, g->small));
      TRY(to_host(g, cf.data(), g->small, B.nd));
      for (int m = 0; m < B.nd; ++m) y[m] = cf[m] / B.mu[m];
      TRY(to_dev(g, g->small, y.data(), B.nd));
      TRY(basis_expand(g, g->small, 1.0, g->xo));
      TRY(to_dev(g, g->small, cf.data(), B.nd));
      TRY(basis_expand(g, g->small, -1.0, g->ro));
    } else if (gal) {
      TRY(basis_project(g, g->ro, g->small));
      TRY(small_matvec(g, B.Einv, g->small, B.nd, g->small2));
      TRY(basis_expand(g, g->small2, 1.0, g->xo));
      TRY(expand(g, B.AW, B.nd, g->small2, -1.0, g->ro));
    }
    TRY(dot_async(g, g->ro, g->ro, S_TMP2));
    TRY(fetch_scalars(g));
    const double rr = g->scal_host[S_TMP2];
    InnerResult Ri;
    const double itol = fp64_res ? correction_tol(inner_tol, p->tol, R.rel, outer)
                                 : p->tol * sqrt(bb / std::max(rr, 1e-300));
    TRY(inner_solve(c, method, p, g->ro, rr, false, itol, p->maxit - its, nullptr, &Ri));
    if (log_on())
      fprintf(stderr, "[whv]   inner solve: %d iterations, rel %.3e (target %.1e)%s%s\n", Ri.iters, Ri.rel, itol,
              Ri.converged ? "" : " not converged", Ri.breakdown ? " BREAKDOWN" : "");
    its += Ri.iters;
    ++outer;
    TRY(axpby(g, N, 1.0, g->x, 1.0, g->xo));
    have_x = true;
    if (Ri.breakdown) { R.breakdown = true; break; }
    if (!fp64_res) {   // single pass: the inner solve's own residual is the answer
      R.converged = Ri.converged;
      R.rel = Ri.rel * sqrt(rr / bb);
      break;
    }
  }
  R.iters = its;
  *res = R;
  *n_outer = outer;
  return WHV_OK;
}

}  // namespace whv

using namespace whv;

// pre_fd: the forcing already deflated by the caller (whv_solve_many); the DEVD projection and
// the inflation are then left to the caller as well
static whv_status solve_impl(whv_grid g, const whv_params* p, const double* f, int use_guess, double* u,
                             whv_info* info, const double* pre_fd = nullptr) {
  const double t0 = now_s();
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!f || !u) return fail(g, WHV_ERR_INVALID, "f_dev and u_dev must not be NULL");
  TimeGridH tg;
  TRY(make_time_grid(g, p, &tg));
  if (!(p->tol >= 0.0) || p->maxit < 0) return fail(g, WHV_ERR_INVALID, "tol must be >= 0, maxit >= 0");
  const int method = p->method;
  if (method < WHV_FPI || method > WHV_ABICGSTAB) return fail(g, WHV_ERR_INVALID, "unknown method");
  Basis& B = g->basis;
  const bool has_basis = B.nd > 0;
  if (has_basis && (B.omega != p->omega || B.periods != p->periods ||
                    B.adjust != (p->adjust_omega ? 1 : 0) || B.cfl != tg.cfl))
    return fail(g, WHV_ERR_INVALID, "deflation basis was set for another frequency / time grid");
  if (method == WHV_DCG && !has_basis) return fail(g, WHV_ERR_INVALID, "DCG needs a deflation basis");
  const bool refine = (p->flags & WHV_REFINE_FP64) != 0;
  if (refine && method == WHV_FPI)
    return fail(g, WHV_ERR_INVALID, "FP64 residual correction needs a Krylov method (CG, DCG, (A)GMRES, ABICGSTAB)");
  // DCG and AGMRES use the basis inside the iteration; the others deflate the forcing (DEVD)
  const bool devd = has_basis && method != WHV_DCG && !augmented(method);
  const int64_t N = g->N;
  SolveCtx c{g, tg, has_basis && (B.flags & WHV_BASIS_REDEFLATE) != 0 && !augmented(method)};
  if (refine && (p->flags & WHV_RESIDUAL_DF64) && !g->cons) c.res_prec = kPrecDF64;
  double* b = g->t;  // b of the iterated system

  // ---- forcing (Algorithm 2: deflate the forcing)
  const double* fuse = f;
  if (devd && !refine && pre_fd) {
    fuse = pre_fd;
  } else if (devd && !refine) {
    TRY(basis_project(g, f, B.d_coef));
    TRY(copy_dev(g, g->fd, f, N));
    TRY(basis_expand(g, B.d_coef, -1.0, g->fd));
    fuse = g->fd;
  }

  InnerResult R;
  int outer = 0;
  if (!refine) {
    TRY(wave_solve(g, tg, nullptr, fuse, b, 0));
    c.ws++;
    TRY(dot_async(g, b, b, S_RR0));
    TRY(fetch_scalars(g));
    const double bb = g->scal_host[S_RR0];
    if (!isfinite(bb)) return fail(g, WHV_ERR_BREAKDOWN, "non-finite right-hand side b (NaN/Inf in f?)");
    if (use_guess) {
      TRY(copy_dev(g, g->x, u, N));
      if (devd) TRY(deflate_vec(g, g->x));
    }
    TRY(inner_solve(c, method, p, b, bb, use_guess != 0, p->tol, p->maxit, fuse, &R));
  } else {
    // ---- iterative refinement with FP64 residuals on the full system b = Pi_h(0; f): b in the
    // stepping precision (the first pass's right-hand side and |b|), every residual
    // r = Pi_h(x; f) - x by one FP64 (or double-float) forced wave solve
    TRY(ensure_fp64_buffers(g));
    TRY(wave_solve(g, tg, nullptr, f, g->bo, 0));
    c.ws++;
    TRY(dot_async(g, g->bo, g->bo, S_RR0));
    TRY(fetch_scalars(g));
    const double bb = g->scal_host[S_RR0];
    if (!isfinite(bb)) return fail(g, WHV_ERR_BREAKDOWN, "non-finite right-hand side b (NaN/Inf in f?)");
    if (use_guess) TRY(copy_dev(g, g->xo, u, N));
    TRY(outer_solve(c, method, p, g->bo, bb, true, use_guess != 0, &R, &outer, f));
    TRY(copy_dev(g, g->x, g->xo, N));
  }

  // ---- inflate (Algorithm 2): u = x + W diag(1/(omega_eff^2 - lambda^2)) W^T M f
  if (devd && !refine && !pre_fd) {
    std::vector<double> cf(B.nd);
    TRY(to_host(g, cf.data(), B.d_coef, B.nd));
    const double om2 = tg.omega_eff * tg.omega_eff;
    for (int m = 0; m < B.nd; ++m) cf[m] = cf[m] / (om2 - B.lambda2[m]);
    TRY(to_dev(g, g->small, cf.data(), B.nd));
    TRY(basis_expand(g, g->small, 1.0, g->x));
  }
  TRY(copy_dev(g, u, g->x, N));

  double true_rel = -1.0;
  if (p->flags & WHV_TRUE_RESIDUAL) {
    // ||Pi_h(u; f) - u|| / ||Pi_h(0; f)||, in FP64 when the grid has FP64 buffers
    const int tp = (refine || g->precision == WHV_FP64) ? WHV_FP64 : g->precision;
    TRY(wave_solve(g, tg, u, f, g->q, 0, tp));
    TRY(copy_dev(g, g->r, g->q, N));
    TRY(axpby(g, N, -1.0, u, 1.0, g->r));
    TRY(dot_async(g, g->r, g->r, S_TMP));
    TRY(wave_solve(g, tg, nullptr, f, g->q, 0, tp));
    TRY(dot_async(g, g->q, g->q, S_TMP2));
    if (tp == WHV_FP64 && g->precision != WHV_FP64) c.ws64 += 2; else c.ws += 2;
    TRY(fetch_scalars(g));
    true_rel = sqrt(g->scal_host[S_TMP] / g->scal_host[S_TMP2]);
  }
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  if (info) {
    info->iterations = R.iters;
    info->wave_solves = c.ws + c.ws64;
    info->nt = tg.nt;
    info->dt = tg.dt;
    info->omega_hat = tg.omega_hat;
    info->omega_eff = tg.omega_eff;
    info->rel_residual = R.rel;
    info->true_rel_residual = true_rel;
    info->seconds = now_s() - t0;
    info->outer_iterations = outer;
    info->wave_solves_fp64 = (g->precision == WHV_FP64) ? c.ws + c.ws64 : c.ws64;
  }
  if (R.breakdown) return fail(g, WHV_ERR_BREAKDOWN, "Krylov breakdown (non-finite or non-positive scalar)");
  if (!R.converged) return fail(g, WHV_ERR_NOT_CONVERGED, "maxit reached before the tolerance");
  return WHV_OK;
}

// ------------------------------------------------------------------ adjoint
namespace whv {
whv_status adjoint_gradients(whv_grid g, const TimeGridH& tg, const double* u, const double* f,
                             const double* lam, double* gc2, double* gf, int K, int prec);
whv_status scale_by(whv_grid g, const double* x, const double* y, double a, double* out);
}  // namespace whv

static whv_status adjoint_impl(whv_grid g, const whv_params* p, const double* f, const double* u,
                               const double* dLdu, double* z, double* grad_c2, double* grad_f,
                               int checkpoint_every, whv_info* info) {
  const double t0 = now_s();
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!u || !dLdu || !z) return fail(g, WHV_ERR_INVALID, "u_dev, dLdu_dev and z_dev must not be NULL");
  TimeGridH tg;
  TRY(make_time_grid(g, p, &tg));
  const int method = p->method;
  if (method == WHV_FPI || method < 0 || method > WHV_ABICGSTAB)
    return fail(g, WHV_ERR_INVALID, "the adjoint solve needs a Krylov method (CG, DCG, (A)GMRES, ABICGSTAB)");
  const Basis& B = g->basis;
  if (B.nd > 0 && (B.omega != p->omega || B.periods != p->periods || B.adjust != (p->adjust_omega ? 1 : 0) ||
                   B.cfl != tg.cfl))
    return fail(g, WHV_ERR_INVALID, "deflation basis was set for another frequency / time grid");
  if (method == WHV_DCG && B.nd == 0) return fail(g, WHV_ERR_INVALID, "DCG needs a deflation basis");
  const int K = checkpoint_every > 0 ? checkpoint_every : 16;
  if (K > 1024) return fail(g, WHV_ERR_INVALID, "checkpoint_every must be <= 1024");
  if (g->cons) return fail(g, WHV_ERR_INVALID, "the adjoint differentiates the non-conservative operator c^2 Delta_h");
  const bool refine = (p->flags & WHV_REFINE_FP64) != 0;
  const int64_t N = g->N;
  TRY(ensure_fp64_buffers(g));
  SolveCtx c{g, tg, B.nd > 0 && (B.flags & WHV_BASIS_REDEFLATE) != 0 && !augmented(method)};
  // (I - S)^T lambda = g  <=>  (I - S) y = c^2 g,  lambda = y / c^2
  TRY(scale_by(g, dLdu, g->c2, 1.0, g->t));
  TRY(dot_async(g, g->t, g->t, S_RR0));
  TRY(fetch_scalars(g));
  const double bb = g->scal_host[S_RR0];
  if (!isfinite(bb)) return fail(g, WHV_ERR_BREAKDOWN, "non-finite dL/du");
  InnerResult R;
  int outer = 0;
  TRY(outer_solve(c, method, p, g->t, bb, refine, false, &R, &outer));
  TRY(scale_by(g, g->xo, g->mw, 1.0, z));
  // lambda^T dPi_h(u; f, c^2) / d(c^2, f): checkpointed reverse sweep -- like a residual it is a
  // single pass whose rounding is not corrected afterwards, so with the FP64 residual correction
  // it runs in FP64 (an FP32 sweep over a few hundred steps carries ~1e-3 relative errors)
  if (grad_c2 || grad_f)
    TRY(adjoint_gradients(g, tg, u, f, z, grad_c2, grad_f, K, refine ? WHV_FP64 : g->precision));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  if (info) {
    info->iterations = R.iters;
    info->wave_solves = c.ws + c.ws64 + ((grad_c2 || grad_f) ? 2 : 0);
    info->nt = tg.nt;
    info->dt = tg.dt;
    info->omega_hat = tg.omega_hat;
    info->omega_eff = tg.omega_eff;
    info->rel_residual = R.rel;
    info->true_rel_residual = -1.0;
    info->seconds = now_s() - t0;
    info->outer_iterations = outer;
    info->wave_solves_fp64 = (g->precision == WHV_FP64) ? info->wave_solves : c.ws64;
  }
  (void)N;
  if (R.breakdown) return fail(g, WHV_ERR_BREAKDOWN, "Krylov breakdown in the adjoint solve");
  if (!R.converged) return fail(g, WHV_ERR_NOT_CONVERGED, "adjoint solve: maxit reached before the tolerance");
  return WHV_OK;
}

extern "C" whv_status whv_solve(whv_grid g, const whv_params* p, const double* f, int use_guess,
                                double* u, whv_info* info) {
  return solve_impl(g, p, f, use_guess, u, info);
}

extern "C" whv_status whv_solve_adjoint(whv_grid g, const whv_params* p, const double* f, const double* u,
                                        const double* dLdu, double* z, double* grad_c2, double* grad_f,
                                        int checkpoint_every, whv_info* info) {
  return adjoint_impl(g, p, f, u, dLdu, z, grad_c2, grad_f, checkpoint_every, info);
}

// Vector-Jacobian product of out = Pi_h(v; f, c^2) (the reverse sweep on its own): for the seed
// abar, vbar = S_h^T abar = M S_h (M^{-1} abar) by one forward wave solve, (c2bar, fbar) =
// abar^T dPi_h/d(c^2, f) by the checkpointed transposed sweep from v.
static whv_status vjp_impl(whv_grid g, const whv_params* p, const double* v, const double* f, const double* abar,
                           double* vbar, double* c2bar, double* fbar, int checkpoint_every) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!v || !abar) return fail(g, WHV_ERR_INVALID, "v_dev and abar_dev must not be NULL");
  if (vbar && (vbar == abar || vbar == v)) return fail(g, WHV_ERR_INVALID, "vbar_dev must not alias v_dev or abar_dev");
  if (g->cons) return fail(g, WHV_ERR_INVALID, "the adjoint differentiates the non-conservative operator c^2 Delta_h");
  TimeGridH tg;
  TRY(make_time_grid(g, p, &tg));
  const int K = checkpoint_every > 0 ? checkpoint_every : 16;
  if (K > 1024) return fail(g, WHV_ERR_INVALID, "checkpoint_every must be <= 1024");
  const int prec = (p->flags & WHV_REFINE_FP64) ? WHV_FP64 : g->precision;
  if (prec == WHV_FP64 && g->precision != WHV_FP64) TRY(ensure_fp64_buffers(g));
  if (c2bar || fbar) TRY(adjoint_gradients(g, tg, v, f, abar, c2bar, fbar, K, prec));
  if (vbar) {
    TRY(scale_by(g, abar, g->c2, 1.0, g->t));                // c^2 abar
    TRY(wave_solve(g, tg, g->t, nullptr, vbar, 0, prec));     // S_h (c^2 abar)
    TRY(scale_by(g, vbar, g->mw, 1.0, vbar));                // / c^2
  }
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

extern "C" whv_status whv_apply_pi_vjp(whv_grid g, const whv_params* p, const double* v, const double* f,
                                       const double* abar, double* vbar, double* c2bar, double* fbar,
                                       int checkpoint_every) {
  return vjp_impl(g, p, v, f, abar, vbar, c2bar, fbar, checkpoint_every);
}

extern "C" whv_status whv_inject_barrier_error(whv_grid g) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  g->barrier_fault = true;
  return WHV_OK;
}

// Several right-hand sides on one grid: column j of F (leading dimension ld) -> column j of U,
// each by whv_solve with the same parameters; the basis, its derived quantities (A W, QR factors)
// and the captured CUDA graphs are built for the first and reused by the others.
extern "C" whv_status whv_solve_many(whv_grid g, const whv_params* p, int nrhs, int64_t ld, const double* F,
                                     int use_guess, double* U, whv_info* infos) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (nrhs < 0 || (nrhs > 0 && (!F || !U)) || ld < g->N)
    return fail(g, WHV_ERR_INVALID, "need nrhs >= 0, ld >= N and non-NULL F, U");
  whv_status worst = WHV_OK;
  const Basis& B = g->basis;
  const int method = p ? p->method : -1;
  // DEVD with a dense basis (Algorithm 2 with FPI / CG / GMRES, no FP64 correction, no initial
  // guesses, no true-residual check): the forcings are deflated and the solutions inflated all at
  // once -- W^T M F, F_d = F - W C and U += W diag(1/(omega_eff^2 - lambda^2)) C each read W once
  // for all columns -- and the columns are solved on F_d (written into U, which receives the
  // solution in place).
  const bool many = nrhs > 1 && !use_guess && B.nd > 0 && B.V && p && method != WHV_DCG &&
                    method != WHV_AGMRES && method != WHV_ABICGSTAB &&
                    !(p->flags & (WHV_REFINE_FP64 | WHV_TRUE_RESIDUAL));
  if (many) {
    TimeGridH tg;
    TRY(make_time_grid(g, p, &tg));
    if (B.omega != p->omega || B.periods != p->periods || B.adjust != (p->adjust_omega ? 1 : 0) || B.cfl != tg.cfl)
      return fail(g, WHV_ERR_INVALID, "deflation basis was set for another frequency / time grid");
    const int nd = B.nd;
    const int64_t N = g->N;
    std::vector<void*> tmp;
    auto cleanup = [&]() {
      cudaStreamSynchronize(g->stream);
      for (void* q : tmp) cudaFree(q);
    };
    auto alloc = [&](void** q, size_t bytes) {
      const cudaError_t e = cudaMalloc(q, bytes);
      if (e == cudaSuccess) tmp.push_back(*q);
      return e;
    };
    double *C = nullptr, *part = nullptr, *scale = nullptr;
    const double** fp = nullptr;
    double** up = nullptr;
    cudaError_t e = alloc((void**)&C, (size_t)nd * nrhs * 8);
    if (e == cudaSuccess) e = alloc((void**)&part, (size_t)project_many_scratch(N, nd, nrhs) * 8);
    if (e == cudaSuccess) e = alloc((void**)&scale, (size_t)nd * 8);
    if (e == cudaSuccess) e = alloc((void**)&fp, (size_t)nrhs * sizeof(double*));
    if (e == cudaSuccess) e = alloc((void**)&up, (size_t)nrhs * sizeof(double*));
    std::vector<const double*> hf(nrhs);
    std::vector<double*> hu(nrhs);
    std::vector<double> hs(nd);
    const double om2 = tg.omega_eff * tg.omega_eff;
    for (int m = 0; m < nd; ++m) hs[m] = 1.0 / (om2 - B.lambda2[m]);
    for (int j = 0; j < nrhs; ++j) {
      hf[j] = F + (size_t)j * ld;
      hu[j] = U + (size_t)j * ld;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(fp, hf.data(), nrhs * sizeof(double*), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(up, hu.data(), nrhs * sizeof(double*), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scale, hs.data(), nd * 8, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = project_many(g->stream, B.V, N, nd, nrhs, fp, g->mw, part, C);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(U, ld * 8, F, ld * 8, N * 8, nrhs, cudaMemcpyDeviceToDevice, g->stream);
    if (e == cudaSuccess) e = expand_many(g->stream, B.V, N, nd, nrhs, C, nullptr, -1.0, up);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(g, e, "whv_solve_many: deflation of the forcings"); }
    for (int j = 0; j < nrhs; ++j) {
      const whv_status st = solve_impl(g, p, hf[j], 0, hu[j], infos ? infos + j : nullptr, hu[j]);
      if (st == WHV_ERR_NOT_CONVERGED) { worst = st; continue; }
      if (st != WHV_OK) { cleanup(); return st; }
    }
    e = expand_many(g->stream, B.V, N, nd, nrhs, C, scale, 1.0, up);   // inflate every column
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(g, e, "whv_solve_many: inflation");
  } else {
    for (int j = 0; j < nrhs; ++j) {
      const whv_status s = whv_solve(g, p, F + (size_t)j * ld, use_guess, U + (size_t)j * ld,
                                     infos ? infos + j : nullptr);
      if (s == WHV_ERR_NOT_CONVERGED) { worst = s; continue; }   // keep going: the iterate is written
      if (s != WHV_OK) return s;
    }
  }
  if (worst != WHV_OK) return fail(g, worst, "whv_solve_many: some right-hand sides did not reach tol");
  return WHV_OK;
}
