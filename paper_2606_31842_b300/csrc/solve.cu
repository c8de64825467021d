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
//  * FPI (Algorithm 1).
#include <math.h>

#include <chrono>
#include <vector>

#include "whv_internal.cuh"

namespace whv {

struct SolveCtx {
  whv_grid g;
  const TimeGridH& tg;
  int ws = 0;
};

static whv_status copy_dev(whv_grid g, double* dst, const double* src, int64_t n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  return WHV_OK;
}

static whv_status to_host(whv_grid g, double* dst, const double* src, int n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

static whv_status to_dev(whv_grid g, double* dst, const double* src, int n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  // src is pageable host memory that may be reused right after: wait for the copy
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

#define TRY(expr)                          \
  do {                                     \
    whv_status _s = (expr);                \
    if (_s != WHV_OK) return _s;           \
  } while (0)

// out = out - W (W^T M out)
static whv_status deflate_vec(whv_grid g, double* vec) {
  const Basis& B = g->basis;
  TRY(project(g, B.V, B.nd, vec, g->small));
  return expand(g, B.V, B.nd, g->small, -1.0, vec);
}

// q = A v (+ re-deflation); scal[S_PQ] = <v, q>_M
static whv_status apply_A(SolveCtx& c, const double* v, double* q, bool redefl) {
  whv_grid g = c.g;
  TRY(wave_solve(g, c.tg, v, nullptr, q, 1));
  c.ws++;
  if (redefl) {
    TRY(deflate_vec(g, q));
    TRY(dot_async(g, v, q, S_PQ));
  }
  return WHV_OK;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace whv

using namespace whv;

extern "C" whv_status whv_solve(whv_grid g, const whv_params* p, const double* f, int use_guess,
                                double* u, whv_info* info) {
  const double t0 = now_s();
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!f || !u) return fail(g, WHV_ERR_INVALID, "f_dev and u_dev must not be NULL");
  TimeGridH tg;
  TRY(make_time_grid(g, p, &tg));
  if (!(p->tol >= 0.0) || p->maxit < 0) return fail(g, WHV_ERR_INVALID, "tol must be >= 0, maxit >= 0");
  const int method = p->method;
  if (method < WHV_FPI || method > WHV_GMRES) return fail(g, WHV_ERR_INVALID, "unknown method");
  Basis& B = g->basis;
  const bool has_basis = B.nd > 0;
  if (has_basis && (B.omega != p->omega || B.periods != p->periods ||
                    B.adjust != (p->adjust_omega ? 1 : 0) || B.cfl != tg.cfl))
    return fail(g, WHV_ERR_INVALID, "deflation basis was set for another frequency / time grid");
  if (method == WHV_DCG && !has_basis) return fail(g, WHV_ERR_INVALID, "DCG needs a deflation basis");
  if (method == WHV_DCG && !(B.flags & WHV_BASIS_EXACT))
    return fail(g, WHV_ERR_INVALID, "DCG is built for exact eigenvector bases (WHV_BASIS_EXACT)");
  const bool devd = has_basis && method != WHV_DCG;
  const bool redefl = has_basis && (B.flags & WHV_BASIS_REDEFLATE);
  const int check = p->check_every > 0 ? p->check_every : 1;
  const int64_t N = g->N;
  SolveCtx c{g, tg};
  double* b = g->t;  // b of the iterated system

  // ---- forcing (Algorithm 2: deflate the forcing)
  const double* fuse = f;
  if (devd) {
    TRY(project(g, B.V, B.nd, f, B.d_coef));
    TRY(copy_dev(g, g->fd, f, N));
    TRY(expand(g, B.V, B.nd, B.d_coef, -1.0, g->fd));
    fuse = g->fd;
  }
  TRY(wave_solve(g, tg, nullptr, fuse, b, 0));
  c.ws++;
  TRY(dot_async(g, b, b, S_RR0));
  TRY(fetch_scalars(g));
  double bb = g->scal_host[S_RR0];
  if (!isfinite(bb)) return fail(g, WHV_ERR_BREAKDOWN, "non-finite right-hand side b (NaN/Inf in f?)");

  // ---- initial guess
  if (use_guess) {
    TRY(copy_dev(g, g->x, u, N));
    if (devd) TRY(deflate_vec(g, g->x));
    TRY(apply_A(c, g->x, g->q, redefl));
    TRY(copy_dev(g, g->r, b, N));
    TRY(axpby(g, N, -1.0, g->q, 1.0, g->r));
  } else {
    WHV_CUDA(g, cudaMemsetAsync(g->x, 0, N * sizeof(double), g->stream));
    TRY(copy_dev(g, g->r, b, N));
  }

  int iters = 0;
  bool converged = false, breakdown = false;
  double rel = 1.0;

  if (bb == 0.0) {
    converged = true;
    rel = 0.0;
  } else if (method == WHV_CG || method == WHV_DCG) {
    double rr0 = bb;
    if (method == WHV_DCG) {
      // x_0 = x_{-1} + W diag(1/mu) W^T M r_{-1};  r_0 = r_{-1} - W W^T M r_{-1}  (A W = W diag(mu))
      std::vector<double> cf(B.nd);
      TRY(project(g, B.V, B.nd, g->r, g->small));
      TRY(to_host(g, cf.data(), g->small, B.nd));
      std::vector<double> y(B.nd);
      for (int m = 0; m < B.nd; ++m) y[m] = cf[m] / B.mu[m];
      TRY(to_dev(g, g->small, y.data(), B.nd));
      TRY(expand(g, B.V, B.nd, g->small, 1.0, g->x));
      TRY(to_dev(g, g->small, cf.data(), B.nd));
      TRY(expand(g, B.V, B.nd, g->small, -1.0, g->r));
    }
    TRY(copy_dev(g, g->p, g->r, N));
    TRY(dot_async(g, g->r, g->r, S_RR));
    TRY(fetch_scalars(g));
    const double rrs = g->scal_host[S_RR];
    if (method == WHV_DCG) rr0 = rrs;  // Algorithm 4: relative to the deflated start residual
    WHV_CUDA(g, cudaMemsetAsync(g->scal + S_FLAG, 0, sizeof(double), g->stream));
    rel = rr0 > 0.0 ? sqrt(rrs / rr0) : 0.0;
    if (rel <= p->tol) converged = true;
    while (!converged && iters < p->maxit) {
      TRY(apply_A(c, g->p, g->q, redefl));
      TRY(cg_update(g));
      TRY(cg_direction(g));
      ++iters;
      if (iters % check == 0 || iters == p->maxit) {
        TRY(fetch_scalars(g));
        if (g->scal_host[S_FLAG] != 0.0) { breakdown = true; break; }
        rel = sqrt(g->scal_host[S_RR] / rr0);
        if (rel <= p->tol) converged = true;
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
      if (!isfinite(beta0)) { breakdown = true; break; }
      rel = beta0 / bnorm;
      if (rel <= p->tol) { converged = true; break; }
      if (iters >= p->maxit) break;
      TRY(axpby(g, N, 1.0 / beta0, g->r, 0.0, K));
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = beta0;
      int k = 0;
      bool lucky = false;
      for (int j = 0; j < m; ++j) {
        double* w = K + (size_t)(j + 1) * N;
        TRY(apply_A(c, K + (size_t)j * N, w, redefl));
        ++iters;
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
        if (!isfinite(hn)) { breakdown = true; break; }
        Hc(j + 1, j) = hn;
        lucky = !(hn > 0.0);
        if (!lucky) TRY(axpby(g, N, 1.0 / hn, w, 0.0, w));
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
          Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
          Hc(i, j) = t;
        }
        const double den = hypot(Hc(j, j), Hc(j + 1, j));
        if (!(den > 0.0)) { breakdown = true; break; }
        cs[j] = Hc(j, j) / den;
        sn[j] = Hc(j + 1, j) / den;
        Hc(j, j) = den;
        Hc(j + 1, j) = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        k = j + 1;
        rel = fabs(gv[k]) / bnorm;
        if (rel <= p->tol || iters >= p->maxit || lucky) break;
      }
      if (breakdown && k == 0) break;
      for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= Hc(i, l) * y[l];
        y[i] = s / Hc(i, i);
      }
      TRY(to_dev(g, g->small, y.data(), k));
      TRY(expand(g, K, k, g->small, 1.0, g->x));
      if (breakdown) break;
      if (rel <= p->tol || lucky) { converged = true; break; }
      // restart: r = b - A x
      TRY(apply_A(c, g->x, g->q, redefl));
      TRY(copy_dev(g, g->r, b, N));
      TRY(axpby(g, N, -1.0, g->q, 1.0, g->r));
    }
  } else {  // FPI, Algorithm 1: v <- Pi_h(v; f_d)
    const double bnorm = sqrt(bb);
    while (iters < p->maxit) {
      TRY(wave_solve(g, tg, g->x, fuse, g->q, 0));
      c.ws++;
      if (redefl) TRY(deflate_vec(g, g->q));
      TRY(copy_dev(g, g->r, g->q, N));
      TRY(axpby(g, N, -1.0, g->x, 1.0, g->r));
      TRY(copy_dev(g, g->x, g->q, N));
      ++iters;
      if (iters % check == 0 || iters == p->maxit) {
        TRY(dot_async(g, g->r, g->r, S_TMP));
        TRY(fetch_scalars(g));
        rel = sqrt(g->scal_host[S_TMP]) / bnorm;
        if (!isfinite(rel)) { breakdown = true; break; }
        if (rel <= p->tol) { converged = true; break; }
      }
    }
  }

  // ---- inflate (Algorithm 2): u = x + W diag(1/(omega_eff^2 - lambda^2)) W^T M f
  if (devd) {
    std::vector<double> cf(B.nd);
    TRY(to_host(g, cf.data(), B.d_coef, B.nd));
    const double om2 = tg.omega_eff * tg.omega_eff;
    for (int m = 0; m < B.nd; ++m) cf[m] = cf[m] / (om2 - B.lambda2[m]);
    TRY(to_dev(g, g->small, cf.data(), B.nd));
    TRY(expand(g, B.V, B.nd, g->small, 1.0, g->x));
  }
  TRY(copy_dev(g, u, g->x, N));

  double true_rel = -1.0;
  if (p->flags & WHV_TRUE_RESIDUAL) {
    // ||Pi_h(u; f) - u|| / ||Pi_h(0; f)||
    TRY(wave_solve(g, tg, u, f, g->q, 0));
    TRY(copy_dev(g, g->r, g->q, N));
    TRY(axpby(g, N, -1.0, u, 1.0, g->r));
    TRY(dot_async(g, g->r, g->r, S_TMP));
    TRY(wave_solve(g, tg, nullptr, f, g->q, 0));
    TRY(dot_async(g, g->q, g->q, S_TMP2));
    c.ws += 2;
    TRY(fetch_scalars(g));
    true_rel = sqrt(g->scal_host[S_TMP] / g->scal_host[S_TMP2]);
  }
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  if (info) {
    info->iterations = iters;
    info->wave_solves = c.ws;
    info->nt = tg.nt;
    info->dt = tg.dt;
    info->omega_hat = tg.omega_hat;
    info->omega_eff = tg.omega_eff;
    info->rel_residual = rel;
    info->true_rel_residual = true_rel;
    info->seconds = now_s() - t0;
  }
  if (breakdown) return fail(g, WHV_ERR_BREAKDOWN, "Krylov breakdown (non-finite or non-positive scalar)");
  if (!converged) return fail(g, WHV_ERR_NOT_CONVERGED, "maxit reached before the tolerance");
  return WHV_OK;
}
