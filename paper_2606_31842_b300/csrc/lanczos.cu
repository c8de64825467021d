// Device eigen-solve for the deflation basis (EigenWave idea, Sec. 4.1): Lanczos on the
// WaveHoltz operator S_h.  Eigenvectors of L_h are eigenvectors of S_h with eigenvalue
// beta_h(lambda); the ones to deflate (lambda nearest the frequency, beta_h near 1) are the
// top of the spectrum of S_h, so they are the extremal Ritz pairs of a Krylov space of S_h.
//
//  * m steps of the Lanczos recurrence in the M inner product (S_h is M-self-adjoint); every
//    matrix-vector product is one f = 0 wave solve on the device; every new vector is
//    re-orthogonalised against all previous ones with classical Gram-Schmidt applied twice,
//    in FP64, with the tall-skinny contraction kernels of the deflation path.
//  * The m x m tridiagonal matrix: its nd largest eigenvalues by Sturm-sequence bisection,
//    their eigenvectors by inverse iteration (tridiagonal LU with partial pivoting),
//    re-orthogonalised inside clusters (host, O(nd m)).
//  * Ritz vectors Y = Q S on the device (k_ritz), lambda^2 = -<y, L_h y>_M / <y, y>_M with an
//    FP64 application of L_h, residuals ||L_h y + lambda^2 y||_M / lambda^2.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "stencil_ops.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

// SplitMix64 (Steele, Lea and Flood, 2014) as a counter-based generator: value i of stream seed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_start_vector(double* __restrict__ v, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = splitmix64(seed * 0x100000001B3ull + (uint64_t)i);
    v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;   // uniform in [-1, 1)
  }
}

// Y[:, j0 + c] = sum_k Q[:, k] S[k, j0 + c], c < JC (S column-major m x nd)
constexpr int kRitzJC = 8;
__global__ void __launch_bounds__(256) k_ritz(const double* __restrict__ Q, int64_t N, int m,
                                              const double* __restrict__ S, int nd, int j0,
                                              double* __restrict__ Y) {
  extern __shared__ double sS[];   // m x JC
  const int jc = min(kRitzJC, nd - j0);
  for (int t = threadIdx.x; t < m * kRitzJC; t += blockDim.x) {
    const int k = t / kRitzJC, c = t % kRitzJC;
    sS[t] = c < jc ? S[(int64_t)(j0 + c) * m + k] : 0.0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc[kRitzJC];
#pragma unroll
    for (int c = 0; c < kRitzJC; ++c) acc[c] = 0.0;
    for (int k = 0; k < m; ++k) {
      const double q = Q[i + (int64_t)k * N];
#pragma unroll
      for (int c = 0; c < kRitzJC; ++c) acc[c] = fma(q, sS[k * kRitzJC + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kRitzJC; ++c)
      if (c < jc) Y[i + (int64_t)(j0 + c) * N] = acc[c];
  }
}

// out = c^2 Delta_h y (FP64)
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_apply_L(const double* __restrict__ y, const double* __restrict__ c2,
                                                 double* __restrict__ out, int nx, int ny, int nz,
                                                 StepCoef<double> cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int yy = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || yy >= ny) return;
  const int64_t idx = x + (int64_t)nx * (yy + (int64_t)ny * z);
  double L = lap<DIM, ORDER, double>(y, idx, x, yy, z, nx, ny, nz, cf, y[idx]);
  if (c2) L *= c2[idx];
  out[idx] = L;
}

// out = div_h(c^2 grad_h) y (FP64, conservative form)
template <int DIM>
__global__ void __launch_bounds__(256) k_apply_L_cons(const double* __restrict__ y, ConsFaces<double> fc,
                                                      double* __restrict__ out, int nx, int ny, int nz,
                                                      StepCoef<double> cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int yy = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || yy >= ny) return;
  const int64_t idx = x + (int64_t)nx * (yy + (int64_t)ny * z);
  out[idx] = lap_cons<DIM, double>(y, idx, x, yy, z, nx, ny, nz, fc, cf, y[idx]);
}

static whv_status apply_L_fp64(whv_grid g, const double* y, double* out) {
  StepCoef<double> cf{};
  for (int m = 0; m < 3; ++m) {
    const double h2 = g->h[m] * g->h[m];
    cf.ih2[m] = g->order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2);
  }
  dim3 block, grid;
  if (g->dim == 1) { block = dim3(256, 1, 1); grid = dim3((g->n[0] + 255) / 256, 1, 1); }
  else { block = dim3(32, 8, 1); grid = dim3((g->n[0] + 31) / 32, (g->n[1] + 7) / 8, g->dim > 2 ? g->n[2] : 1); }
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  if (g->cons) {
    ConsFaces<double> fc{{g->face64[0], g->face64[1], g->face64[2]}, g->c2};
    if (g->dim == 1) k_apply_L_cons<1><<<grid, block, 0, g->stream>>>(y, fc, out, nx, ny, nz, cf);
    else if (g->dim == 2) k_apply_L_cons<2><<<grid, block, 0, g->stream>>>(y, fc, out, nx, ny, nz, cf);
    else k_apply_L_cons<3><<<grid, block, 0, g->stream>>>(y, fc, out, nx, ny, nz, cf);
    count_launches(1);
    WHV_CUDA(g, cudaGetLastError());
    return WHV_OK;
  }
  switch (g->dim * 10 + g->order) {
    case 12: k_apply_L<1, 2><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    case 14: k_apply_L<1, 4><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    case 22: k_apply_L<2, 2><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    case 24: k_apply_L<2, 4><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    case 32: k_apply_L<3, 2><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    case 34: k_apply_L<3, 4><<<grid, block, 0, g->stream>>>(y, g->c2, out, nx, ny, nz, cf); break;
    default: return fail(g, WHV_ERR_INVALID, "unsupported dim/order");
  }
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

// ------------------------------------------------------------------ host: tridiagonal problem
// number of eigenvalues of the symmetric tridiagonal (a, b) smaller than x (Sturm count)
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  const double tiny = 1e-300;
  for (int i = 0; i < k; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -tiny;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Solve (T - theta I) x = rhs in place with Gaussian elimination with partial pivoting.
static void tridiag_shift_solve(const std::vector<double>& a, const std::vector<double>& b, int k,
                                double theta, std::vector<double>& x, double tiny) {
  std::vector<double> d(k), du(k, 0.0), du2(k, 0.0), dl(k, 0.0);
  std::vector<int> piv(k);
  for (int i = 0; i < k; ++i) d[i] = a[i] - theta;
  for (int i = 0; i + 1 < k; ++i) { du[i] = b[i]; dl[i] = b[i]; }
  for (int i = 0; i + 1 < k; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) {
      if (d[i] == 0.0) d[i] = tiny;
      const double fct = dl[i] / d[i];
      dl[i] = fct;
      d[i + 1] -= fct * du[i];
      piv[i] = i;
    } else {
      const double fct = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = fct;
      const double tmp = du[i];
      du[i] = d[i + 1];
      d[i + 1] = tmp - fct * d[i + 1];
      if (i + 2 < k) {
        du2[i] = du[i + 1];
        du[i + 1] = -fct * du[i + 1];
      }
      piv[i] = i + 1;
    }
  }
  if (d[k - 1] == 0.0) d[k - 1] = tiny;
  // forward: apply row interchanges and L
  for (int i = 0; i + 1 < k; ++i) {
    if (piv[i] == i) {
      x[i + 1] -= dl[i] * x[i];
    } else {
      const double t = x[i];
      x[i] = x[i + 1];
      x[i + 1] = t - dl[i] * x[i];
    }
  }
  // back substitution with U (diagonal d, super du, second super du2)
  for (int i = k - 1; i >= 0; --i) {
    double s = x[i];
    if (i + 1 < k) s -= du[i] * x[i + 1];
    if (i + 2 < k) s -= du2[i] * x[i + 2];
    x[i] = s / d[i];
  }
}

// nd largest eigenpairs of the tridiagonal (a, b) of order k: values (descending) and
// eigenvectors S (column-major k x nd)
static void top_eigenpairs(const std::vector<double>& a, const std::vector<double>& b, int k, int nd,
                           std::vector<double>& theta, std::vector<double>& S) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const double tnorm = std::max(fabs(lo), fabs(hi));
  theta.assign(nd, 0.0);
  for (int j = 0; j < nd; ++j) {
    // eigenvalue number k-1-j in ascending order: count(x) <= idx < count(x') ...
    const int idx = k - 1 - j;
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 4e-16 * tnorm; ++it) {
      const double mid = 0.5 * (l + h);
      if (sturm_count(a, b, k, mid) <= idx) l = mid; else h = mid;
    }
    theta[j] = 0.5 * (l + h);
  }
  S.assign((size_t)k * nd, 0.0);
  const double tiny = 1e-14 * tnorm + 1e-300;
  uint64_t st = 88172645463325252ull;
  for (int j = 0; j < nd; ++j) {
    std::vector<double> x(k);
    for (int i = 0; i < k; ++i) {   // xorshift64 start vector
      st ^= st << 13; st ^= st >> 7; st ^= st << 17;
      x[i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    for (int it = 0; it < 4; ++it) {
      tridiag_shift_solve(a, b, k, theta[j], x, tiny);
      // orthogonalise against earlier vectors of the same cluster
      for (int p = 0; p < j; ++p) {
        if (fabs(theta[p] - theta[j]) > 1e-3 * tnorm) continue;
        double dp = 0.0;
        for (int i = 0; i < k; ++i) dp += x[i] * S[(size_t)p * k + i];
        for (int i = 0; i < k; ++i) x[i] -= dp * S[(size_t)p * k + i];
      }
      double nrm = 0.0;
      for (int i = 0; i < k; ++i) nrm += x[i] * x[i];
      nrm = sqrt(nrm);
      for (int i = 0; i < k; ++i) x[i] /= nrm;
    }
    for (int i = 0; i < k; ++i) S[(size_t)j * k + i] = x[i];
  }
}

}  // namespace whv

using namespace whv;

// Rayleigh quotients lambda^2 = -<y, L_h y>_M / <y, y>_M and residuals ||L_h y + lambda^2 y||_M /
// lambda^2 in FP64 for the nd Ritz vectors Y (N x nd, device, owned by the caller until this
// returns WHV_OK, then by the basis), and install them as the grid's WHV_BASIS_LANCZOS basis.
static whv_status install_ritz_basis(whv_grid g, const whv_params* p, const TimeGridH& tg, double* Y, int nd,
                                     const std::vector<double>& theta, int flags, double* theta_host,
                                     double* resid_host) {
  const int64_t N = g->N;
#define LZ_TRY(expr)                                \
  do {                                              \
    whv_status _s = (expr);                         \
    if (_s != WHV_OK) { cudaFree(Y); return _s; }   \
  } while (0)
  std::vector<double> lam2(nd), res(nd);
  for (int j = 0; j < nd; ++j) {
    const double* y = Y + (size_t)j * N;
    LZ_TRY(apply_L_fp64(g, y, g->q));
    LZ_TRY(dot_async(g, y, g->q, S_TMP));
    LZ_TRY(dot_async(g, y, y, S_TMP2));
    LZ_TRY(fetch_scalars(g));
    lam2[j] = -g->scal_host[S_TMP] / g->scal_host[S_TMP2];
    LZ_TRY(axpby(g, N, lam2[j], y, 1.0, g->q));   // q = L y + lambda^2 y
    LZ_TRY(dot_async(g, g->q, g->q, S_TMP));
    LZ_TRY(fetch_scalars(g));
    res[j] = sqrt(g->scal_host[S_TMP]) / fabs(lam2[j]);
  }
  if (getenv("WHV_LOG") && getenv("WHV_LOG")[0] == '1')
    for (int j = 0; j < nd; ++j)
      fprintf(stderr, "[whv] Lanczos pair %d: theta %.6f lambda^2 %.6e residual %.2e\n", j, theta[j], lam2[j], res[j]);
  if (theta_host) std::copy(theta.begin(), theta.end(), theta_host);
  if (resid_host) std::copy(res.begin(), res.end(), resid_host);
  // install as the deflation basis (approximate eigenvectors)
  Basis b;
  b.nd = nd; b.mode = WHV_BASIS_LANCZOS; b.flags = flags & ~WHV_BASIS_EXACT;
  b.omega = p->omega; b.periods = p->periods; b.adjust = p->adjust_omega ? 1 : 0; b.cfl = tg.cfl;
  b.V = Y;
  b.lambda2 = lam2;
  b.mu.resize(nd);
  for (int j = 0; j < nd; ++j) {
    const double x = 1.0 - 0.5 * tg.dt * tg.dt * lam2[j];
    const double th = acos(std::max(-1.0, std::min(1.0, x)));
    double be = 0.0;
    for (int n = 0; n <= tg.nt; ++n) be += tg.weight[n] * cos(n * th);
    b.mu[j] = 1.0 - be;
  }
  b.modes.assign((size_t)nd * g->dim, 0);
  cudaError_t e = cudaMalloc(&b.d_coef, (size_t)kMaxND * sizeof(double));
  if (e != cudaSuccess) { cudaFree(Y); return cuda_fail(g, e, "cudaMalloc"); }
  hold_vectors(b);
  free_basis(g);
  g->basis = std::move(b);
#undef LZ_TRY
  return WHV_OK;
}

static whv_status lanczos_impl(whv_grid g, const whv_params* p, int nd, int m, const double* v0_dev,
                                  int fp64_stepping, int flags, double* theta_host, double* resid_host) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  if (nd < 1 || nd > kMaxND || m < nd || m > kMaxND || m > g->N)
    return fail(g, WHV_ERR_INVALID, "need 1 <= nd <= m <= min(N, 1024)");
  const int prec = fp64_stepping ? WHV_FP64 : g->precision;
  if (prec == WHV_FP64 && g->precision != WHV_FP64) {
    s = ensure_fp64_buffers(g);
    if (s != WHV_OK) return s;
  }
  const int64_t N = g->N;
  double* Q = nullptr;
  double* Y = nullptr;
  double* dS = nullptr;
  auto cleanup = [&]() {
    if (Q) cudaFree(Q);
    if (dS) cudaFree(dS);
  };
#define LZ_TRY(expr)                                \
  do {                                              \
    whv_status _s = (expr);                         \
    if (_s != WHV_OK) { cleanup(); if (Y) cudaFree(Y); return _s; } \
  } while (0)
#define LZ_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) { cleanup(); if (Y) cudaFree(Y); return cuda_fail(g, _e, #call); } \
  } while (0)
  LZ_CUDA(cudaMalloc(&Q, (size_t)m * N * sizeof(double)));
  // start vector
  if (v0_dev) {
    LZ_CUDA(cudaMemcpyAsync(Q, v0_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  } else {
    k_start_vector<<<148 * 4, 256, 0, g->stream>>>(Q, N, 1ull);
    count_launches(1);
    LZ_CUDA(cudaGetLastError());
  }
  LZ_TRY(dot_async(g, Q, Q, S_TMP));
  LZ_TRY(fetch_scalars(g));
  if (!(g->scal_host[S_TMP] > 0.0)) { cleanup(); return fail(g, WHV_ERR_INVALID, "zero start vector"); }
  LZ_TRY(axpby(g, N, 1.0 / sqrt(g->scal_host[S_TMP]), Q, 0.0, Q));
  std::vector<double> alpha(m, 0.0), beta(m, 0.0), h1(m), h2(m);
  int k = 0;
  for (int j = 0; j < m; ++j) {
    double* qj = Q + (size_t)j * N;
    double* z = j + 1 < m ? Q + (size_t)(j + 1) * N : g->q;
    // z = S_h q_j through fixed buffers, so that every step replays one cached CUDA graph
    LZ_CUDA(cudaMemcpyAsync(g->p, qj, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    LZ_TRY(wave_solve(g, tg, g->p, nullptr, g->t, 0, prec));
    LZ_CUDA(cudaMemcpyAsync(z, g->t, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    LZ_TRY(project(g, Q, j + 1, z, g->small));
    LZ_TRY(expand(g, Q, j + 1, g->small, -1.0, z));
    cudaMemcpyAsync(h1.data(), g->small, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, g->stream);
    LZ_TRY(project(g, Q, j + 1, z, g->small));
    LZ_TRY(expand(g, Q, j + 1, g->small, -1.0, z));
    cudaMemcpyAsync(h2.data(), g->small, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, g->stream);
    LZ_TRY(dot_async(g, z, z, S_TMP));
    LZ_TRY(fetch_scalars(g));   // synchronises: h1, h2 are on the host too
    alpha[j] = h1[j] + h2[j];
    k = j + 1;
    const double bn = sqrt(g->scal_host[S_TMP]);
    if (!isfinite(bn)) { cleanup(); return fail(g, WHV_ERR_BREAKDOWN, "non-finite Lanczos vector"); }
    if (j + 1 < m) {
      beta[j] = bn;
      if (!(bn > 1e-14)) break;   // invariant subspace found
      LZ_TRY(axpby(g, N, 1.0 / bn, z, 0.0, z));
    }
  }
  if (k < nd) { cleanup(); return fail(g, WHV_ERR_INVALID, "Krylov space smaller than nd (invariant subspace)"); }
  std::vector<double> theta, S;
  top_eigenpairs(alpha, beta, k, nd, theta, S);
  LZ_CUDA(cudaMalloc(&dS, S.size() * sizeof(double)));
  LZ_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  LZ_CUDA(cudaMalloc(&Y, (size_t)nd * N * sizeof(double)));
  LZ_CUDA(cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kMaxND * kRitzJC * sizeof(double))));
  for (int j0 = 0; j0 < nd; j0 += kRitzJC) {
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, 148 * 8);
    k_ritz<<<blocks, 256, (size_t)k * kRitzJC * sizeof(double), g->stream>>>(Q, N, k, dS, nd, j0, Y);
    count_launches(1);
    LZ_CUDA(cudaGetLastError());
  }
  LZ_CUDA(cudaStreamSynchronize(g->stream));
  cleanup();
  Q = nullptr; dS = nullptr;
  return install_ritz_basis(g, p, tg, Y, nd, theta, flags, theta_host, resid_host);
#undef LZ_TRY
#undef LZ_CUDA
  return WHV_OK;
}

// ------------------------------------------------------------------ thick-restart Lanczos
static bool log_on_lz() {
  static const bool on = [] { const char* e = getenv("WHV_LOG"); return e && e[0] == '1'; }();
  return on;
}

// Top kw eigenpairs of the dense symmetric n x n matrix H (row-major): Householder reduction to
// tridiagonal form H = P T P^T, the tridiagonal eigenpairs by bisection and inverse iteration,
// eigenvectors S = P S_T (n x kw, column-major).
static void dense_top_eigenpairs(std::vector<double> A, int n, int kw, std::vector<double>& theta,
                                 std::vector<double>& S);

namespace whv {
// exported for the SVD compression (compress.cu)
void host_sym_top_eigenpairs(const std::vector<double>& A, int n, int kw, std::vector<double>& theta,
                             std::vector<double>& S) {
  dense_top_eigenpairs(A, n, kw, theta, S);
}
}  // namespace whv

static void dense_top_eigenpairs(std::vector<double> A, int n, int kw, std::vector<double>& theta,
                                 std::vector<double>& S) {
  std::vector<double> P((size_t)n * n, 0.0);   // row-major
  for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), pv(n), q(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;   // length of the column below the diagonal
    double nx = 0.0;
    for (int i = 0; i < m; ++i) nx += A[(size_t)(k + 1 + i) * n + k] * A[(size_t)(k + 1 + i) * n + k];
    nx = sqrt(nx);
    if (nx == 0.0) continue;
    const double x0 = A[(size_t)(k + 1) * n + k];
    const double alpha = x0 >= 0.0 ? -nx : nx;
    for (int i = 0; i < m; ++i) v[i] = A[(size_t)(k + 1 + i) * n + k];
    v[0] -= alpha;
    double nv = 0.0;
    for (int i = 0; i < m; ++i) nv += v[i] * v[i];
    nv = sqrt(nv);
    if (nv == 0.0) continue;
    for (int i = 0; i < m; ++i) v[i] /= nv;
    // trailing block: A22 <- (I - 2 v v^T) A22 (I - 2 v v^T) = A22 - 2 (v q^T + q v^T)
    for (int i = 0; i < m; ++i) {
      double sacc = 0.0;
      for (int j = 0; j < m; ++j) sacc += A[(size_t)(k + 1 + i) * n + (k + 1 + j)] * v[j];
      pv[i] = sacc;
    }
    double K = 0.0;
    for (int i = 0; i < m; ++i) K += v[i] * pv[i];
    for (int i = 0; i < m; ++i) q[i] = pv[i] - K * v[i];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[(size_t)(k + 1 + i) * n + (k + 1 + j)] -= 2.0 * (v[i] * q[j] + q[i] * v[j]);
    A[(size_t)(k + 1) * n + k] = A[(size_t)k * n + (k + 1)] = alpha;
    for (int i = 1; i < m; ++i) A[(size_t)(k + 1 + i) * n + k] = A[(size_t)k * n + (k + 1 + i)] = 0.0;
    // P <- P (I - 2 v v^T) on columns k+1 .. n-1
    for (int r = 0; r < n; ++r) {
      double sacc = 0.0;
      for (int j = 0; j < m; ++j) sacc += P[(size_t)r * n + (k + 1 + j)] * v[j];
      for (int j = 0; j < m; ++j) P[(size_t)r * n + (k + 1 + j)] -= 2.0 * sacc * v[j];
    }
  }
  std::vector<double> a(n), b(n, 0.0), St;
  for (int i = 0; i < n; ++i) a[i] = A[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) b[i] = A[(size_t)(i + 1) * n + i];
  top_eigenpairs(a, b, n, kw, theta, St);
  S.assign((size_t)n * kw, 0.0);
  for (int j = 0; j < kw; ++j)
    for (int r = 0; r < n; ++r) {
      double sacc = 0.0;
      for (int c = 0; c < n; ++c) sacc += P[(size_t)r * n + c] * St[(size_t)j * n + c];
      S[(size_t)j * n + r] = sacc;
    }
}

// Thick-restart Lanczos (Wu and Simon 2000) on S_h in the M inner product: basis of at most m
// vectors, the `keep` largest Ritz vectors and the residual vector carried over a restart.  Every
// step re-orthogonalises against the whole basis (classical Gram-Schmidt twice, FP64), so the
// projected matrix H = Q^T M S_h Q is filled from the Gram-Schmidt coefficients; the Ritz
// residual of pair i is |b s_{m,i}| with b the norm of the last, unnormalised vector.
static whv_status lanczos_thick_impl(whv_grid g, const whv_params* p, int nd, int m, int keep, int max_restarts,
                                     double tol, const double* v0_dev, int fp64_stepping, int flags,
                                     double* theta_host, double* resid_host, int* stats) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  if (keep <= 0) keep = std::min(m - 2, nd + std::max(nd / 2, 8));
  if (nd < 1 || keep < nd || keep > m - 2 || m > kMaxND || m > g->N || max_restarts < 0 || !(tol > 0.0))
    return fail(g, WHV_ERR_INVALID, "need 1 <= nd <= keep <= m - 2, m <= min(N, 1024), max_restarts >= 0, tol > 0");
  const int prec = fp64_stepping ? WHV_FP64 : g->precision;
  if (prec == WHV_FP64 && g->precision != WHV_FP64) {
    s = ensure_fp64_buffers(g);
    if (s != WHV_OK) return s;
  }
  const int64_t N = g->N;
  double *Q = nullptr, *Y = nullptr, *dS = nullptr;
  auto cleanup = [&]() { for (double* x : {Q, Y, dS}) if (x) cudaFree(x); };
#define TL_TRY(expr) do { whv_status _s = (expr); if (_s != WHV_OK) { cleanup(); return _s; } } while (0)
#define TL_CUDA(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) { cleanup(); return cuda_fail(g, _e, #call); } } while (0)
  TL_CUDA(cudaMalloc(&Q, (size_t)m * N * sizeof(double)));
  TL_CUDA(cudaMalloc(&Y, (size_t)keep * N * sizeof(double)));
  TL_CUDA(cudaMalloc(&dS, (size_t)m * keep * sizeof(double)));
  TL_CUDA(cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kMaxND * kRitzJC * sizeof(double))));
  if (v0_dev) {
    TL_CUDA(cudaMemcpyAsync(Q, v0_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  } else {
    k_start_vector<<<148 * 4, 256, 0, g->stream>>>(Q, N, 1ull);
    count_launches(1);
    TL_CUDA(cudaGetLastError());
  }
  TL_TRY(dot_async(g, Q, Q, S_TMP));
  TL_TRY(fetch_scalars(g));
  if (!(g->scal_host[S_TMP] > 0.0)) { cleanup(); return fail(g, WHV_ERR_INVALID, "zero start vector"); }
  TL_TRY(axpby(g, N, 1.0 / sqrt(g->scal_host[S_TMP]), Q, 0.0, Q));
  std::vector<double> H((size_t)m * m, 0.0), h1(m), h2(m), theta, S;
  int j0 = 0, restarts = 0, nws = 0, conv = 0;
  double bres = 0.0;
  while (true) {
    for (int j = j0; j < m; ++j) {
      double* qj = Q + (size_t)j * N;
      double* z = j + 1 < m ? Q + (size_t)(j + 1) * N : g->q;
      TL_CUDA(cudaMemcpyAsync(g->p, qj, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      TL_TRY(wave_solve(g, tg, g->p, nullptr, g->t, 0, prec));
      ++nws;
      TL_CUDA(cudaMemcpyAsync(z, g->t, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      TL_TRY(project(g, Q, j + 1, z, g->small));
      TL_TRY(expand(g, Q, j + 1, g->small, -1.0, z));
      cudaMemcpyAsync(h1.data(), g->small, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, g->stream);
      TL_TRY(project(g, Q, j + 1, z, g->small));
      TL_TRY(expand(g, Q, j + 1, g->small, -1.0, z));
      cudaMemcpyAsync(h2.data(), g->small, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, g->stream);
      TL_TRY(dot_async(g, z, z, S_TMP));
      TL_TRY(fetch_scalars(g));   // synchronises: h1, h2 are on the host too
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = H[(size_t)j * m + i] = h1[i] + h2[i];
      bres = sqrt(g->scal_host[S_TMP]);
      if (!isfinite(bres)) { cleanup(); return fail(g, WHV_ERR_BREAKDOWN, "non-finite Lanczos vector"); }
      if (bres > 1e-14) {
        TL_TRY(axpby(g, N, 1.0 / bres, z, 0.0, z));
      } else if (j + 1 < m) {
        cleanup();
        return fail(g, WHV_ERR_BREAKDOWN, "invariant subspace before the basis filled");
      }   // else: the full basis is invariant, every Ritz pair is exact (residual estimates 0)
      if (j + 1 < m) H[(size_t)(j + 1) * m + j] = H[(size_t)j * m + (j + 1)] = bres;
    }
    dense_top_eigenpairs(H, m, keep, theta, S);
    conv = 0;
    for (int i = 0; i < nd; ++i) conv += fabs(bres * S[(size_t)i * m + (m - 1)]) <= tol ? 1 : 0;
    if (log_on_lz())
      fprintf(stderr, "[whv] thick-restart Lanczos: restart %d, %d wave solves, %d of %d converged\n", restarts, nws,
              conv, nd);
    if (conv == nd || restarts == max_restarts) break;
    ++restarts;
    // keep the `keep` largest Ritz vectors and the residual vector (normalised, in g->q)
    TL_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    for (int c0 = 0; c0 < keep; c0 += kRitzJC) {
      const int blocks = (int)std::min<int64_t>((N + 255) / 256, 148 * 8);
      k_ritz<<<blocks, 256, (size_t)m * kRitzJC * sizeof(double), g->stream>>>(Q, N, m, dS, keep, c0, Y);
      count_launches(1);
      TL_CUDA(cudaGetLastError());
    }
    TL_CUDA(cudaMemcpyAsync(Q, Y, (size_t)keep * N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    TL_CUDA(cudaMemcpyAsync(Q + (size_t)keep * N, g->q, N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    TL_CUDA(cudaStreamSynchronize(g->stream));   // dS is read from the pageable S before it changes
    std::fill(H.begin(), H.end(), 0.0);
    for (int i = 0; i < keep; ++i) {
      H[(size_t)i * m + i] = theta[i];
      H[(size_t)i * m + keep] = H[(size_t)keep * m + i] = bres * S[(size_t)i * m + (m - 1)];
    }
    j0 = keep;
  }
  // the nd wanted Ritz vectors
  std::vector<double> Snd(S.begin(), S.begin() + (size_t)nd * m), th(theta.begin(), theta.begin() + nd);
  TL_CUDA(cudaMemcpyAsync(dS, Snd.data(), Snd.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  double* Yf = nullptr;
  TL_CUDA(cudaMalloc(&Yf, (size_t)nd * N * sizeof(double)));
  for (int c0 = 0; c0 < nd; c0 += kRitzJC) {
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, 148 * 8);
    k_ritz<<<blocks, 256, (size_t)m * kRitzJC * sizeof(double), g->stream>>>(Q, N, m, dS, nd, c0, Yf);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { cudaFree(Yf); cleanup(); return cuda_fail(g, e, "k_ritz"); }
  }
  const cudaError_t e = cudaStreamSynchronize(g->stream);
  cleanup();
  if (e != cudaSuccess) { cudaFree(Yf); return cuda_fail(g, e, "thick-restart Lanczos"); }
  if (stats) { stats[0] = restarts; stats[1] = nws; stats[2] = conv; }
#undef TL_TRY
#undef TL_CUDA
  return install_ritz_basis(g, p, tg, Yf, nd, th, flags, theta_host, resid_host);
}

extern "C" whv_status whv_lanczos(whv_grid g, const whv_params* p, int nd, int m, const double* v0_dev,
                                  int fp64_stepping, int flags, double* theta_host, double* resid_host) {
  return lanczos_impl(g, p, nd, m, v0_dev, fp64_stepping, flags, theta_host, resid_host);
}

extern "C" whv_status whv_lanczos_restarted(whv_grid g, const whv_params* p, int nd, int m, int keep,
                                            int max_restarts, double tol, const double* v0_dev, int fp64_stepping,
                                            int flags, double* theta_host, double* resid_host, int* stats_host) {
  return lanczos_thick_impl(g, p, nd, m, keep, max_restarts, tol, v0_dev, fp64_stepping, flags, theta_host,
                            resid_host, stats_host);
}
