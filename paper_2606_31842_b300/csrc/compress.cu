// SVD compression of the deflation basis (Sec. 4.3, experiment with compressed eigenvectors).
//
// A 2-D basis vector phi_m is an ny x nx matrix (row y, column x).  whv_compress_basis replaces
// every vector by its smallest-rank truncated SVD with Frobenius error < tau,
//     phi_m ~ U_m diag(s_m) V_m^T,  U_m: ny x r_m,  V_m: nx x r_m,
// and frees the dense basis: storage sum_m r_m (nx + ny + 1) doubles instead of nd nx ny.  The
// factors of all vectors are concatenated column-wise (R = sum_m r_m columns, column-major).
// The basis contractions then become two GEMM-shaped steps (FP64, tiled in shared memory):
//     projection  coef_m = sum_{k in m} s_k u_k^T (M o r) v_k:   T = (M o r) V  (ny x R), then one
//                 block per vector sums s_k u_k . T_k in fixed order
//     expansion   out += alpha U diag(c) V^T,  c_k = coef_{m(k)} s_k                 (ny x nx)
// The truncated SVD is computed by a randomized range finder with two power iterations
// (Halko, Martinsson and Tropp 2011): Y = phi Omega (Gaussian Omega, l columns), Q = orth(Y),
// B = Q^T phi; the SVD of the small B (l x nx) comes from the eigen-decomposition of B B^T (cyclic
// Householder reduction, bisection and inverse iteration on the host); the range error ||phi - Q Q^T phi||_F^2 = ||phi||_F^2 - ||B||_F^2 is added
// to the discarded singular values, and l doubles until the tolerance is met.  Singular values
// below ~1e-7 ||phi|| are not resolved by the B B^T eigenvalues: tau must be at least that.
#include <math.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

// ------------------------------------------------------------------ FP64 GEMM (strided)
// C(i, j) = alpha sum_k A(i, k) kscale(k) B(k, j) + beta C(i, j), with
// A(i, k) = A[i ai + k ak], B(k, j) = B[k bk + j bj], C(i, j) = C[i ci + j cj]; kscale may be null.
constexpr int kGT = 32;
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const double* __restrict__ A, int64_t ai,
                                              int64_t ak, const double* __restrict__ B, int64_t bk, int64_t bj,
                                              double* __restrict__ C, int64_t ci, int64_t cj, double alpha,
                                              double beta, const double* __restrict__ kscale) {
  __shared__ double As[kGT][kGT + 1];
  __shared__ double Bs[kGT][kGT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 2 x 2 outputs each
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += kGT) {
    for (int e = threadIdx.x; e < kGT * kGT; e += blockDim.x) {
      const int r = e / kGT, c = e % kGT;
      const int gi = i0 + r, gk = k0 + c;
      double a = 0.0;
      if (gi < M && gk < K) {
        a = A[gi * ai + gk * ak];
        if (kscale) a *= kscale[gk];
      }
      As[r][c] = a;
      const int gk2 = k0 + r, gj = j0 + c;
      Bs[r][c] = (gk2 < K && gj < N) ? B[gk2 * bk + gj * bj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGT; ++kk) {
      const double a0 = As[2 * ty][kk], a1 = As[2 * ty + 1][kk];
      const double b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int gi = i0 + 2 * ty + a, gj = j0 + 2 * tx + b;
      if (gi < M && gj < N) {
        double* c = C + gi * ci + gj * cj;
        *c = beta == 0.0 ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * *c);
      }
    }
}

static whv_status gemm(whv_grid g, int M, int N, int K, const double* A, int64_t ai, int64_t ak, const double* B,
                       int64_t bk, int64_t bj, double* C, int64_t ci, int64_t cj, double alpha, double beta,
                       const double* kscale = nullptr) {
  if (M <= 0 || N <= 0) return WHV_OK;
  dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
  k_gemm<<<grid, 256, 0, g->stream>>>(M, N, K, A, ai, ak, B, bk, bj, C, ci, cj, alpha, beta, kscale);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

// out = w o r  (w = M weights, null: copy)
__global__ void k_weighted(const double* __restrict__ r, const double* __restrict__ w, int64_t n,
                           double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = w ? w[i] * r[i] : r[i];
}

// coef_m = sum_{k in [off_m, off_{m+1})} s_k sum_y U[k ny + y] T[k ny + y]   (one block per m)
__global__ void __launch_bounds__(256) k_comp_coef(const double* __restrict__ U, const double* __restrict__ T,
                                                   const double* __restrict__ s, const int* __restrict__ off,
                                                   int ny, double* __restrict__ coef) {
  const int m = blockIdx.x;
  double acc = 0.0;
  for (int k = off[m]; k < off[m + 1]; ++k) {
    double d = 0.0;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) d = fma(U[(int64_t)k * ny + y], T[(int64_t)k * ny + y], d);
    acc = fma(s[k], d, acc);   // per-thread partial sums, added in fixed order below
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) coef[m] = acc;
}

// c_k = alpha coef_{m(k)} s_k
__global__ void k_comp_scale(const double* __restrict__ coef, const double* __restrict__ s,
                             const int* __restrict__ owner, int R, double alpha, double* __restrict__ c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < R) c[k] = alpha * coef[owner[k]] * s[k];
}

// ------------------------------------------------------------------ basis contractions
whv_status basis_project(whv_grid g, const double* r, double* coef) {
  const Basis& B = g->basis;
  if (B.V) return project(g, B.V, B.nd, r, coef);
  if (!B.cU) return fail(g, WHV_ERR_INVALID, "no deflation basis");
  const int nx = g->n[0], ny = g->n[1];
  k_weighted<<<(int)std::min<int64_t>((g->N + 255) / 256, 4096), 256, 0, g->stream>>>(r, g->mw, g->N, B.cR);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  // T (ny x R, column-major) = (M o r) (ny x nx, row-major) V (nx x R, column-major)
  TRY(gemm(g, ny, B.comp_R, nx, B.cR, nx, 1, B.cV, 1, nx, B.cT, 1, ny, 1.0, 0.0));
  k_comp_coef<<<B.nd, 256, 0, g->stream>>>(B.cU, B.cT, B.cs, B.coff, ny, coef);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status basis_expand(whv_grid g, const double* coef, double alpha, double* out) {
  const Basis& B = g->basis;
  if (B.V) return expand(g, B.V, B.nd, coef, alpha, out);
  if (!B.cU) return fail(g, WHV_ERR_INVALID, "no deflation basis");
  const int nx = g->n[0], ny = g->n[1];
  k_comp_scale<<<(B.comp_R + 255) / 256, 256, 0, g->stream>>>(coef, B.cs, B.cowner, B.comp_R, alpha, B.cc);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  // out (ny x nx, row-major) += U (ny x R) diag(c) V^T (R x nx)
  return gemm(g, ny, nx, B.comp_R, B.cU, 1, ny, B.cV, nx, 1, out, nx, 1, 1.0, 1.0, B.cc);
}

// dst = basis vector m (dense), through the expansion with a unit coefficient
whv_status basis_column(whv_grid g, int m, double* dst) {
  const Basis& B = g->basis;
  if (B.V) {
    WHV_CUDA(g, cudaMemcpyAsync(dst, B.V + (size_t)m * g->N, g->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                g->stream));
    return WHV_OK;
  }
  std::vector<double> e(B.nd, 0.0);
  e[m] = 1.0;
  WHV_CUDA(g, cudaMemsetAsync(dst, 0, g->N * sizeof(double), g->stream));
  WHV_CUDA(g, cudaMemcpyAsync(g->small2, e.data(), B.nd * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));   // e is a host temporary
  return basis_expand(g, g->small2, 1.0, dst);
}

const void* basis_key(const Basis& B) { return B.V ? (const void*)B.V : (const void*)B.cU; }

// ------------------------------------------------------------------ host linear algebra
// Gaussian numbers from a counter-based generator: splitmix64 (Steele, Lea and Flood 2014) of
// (seed, index) feeding the Box-Muller transform.
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double gauss(uint64_t seed, uint64_t i) {
  const double u1 = ((splitmix64(seed * 0x100000001B3ull + 2 * i) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (splitmix64(seed * 0x100000001B3ull + 2 * i + 1) >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Orthonormalise the columns of X (n x l, column-major) by classical Gram-Schmidt applied twice;
// returns the number of columns kept (columns that vanish are dropped).
static int orthonormalise(std::vector<double>& X, int n, int l) {
  int kept = 0;
  for (int j = 0; j < l; ++j) {
    double* x = &X[(size_t)j * n];
    const double n0 = sqrt(std::inner_product(x, x + n, x, 0.0));
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<double> h(kept);
      for (int i = 0; i < kept; ++i) h[i] = std::inner_product(&X[(size_t)i * n], &X[(size_t)i * n] + n, x, 0.0);
      for (int i = 0; i < kept; ++i)
        for (int t = 0; t < n; ++t) x[t] -= h[i] * X[(size_t)i * n + t];
    }
    const double nn = sqrt(std::inner_product(x, x + n, x, 0.0));
    if (!(nn > 1e-12 * n0) || nn == 0.0) continue;
    for (int t = 0; t < n; ++t) X[(size_t)kept * n + t] = x[t] / nn;
    ++kept;
  }
  return kept;
}

}  // namespace whv

using namespace whv;

extern "C" whv_status whv_compress_basis(whv_grid g, double tau, int* ranks_host) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  Basis& B = g->basis;
  if (g->dim != 2) return fail(g, WHV_ERR_INVALID, "SVD compression needs a 2-D grid");
  if (!B.V || B.nd < 1) return fail(g, WHV_ERR_INVALID, "no dense deflation basis to compress");
  if (!(tau > 0.0)) return fail(g, WHV_ERR_INVALID, "tau must be > 0");
  const int nx = g->n[0], ny = g->n[1], nd = B.nd;
  // ranks beyond ~half the shorter side store more than the dense vector: the sketch stops at
  // kCompMaxRank, and a vector that needs more at this tolerance is reported as not compressible
  constexpr int kCompMaxRank = 256;
  const int lmax = std::min({nx, ny, kCompMaxRank});
  const int64_t N = g->N;
  // device scratch for the range finder (largest l = lmax)
  double *Y = nullptr, *Zd = nullptr, *Bd = nullptr;
  auto cleanup = [&]() { for (double* p : {Y, Zd, Bd}) if (p) cudaFree(p); };
  if (cudaMalloc(&Y, (size_t)ny * lmax * 8) != cudaSuccess || cudaMalloc(&Zd, (size_t)nx * lmax * 8) != cudaSuccess ||
      cudaMalloc(&Bd, (size_t)lmax * nx * 8) != cudaSuccess) {
    cleanup();
    return fail(g, WHV_ERR_OOM, "cudaMalloc (compression scratch)");
  }
  std::vector<double> Uall, Vall, sall;
  std::vector<int> off(nd + 1, 0), ranks(nd);
  whv_status st = WHV_OK;
  for (int m = 0; m < nd && st == WHV_OK; ++m) {
    const double* phi = B.V + (size_t)m * N;
    // ||phi||_F^2 (plain: the compression is of the values, independent of M)
    std::vector<double> ph(N);
    if (cudaMemcpy(ph.data(), phi, N * 8, cudaMemcpyDeviceToHost) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
    const double fro2 = std::inner_product(ph.begin(), ph.end(), ph.begin(), 0.0);
    int l = std::min(16, lmax);
    while (true) {
      // Omega (nx x l, column-major), Y = phi Omega (ny x l)
      std::vector<double> Om((size_t)nx * l);
      for (size_t e = 0; e < Om.size(); ++e) Om[e] = gauss(1000003ull * (m + 1) + l, e);
      if (cudaMemcpy(Zd, Om.data(), Om.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
      st = gemm(g, ny, l, nx, phi, nx, 1, Zd, 1, nx, Y, 1, ny, 1.0, 0.0);
      std::vector<double> Yh((size_t)ny * l), Zh((size_t)nx * l);
      int kept = l;
      for (int it = 0; it < 2 && st == WHV_OK; ++it) {   // power iterations with re-orthonormalisation
        if (cudaMemcpy(Yh.data(), Y, Yh.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
        kept = orthonormalise(Yh, ny, l);
        std::fill(Yh.begin() + (size_t)kept * ny, Yh.end(), 0.0);
        cudaMemcpy(Y, Yh.data(), Yh.size() * 8, cudaMemcpyHostToDevice);
        st = gemm(g, nx, l, ny, phi, 1, nx, Y, 1, ny, Zd, 1, nx, 1.0, 0.0);   // Z = phi^T Y
        if (st != WHV_OK) break;
        if (cudaMemcpy(Zh.data(), Zd, Zh.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
        const int kz = orthonormalise(Zh, nx, l);
        std::fill(Zh.begin() + (size_t)kz * nx, Zh.end(), 0.0);
        cudaMemcpy(Zd, Zh.data(), Zh.size() * 8, cudaMemcpyHostToDevice);
        st = gemm(g, ny, l, nx, phi, nx, 1, Zd, 1, nx, Y, 1, ny, 1.0, 0.0);   // Y = phi Z
      }
      if (st != WHV_OK) break;
      if (cudaMemcpy(Yh.data(), Y, Yh.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
      kept = orthonormalise(Yh, ny, l);
      cudaMemcpy(Y, Yh.data(), (size_t)ny * std::max(kept, 1) * 8, cudaMemcpyHostToDevice);
      // B = Q^T phi (kept x nx, row-major)
      std::vector<double> Bh((size_t)std::max(kept, 1) * nx, 0.0);
      if (kept > 0) {
        st = gemm(g, kept, nx, ny, Y, ny, 1, phi, nx, 1, Bd, nx, 1, 1.0, 0.0);
        if (st != WHV_OK) break;
        if (cudaMemcpy(Bh.data(), Bd, (size_t)kept * nx * 8, cudaMemcpyDeviceToHost) != cudaSuccess) { st = fail(g, WHV_ERR_CUDA, "copy"); break; }
      }
      // B B^T = Z diag(sigma^2) Z^T
      std::vector<double> G((size_t)kept * kept), ev, Z;
      for (int a = 0; a < kept; ++a)
        for (int b = 0; b <= a; ++b) {
          const double v = std::inner_product(&Bh[(size_t)a * nx], &Bh[(size_t)a * nx] + nx, &Bh[(size_t)b * nx], 0.0);
          G[(size_t)a * kept + b] = G[(size_t)b * kept + a] = v;
        }
      double bfro2 = 0.0;
      for (double v : Bh) bfro2 += v * v;
      if (kept > 0) host_sym_top_eigenpairs(G, kept, kept, ev, Z);
      const double range2 = std::max(fro2 - bfro2, 0.0);   // ||phi - Q Q^T phi||_F^2
      // smallest r with sum_{k >= r} sigma_k^2 + range error < tau^2
      std::vector<double> tail(kept + 1, 0.0);
      for (int k = kept - 1; k >= 0; --k) tail[k] = tail[k + 1] + std::max(ev[k], 0.0);
      int r = -1;
      for (int k = 0; k <= kept; ++k)
        if (tail[k] + range2 < tau * tau) { r = k; break; }
      if (r < 0 && l < lmax) {   // the sketch misses part of the range: enlarge it
        l = std::min(2 * l, lmax);
        continue;
      }
      if (r < 0) {
        if (lmax == std::min(nx, ny)) {
          r = kept;   // the sketch spans the whole column space: keep everything it resolved
        } else {
          st = fail(g, WHV_ERR_INVALID, "whv_compress_basis: a basis vector needs rank > 256 at this tolerance "
                                        "(not compressible; the basis is left dense)");
          break;
        }
      }
      // U = Q Z_r (ny x r), s = sqrt(ev), V = B^T Z_r / s (nx x r)
      for (int k = 0; k < r; ++k) {
        const double sk = sqrt(std::max(ev[k], 0.0));
        std::vector<double> u(ny, 0.0), v(nx, 0.0);
        for (int a = 0; a < kept; ++a) {
          const double z = Z[(size_t)k * kept + a];
          for (int y = 0; y < ny; ++y) u[y] += Yh[(size_t)a * ny + y] * z;
          for (int x = 0; x < nx; ++x) v[x] += Bh[(size_t)a * nx + x] * z;
        }
        for (int x = 0; x < nx; ++x) v[x] = sk > 0 ? v[x] / sk : 0.0;
        Uall.insert(Uall.end(), u.begin(), u.end());
        Vall.insert(Vall.end(), v.begin(), v.end());
        sall.push_back(sk);
      }
      ranks[m] = r;
      off[m + 1] = off[m] + r;
      break;
    }
  }
  cleanup();
  if (st != WHV_OK) return st;
  const int R = off[nd];
  if (R < 1) return fail(g, WHV_ERR_INVALID, "every basis vector compressed to rank 0 (tau too large)");
  std::vector<int> owner(R);
  for (int m = 0; m < nd; ++m)
    for (int k = off[m]; k < off[m + 1]; ++k) owner[k] = m;
  Basis nb = B;   // keep everything but the dense vectors
  nb.comp_R = R;
  nb.comp_tau = tau;
  auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
  if (!A((void**)&nb.cU, (size_t)ny * R * 8) || !A((void**)&nb.cV, (size_t)nx * R * 8) || !A((void**)&nb.cs, R * 8) ||
      !A((void**)&nb.cT, (size_t)ny * R * 8) || !A((void**)&nb.cc, R * 8) || !A((void**)&nb.cR, N * 8) ||
      !A((void**)&nb.coff, (nd + 1) * sizeof(int)) || !A((void**)&nb.cowner, R * sizeof(int))) {
    for (void* p : {(void*)nb.cU, (void*)nb.cV, (void*)nb.cs, (void*)nb.cT, (void*)nb.cc, (void*)nb.cR, (void*)nb.coff,
                    (void*)nb.cowner})
      if (p) cudaFree(p);
    return fail(g, WHV_ERR_OOM, "cudaMalloc (compressed basis)");
  }
  cudaMemcpy(nb.cU, Uall.data(), Uall.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(nb.cV, Vall.data(), Vall.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(nb.cs, sall.data(), sall.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(nb.coff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(nb.cowner, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice);
  // the dense vectors (and what was built from them: graphs, A W, QR) go
  cudaStreamSynchronize(g->stream);
  free_plan(g);
  nb.vhold.reset();   // the dense vectors: freed unless another grid shares them
  for (void* p : {(void*)B.AW, (void*)B.Einv, (void*)B.QAW})
    if (p) cudaFree(p);
  nb.V = nullptr;
  nb.AW = nullptr;
  nb.Einv = nullptr;
  nb.QAW = nullptr;
  nb.Raw.clear();
  B = nb;
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(g, WHV_ERR_CUDA, "compressed basis upload");
  if (ranks_host) std::copy(ranks.begin(), ranks.end(), ranks_host);
  return WHV_OK;
}
