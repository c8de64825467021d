// Tall-skinny deflation contractions (W^T M r and W y) and the closed-form deflation basis.
//
// W is N x nd, column-major, FP64.  project reads W exactly once: each block stages a chunk of
// M r in shared memory and its warps sweep the columns of that chunk with coalesced loads; the
// per-block partial sums are then added in block order by a second kernel (deterministic).
// expand reads W once with one thread per row.  Both are HBM-bound: N nd 8 bytes per call.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

constexpr int kProjThreads = 256;
constexpr int kProjRows = 2048;   // rows of r staged per block (16 KB of shared memory)

__global__ void __launch_bounds__(kProjThreads) k_project(const double* __restrict__ W, int64_t N, int nd,
                                                          const double* __restrict__ r,
                                                          const double* __restrict__ mw,
                                                          double* __restrict__ partials) {
  __shared__ double sr[kProjRows];
  const int64_t row0 = (int64_t)blockIdx.x * kProjRows;
  const int rows = (int)min((int64_t)kProjRows, N - row0);
  for (int i = threadIdx.x; i < rows; i += kProjThreads)
    sr[i] = mw ? r[row0 + i] * mw[row0 + i] : r[row0 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int m = warp; m < nd; m += kProjThreads / 32) {
    const double* col = W + (int64_t)m * N + row0;
    double s = 0.0;
#pragma unroll 8
    for (int i = lane; i < rows; i += 32) s = fma(col[i], sr[i], s);
    s = warp_sum(s);
    if (lane == 0) partials[(int64_t)blockIdx.x * nd + m] = s;
  }
}

__global__ void __launch_bounds__(256) k_project_finish(const double* __restrict__ partials, int nblocks, int nd,
                                                        double* __restrict__ coef) {
  const int m = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(int64_t)b * nd + m];
  s = block_sum(s);
  if (threadIdx.x == 0) coef[m] = s;
}

// out_i += alpha sum_m W[i + m N] y_m
__global__ void __launch_bounds__(256) k_expand(const double* __restrict__ W, int64_t N, int nd,
                                                const double* __restrict__ y, double alpha,
                                                double* __restrict__ out) {
  __shared__ double sy[kMaxND];
  for (int m = threadIdx.x; m < nd; m += blockDim.x) sy[m] = alpha * y[m];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    double s = 0.0;
    for (int m = 0; m < nd; ++m) s = fma(W[i + (int64_t)m * N], sy[m], s);
    out[i] += s;
  }
}

whv_status project(whv_grid g, const double* W, int nd, const double* r, double* coef) {
  if (nd < 1 || nd > kMaxND) return fail(g, WHV_ERR_INVALID, "project: bad nd");
  const int64_t nb64 = (g->N + kProjRows - 1) / kProjRows;
  if (nb64 * nd > chan_cap(g, CH_PROJ)) return fail(g, WHV_ERR_INVALID, "project: N * nd too large");
  const int nb = (int)nb64;
  double* part = chan(g, CH_PROJ);
  k_project<<<nb, kProjThreads, 0, g->stream>>>(W, g->N, nd, r, g->mw, part);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  k_project_finish<<<nd, 256, 0, g->stream>>>(part, nb, nd, coef);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status expand(whv_grid g, const double* W, int nd, const double* coef, double alpha, double* out) {
  if (nd < 1 || nd > kMaxND) return fail(g, WHV_ERR_INVALID, "expand: bad nd");
  int64_t b = (g->N + 255) / 256;
  const int blocks = (int)std::min<int64_t>(b, 148 * 8);
  k_expand<<<blocks, 256, 0, g->stream>>>(W, g->N, nd, coef, alpha, out);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

// ------------------------------------------------------------------ many right-hand sides
// The same contractions for k right-hand sides that share one basis W (several forcings on one
// grid, or batched problems whose grids share a basis): W is read once for all of them.
//   project_many:  C[j nd + m] = sum_i W[i + m N] M_i r_j[i]            (j < k, m < nd)
//   expand_many:   out_j[i]  += alpha sum_m W[i + m N] s_m C[j nd + m]  (s = scale or 1)
// Both are FP64-FMA bound on this GPU once k is more than a few (nd k FMAs per row against
// (nd + k) 8 bytes), so a block takes up to kMK right-hand sides at a time (grid.y covers more)
// and the template width KB keeps the FMA count at the actual k when k is small.
constexpr int kMThreads = 256;
constexpr int kMRows = 512;    // rows staged per block by project_many
constexpr int kMK = 16;        // right-hand sides per block

template <int KB>
__global__ void __launch_bounds__(kMThreads) k_project_many(const double* __restrict__ W, int64_t N, int nd, int k,
                                                            const double* const* __restrict__ R,
                                                            const double* __restrict__ mw,
                                                            double* __restrict__ partials) {
  extern __shared__ __align__(16) double sr[];   // KB x kMRows: the block's rows of M r_j
  const int j0 = blockIdx.y * KB;
  const int kb = min(KB, k - j0);
  const int64_t row0 = (int64_t)blockIdx.x * kMRows;
  const int rows = (int)min((int64_t)kMRows, N - row0);
  for (int j = 0; j < KB; ++j) {
    const double* r = j < kb ? R[j0 + j] + row0 : nullptr;
    for (int i = threadIdx.x; i < rows; i += kMThreads)
      sr[j * kMRows + i] = r ? (mw ? r[i] * mw[row0 + i] : r[i]) : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int m = warp; m < nd; m += kMThreads / 32) {
    const double* col = W + (int64_t)m * N + row0;
    double acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = 0.0;
    for (int i = lane; i < rows; i += 32) {
      const double v = __ldcs(col + i);   // W is streamed once: do not keep it in L2
#pragma unroll
      for (int j = 0; j < KB; ++j) acc[j] = fma(v, sr[j * kMRows + i], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const double s = warp_sum(acc[j]);
      if (lane == 0 && j < kb) partials[((int64_t)blockIdx.x * k + j0 + j) * nd + m] = s;
    }
  }
}

// C[j nd + m] = sum over blocks b (in order) of partials[(b k + j) nd + m]: one block per (j, m)
__global__ void __launch_bounds__(256) k_project_many_finish(const double* __restrict__ partials, int nblocks,
                                                             int nd, int k, double* __restrict__ C) {
  const int jm = blockIdx.x;   // j nd + m
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(int64_t)b * k * nd + jm];
  s = block_sum(s);
  if (threadIdx.x == 0) C[jm] = s;
}

template <int KB>
__global__ void __launch_bounds__(kMThreads) k_expand_many(const double* __restrict__ W, int64_t N, int nd, int k,
                                                           const double* __restrict__ C,
                                                           const double* __restrict__ scale, double alpha,
                                                           double* const* __restrict__ out) {
  constexpr int kSlab = 256;   // coefficients staged per pass
  __shared__ double sc[kSlab * KB];
  const int j0 = blockIdx.y * KB;
  const int kb = min(KB, k - j0);
  const int64_t stride = (int64_t)gridDim.x * kMThreads;
  for (int m0 = 0; m0 < nd; m0 += kSlab) {
    const int mb = min(kSlab, nd - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mb * KB; t += kMThreads) {
      const int m = t / KB, j = t % KB;
      sc[t] = j < kb ? (alpha * (scale ? scale[m0 + m] : 1.0)) * C[(int64_t)(j0 + j) * nd + m0 + m] : 0.0;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kMThreads + threadIdx.x; i < N; i += stride) {
      double acc[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) acc[j] = 0.0;
      for (int m = 0; m < mb; ++m) {
        const double w = __ldcs(W + i + (int64_t)(m0 + m) * N);
#pragma unroll
        for (int j = 0; j < KB; ++j) acc[j] = fma(w, sc[m * KB + j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < kb) out[j0 + j][i] += acc[j];
    }
  }
}

template <int KB>
static cudaError_t project_many_kb(cudaStream_t st, const double* W, int64_t N, int nd, int k,
                                   const double* const* R, const double* mw, double* partials, double* C) {
  const int nb = (int)((N + kMRows - 1) / kMRows);
  const size_t smem = (size_t)KB * kMRows * sizeof(double);
  static bool attr = false;   // opt into > 48 KB of dynamic shared memory once
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_project_many<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_project_many<KB><<<dim3(nb, (k + KB - 1) / KB), kMThreads, smem, st>>>(W, N, nd, k, R, mw, partials);
  k_project_many_finish<<<nd * k, 256, 0, st>>>(partials, nb, nd, k, C);
  count_launches(2);
  return cudaGetLastError();
}

template <int KB>
static cudaError_t expand_many_kb(cudaStream_t st, const double* W, int64_t N, int nd, int k, const double* C,
                                  const double* scale, double alpha, double* const* out) {
  const int blocks = (int)std::min<int64_t>((N + kMThreads - 1) / kMThreads, 148 * 8);
  k_expand_many<KB><<<dim3(blocks, (k + KB - 1) / KB), kMThreads, 0, st>>>(W, N, nd, k, C, scale, alpha, out);
  count_launches(1);
  return cudaGetLastError();
}

int64_t project_many_scratch(int64_t N, int nd, int k) { return ((N + kMRows - 1) / kMRows) * (int64_t)nd * k; }

cudaError_t project_many(cudaStream_t st, const double* W, int64_t N, int nd, int k, const double* const* R,
                         const double* mw, double* partials, double* C) {
  if (k <= 1) return project_many_kb<1>(st, W, N, nd, k, R, mw, partials, C);
  if (k <= 2) return project_many_kb<2>(st, W, N, nd, k, R, mw, partials, C);
  if (k <= 4) return project_many_kb<4>(st, W, N, nd, k, R, mw, partials, C);
  if (k <= 8) return project_many_kb<8>(st, W, N, nd, k, R, mw, partials, C);
  return project_many_kb<kMK>(st, W, N, nd, k, R, mw, partials, C);
}

cudaError_t expand_many(cudaStream_t st, const double* W, int64_t N, int nd, int k, const double* C,
                        const double* scale, double alpha, double* const* out) {
  if (k <= 1) return expand_many_kb<1>(st, W, N, nd, k, C, scale, alpha, out);
  if (k <= 2) return expand_many_kb<2>(st, W, N, nd, k, C, scale, alpha, out);
  if (k <= 4) return expand_many_kb<4>(st, W, N, nd, k, C, scale, alpha, out);
  if (k <= 8) return expand_many_kb<8>(st, W, N, nd, k, C, scale, alpha, out);
  return expand_many_kb<kMK>(st, W, N, nd, k, C, scale, alpha, out);
}

// ------------------------------------------------------------------ closed-form basis
// beta_h of every tensor-product sine mode: lambda^2 is the sum of the per-direction values in
// ascending order (so permuted tuples tie exactly), cos(theta) = 1 - dt^2 lambda^2/2,
// beta_h = sum_n w_n cos(n theta) (the exact transfer of the leapfrog + trapezoid filter).
__global__ void k_mode_beta(const double* __restrict__ l1x, const double* __restrict__ l1y,
                            const double* __restrict__ l1z, int nx, int ny, int nz, double dt2,
                            const double* __restrict__ w, int nt, double* __restrict__ beta) {
  const int64_t total = (int64_t)nx * ny * nz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(t % nx);
    const int ky = (int)((t / nx) % ny);
    const int kz = (int)(t / ((int64_t)nx * ny));
    // per-direction values padded with zeros, sorted ascending, summed from the smallest
    double a = l1x[kx], b = l1y ? l1y[ky] : 0.0, c = l1z ? l1z[kz] : 0.0, tmp;
    if (a > b) { tmp = a; a = b; b = tmp; }
    if (b > c) { tmp = b; b = c; c = tmp; }
    if (a > b) { tmp = a; a = b; b = tmp; }
    const double lam2 = (a + b) + c;
    const double x = 1.0 - 0.5 * dt2 * lam2;
    const double th = acos(fmax(-1.0, fmin(1.0, x)));
    double s = 0.0;
    for (int n = 0; n <= nt; ++n) s += w[n] * cos(n * th);
    beta[t] = s;
  }
}

// column m of the basis: prod_d sqrt(2/(n_d+1)) sin(pi k_d (i_d+1)/(n_d+1))
__global__ void k_sine_basis(double* __restrict__ V, int64_t N, int nx, int ny, int nz,
                             const int* __restrict__ modes, int dim, int nd) {
  const int m = blockIdx.y;
  const int kx = modes[m * dim + 0];
  const int ky = dim > 1 ? modes[m * dim + 1] : 0;
  const int kz = dim > 2 ? modes[m * dim + 2] : 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx);
    const int iy = (int)((i / nx) % ny);
    const int iz = (int)(i / ((int64_t)nx * ny));
    // exact argument reduction: sin(pi k j / L) with k j mod 2L
    const int64_t Lx = nx + 1;
    double v = sqrt(2.0 / Lx) * sinpi((double)(((int64_t)kx * (ix + 1)) % (2 * Lx)) / (double)Lx);
    if (dim > 1) {
      const int64_t Ly = ny + 1;
      v *= sqrt(2.0 / Ly) * sinpi((double)(((int64_t)ky * (iy + 1)) % (2 * Ly)) / (double)Ly);
    }
    if (dim > 2) {
      const int64_t Lz = nz + 1;
      v *= sqrt(2.0 / Lz) * sinpi((double)(((int64_t)kz * (iz + 1)) % (2 * Lz)) / (double)Lz);
    }
    V[i + (int64_t)m * N] = v;
  }
}

static std::vector<double> eig1d(int n_interior, double h, int order) {
  // lambda_k^2 of the 1-D Dirichlet stencil, k = 1..n (Sec. 4.3 sine vectors)
  std::vector<double> l(n_interior);
  const double pi = 3.14159265358979323846;
  for (int k = 1; k <= n_interior; ++k) {
    const double th = pi * k / (double)(n_interior + 1);
    l[k - 1] = order == 2 ? (2.0 - 2.0 * cos(th)) / (h * h)
                          : (30.0 - 32.0 * cos(th) + 2.0 * cos(2.0 * th)) / (12.0 * h * h);
  }
  return l;
}

whv_status closed_form_basis(whv_grid g, const TimeGridH& tg, int nd, Basis* b) {
  const int nx = g->n[0], ny = g->dim > 1 ? g->n[1] : 1, nz = g->dim > 2 ? g->n[2] : 1;
  const int64_t total = (int64_t)nx * ny * nz;
  std::vector<double> lx = eig1d(nx, g->h[0], g->order);
  std::vector<double> ly = g->dim > 1 ? eig1d(ny, g->h[1], g->order) : std::vector<double>();
  std::vector<double> lz = g->dim > 2 ? eig1d(nz, g->h[2], g->order) : std::vector<double>();
  double *d_lx = nullptr, *d_ly = nullptr, *d_lz = nullptr, *d_w = nullptr, *d_beta = nullptr;
  int* d_modes = nullptr;
  whv_status st = WHV_OK;
  auto cleanup = [&]() {
    for (void* p : {(void*)d_lx, (void*)d_ly, (void*)d_lz, (void*)d_w, (void*)d_beta, (void*)d_modes})
      if (p) cudaFree(p);
  };
#define CF_CUDA(call)                                            \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) { st = cuda_fail(g, _e, #call); cleanup(); return st; } \
  } while (0)
  CF_CUDA(cudaMalloc(&d_lx, nx * 8));
  CF_CUDA(cudaMemcpyAsync(d_lx, lx.data(), nx * 8, cudaMemcpyHostToDevice, g->stream));
  if (g->dim > 1) {
    CF_CUDA(cudaMalloc(&d_ly, ny * 8));
    CF_CUDA(cudaMemcpyAsync(d_ly, ly.data(), ny * 8, cudaMemcpyHostToDevice, g->stream));
  }
  if (g->dim > 2) {
    CF_CUDA(cudaMalloc(&d_lz, nz * 8));
    CF_CUDA(cudaMemcpyAsync(d_lz, lz.data(), nz * 8, cudaMemcpyHostToDevice, g->stream));
  }
  CF_CUDA(cudaMalloc(&d_w, (tg.nt + 1) * 8));
  CF_CUDA(cudaMemcpyAsync(d_w, tg.weight.data(), (tg.nt + 1) * 8, cudaMemcpyHostToDevice, g->stream));
  CF_CUDA(cudaMalloc(&d_beta, total * 8));
  {
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
    k_mode_beta<<<blocks, 256, 0, g->stream>>>(d_lx, d_ly, d_lz, nx, ny, nz, tg.dt * tg.dt, d_w,
                                               tg.nt, d_beta);
    count_launches(1);
    CF_CUDA(cudaGetLastError());
  }
  std::vector<double> beta(total);
  CF_CUDA(cudaMemcpyAsync(beta.data(), d_beta, total * 8, cudaMemcpyDeviceToHost, g->stream));
  CF_CUDA(cudaStreamSynchronize(g->stream));
  // the nd modes with the smallest |1 - beta_h|; ties by (kx, ky, kz) ascending
  std::vector<int64_t> idx(total);
  std::iota(idx.begin(), idx.end(), (int64_t)0);
  auto tuple_of = [&](int64_t t, int* k) {
    k[0] = (int)(t % nx); k[1] = (int)((t / nx) % ny); k[2] = (int)(t / ((int64_t)nx * ny));
  };
  auto less = [&](int64_t a, int64_t c) {
    const double ka = fabs(1.0 - beta[a]), kc = fabs(1.0 - beta[c]);
    if (ka != kc) return ka < kc;
    int ta[3], tc[3];
    tuple_of(a, ta); tuple_of(c, tc);
    for (int d = 0; d < 3; ++d)
      if (ta[d] != tc[d]) return ta[d] < tc[d];
    return false;
  };
  std::partial_sort(idx.begin(), idx.begin() + nd, idx.end(), less);
  b->modes.assign((size_t)nd * g->dim, 0);
  b->lambda2.resize(nd);
  b->mu.resize(nd);
  for (int m = 0; m < nd; ++m) {
    int k[3];
    tuple_of(idx[m], k);
    double parts[3] = {lx[k[0]], g->dim > 1 ? ly[k[1]] : 0.0, g->dim > 2 ? lz[k[2]] : 0.0};
    std::sort(parts, parts + g->dim);
    double l2 = 0.0;
    for (int d = 0; d < g->dim; ++d) l2 += parts[d];
    for (int d = 0; d < g->dim; ++d) b->modes[m * g->dim + d] = k[d] + 1;
    b->lambda2[m] = l2;
    b->mu[m] = 1.0 - beta[idx[m]];
  }
  CF_CUDA(cudaMalloc(&d_modes, (size_t)nd * g->dim * sizeof(int)));
  CF_CUDA(cudaMemcpyAsync(d_modes, b->modes.data(), (size_t)nd * g->dim * sizeof(int),
                          cudaMemcpyHostToDevice, g->stream));
  CF_CUDA(cudaMalloc(&b->V, (size_t)g->N * nd * 8));
  {
    dim3 grid((unsigned)std::min<int64_t>((g->N + 255) / 256, 1024), nd);
    k_sine_basis<<<grid, 256, 0, g->stream>>>(b->V, g->N, nx, ny, nz, d_modes, g->dim, nd);
    count_launches(1);
    CF_CUDA(cudaGetLastError());
  }
  CF_CUDA(cudaStreamSynchronize(g->stream));
  cleanup();
#undef CF_CUDA
  return WHV_OK;
}

}  // namespace whv

// ------------------------------------------------------------------ allocation-free projection
// A variant of the W^T M r projection for callers that must not allocate device memory: its
// per-block partial sums live in this file-scope array instead of a grid's scratch.  Every GPU
// that loads the library holds the array (2 MiB) until the process exits.
namespace whv {

constexpr int64_t kNoAllocPartials = (int64_t)1 << 18;   // 262144 doubles = 2 MiB
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

constexpr int kNoAllocMaxDevices = 64;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_partials on the current device.  In host code the symbol's name
// is only a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached.
static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace whv

extern "C" whv_status whv_project_noalloc(int64_t n, int nd, const double* W_dev, const double* r_dev,
                                          const double* w_dev, double* coef_dev, void* cuda_stream) {
  using namespace whv;
  if (n < 1 || nd < 1 || nd > kMaxND)
    return fail(nullptr, WHV_ERR_INVALID, "whv_project_noalloc: need n >= 1 and 1 <= nd <= 1024");
  if (!W_dev || !r_dev || !coef_dev) return fail(nullptr, WHV_ERR_INVALID, "whv_project_noalloc: NULL pointer");
  const int64_t nb = (n + kProjRows - 1) / kProjRows;
  if (nb * nd > kNoAllocPartials)
    return fail(nullptr, WHV_ERR_INVALID,
                "whv_project_noalloc: ceil(n/2048)*nd exceeds the 262144-entry static scratch "
                "(use whv_project on a grid for larger problems)");
  double* part = nullptr;
  cudaError_t e = noalloc_scratch(&part);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(static scratch)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // every partial the finishing kernel reads is written by k_project first: nothing to clear
  k_project<<<(unsigned)nb, kProjThreads, 0, st>>>(W_dev, n, nd, r_dev, w_dev, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_project launch");
  k_project_finish<<<nd, 256, 0, st>>>(part, (int)nb, nd, coef_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_project_finish launch");
  count_launches(2);
  return WHV_OK;
}
