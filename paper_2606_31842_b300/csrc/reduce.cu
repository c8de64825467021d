// Krylov reductions and vector updates (FP64, deterministic): the M-weighted dot product,
// the fused CG update x += a p, r -= a q with r^T M r, the direction update p = r + b p.
#include <math.h>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

__global__ void __launch_bounds__(256) k_dot(const double* __restrict__ x, const double* __restrict__ y,
                                             const double* __restrict__ mw, int64_t n,
                                             double* partials, unsigned* counter, double* out) {
  double s = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (mw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
      s = fma(x[i] * mw[i], y[i], s);
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
      s = fma(x[i], y[i], s);
  }
  s = block_sum(s);
  double total;
  if (grid_reduce(s, partials, counter, &total) && threadIdx.x == 0) *out = total;
}

// alpha = rr / pq; x += alpha p; r -= alpha q; rr' = r^T M r; beta = rr'/rr; rr <- rr'.
// Breakdown (pq = 0 or non-finite scalars) raises scal[S_FLAG].  A negative pq is allowed: the
// discrete filter transfer beta_h can exceed 1 by a few 1e-7 right at resonance, so A = I - S_h
// may have tiny negative eigenvalues, and CG remains the Galerkin (Lanczos) iteration there.
__global__ void __launch_bounds__(256) k_cg_update(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p,
                                                   const double* __restrict__ q,
                                                   const double* __restrict__ mw, int64_t n,
                                                   double* scal, double* partials,
                                                   unsigned* counter) {
  if (scal[S_HALT] != 0.0) return;   // a stopped problem of a batched solve
  const double rr = scal[S_RR];
  const double pq = scal[S_PQ];
  const double alpha = rr / pq;
  const bool ok = (pq != 0.0) && isfinite(alpha);
  const double a = ok ? alpha : 0.0;
  double s = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    s = fma(mw ? ri * mw[i] : ri, ri, s);
  }
  s = block_sum(s);
  double total;
  if (grid_reduce(s, partials, counter, &total) && threadIdx.x == 0) {
    scal[S_ALPHA] = a;
    scal[S_BETA] = total / rr;
    scal[S_RR] = total;
    if (!ok || !isfinite(total)) scal[S_FLAG] = 1.0;
  }
}

__global__ void __launch_bounds__(256) k_cg_direction(double* __restrict__ p, const double* __restrict__ r,
                                                      const double* __restrict__ scal, int64_t n) {
  if (scal[S_HALT] != 0.0) return;
  const double beta = scal[S_BETA];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    p[i] = fma(beta, p[i], r[i]);
}

__global__ void __launch_bounds__(256) k_axpby(int64_t n, double a, const double* __restrict__ x,
                                               double b, double* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (b == 0.0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
      y[i] = a * x[i];
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
      y[i] = fma(a, x[i], b * y[i]);
  }
}

static int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks);
}

whv_status dot_async(whv_grid g, const double* x, const double* y, int slot) {
  k_dot<<<grid_for(g->N), 256, 0, g->stream>>>(x, y, g->mw, g->N, chan(g, CH_DOT),
                                               g->counters + CH_DOT, g->scal + slot);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status cg_update(whv_grid g) {
  k_cg_update<<<grid_for(g->N), 256, 0, g->stream>>>(g->x, g->r, g->p, g->q, g->mw, g->N, g->scal,
                                                     chan(g, CH_UPDATE),
                                                     g->counters + CH_UPDATE);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status cg_direction(whv_grid g) {
  k_cg_direction<<<grid_for(g->N), 256, 0, g->stream>>>(g->p, g->r, g->scal, g->N);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status axpby(whv_grid g, int64_t n, double a, const double* x, double b, double* y) {
  k_axpby<<<grid_for(n), 256, 0, g->stream>>>(n, a, x, b, y);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

whv_status fetch_scalars(whv_grid g) {
  WHV_CUDA(g, cudaMemcpyAsync(g->scal_host, g->scal, S_NSLOTS * sizeof(double),
                              cudaMemcpyDeviceToHost, g->stream));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

}  // namespace whv
