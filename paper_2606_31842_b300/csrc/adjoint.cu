// Discrete adjoint of the WaveHoltz solve: gradients of L = 1/2 ||u - u_obs||^2 with respect
// to the forcing f and the squared speed c^2 (the differentiation path of the library).
//
// u is the fixed point u = Pi_h(u; f, c^2) (Sec. 2.1-2.2).  With g = dL/du and lambda solving
// (I - S_h)^T lambda = g, dL/dtheta = lambda^T dPi_h(u; f, c^2)/dtheta.
//  * Adjoint system: S_h is self-adjoint in <.,.>_M, M = diag(1/c^2) (the mass-matrix
//    symmetrisation of Sec. 4.1), so S_h^T = M S_h M^{-1} and (I - S_h)^T lambda = g is
//    (I - S_h) y = c^2 g, lambda = y / c^2: the forward solver (any method, deflation, FP64
//    residual correction) does it.
//  * lambda^T dPi/dtheta: the transpose of one wave solve at the fixed point -- the leapfrog run
//    backwards with the filter weights as source:
//        Wb^n += w_n lambda;  for n = Nt-1 .. 1:
//        Wb^n += 2 Wb^{n+1} + dt^2 Delta(c^2 Wb^{n+1}),  Wb^{n-1} -= Wb^{n+1},
//        dL/dc^2 += dt^2 (Delta W^n) Wb^{n+1},  dL/df -= dt^2 cos(w t^n) Wb^{n+1},
//    and the first (Taylor) step with half weights.  The forward states W^n are needed in
//    reverse order: they are checkpointed every K steps during one forward sweep and each
//    segment is recomputed from its checkpoint into a (K+1)-state buffer before it is reversed.
#include <math.h>

#include <algorithm>
#include <vector>

#include "stencil_ops.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

// one forward step out of place: wn = 2 wc - wp + dt^2 (c^2 Delta wc - f cos)   (first: Taylor)
template <typename T, int DIM, int ORDER, bool FIRST>
__global__ void __launch_bounds__(256) k_fwd_state(const T* __restrict__ wp, const T* __restrict__ wc,
                                                   T* __restrict__ wn, const T* __restrict__ c2,
                                                   const double* __restrict__ f, int nx, int ny, int nz,
                                                   StepCoef<T> cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  const T c = wc[idx];
  T L = lap<DIM, ORDER, T>(wc, idx, x, y, z, nx, ny, nz, cf, c);
  if (c2) L *= c2[idx];
  if (f) L = fma(-(T)f[idx], cf.fph, L);
  wn[idx] = FIRST ? fma(T(0.5) * cf.dt2, L, c) : fma(cf.dt2, L, fma(T(2), c, -wp[idx]));
}

// FP64 -> T copy (the fixed point u is the forward initial state)
template <typename T>
__global__ void k_to_state(const double* __restrict__ u, T* __restrict__ w, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (T)u[i];
}

// Delta(c^2 a) at idx, with c^2 a formed on the fly at the neighbours
template <int DIM, int ORDER, typename T>
__device__ __forceinline__ T lap_c2(const T* __restrict__ a, const T* __restrict__ c2, int64_t idx, int x,
                                    int y, int z, int nx, int ny, int nz, const StepCoef<T>& cf) {
  auto val = [&](int64_t j) -> T { return c2 ? a[j] * c2[j] : a[j]; };
  auto d2c = [&](int i, int n, int64_t s) -> T {
    const T c = val(idx);
    const T m1 = i > 0 ? val(idx - s) : T(0);
    const T p1 = i < n - 1 ? val(idx + s) : T(0);
    if (ORDER == 2) return fma(T(-2), c, m1 + p1);
    const T m2 = i > 1 ? val(idx - 2 * s) : (i == 1 ? T(0) : -c);
    const T p2 = i < n - 2 ? val(idx + 2 * s) : (i == n - 2 ? T(0) : -c);
    return fma(T(-30), c, fma(T(16), m1 + p1, -(m2 + p2)));
  };
  T l = d2c(x, nx, 1) * cf.ih2[0];
  if (DIM > 1) l = fma(d2c(y, ny, (int64_t)nx), cf.ih2[1], l);
  if (DIM > 2) l = fma(d2c(z, nz, (int64_t)nx * ny), cf.ih2[2], l);
  return l;
}

// Reverse of step n (W^{n+1} from W^n, W^{n-1}); FIRST: reverse of the Taylor step (n = 0).
//   bcur  (Wb^n)     += 2 bnext + dt^2 Delta(c^2 bnext)        (FIRST: bnext + dt^2/2 Delta(...))
//   bprev (Wb^{n-1})  = w_{n-1} lambda - bnext                  (not FIRST)
//   gc2 += s dt^2 (Delta W^n) bnext,  gf -= s dt^2 cos(w t^n) bnext,   s = 1 (FIRST: 1/2)
template <typename T, int DIM, int ORDER, bool FIRST>
__global__ void __launch_bounds__(256) k_reverse(const T* __restrict__ bnext, T* __restrict__ bcur,
                                                 T* __restrict__ bprev, const T* __restrict__ wstate,
                                                 const double* __restrict__ lam, const T* __restrict__ c2,
                                                 double* __restrict__ gc2, double* __restrict__ gf,
                                                 int nx, int ny, int nz, StepCoef<T> cf, T wprev_weight) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  const T bn = bnext[idx];
  const T s = FIRST ? T(0.5) : T(1);
  const T lc = lap_c2<DIM, ORDER, T>(bnext, c2, idx, x, y, z, nx, ny, nz, cf);
  bcur[idx] += (FIRST ? bn : T(2) * bn) + s * cf.dt2 * lc;
  if (!FIRST) bprev[idx] = fma(wprev_weight, (T)lam[idx], -bn);
  if (gc2) {
    const T lw = lap<DIM, ORDER, T>(wstate, idx, x, y, z, nx, ny, nz, cf, wstate[idx]);
    gc2[idx] += (double)(s * cf.dt2) * (double)lw * (double)bn;
  }
  if (gf) gf[idx] -= (double)(s * cf.dt2) * (double)cf.fph * (double)bn;
}

template <typename T>
__global__ void k_init_adj(T* __restrict__ bN, T* __restrict__ bN1, const double* __restrict__ lam, T wN,
                           T wN1, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bN[i] = wN * (T)lam[i];
    bN1[i] = wN1 * (T)lam[i];
  }
}

template <typename T, int DIM, int ORDER>
static whv_status reverse_sweep(whv_grid g, const TimeGridH& tg, const double* u, const double* f,
                                const double* lam, double* gc2, double* gf, int K) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t N = g->N;
  const int nt = tg.nt;
  dim3 block, grid;
  if (DIM == 1) { block = dim3(256, 1, 1); grid = dim3((nx + 255) / 256, 1, 1); }
  else { block = dim3(32, 8, 1); grid = dim3((nx + 31) / 32, (ny + 7) / 8, DIM > 2 ? nz : 1); }
  const int rb = (int)std::min<int64_t>((N + 255) / 256, 148 * 8);
  const T* c2 = g->c2 ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  StepCoef<T> cf{};
  for (int m = 0; m < 3; ++m) {
    const double h2 = g->h[m] * g->h[m];
    cf.ih2[m] = (T)(g->order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2));
  }
  cf.dt2 = (T)(tg.dt * tg.dt);
  const int nck = (nt + K - 1) / K;   // checkpoints at n = 0, K, 2K, ... (pairs W^{sK}, W^{sK+1})
  const size_t es = sizeof(T);
  T *ck = nullptr, *seg = nullptr, *adj = nullptr;
  auto cleanup = [&]() { if (ck) cudaFree(ck); if (seg) cudaFree(seg); if (adj) cudaFree(adj); };
#define AD_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) { cleanup(); return cuda_fail(g, _e, #call); }    \
  } while (0)
  AD_CUDA(cudaMalloc(&ck, (size_t)nck * 2 * N * es));
  AD_CUDA(cudaMalloc(&seg, (size_t)(K + 2) * N * es));
  AD_CUDA(cudaMalloc(&adj, (size_t)3 * N * es));
  int launches = 0;
  // ---- forward sweep: W^0 = u, W^1 (Taylor), ..., keeping pairs (W^{sK}, W^{sK+1})
  T* s0 = seg;            // rolling three states in the segment buffer
  T* s1 = seg + N;
  T* s2 = seg + 2 * N;
  k_to_state<T><<<rb, 256, 0, g->stream>>>(u, s0, N);
  cf.fph = T(1);
  k_fwd_state<T, DIM, ORDER, true><<<grid, block, 0, g->stream>>>(nullptr, s0, s1, c2, f, nx, ny, nz, cf);
  launches += 2;
  AD_CUDA(cudaGetLastError());
  for (int n = 1; n <= nt; ++n) {
    // s0 = W^{n-1}, s1 = W^n
    if ((n - 1) % K == 0) {
      const int s = (n - 1) / K;
      AD_CUDA(cudaMemcpyAsync(ck + (size_t)(2 * s) * N, s0, N * es, cudaMemcpyDeviceToDevice, g->stream));
      AD_CUDA(cudaMemcpyAsync(ck + (size_t)(2 * s + 1) * N, s1, N * es, cudaMemcpyDeviceToDevice, g->stream));
    }
    if (n == nt) break;
    cf.fph = (T)tg.phase[n];
    k_fwd_state<T, DIM, ORDER, false><<<grid, block, 0, g->stream>>>(s0, s1, s2, c2, f, nx, ny, nz, cf);
    ++launches;
    T* t = s0; s0 = s1; s1 = s2; s2 = t;
  }
  AD_CUDA(cudaGetLastError());
  // ---- reverse sweep, segment by segment (last first)
  T* bnext = adj;          // Wb^{n+1}
  T* bcur = adj + N;       // Wb^n
  T* bprev = adj + 2 * N;  // Wb^{n-1}
  k_init_adj<T><<<rb, 256, 0, g->stream>>>(bnext, bcur, lam, (T)tg.weight[nt], (T)tg.weight[nt - 1], N);
  ++launches;
  AD_CUDA(cudaGetLastError());
  // bnext = Wb^{nt} (complete), bcur = Wb^{nt-1} (partial)
  for (int s = nck - 1; s >= 0; --s) {
    const int n0 = s * K, n1 = std::min(nt, n0 + K);   // states W^{n0} .. W^{n1} in seg[0 .. n1-n0]
    AD_CUDA(cudaMemcpyAsync(seg, ck + (size_t)(2 * s) * N, N * es, cudaMemcpyDeviceToDevice, g->stream));
    AD_CUDA(cudaMemcpyAsync(seg + N, ck + (size_t)(2 * s + 1) * N, N * es, cudaMemcpyDeviceToDevice, g->stream));
    for (int n = n0 + 1; n < n1 - 1; ++n) {   // W^{n0+2} .. W^{n1-1}
      cf.fph = (T)tg.phase[n];
      k_fwd_state<T, DIM, ORDER, false><<<grid, block, 0, g->stream>>>(
          seg + (size_t)(n - 1 - n0) * N, seg + (size_t)(n - n0) * N, seg + (size_t)(n + 1 - n0) * N, c2, f,
          nx, ny, nz, cf);
      ++launches;
    }
    AD_CUDA(cudaGetLastError());
    // reverse steps n = n1-1 .. max(n0, 1) of this segment use W^n = seg[n - n0]
    for (int n = n1 - 1; n >= std::max(n0, 1); --n) {
      cf.fph = (T)tg.phase[n];
      k_reverse<T, DIM, ORDER, false><<<grid, block, 0, g->stream>>>(
          bnext, bcur, bprev, seg + (size_t)(n - n0) * N, lam, c2, gc2, gf, nx, ny, nz, cf,
          (T)tg.weight[n - 1]);
      ++launches;
      T* t = bnext; bnext = bcur; bcur = bprev; bprev = t;
    }
    AD_CUDA(cudaGetLastError());
  }
  // now bnext = Wb^1 (complete), bcur = Wb^0 (partial); reverse of the Taylor step with W^0 = seg[0]
  // (segment 0 is the last one loaded)
  cf.fph = (T)tg.phase[0];
  k_reverse<T, DIM, ORDER, true><<<grid, block, 0, g->stream>>>(bnext, bcur, nullptr, seg, lam, c2, gc2, gf,
                                                                 nx, ny, nz, cf, T(0));
  ++launches;
  AD_CUDA(cudaGetLastError());
  AD_CUDA(cudaStreamSynchronize(g->stream));
  count_launches(launches);
  cleanup();
#undef AD_CUDA
  return WHV_OK;
}

template <typename T>
static whv_status reverse_dispatch(whv_grid g, const TimeGridH& tg, const double* u, const double* f,
                                   const double* lam, double* gc2, double* gf, int K) {
  switch (g->dim * 10 + g->order) {
    case 12: return reverse_sweep<T, 1, 2>(g, tg, u, f, lam, gc2, gf, K);
    case 14: return reverse_sweep<T, 1, 4>(g, tg, u, f, lam, gc2, gf, K);
    case 22: return reverse_sweep<T, 2, 2>(g, tg, u, f, lam, gc2, gf, K);
    case 24: return reverse_sweep<T, 2, 4>(g, tg, u, f, lam, gc2, gf, K);
    case 32: return reverse_sweep<T, 3, 2>(g, tg, u, f, lam, gc2, gf, K);
    case 34: return reverse_sweep<T, 3, 4>(g, tg, u, f, lam, gc2, gf, K);
  }
  return fail(g, WHV_ERR_INVALID, "unsupported dim/order");
}

// out = a * x * y (elementwise; y = nullptr => ones)
__global__ void k_scale_by(const double* __restrict__ x, const double* __restrict__ y, double a, int64_t n,
                           double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] * (y ? y[i] : 1.0);
}

whv_status adjoint_gradients(whv_grid g, const TimeGridH& tg, const double* u, const double* f,
                             const double* lam, double* gc2, double* gf, int K, int prec) {
  if (gc2) WHV_CUDA(g, cudaMemsetAsync(gc2, 0, g->N * sizeof(double), g->stream));
  if (gf) WHV_CUDA(g, cudaMemsetAsync(gf, 0, g->N * sizeof(double), g->stream));
  return prec == WHV_FP64 ? reverse_dispatch<double>(g, tg, u, f, lam, gc2, gf, K)
                          : reverse_dispatch<float>(g, tg, u, f, lam, gc2, gf, K);
}

whv_status scale_by(whv_grid g, const double* x, const double* y, double a, double* out) {
  const int rb = (int)std::min<int64_t>((g->N + 255) / 256, 148 * 8);
  k_scale_by<<<rb, 256, 0, g->stream>>>(x, y, a, g->N, out);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  return WHV_OK;
}

}  // namespace whv
