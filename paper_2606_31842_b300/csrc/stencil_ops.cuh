// Stencil pieces shared by the stepping kernels and the eigen-solve: step coefficients and the
// p-th order second differences with the Dirichlet / odd-reflection closure.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace whv {

template <typename T>
struct StepCoef {
  T ih2[3];   // 1/h^2 per direction (order 4: 1/(12 h^2))
  T dt2;      // dt^2
  T fph;      // cos(omega_hat t^n) of the step (first step: 1)
  T w0, w1;   // first step: w_0, w_1; other steps: w1 = w_{n+1}
  // 2nd order, c = 1: W^{n+1} = sum_m a_m (W_{+e_m} + W_{-e_m}) + b W^n - W^{n-1} (- dt^2 f cos)
  T a[3];     // dt^2 / h_m^2
  T b;        // 2 - 2 sum_m a_m
};

// Second difference along one axis at interior index i of n, without the 1/h^2 factor.
// Dirichlet nodes hold 0; order 4 uses the odd reflection u_{-1} = -u_1 beyond the boundary.
template <int ORDER, typename T, typename S>
__device__ __forceinline__ T d2(const S* __restrict__ w, int64_t idx, int i, int n, int64_t s, T c) {
  const T m1 = (i > 0) ? (T)__ldg(w + idx - s) : T(0);
  const T p1 = (i < n - 1) ? (T)__ldg(w + idx + s) : T(0);
  if (ORDER == 2) {
    return fma(T(-2), c, m1 + p1);
  } else {
    const T m2 = (i > 1) ? (T)__ldg(w + idx - 2 * s) : (i == 1 ? T(0) : -c);
    const T p2 = (i < n - 2) ? (T)__ldg(w + idx + 2 * s) : (i == n - 2 ? T(0) : -c);
    return fma(T(-30), c, fma(T(16), m1 + p1, -(m2 + p2)));
  }
}

// The same second difference with L2-coherent loads (ld.global.cg): for kernels that read data
// written earlier in the same launch (the persistent batched kernel), where the read-only path
// could serve stale L1 lines.
template <int ORDER, typename T>
__device__ __forceinline__ T d2_cg(const T* w, int64_t idx, int i, int n, int64_t s, T c) {
  const T m1 = (i > 0) ? __ldcg(w + idx - s) : T(0);
  const T p1 = (i < n - 1) ? __ldcg(w + idx + s) : T(0);
  if (ORDER == 2) return fma(T(-2), c, m1 + p1);
  const T m2 = (i > 1) ? __ldcg(w + idx - 2 * s) : (i == 1 ? T(0) : -c);
  const T p2 = (i < n - 2) ? __ldcg(w + idx + 2 * s) : (i == n - 2 ? T(0) : -c);
  return fma(T(-30), c, fma(T(16), m1 + p1, -(m2 + p2)));
}

template <int DIM, int ORDER, typename T>
__device__ __forceinline__ T lap_cg(const T* w, int64_t idx, int x, int y, int z, int nx, int ny, int nz,
                                    const StepCoef<T>& cf, T c) {
  T l = d2_cg<ORDER, T>(w, idx, x, nx, 1, c) * cf.ih2[0];
  if (DIM > 1) l = fma(d2_cg<ORDER, T>(w, idx, y, ny, (int64_t)nx, c), cf.ih2[1], l);
  if (DIM > 2) l = fma(d2_cg<ORDER, T>(w, idx, z, nz, (int64_t)nx * ny, c), cf.ih2[2], l);
  return l;
}

template <int DIM, int ORDER, typename T, typename S>
__device__ __forceinline__ T lap(const S* __restrict__ w, int64_t idx, int x, int y, int z, int nx,
                                 int ny, int nz, const StepCoef<T>& cf, T c) {
  T l = d2<ORDER, T>(w, idx, x, nx, 1, c) * cf.ih2[0];
  if (DIM > 1) l = fma(d2<ORDER, T>(w, idx, y, ny, (int64_t)nx, c), cf.ih2[1], l);
  if (DIM > 2) l = fma(d2<ORDER, T>(w, idx, z, nz, (int64_t)nx * ny, c), cf.ih2[2], l);
  return l;
}

// Conservative second-order operator div_h(c^2 grad_h) at interior index idx (x fastest): per
// axis m, (F+ (u+ - u) - F- (u - u-)) / h^2, where F+ = face[m][idx] is the face value towards the
// + neighbour (mean of the two nodes' c^2, or the node's own c^2 on the face to the boundary
// node) and F- the face towards the - neighbour (face[m] of that neighbour, or the node's own
// c^2 at the first node); boundary nodes hold 0.
template <typename T>
struct ConsFaces {
  const T* f[3];   // face values per axis
  const T* c2;     // node values (the - face of the first node)
};

template <int DIM, typename T, typename S>
__device__ __forceinline__ T lap_cons(const S* __restrict__ w, int64_t idx, int x, int y, int z, int nx, int ny,
                                      int nz, const ConsFaces<T>& fc, const StepCoef<T>& cf, T c) {
  T L = T(0);
#pragma unroll
  for (int m = 0; m < DIM; ++m) {
    const int i = m == 0 ? x : (m == 1 ? y : z);
    const int n = m == 0 ? nx : (m == 1 ? ny : nz);
    const int64_t st = m == 0 ? 1 : (m == 1 ? (int64_t)nx : (int64_t)nx * ny);
    const T up = i < n - 1 ? (T)__ldg(w + idx + st) : T(0);
    const T um = i > 0 ? (T)__ldg(w + idx - st) : T(0);
    const T Fp = __ldg(fc.f[m] + idx);
    const T Fm = i > 0 ? __ldg(fc.f[m] + idx - st) : __ldg(fc.c2 + idx);
    L = fma(fma(Fp, up - c, -Fm * (c - um)), cf.ih2[m], L);
  }
  return L;
}

}  // namespace whv
