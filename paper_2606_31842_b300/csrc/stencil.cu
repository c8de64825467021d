// Fused explicit leapfrog step + trapezoid time filter: one wave solve = Pi_h (eq.
// discreteWaveExplicit with the filter of eq. quadrature accumulated in the same pass).
//
//   first step  W^1 = W^0 + dt^2/2 (c^2 Delta_h W^0 - f)                 (D0t W^0 = 0)
//               acc = w_0 W^0 + w_1 W^1
//   step n      W^{n+1} = 2 W^n - W^{n-1} + dt^2 (c^2 Delta_h W^n - f cos(omega_hat t^n))
//               acc += w_{n+1} W^{n+1}            (W^{n+1} overwrites W^{n-1} in place)
//   last step   as step n = Nt-1, but instead of storing W^Nt and acc it writes the FP64
//               result: out = acc (Pi_h v) or out = v - acc (= A v for f = 0) together with the
//               M-weighted partial sums of <v, out> (the CG denominator p^T A p).
//
// One thread per interior node; x is the fastest axis and maps to threadIdx.x so every load of
// a row is coalesced; neighbour loads go through the read-only path.  Element type T is double
// (FP64 stepping) or float (FP32 stepping: state, speed and filter accumulator in FP32, the
// Krylov-side input v and output in FP64).
#include <math.h>

#include <type_traits>
#include <vector>

#include "df64.cuh"
#include "stencil_ops.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

enum Kind { K_STEP = 0, K_LAST_OUT = 1, K_LAST_AV = 2 };

// First step from W^0 = v (FP64 in; nullptr => 0).  Writes W^0 -> w0, W^1 -> w1, acc.
template <typename T, int DIM, int ORDER, bool VARC, bool FORCE, bool ZERO_V>
__global__ void __launch_bounds__(256) k_first(const double* __restrict__ v, T* __restrict__ w0,
                                               T* __restrict__ w1, T* __restrict__ acc,
                                               const T* __restrict__ c2,
                                               const double* __restrict__ f, int nx, int ny, int nz,
                                               StepCoef<T> cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  T W0 = T(0), L = T(0);
  if (!ZERO_V) {
    W0 = (T)v[idx];
    L = lap<DIM, ORDER, T>(v, idx, x, y, z, nx, ny, nz, cf, W0);
    if (VARC) L *= c2[idx];
  }
  if (FORCE) L -= (T)f[idx];  // cos(0) = 1
  const T W1 = fma(T(0.5) * cf.dt2, L, W0);
  w0[idx] = W0;
  w1[idx] = W1;
  acc[idx] = fma(cf.w1, W1, cf.w0 * W0);
}

template <typename T, int DIM, int ORDER, bool VARC, bool FORCE, int KIND>
__global__ void __launch_bounds__(256) k_step(const T* __restrict__ wc, T* __restrict__ wp,
                                              T* __restrict__ acc, const T* __restrict__ c2,
                                              const double* __restrict__ f,
                                              const double* __restrict__ v,
                                              const double* __restrict__ mw,
                                              double* __restrict__ out, int nx, int ny, int nz,
                                              StepCoef<T> cf, double* partials, unsigned* counter,
                                              double* scal_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool in = (x < nx) && (y < ny);
  double part = 0.0;
  if (in) {
    const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
    const T c = __ldg(wc + idx);
    T wn;
    if constexpr (ORDER == 2 && !VARC) {
      // 6 (2-D) / 8 (3-D) floating-point instructions per update instead of 9 / 12
      T u = fma(cf.b, c, -wp[idx]);
      u = fma(cf.a[0], (x > 0 ? __ldg(wc + idx - 1) : T(0)) + (x < nx - 1 ? __ldg(wc + idx + 1) : T(0)), u);
      if (DIM > 1)
        u = fma(cf.a[1], (y > 0 ? __ldg(wc + idx - nx) : T(0)) + (y < ny - 1 ? __ldg(wc + idx + nx) : T(0)), u);
      if (DIM > 2) {
        const int64_t pl = (int64_t)nx * ny;
        u = fma(cf.a[2], (z > 0 ? __ldg(wc + idx - pl) : T(0)) + (z < nz - 1 ? __ldg(wc + idx + pl) : T(0)), u);
      }
      if (FORCE) u = fma(-cf.dt2 * cf.fph, (T)f[idx], u);
      wn = u;
    } else {
      T L = lap<DIM, ORDER, T>(wc, idx, x, y, z, nx, ny, nz, cf, c);
      if (VARC) L *= c2[idx];
      if (FORCE) L = fma(-(T)f[idx], cf.fph, L);
      wn = fma(cf.dt2, L, fma(T(2), c, -wp[idx]));
    }
    const T a = fma(cf.w1, wn, acc[idx]);
    if (KIND == K_STEP) {
      wp[idx] = wn;
      acc[idx] = a;
    } else if (KIND == K_LAST_OUT) {
      out[idx] = (double)a;
    } else {
      const double vi = v[idx];
      const double o = vi - (double)a;
      out[idx] = o;
      part = (mw ? vi * mw[idx] : vi) * o;
    }
  }
  if (KIND == K_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// Conservative operator div_h(c^2 grad_h) (second order): first step and step kernels, same
// structure and epilogues as k_first / k_step with lap_cons in place of c^2 Delta_h.
template <typename T, int DIM, bool FORCE, bool ZERO_V>
__global__ void __launch_bounds__(256) k_first_cons(const double* __restrict__ v, T* __restrict__ w0,
                                                    T* __restrict__ w1, T* __restrict__ acc, ConsFaces<T> fc,
                                                    const double* __restrict__ f, int nx, int ny, int nz,
                                                    StepCoef<T> cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  T W0 = T(0), L = T(0);
  if (!ZERO_V) {
    W0 = (T)v[idx];
    L = lap_cons<DIM, T>(v, idx, x, y, z, nx, ny, nz, fc, cf, W0);
  }
  if (FORCE) L -= (T)f[idx];
  const T W1 = fma(T(0.5) * cf.dt2, L, W0);
  w0[idx] = W0;
  w1[idx] = W1;
  acc[idx] = fma(cf.w1, W1, cf.w0 * W0);
}

template <typename T, int DIM, bool FORCE, int KIND>
__global__ void __launch_bounds__(256) k_step_cons(const T* __restrict__ wc, T* __restrict__ wp,
                                                   T* __restrict__ acc, ConsFaces<T> fc,
                                                   const double* __restrict__ f, const double* __restrict__ v,
                                                   double* __restrict__ out, int nx, int ny, int nz, StepCoef<T> cf,
                                                   double* partials, unsigned* counter, double* scal_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool in = (x < nx) && (y < ny);
  double part = 0.0;
  if (in) {
    const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
    const T c = __ldg(wc + idx);
    T L = lap_cons<DIM, T>(wc, idx, x, y, z, nx, ny, nz, fc, cf, c);
    if (FORCE) L = fma(-(T)f[idx], cf.fph, L);
    const T wn = fma(cf.dt2, L, fma(T(2), c, -wp[idx]));
    const T a = fma(cf.w1, wn, acc[idx]);
    if (KIND == K_STEP) {
      wp[idx] = wn;
      acc[idx] = a;
    } else if (KIND == K_LAST_OUT) {
      out[idx] = (double)a;
    } else {   // Euclidean inner product (the conservative operator is symmetric without M)
      const double vi = v[idx];
      const double o = vi - (double)a;
      out[idx] = o;
      part = vi * o;
    }
  }
  if (KIND == K_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// Double-float wave solves (second order): the residual wave solves of the FP64 residual
// correction with WHV_RESIDUAL_DF64 -- same recurrence, filter and epilogues as k_first / k_step,
// each value the pair hi + lo of FP32 numbers (df64.cuh), stored as 8-byte pairs.
// second order: ih2 ((W_- + W_+) - 2 W) per axis; fourth order (ih2 = 1 / 12 h^2):
// ih2 ((16 (W_-1 + W_+1) - (W_-2 + W_+2)) - 30 W) with the odd-reflection closure of the FP32 / FP64
// kernels (the value two nodes outside the first or last interior node is minus that node)
template <int DIM, int ORDER, typename LD>
__device__ __forceinline__ dfl lap_df(LD load, int x, int y, int z, int nx, int ny, int nz, int64_t idx,
                                      const DfCoef& cf, dfl c) {
  const dfl c2x = {2.0f * c.hi, 2.0f * c.lo};   // exact
  dfl L = df_zero();
#pragma unroll
  for (int m = 0; m < DIM; ++m) {
    const int i = m == 0 ? x : (m == 1 ? y : z);
    const int n = m == 0 ? nx : (m == 1 ? ny : nz);
    const int64_t st = m == 0 ? 1 : (m == 1 ? (int64_t)nx : (int64_t)nx * ny);
    const dfl s = df_add(i > 0 ? load(idx - st) : df_zero(), i < n - 1 ? load(idx + st) : df_zero());
    dfl t;
    if (ORDER == 2) {
      t = df_sub(s, c2x);
    } else {
      const dfl m2 = i > 1 ? load(idx - 2 * st) : (i == 1 ? df_zero() : df_neg(c));
      const dfl p2 = i < n - 2 ? load(idx + 2 * st) : (i == n - 2 ? df_zero() : df_neg(c));
      t = df_sub(dfl{16.0f * s.hi, 16.0f * s.lo}, df_add(m2, p2));   // 16 s exact
      t = df_sub(t, df_mul(dfl{30.0f, 0.0f}, c));
    }
    L = df_add(L, df_mul(cf.ih2[m], t));
  }
  return L;
}

template <int DIM, int ORDER, bool VARC, bool FORCE, bool ZERO_V>
__global__ void __launch_bounds__(256) k_first_df(const double* __restrict__ v, dfl* __restrict__ w0,
                                                  dfl* __restrict__ w1, dfl* __restrict__ acc,
                                                  const double* __restrict__ c2, const double* __restrict__ f,
                                                  int nx, int ny, int nz, DfCoef cf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  dfl W0 = df_zero(), L = df_zero();
  if (!ZERO_V) {
    W0 = df_from(v[idx]);
    L = lap_df<DIM, ORDER>([&](int64_t j) { return df_from(__ldg(v + j)); }, x, y, z, nx, ny, nz, idx, cf, W0);
    if (VARC) L = df_mul(L, df_from(c2[idx]));
  }
  if (FORCE) L = df_sub(L, df_from(f[idx]));   // cos(0) = 1
  const dfl W1 = df_add(W0, df_mul(cf.hdt2, L));
  w0[idx] = W0;
  w1[idx] = W1;
  acc[idx] = df_add(df_mul(cf.w0, W0), df_mul(cf.w1, W1));
}

template <int DIM, int ORDER, bool VARC, bool FORCE, int KIND>
__global__ void __launch_bounds__(256) k_step_df(const dfl* __restrict__ wc, dfl* __restrict__ wp,
                                                 dfl* __restrict__ acc, const double* __restrict__ c2,
                                                 const double* __restrict__ f, const double* __restrict__ v,
                                                 const double* __restrict__ mw, double* __restrict__ out, int nx,
                                                 int ny, int nz, DfCoef cf, double* partials, unsigned* counter,
                                                 double* scal_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool in = (x < nx) && (y < ny);
  double part = 0.0;
  if (in) {
    const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
    const dfl c = wc[idx];
    auto load = [&](int64_t j) { return wc[j]; };
    dfl wn;
    if (!VARC && ORDER == 2) {   // sum_m a_m (W_{+m} + W_{-m}) + b W^n - W^{n-1}
      wn = df_sub(df_mul(cf.b, c), wp[idx]);
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        const int i = m == 0 ? x : (m == 1 ? y : z);
        const int n = m == 0 ? nx : (m == 1 ? ny : nz);
        const int64_t st = m == 0 ? 1 : (m == 1 ? (int64_t)nx : (int64_t)nx * ny);
        const dfl s = df_add(i > 0 ? load(idx - st) : df_zero(), i < n - 1 ? load(idx + st) : df_zero());
        wn = df_add(wn, df_mul(cf.a[m], s));
      }
      if (FORCE) wn = df_sub(wn, df_mul(cf.fph, df_from(f[idx])));   // fph = dt^2 cos(omega_hat t^n)
    } else {
      dfl L = lap_df<DIM, ORDER>(load, x, y, z, nx, ny, nz, idx, cf, c);
      if (VARC) L = df_mul(L, df_from(c2[idx]));
      if (FORCE) L = df_sub(L, df_mul(cf.fph, df_from(f[idx])));   // fph = cos(omega_hat t^n)
      const dfl t = df_sub(dfl{2.0f * c.hi, 2.0f * c.lo}, wp[idx]);
      wn = df_add(t, df_mul(cf.dt2, L));
    }
    const dfl a = df_add(acc[idx], df_mul(cf.w1, wn));
    if (KIND == K_STEP) {
      wp[idx] = wn;
      acc[idx] = a;
    } else if (KIND == K_LAST_OUT) {
      out[idx] = df_to(a);
    } else {
      const double vi = v[idx];
      const double o = vi - df_to(a);
      out[idx] = o;
      part = (mw ? vi * mw[idx] : vi) * o;
    }
  }
  if (KIND == K_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// 3-D 7-point variant: each thread marches through a column of `zc` planes, keeping W^n at
// z-1, z, z+1 in registers (the z neighbours cost no extra load) and loading the next plane
// one iteration ahead; x / y neighbours come through L1.  Same arithmetic and summation order
// as k_step.
template <typename T, bool VARC, bool FORCE, int KIND>
__global__ void __launch_bounds__(256) k_step3d(const T* __restrict__ wc, T* __restrict__ wp,
                                                T* __restrict__ acc, const T* __restrict__ c2,
                                                const double* __restrict__ f,
                                                const double* __restrict__ v,
                                                const double* __restrict__ mw,
                                                double* __restrict__ out, int nx, int ny, int nz,
                                                int zc, StepCoef<T> cf, double* partials,
                                                unsigned* counter, double* scal_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const bool in = (x < nx) && (y < ny);
  const int64_t plane = (int64_t)nx * ny;
  int64_t idx = x + (int64_t)nx * y + plane * z0;
  double part = 0.0;
  if (in) {
    T wzm = z0 > 0 ? __ldg(wc + idx - plane) : T(0);
    T wz = __ldg(wc + idx);
    T wzp = z0 + 1 < nz ? __ldg(wc + idx + plane) : T(0);
    // W^{n-1} and acc of the current plane, loaded one plane ahead (KIND == K_LAST_AV reads v
    // instead of storing: the extra loads stay the same)
    T wpc = wp[idx];
    T acc_c = acc[idx];
    for (int z = z0; z < z1; ++z) {
      const bool more = z + 1 < z1;
      // prefetch: W^n two planes ahead, W^{n-1} and acc one plane ahead
      const T wzpp = z + 2 < nz ? __ldg(wc + idx + 2 * plane) : T(0);
      const T wpn = more ? wp[idx + plane] : T(0);
      const T accn = more ? acc[idx + plane] : T(0);
      const T xm = x > 0 ? __ldg(wc + idx - 1) : T(0);
      const T xp = x < nx - 1 ? __ldg(wc + idx + 1) : T(0);
      const T ym = y > 0 ? __ldg(wc + idx - nx) : T(0);
      const T yp = y < ny - 1 ? __ldg(wc + idx + nx) : T(0);
      T wn;
      if constexpr (!VARC) {
        T u = fma(cf.b, wz, -wpc);
        u = fma(cf.a[0], xm + xp, u);
        u = fma(cf.a[1], ym + yp, u);
        u = fma(cf.a[2], wzm + wzp, u);
        if (FORCE) u = fma(-cf.dt2 * cf.fph, (T)f[idx], u);
        wn = u;
      } else {
        T L = fma(T(-2), wz, xm + xp) * cf.ih2[0];
        L = fma(fma(T(-2), wz, ym + yp), cf.ih2[1], L);
        L = fma(fma(T(-2), wz, wzm + wzp), cf.ih2[2], L);
        L *= c2[idx];
        if (FORCE) L = fma(-(T)f[idx], cf.fph, L);
        wn = fma(cf.dt2, L, fma(T(2), wz, -wpc));
      }
      const T a = fma(cf.w1, wn, acc_c);
      if (KIND == K_STEP) {
        wp[idx] = wn;
        acc[idx] = a;
      } else if (KIND == K_LAST_OUT) {
        out[idx] = (double)a;
      } else {
        const double vi = v[idx];
        const double o = vi - (double)a;
        out[idx] = o;
        part = fma(mw ? vi * mw[idx] : vi, o, part);
      }
      wzm = wz;
      wz = wzp;
      wzp = wzpp;
      wpc = wpn;
      acc_c = accn;
      idx += plane;
    }
  }
  if (KIND == K_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// 3-D 7-point, FP32, c = 1, f = 0: TWO leapfrog steps per pass (W^{n-1}, W^n -> W^{n+1}, W^{n+2}
// into the other buffer pair), halving the state traffic of single steps.  A CTA of 32 x 16
// threads covers an xy region R1 = tile + 1-node ring (tile 30 x 14) and marches through a
// chunk of zc planes.  At iteration z, step A computes W^{n+1} on R1 at plane z from W^n at
// z-1, z, z+1 (the plane z with its ring staged in shared memory, the z neighbours in registers)
// and stages it; step B then computes W^{n+2} on the tile at plane z-1 from W^{n+1} at z-2, z-1
// (shared memory, staged one iteration earlier), z (registers).  Step A runs on planes
// z0-1 .. z1 of the chunk [z0, z1), step B on z0 .. z1-1.  Nodes outside the domain are 0 (the
// Dirichlet values).  Same operations in the same order as two k_step3d steps:
//   W^{n+1} = fma(az, zm + zp, fma(ay, ym + yp, fma(ax, xm + xp, fma(b, W^n, -W^{n-1}))))
//   acc = fma(w_{n+2}, W^{n+2}, fma(w_{n+1}, W^{n+1}, acc))
// Global traffic per node and 2 steps: read W^{n-1}, W^n, acc, write W^{n+1}, W^{n+2}, acc
// (24 B instead of 40 B), plus the ring re-reads (mostly L1/L2 hits).
constexpr int k3TX = 32, k3TY = 16;   // threads = R1 extent; tile (k3TX - 2) x (k3TY - 2)

template <int KIND>
__global__ void __launch_bounds__(k3TX * k3TY) k_step3d2(const float* __restrict__ gp, const float* __restrict__ gc,
                                                     float* __restrict__ op, float* __restrict__ oc,
                                                     float* __restrict__ acc, const double* __restrict__ v,
                                                     const double* __restrict__ mw, double* __restrict__ out,
                                                     int nx, int ny, int nz, int zc, StepCoef<float> cf, float w2,
                                                     double* partials, unsigned* counter, double* scal_out) {
  // Double-buffered stages, so that one barrier per plane suffices: at iteration z the CTA writes
  // P[z & 1] (W^n(z) with its ring; corners unused) and Q[z & 1] (W^{n+1}(z) on R1), step A reads
  // P[z & 1] after the barrier, step B reads Q[(z - 1) & 1], written before it.
  __shared__ float P[2][k3TY + 2][k3TX + 2];
  __shared__ float Q[2][k3TY][k3TX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int xb = blockIdx.x * (k3TX - 2) - 1, yb = blockIdx.y * (k3TY - 2) - 1;   // R1 origin
  const int x = xb + tx, y = yb + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const bool xin = x >= 0 && x < nx, yin = y >= 0 && y < ny;
  const bool inxy = xin && yin;
  const bool tile = inxy && tx >= 1 && tx < k3TX - 1 && ty >= 1 && ty < k3TY - 1;
  const int64_t plane = (int64_t)nx * ny;
  // the ring node this thread stages, if any: the row above (ty = 0) / below (ty = last) its
  // column, the column left (tx = 0) / right (tx = last) of its row
  int64_t ringv = -1, ringh = -1;
  if (ty == 0 && xin && yb - 1 >= 0) ringv = x + (int64_t)nx * (yb - 1);
  if (ty == k3TY - 1 && xin && yb + k3TY < ny) ringv = x + (int64_t)nx * (yb + k3TY);
  if (tx == 0 && yin && xb - 1 >= 0) ringh = (xb - 1) + (int64_t)nx * y;
  if (tx == k3TX - 1 && yin && xb + k3TX < nx) ringh = (xb + k3TX) + (int64_t)nx * y;
  const int pvy = ty == 0 ? 0 : k3TY + 1, phx = tx == 0 ? 0 : k3TX + 1;
  const bool hasv = ty == 0 || ty == k3TY - 1, hash = tx == 0 || tx == k3TX - 1;
  const int64_t col = inxy ? (int64_t)x + (int64_t)nx * y : 0;
  auto ldc = [&](int z) { return (inxy && z >= 0 && z < nz) ? __ldg(gc + col + plane * z) : 0.0f; };
  float cm = ldc(z0 - 2), c0 = ldc(z0 - 1), cp = ldc(z0);   // W^n at z - 1, z, z + 1 for z = z0 - 1
  float q2 = 0.0f, q1 = 0.0f;   // W^{n+1} of this column at z - 2, z - 1
  float accA = 0.0f;            // acc(z - 1) after step n + 1
  double part = 0.0;
  // running pointers of plane z (valid only where dereferenced: z in range)
  int64_t zo = plane * (z0 - 1);
  for (int z = z0 - 1; z <= z1; ++z, zo += plane) {
    const int b = z & 1;
    const bool zin = z >= 0 && z < nz;
    P[b][ty + 1][tx + 1] = c0;
    if (hasv) P[b][pvy][tx + 1] = (zin && ringv >= 0) ? __ldg(gc + ringv + zo) : 0.0f;
    if (hash) P[b][ty + 1][phx] = (zin && ringh >= 0) ? __ldg(gc + ringh + zo) : 0.0f;
    const bool act = inxy && zin;
    const float cpp = (inxy && z + 2 < nz) ? __ldg(gc + col + zo + 2 * plane) : 0.0f;
    const float wpz = act ? __ldg(gp + col + zo) : 0.0f;
    const float accz = (tile && zin) ? acc[col + zo] : 0.0f;
    __syncthreads();
    // step A: W^{n+1}(z) on R1
    float a1 = 0.0f;
    if (act) {
      float u = fmaf(cf.b, c0, -wpz);
      u = fmaf(cf.a[0], P[b][ty + 1][tx] + P[b][ty + 1][tx + 2], u);
      u = fmaf(cf.a[1], P[b][ty][tx + 1] + P[b][ty + 2][tx + 1], u);
      u = fmaf(cf.a[2], cm + cp, u);
      a1 = u;
    }
    Q[b][ty][tx] = a1;
    const float accN = fmaf(cf.w1, a1, accz);
    // step B: W^{n+2}(z - 1) on the tile, from Q[(z - 1) & 1] (written before the barrier)
    if (z > z0 && tile) {
      const float(*R)[k3TX] = Q[b ^ 1];
      float u = fmaf(cf.b, q1, -cm);
      u = fmaf(cf.a[0], R[ty][tx - 1] + R[ty][tx + 1], u);
      u = fmaf(cf.a[1], R[ty - 1][tx] + R[ty + 1][tx], u);
      u = fmaf(cf.a[2], q2 + a1, u);
      const float a = fmaf(w2, u, accA);
      const int64_t idx = col + zo - plane;
      if (KIND == K_STEP) {
        op[idx] = q1;
        oc[idx] = u;
        acc[idx] = a;
      } else if (KIND == K_LAST_OUT) {
        out[idx] = (double)a;
      } else {
        const double vi = v[idx];
        const double o = vi - (double)a;
        out[idx] = o;
        part = fma(mw ? vi * mw[idx] : vi, o, part);
      }
    }
    q2 = q1;
    q1 = a1;
    accA = accN;
    cm = c0;
    c0 = cp;
    cp = cpp;
  }
  if (KIND == K_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// --------------------------------------------------------------------------- host side
struct LaunchShape {
  dim3 grid, block;
};

constexpr int kZChunk = 16;   // planes per thread of the 3-D 7-point kernel

static bool use_zmarch(whv_grid g) { return g->dim == 3 && g->order == 2; }

static LaunchShape shape_of(whv_grid g) {
  LaunchShape s;
  if (use_zmarch(g)) {
    s.block = dim3(32, 8, 1);
    s.grid = dim3((g->n[0] + 31) / 32, (g->n[1] + 7) / 8, (g->n[2] + kZChunk - 1) / kZChunk);
    return s;
  }
  if (g->dim == 1) {
    s.block = dim3(256, 1, 1);
    s.grid = dim3((g->n[0] + 255) / 256, 1, 1);
  } else {
    s.block = dim3(32, 8, 1);
    s.grid = dim3((g->n[0] + 31) / 32, (g->n[1] + 7) / 8, g->dim > 2 ? g->n[2] : 1);
  }
  return s;
}

template <typename T>
static StepCoef<T> coef_of(whv_grid g, const TimeGridH& tg) {
  StepCoef<T> cf;
  for (int m = 0; m < 3; ++m) {
    const double h2 = g->h[m] * g->h[m];
    cf.ih2[m] = (T)(g->order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2));
  }
  cf.dt2 = (T)(tg.dt * tg.dt);
  cf.fph = T(1);
  cf.w0 = (T)tg.weight[0];
  cf.w1 = (T)tg.weight[1];
  double asum = 0.0;
  for (int m = 0; m < 3; ++m) {
    const double am = m < g->dim ? tg.dt * tg.dt / (g->h[m] * g->h[m]) : 0.0;
    cf.a[m] = (T)am;
    asum += am;
  }
  cf.b = (T)(2.0 - 2.0 * asum);
  return cf;
}

template <typename T, int DIM, bool FORCE>
static whv_status launch_solve_cons(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                                    double* out, int epi, int* nlaunch, void* const* bufs, void* accbuf) {
  const LaunchShape ls = shape_of(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  T* b0 = (T*)bufs[0];
  T* b1 = (T*)bufs[1];
  T* acc = (T*)accbuf;
  ConsFaces<T> fc;
  for (int m = 0; m < 3; ++m) fc.f[m] = (const T*)(sizeof(T) == 8 ? (const void*)g->face64[m] : (const void*)g->face32[m]);
  fc.c2 = (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f);
  StepCoef<T> cf = coef_of<T>(g, tg);
  dim3 fgrid = ls.grid;
  if (DIM == 3) fgrid.z = nz;
  if (v)
    k_first_cons<T, DIM, FORCE, false><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, fc, f, nx, ny, nz, cf);
  else
    k_first_cons<T, DIM, FORCE, true><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, fc, f, nx, ny, nz, cf);
  WHV_CUDA(g, cudaGetLastError());
  *nlaunch = tg.nt;
  T* wprev = b0;
  T* wcur = b1;
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  for (int n = 1; n < tg.nt; ++n) {
    cf.fph = (T)tg.phase[n];
    cf.w1 = (T)tg.weight[n + 1];
    const bool last = (n == tg.nt - 1);
    if (!last)
      k_step_cons<T, DIM, FORCE, K_STEP><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, fc, f, nullptr, nullptr,
                                                                            nx, ny, nz, cf, nullptr, nullptr, nullptr);
    else if (epi == 0)
      k_step_cons<T, DIM, FORCE, K_LAST_OUT><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, fc, f, nullptr, out,
                                                                                nx, ny, nz, cf, nullptr, nullptr,
                                                                                nullptr);
    else
      k_step_cons<T, DIM, FORCE, K_LAST_AV><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, fc, f, v, out, nx,
                                                                               ny, nz, cf, part, cnt, g->scal + S_PQ);
    WHV_CUDA(g, cudaGetLastError());
    T* tmp = wprev;
    wprev = wcur;
    wcur = tmp;
  }
  return WHV_OK;
}

template <int DIM, int ORDER, bool VARC, bool FORCE>
static whv_status launch_solve_df(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                                  double* out, int epi, int* nlaunch, void* const* bufs, void* accbuf) {
  const LaunchShape ls = shape_of(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  dfl* b0 = (dfl*)bufs[0];
  dfl* b1 = (dfl*)bufs[1];
  dfl* acc = (dfl*)accbuf;
  DfCoef cf{};
  double asum = 0.0;
  for (int m = 0; m < 3; ++m) {
    const double h2 = g->h[m] * g->h[m];
    cf.ih2[m] = df_from(ORDER == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2));
    const double am = m < g->dim ? tg.dt * tg.dt / h2 : 0.0;
    cf.a[m] = df_from(am);
    asum += am;
  }
  cf.b = df_from(2.0 - 2.0 * asum);
  cf.dt2 = df_from(tg.dt * tg.dt);
  cf.hdt2 = df_from(0.5 * tg.dt * tg.dt);
  cf.w0 = df_from(tg.weight[0]);
  cf.w1 = df_from(tg.weight[1]);
  dim3 fgrid = ls.grid;
  if (DIM == 3) fgrid.z = nz;
  if (v)
    k_first_df<DIM, ORDER, VARC, FORCE, false><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, g->c2, f, nx, ny, nz, cf);
  else
    k_first_df<DIM, ORDER, VARC, FORCE, true><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, g->c2, f, nx, ny, nz, cf);
  WHV_CUDA(g, cudaGetLastError());
  *nlaunch = tg.nt;
  dfl* wprev = b0;
  dfl* wcur = b1;
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  for (int n = 1; n < tg.nt; ++n) {
    // the c = 1 second-order update takes dt^2 cos(omega_hat t^n) whole, the general one cos(...)
    cf.fph = df_from(VARC || ORDER == 4 ? tg.phase[n] : tg.dt * tg.dt * tg.phase[n]);
    cf.w1 = df_from(tg.weight[n + 1]);
    const bool last = (n == tg.nt - 1);
    if (!last)
      k_step_df<DIM, ORDER, VARC, FORCE, K_STEP><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, g->c2, f, nullptr,
                                                                           nullptr, nullptr, nx, ny, nz, cf, nullptr,
                                                                           nullptr, nullptr);
    else if (epi == 0)
      k_step_df<DIM, ORDER, VARC, FORCE, K_LAST_OUT><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, g->c2, f, nullptr,
                                                                               nullptr, out, nx, ny, nz, cf, nullptr,
                                                                               nullptr, nullptr);
    else
      k_step_df<DIM, ORDER, VARC, FORCE, K_LAST_AV><<<fgrid, ls.block, 0, g->stream>>>(wcur, wprev, acc, g->c2, f, v, g->mw,
                                                                              out, nx, ny, nz, cf, part, cnt,
                                                                              g->scal + S_PQ);
    WHV_CUDA(g, cudaGetLastError());
    dfl* tmp = wprev;
    wprev = wcur;
    wcur = tmp;
  }
  return WHV_OK;
}

template <int DIM, int ORDER>
static whv_status dispatch_df_ord(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                                  int epi, int* nl, void* const* bufs, void* acc) {
  const bool varc = g->c2 != nullptr;
  if (varc) return f ? launch_solve_df<DIM, ORDER, true, true>(g, tg, v, f, out, epi, nl, bufs, acc)
                     : launch_solve_df<DIM, ORDER, true, false>(g, tg, v, f, out, epi, nl, bufs, acc);
  return f ? launch_solve_df<DIM, ORDER, false, true>(g, tg, v, f, out, epi, nl, bufs, acc)
           : launch_solve_df<DIM, ORDER, false, false>(g, tg, v, f, out, epi, nl, bufs, acc);
}

template <int DIM>
static whv_status dispatch_df_dim(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                                  int epi, int* nl, void* const* bufs, void* acc) {
  return g->order == 2 ? dispatch_df_ord<DIM, 2>(g, tg, v, f, out, epi, nl, bufs, acc)
                       : dispatch_df_ord<DIM, 4>(g, tg, v, f, out, epi, nl, bufs, acc);
}

constexpr int kZChunk2 = 32;   // planes per CTA of the two-step 3-D kernel

static dim3 grid_3d2(whv_grid g) {
  return dim3((g->n[0] + k3TX - 3) / (k3TX - 2), (g->n[1] + k3TY - 3) / (k3TY - 2),
              (g->n[2] + kZChunk2 - 1) / kZChunk2);
}

// Steps n = 1 .. nt-1 of a 3-D f = 0 FP32 wave solve (c = 1, second order) after the Taylor
// start (W^0 in buf[0], W^1 in buf[1], acc): one single step when their number is odd, then
// two-step passes alternating between the buffer pairs (0, 1) and (2, 3); the last launch writes
// the epilogue.
static whv_status two_step_3d(whv_grid g, const TimeGridH& tg, const double* v, double* out, int epi,
                              int* launches, void* const* bufs, void* accbuf) {
  float* buf[4] = {(float*)bufs[0], (float*)bufs[1], (float*)bufs[2], (float*)bufs[3]};
  float* acc = (float*)accbuf;
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  StepCoef<float> cf = coef_of<float>(g, tg);
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  const dim3 g2 = grid_3d2(g), b2(k3TX, k3TY, 1);
  if ((int64_t)g2.x * g2.y * g2.z > chan_cap(g, CH_STEP)) return fail(g, WHV_ERR_INVALID, "grid too large for the fused reduction");
  const LaunchShape ls = shape_of(g);
  float* wprev = buf[0];
  float* wcur = buf[1];
  int n = 1, nl = 0;
  if ((tg.nt - 1) % 2 == 1) {   // one single step first (the last one when nt = 2)
    cf.w1 = (float)tg.weight[2];
    const bool last = tg.nt == 2;
    if (!last)
      k_step3d<float, false, false, K_STEP><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, nullptr, nullptr, nullptr, nullptr, nullptr, nx, ny, nz, kZChunk, cf, nullptr, nullptr, nullptr);
    else if (epi == 0)
      k_step3d<float, false, false, K_LAST_OUT><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, nullptr, nullptr, nullptr, nullptr, out, nx, ny, nz, kZChunk, cf, nullptr, nullptr, nullptr);
    else
      k_step3d<float, false, false, K_LAST_AV><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, nullptr, nullptr, v, g->mw, out, nx, ny, nz, kZChunk, cf, part, cnt, g->scal + S_PQ);
    WHV_CUDA(g, cudaGetLastError());
    ++nl;
    float* t = wprev; wprev = wcur; wcur = t;
    n = 2;
  }
  while (n < tg.nt) {   // W^n -> W^{n+2}
    cf.w1 = (float)tg.weight[n + 1];
    const float w2 = (float)tg.weight[n + 2];
    const bool last = n + 2 == tg.nt;
    const bool in01 = wprev == buf[0] || wprev == buf[1];   // (wprev, wcur) is one of the pairs
    float* op = in01 ? buf[2] : buf[0];
    float* oc = in01 ? buf[3] : buf[1];
    if (!last)
      k_step3d2<K_STEP><<<g2, b2, 0, g->stream>>>(wprev, wcur, op, oc, acc, nullptr, nullptr, nullptr, nx, ny, nz,
                                                  kZChunk2, cf, w2, nullptr, nullptr, nullptr);
    else if (epi == 0)
      k_step3d2<K_LAST_OUT><<<g2, b2, 0, g->stream>>>(wprev, wcur, op, oc, acc, nullptr, nullptr, out, nx, ny, nz,
                                                      kZChunk2, cf, w2, nullptr, nullptr, nullptr);
    else
      k_step3d2<K_LAST_AV><<<g2, b2, 0, g->stream>>>(wprev, wcur, op, oc, acc, v, g->mw, out, nx, ny, nz, kZChunk2,
                                                     cf, w2, part, cnt, g->scal + S_PQ);
    WHV_CUDA(g, cudaGetLastError());
    ++nl;
    wprev = op;
    wcur = oc;
    n += 2;
  }
  *launches = nl;
  return WHV_OK;
}

template <typename T, int DIM, int ORDER, bool VARC, bool FORCE>
static whv_status launch_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                               double* out, int epi, int* nlaunch, void* const* bufs, void* accbuf,
                               int kb) {
  if constexpr (ORDER == 2 && VARC) {
    if (g->cons) return launch_solve_cons<T, DIM, FORCE>(g, tg, v, f, out, epi, nlaunch, bufs, accbuf);
  }
  const LaunchShape ls = shape_of(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  T* b0 = (T*)bufs[0];
  T* b1 = (T*)bufs[1];
  T* acc = (T*)accbuf;
  const T* c2 = VARC ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  StepCoef<T> cf = coef_of<T>(g, tg);
  dim3 fgrid = ls.grid;
  if (DIM == 3) fgrid.z = nz;   // the first-step kernel takes one plane per z block
  if (v)
    k_first<T, DIM, ORDER, VARC, FORCE, false><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf);
  else
    k_first<T, DIM, ORDER, VARC, FORCE, true><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf);
  WHV_CUDA(g, cudaGetLastError());
  *nlaunch = 1;
  if constexpr (DIM == 2 && !FORCE) {
    if (kb > 1) {
      int nl = 0;
      whv_status s = blocked_steps_2d<T, ORDER, VARC>(g, tg, v, out, epi, kb, &nl, bufs, accbuf);
      *nlaunch += nl;
      return s;
    }
  }
  if constexpr (DIM == 3 && ORDER == 2 && !VARC && !FORCE && sizeof(T) == 4) {
    if (g->kblock >= 2) {   // two steps per launch when set (or chosen by the autotuner)
      int nl = 0;
      whv_status s = two_step_3d(g, tg, v, out, epi, &nl, bufs, accbuf);
      *nlaunch += nl;
      return s;
    }
  }
  *nlaunch += tg.nt - 1;
  // after the first step: W^{n-1} in b0, W^n in b1
  T* wprev = b0;
  T* wcur = b1;
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  for (int n = 1; n < tg.nt; ++n) {
    cf.fph = (T)tg.phase[n];
    cf.w1 = (T)tg.weight[n + 1];
    const bool last = (n == tg.nt - 1);
    if constexpr (DIM == 3 && ORDER == 2) {
      if (!last)
        k_step3d<T, VARC, FORCE, K_STEP><<<ls.grid, ls.block, 0, g->stream>>>(
            wcur, wprev, acc, c2, f, nullptr, nullptr, nullptr, nx, ny, nz, kZChunk, cf, nullptr, nullptr, nullptr);
      else if (epi == 0)
        k_step3d<T, VARC, FORCE, K_LAST_OUT><<<ls.grid, ls.block, 0, g->stream>>>(
            wcur, wprev, acc, c2, f, nullptr, nullptr, out, nx, ny, nz, kZChunk, cf, nullptr, nullptr, nullptr);
      else
        k_step3d<T, VARC, FORCE, K_LAST_AV><<<ls.grid, ls.block, 0, g->stream>>>(
            wcur, wprev, acc, c2, f, v, g->mw, out, nx, ny, nz, kZChunk, cf, part, cnt, g->scal + S_PQ);
    } else if (!last) {
      k_step<T, DIM, ORDER, VARC, FORCE, K_STEP><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, c2, f, nullptr, nullptr, nullptr, nx, ny, nz, cf, nullptr, nullptr, nullptr);
    } else if (epi == 0) {
      k_step<T, DIM, ORDER, VARC, FORCE, K_LAST_OUT><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, c2, f, nullptr, nullptr, out, nx, ny, nz, cf, nullptr, nullptr, nullptr);
    } else {
      k_step<T, DIM, ORDER, VARC, FORCE, K_LAST_AV><<<ls.grid, ls.block, 0, g->stream>>>(
          wcur, wprev, acc, c2, f, v, g->mw, out, nx, ny, nz, cf, part, cnt, g->scal + S_PQ);
    }
    WHV_CUDA(g, cudaGetLastError());
    T* tmp = wprev;
    wprev = wcur;
    wcur = tmp;
  }
  return WHV_OK;
}

struct BufSet {
  void* const* bufs;
  void* acc;
  int kb;
};

template <typename T, int DIM, int ORDER>
static whv_status dispatch_vf(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                              double* out, int epi, int* nl, const BufSet& B) {
  const bool varc = g->c2 != nullptr;
  if (varc) {
    return f ? launch_solve<T, DIM, ORDER, true, true>(g, tg, v, f, out, epi, nl, B.bufs, B.acc, B.kb)
             : launch_solve<T, DIM, ORDER, true, false>(g, tg, v, f, out, epi, nl, B.bufs, B.acc, B.kb);
  }
  return f ? launch_solve<T, DIM, ORDER, false, true>(g, tg, v, f, out, epi, nl, B.bufs, B.acc, B.kb)
           : launch_solve<T, DIM, ORDER, false, false>(g, tg, v, f, out, epi, nl, B.bufs, B.acc, B.kb);
}

template <typename T>
static whv_status dispatch(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                           double* out, int epi, int* nl, const BufSet& B) {
  switch (g->dim * 10 + g->order) {
    case 12: return dispatch_vf<T, 1, 2>(g, tg, v, f, out, epi, nl, B);
    case 14: return dispatch_vf<T, 1, 4>(g, tg, v, f, out, epi, nl, B);
    case 22: return dispatch_vf<T, 2, 2>(g, tg, v, f, out, epi, nl, B);
    case 24: return dispatch_vf<T, 2, 4>(g, tg, v, f, out, epi, nl, B);
    case 32: return dispatch_vf<T, 3, 2>(g, tg, v, f, out, epi, nl, B);
    case 34: return dispatch_vf<T, 3, 4>(g, tg, v, f, out, epi, nl, B);
  }
  return fail(g, WHV_ERR_INVALID, "unsupported dim/order");
}

// default steps per sweep of the blocked 2-D kernel: FP32 stepping is bound by launches and
// L2 traffic (block 8 steps); FP64 stepping is bound by the FP64 pipe, where the redundant halo
// updates of a blocked sweep cost more than the launches they save (one step per launch)
int default_kblock(whv_grid g) { return g->precision == WHV_FP32_STEP ? 8 : 1; }

// outer vectors of the FP64 residual correction, and FP64 stepping buffers on FP32 grids
whv_status ensure_fp64_buffers(whv_grid g) {
  const size_t bytes = (size_t)g->N * sizeof(double);
  if (!g->bo) {
    WHV_CUDA(g, cudaMalloc(&g->xo, bytes));
    WHV_CUDA(g, cudaMalloc(&g->ro, bytes));
    WHV_CUDA(g, cudaMalloc(&g->bo, bytes));
  }
  if (g->precision == WHV_FP64 || g->acc64) return WHV_OK;
  for (int i = 0; i < 4; ++i) WHV_CUDA(g, cudaMalloc(&g->wbuf64[i], bytes));
  WHV_CUDA(g, cudaMalloc(&g->acc64, bytes));
  return WHV_OK;
}

static whv_status launch_wave_solve(whv_grid g, const TimeGridH& tg, const double* v,
                                    const double* f, double* out, int epi, int* nl, int prec) {
  const LaunchShape ls = shape_of(g);
  if ((int64_t)ls.grid.x * ls.grid.y * ls.grid.z > chan_cap(g, CH_STEP))
    return fail(g, WHV_ERR_INVALID, "grid too large for the fused reduction");
  if (prec < 0) prec = g->precision;
  // (the single-CTA kernel steps in FP32 or FP64 only: double-float solves take the general path)
  if (!g->cons && prec != kPrecDF64 && small_grid(g) && g->kblock == 0 && small_tables(g, tg) >= 0) {
    *nl = 1;
    return small_wave_solve(g, tg, v, f, out, epi, prec);
  }
  if (prec == g->precision) {
    const BufSet B{g->wbuf, g->acc, g->cons ? 1 : (g->kblock > 0 ? g->kblock : default_kblock(g))};
    return prec == WHV_FP64 ? dispatch<double>(g, tg, v, f, out, epi, nl, B)
                            : dispatch<float>(g, tg, v, f, out, epi, nl, B);
  }
  if (prec == kPrecDF64) {   // double-float residual wave solves (c^2 Delta_h, order 2 or 4)
    if (g->cons) return fail(g, WHV_ERR_INVALID, "double-float stepping needs the non-conservative operator");
    if (!g->acc64 && g->precision != WHV_FP64) return fail(g, WHV_ERR_INVALID, "FP64 buffers are not allocated");
    void* const* bufs = g->precision == WHV_FP64 ? g->wbuf : g->wbuf64;
    void* acc = g->precision == WHV_FP64 ? g->acc : g->acc64;
    switch (g->dim) {
      case 1: return dispatch_df_dim<1>(g, tg, v, f, out, epi, nl, bufs, acc);
      case 2: return dispatch_df_dim<2>(g, tg, v, f, out, epi, nl, bufs, acc);
      default: return dispatch_df_dim<3>(g, tg, v, f, out, epi, nl, bufs, acc);
    }
  }
  if (prec != WHV_FP64) return fail(g, WHV_ERR_INVALID, "FP32 stepping on an FP64 grid is not provided");
  if (!g->acc64) return fail(g, WHV_ERR_INVALID, "FP64 buffers of the FP32 grid are not allocated");
  const BufSet B{g->wbuf64, g->acc64, 1};   // FP64 stepping is FP64-pipe bound: one step per launch
  return dispatch<double>(g, tg, v, f, out, epi, nl, B);
}

// ------------------------------------------------------------------ CUDA graph cache
// A wave solve is Nt kernel launches; the solvers replay it many times with the same pointers,
// so each (pointers, time grid) combination is captured once into a CUDA graph.
struct PlanEntry {
  const double *v, *f;
  double* out;
  int epi;
  double omega, cfl;
  int periods, adjust, nt, kblock, prec;
  int launches;   // kernels in the graph
  cudaGraphExec_t exec;
  unsigned long long last_use;
};

struct StepPlan {
  std::vector<PlanEntry> entries;
  unsigned long long tick = 0;
};

void free_plan(whv_grid g) {
  // executable graphs must not be destroyed while a launch of them may still be running
  if (g->plan || g->cgloop) cudaStreamSynchronize(g->stream);
  free_cgloop(g);
  if (!g->plan) return;
  for (auto& e : g->plan->entries) cudaGraphExecDestroy(e.exec);
  delete g->plan;
  g->plan = nullptr;
}

static bool uses_tables(whv_grid g) {
  return !g->cons && small_grid(g) && g->kblock == 0;
}

whv_status wave_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                      double* out, int epi, int prec) {
  if (prec < 0) prec = g->precision;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  WHV_CUDA(g, cudaStreamIsCapturing(g->stream, &cs));
  // small grids read the device weight table: a new time grid replaces
  // it, so graphs captured with the old one are dropped before anything is replayed
  if (cs == cudaStreamCaptureStatusNone && uses_tables(g) && small_tables(g, tg) == 1) free_plan(g);
  if (cs != cudaStreamCaptureStatusNone) {  // caller is capturing: record the launches into its graph
    int nl = 0;
    whv_status s = launch_wave_solve(g, tg, v, f, out, epi, &nl, prec);
    count_launches(nl);
    return s;
  }
  if (!g->plan) g->plan = new StepPlan();
  StepPlan* P = g->plan;
  P->tick++;
  for (auto& e : P->entries) {
    if (e.v == v && e.f == f && e.out == out && e.epi == epi && e.omega == tg.omega &&
        e.cfl == tg.cfl && e.periods == tg.periods && e.adjust == tg.adjust && e.nt == tg.nt &&
        e.kblock == g->kblock && e.prec == prec) {
      e.last_use = P->tick;
      WHV_CUDA(g, cudaGraphLaunch(e.exec, g->stream));
      count_launches(e.launches);
      return WHV_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  WHV_CUDA(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  int nl = 0;
  whv_status s = launch_wave_solve(g, tg, v, f, out, epi, &nl, prec);
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (s != WHV_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  WHV_CUDA(g, e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  WHV_CUDA(g, e);
  if (P->entries.size() >= 8) {  // evict the least recently used
    size_t victim = 0;
    for (size_t i = 1; i < P->entries.size(); ++i)
      if (P->entries[i].last_use < P->entries[victim].last_use) victim = i;
    cudaGraphExecDestroy(P->entries[victim].exec);
    P->entries.erase(P->entries.begin() + victim);
  }
  P->entries.push_back(PlanEntry{v, f, out, epi, tg.omega, tg.cfl, tg.periods, tg.adjust, tg.nt,
                                g->kblock, prec, nl, exec, P->tick});
  WHV_CUDA(g, cudaGraphLaunch(exec, g->stream));
  count_launches(nl);
  return WHV_OK;
}

}  // namespace whv

using namespace whv;

extern "C" whv_status whv_apply_pi(whv_grid g, const whv_params* p, const double* v_dev,
                                   const double* f_dev, double* out_dev) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!out_dev) return fail(g, WHV_ERR_INVALID, "out_dev is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  // v and out may alias: the first step has consumed v before the last step writes out.
  // Repeated calls with the same buffers replay one cached CUDA graph.
  return wave_solve(g, tg, v_dev, f_dev, out_dev, 0);
}

extern "C" whv_status whv_set_steps_per_sweep(whv_grid g, int k) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (k < 0 || k > 16) return fail(g, WHV_ERR_INVALID, "steps per sweep must be in [0, 16]");
  g->kblock = k;
  return WHV_OK;
}

extern "C" whv_status whv_get_steps_per_sweep(whv_grid g, int* k) {
  if (!g || !k) return fail(g, WHV_ERR_INVALID, "NULL argument");
  *k = g->kblock != 0 ? g->kblock : (small_grid(g) ? 0 : default_kblock(g));
  return WHV_OK;
}

// Autotuner of the steps per sweep: times two f = 0 wave solves per candidate (graph replay,
// CUDA events on the grid's stream, after one warm-up replay) and keeps the fastest.
extern "C" whv_status whv_autotune(whv_grid g, const whv_params* p, int* best) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  if (small_grid(g) && !g->cons) {   // the whole wave solve runs in one CTA: nothing to tune
    g->kblock = 0;
    if (best) *best = 0;
    return WHV_OK;
  }
  if (g->cons) {   // the conservative operator steps once per launch
    g->kblock = 1;
    if (best) *best = 1;
    return WHV_OK;
  }
  // 2-D: per step and blocked sweeps of k steps; 3-D FP32 (c = 1): per step and two steps per launch
  std::vector<int> cands = {1};
  if (g->dim == 3 && g->order == 2 && !g->c2 && g->precision == WHV_FP32_STEP) cands.push_back(2);
  if (g->dim == 2)
    for (int k : {2, 4, 6, 8, 10, 12, 16}) cands.push_back(k);
  const int nc = (int)cands.size();
  cudaEvent_t e0, e1;
  WHV_CUDA(g, cudaEventCreate(&e0));
  WHV_CUDA(g, cudaEventCreate(&e1));
  int kbest = 1;
  float tbest = 1e30f;
  const int saved = g->kblock;
  WHV_CUDA(g, cudaMemsetAsync(g->x, 0, g->N * sizeof(double), g->stream));
  for (int c = 0; c < nc; ++c) {
    g->kblock = cands[c];
    // v = x (any finite content), out = t; f = 0
    s = wave_solve(g, tg, g->x, nullptr, g->t, 0);
    if (s != WHV_OK) break;
    cudaEventRecord(e0, g->stream);
    for (int r = 0; r < 2 && s == WHV_OK; ++r) s = wave_solve(g, tg, g->x, nullptr, g->t, 0);
    cudaEventRecord(e1, g->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) { s = fail(g, WHV_ERR_CUDA, "autotune timing"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < tbest) { tbest = ms; kbest = cands[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != WHV_OK) { g->kblock = saved; return s; }
  g->kblock = kbest;
  if (best) *best = kbest;
  return WHV_OK;
}
