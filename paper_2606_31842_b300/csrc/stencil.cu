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

#include <algorithm>
#include <type_traits>
#include <vector>

#include <cuda.h>   // CUtensorMap and its encoding enums (the encoder is fetched through the runtime)

#include "df64.cuh"
#include "stencil_ops.cuh"
#include "tma.cuh"
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
                                               StepCoef<T> cf, int wpitch) {
  // (wpitch: row length of the written arrays -- nx, or the padded rows of the 3-D two-step chain)
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const int64_t idx = x + (int64_t)nx * (y + (int64_t)ny * z);
  const int64_t widx = x + (int64_t)wpitch * (y + (int64_t)ny * z);
  T W0 = T(0), L = T(0);
  if (!ZERO_V) {
    W0 = (T)v[idx];
    L = lap<DIM, ORDER, T>(v, idx, x, y, z, nx, ny, nz, cf, W0);
    if (VARC) L *= c2[idx];
  }
  if (FORCE) L -= (T)f[idx];  // cos(0) = 1
  const T W1 = fma(T(0.5) * cf.dt2, L, W0);
  w0[widx] = W0;
  w1[widx] = W1;
  acc[widx] = fma(cf.w1, W1, cf.w0 * W0);
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
      dfs sm[DIM];
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        const int i = m == 0 ? x : (m == 1 ? y : z);
        const int n = m == 0 ? nx : (m == 1 ? ny : nz);
        const int64_t st = m == 0 ? 1 : (m == 1 ? (int64_t)nx : (int64_t)nx * ny);
        sm[m] = df_pair_sum(i > 0 ? load(idx - st) : df_zero(), i < n - 1 ? load(idx + st) : df_zero());
      }
      // fph = dt^2 cos(omega_hat t^n)
      wn = df_leapfrog<DIM, FORCE>(cf.b, c, wp[idx], cf.a, sm, cf.fph, FORCE ? df_from(f[idx]) : df_zero());
    } else {
      dfl L = lap_df<DIM, ORDER>(load, x, y, z, nx, ny, nz, idx, cf, c);
      if (VARC) L = df_mul(L, df_from(c2[idx]));
      if (FORCE) L = df_sub(L, df_mul(cf.fph, df_from(f[idx])));   // fph = cos(omega_hat t^n)
      const dfl t = df_sub(dfl{2.0f * c.hi, 2.0f * c.lo}, wp[idx]);
      wn = df_add(t, df_mul(cf.dt2, L));
    }
    const dfl a = df_fma_acc(acc[idx], cf.w1, wn);
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
// into the other buffer pair), halving the state traffic of single steps.  A CTA of 18 warps
// owns a tile of 64 x 32 nodes in x, y and marches through planes z; lane l of warp row w < 17 holds
// the two adjacent columns x0 + 2l, x0 + 2l + 1 of the two region rows 2w, 2w + 1 (region row r
// is y = y0 - 1 + r: rows 1 .. 32 are the tile, 0 and 33 its ring).  The state lives in
// row-padded ("pitched") FP32 buffers so that every plane of W^n (72 x 36 nodes: the tile, its
// ring, the column beyond the ring and one row beyond it), of W^{n-1} (same box) and of the filter
// sums (the tile) is copied into shared memory by the copy engine (TMA, one elected thread, an
// mbarrier per stage with a bounded wait), two or three planes ahead: W^n in a ring of five
// stages, W^{n-1} and the filter sums in rings of three.  At plane z, step A computes W^{n+1}(z)
// on the tile and its one-node ring into a double-buffered stage (the ring columns x0 - 1 and
// x0 + 64 by the 18th warp, which takes no part in step B); step B computes W^{n+2}(z - 1) on the tile from W^{n+1} at z - 2,
// z - 1 (registers and the stage written at the previous plane) and z, and writes W^{n+1},
// W^{n+2} and the filter sum of plane z - 1.  One barrier per plane.  The grid is persistent: the
// (tile column, plane) pairs are split into equal contiguous ranges, one per CTA, ordered slab by
// slab (slabs of one range's thickness, column by column inside a slab) so that neighbouring tile
// columns pass the same planes at the same time and their halo reads meet in L2.  Nodes outside
// the domain are 0 (copies outside the tensor read as zero).  Same operations in the same order
// as two k_step3d steps:
//   W^{n+1} = fma(az, zm + zp, fma(ay, ym + yp, fma(ax, xm + xp, fma(b, W^n, -W^{n-1}))))
//   acc = fma(w_{n+2}, W^{n+2}, fma(w_{n+1}, W^{n+1}, acc))
// Global traffic per node and 2 steps: read W^{n-1}, W^n, acc, write W^{n+1}, W^{n+2}, acc
// (24 B instead of 40 B), plus the ring re-reads.  If a copy does not arrive within the bounded
// wait, the CTA raises the breakdown flag S_FLAG of the grid and leaves (after a bounded drain).
constexpr int k3W = 64;               // tile columns (two per lane)
constexpr int k3H = 32;               // tile rows
constexpr int k3WR = k3H / 2 + 1;     // warp rows (two region rows each: tile + one ring row per side)
constexpr int k3BX = k3W + 8;         // staged columns x0 - 4 .. x0 + 67 (column c is x0 - 4 + c)
constexpr int k3BY = k3H + 4;         // staged rows y0 - 2 .. y0 + 33 (row pr is region row pr - 1)
constexpr int k3NW = 5, k3NP = 3;     // stages of W^n; of W^{n-1} and of the filter sums
constexpr int k3SPlane = k3BX * k3BY;                       // floats of a W^n / W^{n-1} stage
constexpr int k3APlane = k3W * k3H;                         // floats of a filter-sum stage
constexpr int k3QPlane = k3BX * (k3H + 2);                  // floats of a W^{n+1} stage (rows 0 .. 33)
constexpr int k3Smem = 4 * ((k3NW + k3NP) * k3SPlane + k3NP * k3APlane + 2 * k3QPlane) + 128;

struct Maps3d2 {         // tensor maps of the pitched buffers (one per buffer)
  CUtensorMap w[4];      // 72 x 36 x 1 boxes of the two (W^{n-1}, W^n) pairs
  CUtensorMap acc;       // 64 x 32 x 1 boxes of the filter sums
};

__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

constexpr uint32_t kMbarPolls3 = 1u << 22;   // bound on the polls of one stage's mbarrier
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

struct Geo3d2 {          // per-thread geometry of the current range
  float *op, *oc, *acc;  // pitched outputs
  const double *v, *mw;
  double* out;
  int64_t ppitch, plane;               // pitched plane; unpadded plane (FP64 epilogue)
  int nx, ny, nz, pitch, zs, ze, x0, y0;
  int co[2], uo[2];                    // own pair: pitched / unpadded in-plane offsets
  bool own0[2], own1[2], trow[2], xin0, xin1;
  int pc;                              // staged column of the own pair
};

struct Q3d2 {            // W^{n+1} of the own nodes: q[k & 3] is plane z; filter sums after step n + 1
  float2 q[4][2];
};

template <int PH, int KIND>
__device__ __forceinline__ void s3d2_plane(Q3d2& S, const Geo3d2& G, int z, int wr, const float* SW,
                                           const float* SP, const float* SA, float* SQ, int kw, int kp,
                                           const StepCoef<float>& cf, float w2, double& part) {
  constexpr int Q0 = PH, Q1 = (PH + 3) & 3, Q2 = (PH + 2) & 3;   // W^{n+1}: z, z - 1, z - 2
  const int kwm = kw == 0 ? k3NW - 1 : kw - 1, kwp = kw + 1 == k3NW ? 0 : kw + 1;
  const int kpm = kp == 0 ? k3NP - 1 : kp - 1;
  const float* W0 = SW + kw * k3SPlane;    // W^n(z)
  const float* Wm = SW + kwm * k3SPlane;   // W^n(z - 1)
  const float* Wp = SW + kwp * k3SPlane;   // W^n(z + 1)
  const float* Pp = SP + kp * k3SPlane;    // W^{n-1}(z)
  float* Qz = SQ + (PH & 1) * k3QPlane;    // W^{n+1}(z)
  const bool zin = (unsigned)z < (unsigned)G.nz;
  if (wr == k3WR) {   // the ring warp: step A on the ring columns x0 - 1 and x0 + 64 of the tile rows
    const int r = (threadIdx.x & 31) + 1;   // region row
    const int y = G.y0 - 1 + r;
    const bool yin = y < G.ny;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int c = side == 0 ? 3 : k3W + 4;   // staged column
      const int x = G.x0 - 4 + c;
      const int lr = (r + 1) * k3BX + c;
      float w = fmaf(cf.b, W0[lr], -Pp[lr]);
      w = fmaf(cf.a[0], W0[lr - 1] + W0[lr + 1], w);
      w = fmaf(cf.a[1], W0[lr - k3BX] + W0[lr + k3BX], w);
      w = fmaf(cf.a[2], Wm[lr] + Wp[lr], w);
      Qz[lr - k3BX] = (zin && yin && x >= 0 && x < G.nx) ? w : 0.f;
    }
    return;
  }
  // step A: W^{n+1}(z) of the own nodes (region rows 0 .. 33)
  float2 cm[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int sr = 2 * wr + i + 1;   // staged row of region row 2 wr + i
    const int l = sr * k3BX + G.pc;
    const float2 c0 = lds2(W0 + l), cp = lds2(Wp + l), wpv = lds2(Pp + l);
    cm[i] = lds2(Wm + l);
    const float xm = W0[l - 1], xp = W0[l + 2];
    const float2 up = lds2(W0 + l - k3BX), dn = lds2(W0 + l + k3BX);
    float u0 = fmaf(cf.b, c0.x, -wpv.x);
    u0 = fmaf(cf.a[0], xm + c0.y, u0);
    u0 = fmaf(cf.a[1], up.x + dn.x, u0);
    u0 = fmaf(cf.a[2], cm[i].x + cp.x, u0);
    float u1 = fmaf(cf.b, c0.y, -wpv.y);
    u1 = fmaf(cf.a[0], c0.x + xp, u1);
    u1 = fmaf(cf.a[1], up.y + dn.y, u1);
    u1 = fmaf(cf.a[2], cm[i].y + cp.y, u1);
    S.q[Q0][i] = make_float2((zin && G.own0[i]) ? u0 : 0.f, (zin && G.own1[i]) ? u1 : 0.f);
    *reinterpret_cast<float2*>(Qz + (sr - 1) * k3BX + G.pc) = S.q[Q0][i];
  }
  // step B: W^{n+2}(z - 1) on the tile rows, from Q[(z - 1) & 1]
  if (z > G.zs) {
    const float* R = SQ + ((PH + 1) & 1) * k3QPlane;
    const float* Az = SA + kpm * k3APlane;   // filter sums of plane z - 1
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (!G.trow[i]) continue;
      const int qr = 2 * wr + i;
      const int l = qr * k3BX + G.pc;
      const float2 q1 = S.q[Q1][i], q2 = S.q[Q2][i], a1 = S.q[Q0][i];
      const float xm = R[l - 1], xp = R[l + 2];
      const float2 up = i == 0 ? lds2(R + l - k3BX) : S.q[Q1][0];
      const float2 dn = i == 1 ? lds2(R + l + k3BX) : S.q[Q1][1];
      float u0 = fmaf(cf.b, q1.x, -cm[i].x);
      u0 = fmaf(cf.a[0], xm + q1.y, u0);
      u0 = fmaf(cf.a[1], up.x + dn.x, u0);
      u0 = fmaf(cf.a[2], q2.x + a1.x, u0);
      float u1 = fmaf(cf.b, q1.y, -cm[i].y);
      u1 = fmaf(cf.a[0], q1.x + xp, u1);
      u1 = fmaf(cf.a[1], up.y + dn.y, u1);
      u1 = fmaf(cf.a[2], q2.y + a1.y, u1);
      const float2 ap = lds2(Az + (qr - 1) * k3W + 2 * (threadIdx.x & 31));
      const float2 a = make_float2(fmaf(w2, u0, fmaf(cf.w1, q1.x, ap.x)), fmaf(w2, u1, fmaf(cf.w1, q1.y, ap.y)));
      if (KIND == K_STEP) {
        const int64_t idx = (int64_t)(z - 1) * G.ppitch + G.co[i];
        // pitched rows hold a multiple of 4 floats: a pair's second column past nx is padding
        if (G.xin0) {
          *reinterpret_cast<float2*>(G.op + idx) = q1;
          *reinterpret_cast<float2*>(G.oc + idx) = make_float2(u0, u1);
          *reinterpret_cast<float2*>(G.acc + idx) = a;
        }
      } else {
        const int64_t idx = (int64_t)(z - 1) * G.plane + G.uo[i];
        if (KIND == K_LAST_OUT) {
          if (G.xin0) G.out[idx] = (double)a.x;
          if (G.xin1) G.out[idx + 1] = (double)a.y;
        } else {
          if (G.xin0) {
            const double vi = G.v[idx];
            const double o = vi - (double)a.x;
            G.out[idx] = o;
            part = fma(G.mw ? vi * G.mw[idx] : vi, o, part);
          }
          if (G.xin1) {
            const double vi = G.v[idx + 1];
            const double o = vi - (double)a.y;
            G.out[idx + 1] = o;
            part = fma(G.mw ? vi * G.mw[idx + 1] : vi, o, part);
          }
        }
      }
    }
  }
}

// Buffer indices: in_p / in_c = the W^{n-1} / W^n buffers (0 .. 3) of the maps, outputs op / oc.
template <int KIND>
__global__ void __launch_bounds__(32 * (k3WR + 1), 1) k_step3d2(const Maps3d2* __restrict__ maps, int in_p, int in_c,
                                                         float* __restrict__ op, float* __restrict__ oc,
                                                         float* __restrict__ acc, const double* __restrict__ v,
                                                         const double* __restrict__ mw, double* __restrict__ out,
                                                         int nx, int ny, int nz, int pitch, int cx, int ncol,
                                                         int slab, int64_t units, StepCoef<float> cf, float w2,
                                                         double* partials, unsigned* counter, double* scal_out,
                                                         double* flag) {
  extern __shared__ unsigned char s3raw[];
  float* const SW = reinterpret_cast<float*>(((uintptr_t)s3raw + 127) & ~(uintptr_t)127);   // [5][36][72]
  float* const SP = SW + k3NW * k3SPlane;                                                      // [3][36][72]
  float* const SA = SP + k3NP * k3SPlane;                                                      // [3][32][64]
  float* const SQ = SA + k3NP * k3APlane;                                                      // [2][34][72]
  __shared__ __align__(8) uint64_t barW[k3NW], barP[k3NP], barA[k3NP];
  __shared__ int s_fail;
  const int lane = threadIdx.x, wr = threadIdx.y;
  const bool leader = lane == 0 && wr == 0;
  if (leader) {
    for (int s = 0; s < k3NW; ++s) mbar_init(&barW[s], 1);
    for (int s = 0; s < k3NP; ++s) {
      mbar_init(&barP[s], 1);
      mbar_init(&barA[s], 1);
    }
    mbar_init_fence();
    s_fail = 0;
  }
  // launched as a programmatic dependent of the previous pass: wait for its results before any
  // global access (returns at once when there is no such dependency)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  const CUtensorMap* mapC = &maps->w[in_c];
  const CUtensorMap* mapP = &maps->w[in_p];
  const CUtensorMap* mapA = &maps->acc;
  unsigned parW = 0u, parP = 0u, parA = 0u;   // phase parity of each stage (bit s)
  Geo3d2 G;
  G.op = op; G.oc = oc; G.acc = acc; G.v = v; G.mw = mw; G.out = out;
  G.nx = nx; G.ny = ny; G.nz = nz; G.pitch = pitch;
  G.ppitch = (int64_t)pitch * ny;
  G.plane = (int64_t)nx * ny;
  G.pc = 2 * lane + 4;
  double part = 0.0;
  bool failed = false;
  const int64_t u_end = units * (blockIdx.x + 1) / gridDim.x;
  const int64_t per_slab = (int64_t)ncol * slab;
  for (int64_t u = units * blockIdx.x / gridDim.x; u < u_end && !failed;) {
    // unit u -> (slab, tile column, plane)
    const int64_t sl = u / per_slab;
    const int zlo = (int)(sl * slab);
    const int thick = min(slab, nz - zlo);
    const int64_t rem = u - sl * per_slab;
    const int cid = (int)(rem / thick);
    G.zs = zlo + (int)(rem - (int64_t)cid * thick);
    G.ze = (int)min((int64_t)zlo + thick, (int64_t)G.zs + (u_end - u));
    u += G.ze - G.zs;
    G.x0 = (cid % cx) * k3W;
    G.y0 = (cid / cx) * k3H;
    const int xl = G.x0 + 2 * lane;
    G.xin0 = xl < nx;
    G.xin1 = xl + 1 < nx;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = 2 * wr + i, y = G.y0 - 1 + r;
      const bool yin = y >= 0 && y < ny;
      G.trow[i] = yin && r >= 1 && r <= k3H;
      G.own0[i] = yin && G.xin0;
      G.own1[i] = yin && G.xin1;
      G.co[i] = yin ? xl + pitch * y : 0;
      G.uo[i] = yin ? xl + nx * y : 0;
    }
    const int zb = G.zs - 1;
    // copies of plane zz into its stage (issued by one thread; zz outside the grid reads zeros)
    auto issue_w = [&](int zz, int slot) {
      mbar_arrive_expect_tx(&barW[slot], k3SPlane * 4);
      tma_load_3d(SW + slot * k3SPlane, mapC, G.x0 - 4, G.y0 - 2, zz, &barW[slot]);
    };
    auto issue_p = [&](int zz, int slot) {
      mbar_arrive_expect_tx(&barP[slot], k3SPlane * 4);
      tma_load_3d(SP + slot * k3SPlane, mapP, G.x0 - 4, G.y0 - 2, zz, &barP[slot]);
    };
    auto issue_a = [&](int zz, int slot) {
      mbar_arrive_expect_tx(&barA[slot], k3APlane * 4);
      tma_load_3d(SA + slot * k3APlane, mapA, G.x0, G.y0, zz, &barA[slot]);
    };
    __syncthreads();   // the previous range's reads of the stages are done
    // stage slots: W^n plane zz in (zz - zb + 1) mod 5, W^{n-1} and acc plane zz in (zz - zb) mod 3
    if (leader) {
      issue_w(zb - 1, 0);
      issue_w(zb, 1);
      issue_w(zb + 1, 2);
      if (zb + 2 <= G.ze + 1) issue_w(zb + 2, 3);
      issue_p(zb, 0);
      if (zb + 1 <= G.ze) issue_p(zb + 1, 1);
    }
    Q3d2 S;
#pragma unroll
    for (int d = 0; d < 4; ++d) S.q[d][0] = S.q[d][1] = make_float2(0.f, 0.f);
    int kw = 1, kp = 0;   // stages of W^n(z) and of plane z
    int z = zb;
    // wait for a stage's copies (every thread), flip its parity
    auto wait = [&](uint64_t* bar, unsigned& par, int slot) {
      if (!mbar_wait(&bar[slot], (par >> slot) & 1u, kMbarPolls3)) failed = true;
      par ^= 1u << slot;
    };
    // the planes' stages needed before the loop: W^n(zb - 1), W^n(zb)
    wait(barW, parW, 0);
    wait(barW, parW, 1);
    auto plane = [&](auto ph) {
      constexpr int PH = decltype(ph)::value;
      // W^n(z + 1), W^{n-1}(z) and acc(z - 1) have landed (issued at least two planes ago)
      const int kwp = kw + 1 == k3NW ? 0 : kw + 1;
      wait(barW, parW, kwp);
      wait(barP, parP, kp);
      const int kpm = kp == 0 ? k3NP - 1 : kp - 1;
      if (z > G.zs) wait(barA, parA, kpm);
      if (__syncthreads_or(failed)) {
        failed = true;
        return;
      }
      // the next copies, into stages last read at the previous plane
      if (leader) {
        const int kw3 = kw + 3 >= k3NW ? kw + 3 - k3NW : kw + 3, kp2 = kp + 2 >= k3NP ? kp + 2 - k3NP : kp + 2;
        const int kp1 = kp + 1 == k3NP ? 0 : kp + 1;
        if (z + 3 <= G.ze + 1) issue_w(z + 3, kw3);
        if (z + 2 <= G.ze) issue_p(z + 2, kp2);
        if (z + 1 >= G.zs && z + 1 < G.ze) issue_a(z + 1, kp1);
      }
      s3d2_plane<PH, KIND>(S, G, z, wr, SW, SP, SA, SQ, kw, kp, cf, w2, part);
      kw = kwp;
      kp = kp + 1 == k3NP ? 0 : kp + 1;
      ++z;
    };
    // planes zb .. ze, four at a time (phase k = z - zb: the W^{n+1} stage and registers follow it)
    for (;;) {
      plane(std::integral_constant<int, 0>()); if (failed || z > G.ze) break;
      plane(std::integral_constant<int, 1>()); if (failed || z > G.ze) break;
      plane(std::integral_constant<int, 2>()); if (failed || z > G.ze) break;
      plane(std::integral_constant<int, 3>()); if (failed || z > G.ze) break;
    }
  }
  if (failed) {   // a copy that did not arrive: report, then a bounded drain of the stages
    if (leader) {
      *flag = 1.0;
      for (int s = 0; s < k3NW; ++s) mbar_wait(&barW[s], (parW >> s) & 1u, kMbarPolls3);
      for (int s = 0; s < k3NP; ++s) {
        mbar_wait(&barP[s], (parP >> s) & 1u, kMbarPolls3);
        mbar_wait(&barA[s], (parA >> s) & 1u, kMbarPolls3);
      }
    }
    __syncthreads();
  }
  if (KIND == K_LAST_AV) {   // (also after a failure: the grid's reduction counter stays consistent)
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// unpadded -> pitched copies of the state a two-step chain starts from
__global__ void __launch_bounds__(256) k_to_pitched3(const float* __restrict__ a, const float* __restrict__ b,
                                                     const float* __restrict__ c, float* __restrict__ pa,
                                                     float* __restrict__ pb, float* __restrict__ pc, int nx,
                                                     int64_t n, int pitch) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t x = i % nx, yz = i / nx;
    const int64_t pi = x + (int64_t)pitch * yz;
    pa[pi] = a[i];
    pb[pi] = b[i];
    pc[pi] = c[i];
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

// CTAs of the persistent two-step 3-D kernel: every resident CTA slot of the GPU (one per SM),
// fewer when the grid has fewer than 16 (tile column, plane) pairs per slot
static int s3d2_slots = 0;

void step3d2_init() {
  if (s3d2_slots) return;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fns[] = {(const void*)k_step3d2<K_STEP>, (const void*)k_step3d2<K_LAST_OUT>,
                       (const void*)k_step3d2<K_LAST_AV>};
  for (const void* f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, k3Smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step3d2<K_STEP>, 32 * (k3WR + 1), k3Smem);
  s3d2_slots = std::max(1, sms * std::max(per_sm, 1));
}

struct Grid3d2 {
  int cx, ncol, slab;
  int64_t units;
  int blocks;
};

// tile columns x planes, split into one contiguous range per CTA; slabs as thick as one range
static Grid3d2 grid_3d2(whv_grid g) {
  Grid3d2 q;
  q.cx = (g->n[0] + k3W - 1) / k3W;
  q.ncol = q.cx * ((g->n[1] + k3H - 1) / k3H);
  q.units = (int64_t)q.ncol * g->n[2];
  q.blocks = (int)std::max<int64_t>(1, std::min<int64_t>(s3d2_slots, (q.units + 15) / 16));
  q.slab = (int)std::min<int64_t>(g->n[2], (q.units + q.blocks - 1) / q.blocks);
  return q;
}

typedef CUresult (*EncodeTiled3Fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static bool encode_box3(EncodeTiled3Fn enc, CUtensorMap* map, float* base, int nx, int ny, int nz, int pitch,
                        int bx, int by) {
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)pitch * ny * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// pitched FP32 state of the two-step 3-D kernel (rows padded to a multiple of 4 floats: the copy
// engine needs 16-byte row strides) and its tensor maps; called outside any stream capture
whv_status ensure_pitched3(whv_grid g) {
  if (g->pw3[0]) return WHV_OK;
  const EncodeTiled3Fn enc = (EncodeTiled3Fn)tensor_map_encoder();
  if (!enc) return fail(g, WHV_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int pitch = (nx + 3) / 4 * 4;
  const size_t bytes = (size_t)pitch * ny * nz * sizeof(float);
  float* bufs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < 5 && e == cudaSuccess; ++m) {
    e = cudaMalloc(&bufs[m], bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(bufs[m], 0, bytes, g->stream);   // padding columns stay 0
  }
  Maps3d2 M;
  void* dm = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(Maps3d2));
  bool ok = e == cudaSuccess;
  for (int m = 0; m < 4 && ok; ++m) ok = encode_box3(enc, &M.w[m], bufs[m], nx, ny, nz, pitch, k3BX, k3BY);
  if (ok) ok = encode_box3(enc, &M.acc, bufs[4], nx, ny, nz, pitch, k3W, k3H);
  if (ok) e = cudaMemcpy(dm, &M, sizeof(Maps3d2), cudaMemcpyHostToDevice);
  if (!ok || e != cudaSuccess) {
    for (float* b : bufs) if (b) cudaFree(b);
    if (dm) cudaFree(dm);
    return !ok ? fail(g, WHV_ERR_CUDA, "cuTensorMapEncodeTiled failed (two-step 3-D buffers)")
               : cuda_fail(g, e, "two-step 3-D buffers");
  }
  for (int m = 0; m < 4; ++m) g->pw3[m] = bufs[m];
  g->pacc3 = bufs[4];
  g->maps3 = dm;
  g->pitch3 = pitch;
  return WHV_OK;
}

// Steps n = 1 .. nt-1 of a 3-D f = 0 FP32 wave solve (c = 1, second order) after the Taylor
// start (W^0 in buf[0], W^1 in buf[1], acc): one single step when their number is odd, then
// two-step passes alternating between the buffer pairs (0, 1) and (2, 3); the last launch writes
// the epilogue.
static whv_status two_step_3d(whv_grid g, const TimeGridH& tg, const double* v, double* out, int epi,
                              int* launches, void* const* bufs, void* accbuf, bool prepitched) {
  float* buf[4] = {(float*)bufs[0], (float*)bufs[1], (float*)bufs[2], (float*)bufs[3]};
  float* acc = (float*)accbuf;
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  StepCoef<float> cf = coef_of<float>(g, tg);
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  const Grid3d2 q = grid_3d2(g);
  const dim3 g2(q.blocks), b2(32, k3WR + 1, 1);   // 17 warp rows and the ring warp
  if (q.blocks > chan_cap(g, CH_STEP)) return fail(g, WHV_ERR_INVALID, "grid too large for the fused reduction");
  const LaunchShape ls = shape_of(g);
  float* wprev = buf[0];
  float* wcur = buf[1];
  int n = 1, nl = 0;
  if (!prepitched && (tg.nt - 1) % 2 == 1) {   // one single step first (the last one when nt = 2)
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
  if (n < tg.nt && !prepitched) {   // the chain of two-step passes runs on pitched copies of the state
    const int64_t N = g->N;
    k_to_pitched3<<<(int)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, g->stream>>>(
        wprev, wcur, acc, g->pw3[0], g->pw3[1], g->pacc3, nx, N, g->pitch3);
    WHV_CUDA(g, cudaGetLastError());
    ++nl;
  }
  int ip = 0;   // the pitched pair holding (W^{n-1}, W^n): buffers ip, ip + 1
  while (n < tg.nt) {   // W^n -> W^{n+2}
    cf.w1 = (float)tg.weight[n + 1];
    const float w2 = (float)tg.weight[n + 2];
    const bool last = n + 2 == tg.nt;
    const int oq = 2 - ip;
    float* op = g->pw3[oq];
    float* oc = g->pw3[oq + 1];
    const int kind = !last ? K_STEP : (epi == 0 ? K_LAST_OUT : K_LAST_AV);
    auto kern = kind == K_STEP ? k_step3d2<K_STEP> : (kind == K_LAST_OUT ? k_step3d2<K_LAST_OUT> : k_step3d2<K_LAST_AV>);
    // programmatic dependent launch: the pass's CTAs may be scheduled as the previous kernel's
    // exit; they wait (griddepcontrol.wait) for its completion before touching global memory
    cudaLaunchConfig_t lc = {};
    lc.gridDim = g2;
    lc.blockDim = b2;
    lc.dynamicSmemBytes = k3Smem;
    lc.stream = g->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    const double* vk = kind == K_LAST_AV ? v : nullptr;
    const double* mwk = kind == K_LAST_AV ? g->mw : nullptr;
    double* outk = kind == K_STEP ? nullptr : out;
    WHV_CUDA(g, cudaLaunchKernelEx(&lc, kern, (const Maps3d2*)g->maps3, ip, ip + 1, op, oc, g->pacc3, vk, mwk, outk,
                                   nx, ny, nz, g->pitch3, q.cx, q.ncol, q.slab, q.units, cf, w2, part, cnt,
                                   g->scal + S_PQ, g->scal + S_FLAG));
    ++nl;
    ip = oq;
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
  // the 3-D two-step chain (two steps per launch when set or chosen by the autotuner, planes of
  // < 2^31 nodes) runs on padded rows; with an even number of steps after the first one, the
  // first step writes them directly
  bool two_step = false, prepitched = false;
  if constexpr (DIM == 3 && ORDER == 2 && !VARC && !FORCE && sizeof(T) == 4) {
    two_step = g->kblock >= 2 && g->pw3[0] && (int64_t)g->n[0] * g->n[1] < (int64_t(1) << 31);
    prepitched = two_step && (tg.nt - 1) % 2 == 0 && tg.nt > 1;
    if (prepitched) {
      b0 = (T*)g->pw3[0];
      b1 = (T*)g->pw3[1];
      acc = (T*)g->pacc3;
    }
  }
  const int wpitch = prepitched ? g->pitch3 : nx;
  if (v)
    k_first<T, DIM, ORDER, VARC, FORCE, false><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf,
                                                                                  wpitch);
  else
    k_first<T, DIM, ORDER, VARC, FORCE, true><<<fgrid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf,
                                                                                 wpitch);
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
  if (two_step) {
    int nl = 0;
    whv_status s = two_step_3d(g, tg, v, out, epi, &nl, bufs, accbuf, prepitched);
    *nlaunch += nl;
    return s;
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
  if (k >= 2 && g->dim == 3 && g->order == 2 && !g->c2 && !g->cons && g->precision == WHV_FP32_STEP) {
    const whv_status s = ensure_pitched3(g);   // the two-step kernel's buffers, outside any capture
    if (s != WHV_OK) return s;
  }
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
  if (g->dim == 3 && g->order == 2 && !g->c2 && g->precision == WHV_FP32_STEP && ensure_pitched3(g) == WHV_OK)
    cands.push_back(2);
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
