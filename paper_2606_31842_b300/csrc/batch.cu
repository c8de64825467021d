// Batched solves: many independent problems -- right-hand sides, frequencies and grids of uneven
// size -- advanced together.
//
// A batched wave solve (one role, e.g. q_p = A p_p, for every active problem) is ONE persistent
// cooperative kernel launch:
//  - 2-D grids: k_batch_block2d sweeps k leapfrog steps at a time.  A sweep processes the tiles of
//    every problem that still has steps left; each tile stages a 64 x 64 region (its (64-2kr)^2
//    nodes plus a halo of width kr, r the stencil radius) and advances it k steps in registers
//    and shared memory; then all CTAs meet at a grid barrier.  Global traffic is 3 reads and 3
//    writes per node per k steps (plus the halo) instead of 5 accesses per step.
//  - 2-D, second order, c = 1 (the default path of the batched squares): wavefront kernels in
//    which ONE warp advances a strip of columns several time levels in a single pass down the
//    rows, with the levels' rows in register rings: k_batch_front for the FP32 A p of the CG loop
//    (k = 8, inputs by TMA), k_batch_front2 for the double-float residual roles (4 levels) and the
//    forced FP32 b role (8 levels).  A strip waits only for its own problem's previous sweep
//    (per-problem completion counters) instead of a grid barrier.
//  - 3-D grids: k_batch_wave sweeps one step at a time (tiles of 32 x 8 nodes per z plane).
// Problems are sorted by their number of sweeps, so the active ones are a prefix of the list;
// stopped problems are skipped a whole problem at a time.  The barrier spins with an iteration
// limit: a CTA that gives up raises an error flag and every CTA returns.
//
// The batched CG loop is one CUDA graph: a conditional WHILE node whose body is the batched wave
// solve (q_p = A p_p with per-tile partial sums of p^T M q), a finishing kernel (p^T M q per
// problem, fixed order), each problem's fused CG update and direction update (which return at
// once for stopped problems), a per-problem convergence test and a one-thread kernel that keeps
// the loop running while any problem is active.
//
// Without FP64 residual correction, DEVD (Algorithm 2) deflates each forcing first and inflates
// each solution after the loop.  With it (WHV_REFINE_FP64), the residual r = b - A u of the full
// system is formed by FP64 (or double-float) batched wave solves, its deflated components are
// solved modally and the rest by the batched CG loop in the grids' stepping precision, until every
// problem's FP64 residual meets its tolerance.  The residual is one forced wave solve from u,
// r = Pi_h(u; f) - u (= b - A u, since Pi_h(u; f) = S_h u + b), so b itself is only needed as the
// first pass's right-hand side and for |b| in the stopping test: it is formed by one forced wave
// solve in the stepping precision (its rounding, ~1e-5 relative in FP32, is far inside the first
// pass's inner tolerance and moves the stopping threshold by as little).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <type_traits>
#include <utility>
#include <vector>

#include <cuda.h>   // CUtensorMap and its encoding enums (the encoder is fetched through the runtime)

#include "df64.cuh"
#include "stencil_ops.cuh"
#include "quad2d.cuh"
#include "tma.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

constexpr int kBatchMaxProblems = 1024;

// Work item to continue from so that the CTA's next item (this one + gridDim.x) is the first at
// or after `end`: skips the rest of a stopped problem's tiles.
__device__ __forceinline__ int64_t skip_to(int64_t item, int64_t end) {
  const int64_t G = gridDim.x;
  return item + ((end - item + G - 1) / G - 1) * G;
}

// ------------------------------------------------------------------ 3-D: one step per sweep
template <typename T>
struct BProb {
  T* w0;                 // stepping buffers: W^0, W^1 ... ping-pong
  T* w1;
  T* acc;                // filter accumulator
  const double* v;       // initial state (nullptr: 0)
  const double* f;       // forcing (nullptr: 0)
  double* out;           // epi 0: Pi_h v;  epi 1: v - Pi_h v
  const T* c2;           // squared speed (nullptr: 1)
  const double* mw;      // M weights (nullptr: 1)
  double* partials;      // epi 1: per-tile partial sums of <v, out>_M
  const double* halt;    // problem stopped when *halt != 0 (nullptr: never)
  int64_t tile0;         // first work item of this problem (exclusive prefix over problems)
  int nx, ny, nz, nt, tx, ty, ntiles, epi, wofs;
  StepCoef<T> cf;
};

template <typename T, int DIM, int ORDER, bool VARC>
__global__ void __launch_bounds__(256) k_batch_wave(const BProb<T>* __restrict__ P, const int* __restrict__ nact,
                                                    int S, const T* __restrict__ wtab, const T* __restrict__ ptab,
                                                    unsigned* bar_count, unsigned* bar_gen, int* err) {
  // tile offsets of all problems (and one past the last) in shared memory: each block walks its
  // work items in increasing order, so the problem index only moves forward
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  __shared__ BProb<T> sB;
  const int np = nact[0];
  for (int p = threadIdx.x + blockDim.x * threadIdx.y; p <= np; p += blockDim.x * blockDim.y)
    s_tile0[p] = p < np ? P[p].tile0 : P[np - 1].tile0 + P[np - 1].ntiles;
  __syncthreads();
  const int lx = threadIdx.x, ly = threadIdx.y;
  for (int s = 0; s < S; ++s) {
    const int A = nact[s];
    const int64_t total = s_tile0[A];
    int cur = -1;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
      int p = cur < 0 ? 0 : cur;
      while (s_tile0[p + 1] <= item) ++p;
      if (p != cur) {   // stage the problem's descriptor in shared memory
        __syncthreads();
        if (lx == 0 && ly == 0) sB = P[p];
        __syncthreads();
        cur = p;
      }
      const BProb<T>& B = sB;
      if (B.halt && *B.halt != 0.0) {   // uniform per block: skip the problem
        item = skip_to(item, s_tile0[p + 1]);
        continue;
      }
      const int t = (int)(item - B.tile0);
      const int tx = t % B.tx, ty = (t / B.tx) % B.ty, tz = t / (B.tx * B.ty);
      const int x = tx * 32 + lx, y = ty * 8 + ly, z = tz;
      const bool in = x < B.nx && y < B.ny;
      const int64_t idx = x + (int64_t)B.nx * (y + (int64_t)B.ny * z);
      const T* wtb = wtab + B.wofs;
      double part = 0.0;
      const bool last = (s == B.nt - 1);
      if (s == 0) {
        if (in) {
          const T W0 = B.v ? (T)B.v[idx] : T(0);
          T L = B.v ? lap<DIM, ORDER, T>(B.v, idx, x, y, z, B.nx, B.ny, B.nz, B.cf, W0) : T(0);
          if (VARC) L *= B.c2[idx];
          if (B.f) L -= (T)B.f[idx];
          const T W1 = fma(T(0.5) * B.cf.dt2, L, W0);
          B.w0[idx] = W0;
          B.w1[idx] = W1;
          B.acc[idx] = fma(wtb[1], W1, wtb[0] * W0);
        }
      } else {
        T* wcur = (s & 1) ? B.w1 : B.w0;
        T* wprv = (s & 1) ? B.w0 : B.w1;
        if (in) {
          // wcur was written by other CTAs at the previous step of this launch: coherent loads
          const T c = __ldcg(wcur + idx);
          T L = lap_cg<DIM, ORDER, T>(wcur, idx, x, y, z, B.nx, B.ny, B.nz, B.cf, c);
          if (VARC) L *= B.c2[idx];
          if (B.f) L = fma(-(T)B.f[idx], ptab[B.wofs + s], L);
          const T wn = fma(B.cf.dt2, L, fma(T(2), c, -__ldcg(wprv + idx)));
          const T a = fma(wtb[s + 1], wn, __ldcg(B.acc + idx));
          if (!last) {
            wprv[idx] = wn;
            B.acc[idx] = a;
          } else if (B.epi == 0) {
            B.out[idx] = (double)a;
          } else {
            const double vi = B.v[idx];
            const double o = vi - (double)a;
            B.out[idx] = o;
            part = (B.mw ? vi * B.mw[idx] : vi) * o;
          }
        }
      }
      if (last && B.epi == 1) {
        part = block_sum(part);
        if (lx == 0 && ly == 0) B.partials[t] = part;
      }
    }
    if (!grid_barrier(bar_count, bar_gen, err, gridDim.x)) return;
  }
}

// ------------------------------------------------------------------ 2-D: k steps per sweep
constexpr int kBReg = 64;                  // staged region edge
constexpr int kBThreads = 1024;            // 32 warps
constexpr int kBPitch = kBThreads / 64;    // rows between a thread's cells (16)
constexpr int kBRows = kBReg / kBPitch;    // cells per thread (4)

template <typename T>
struct BTile {
  T* w[4];               // two (W^{n-1}, W^n) pairs: sweep j writes pair j & 1
  T* acc;                // filter accumulator
  const double* v;       // W^0 (nullptr: 0)
  const double* f;       // forcing (FORCED kernels)
  double* out;           // epi 0: Pi_h(v; f);  epi 1: v - Pi_h v
  const T* c2;           // squared speed (VARC kernels)
  const double* mw;      // M weights (nullptr: 1)
  double* partials;      // epi 1: per-tile partial sums of <v, out>_M
  const double* halt;    // problem stopped when *halt != 0 (nullptr: never)
  int64_t tile0;
  int nx, ny, nt, tiles_x, ntiles, epi, wofs;
  T ih2x, ih2y, dt2;
  T ax, ay, b;           // 2nd order, c = 1: W^{n+1} = ax s_x + ay s_y + b W^n - W^{n-1}
};

// second difference at global index gi (of n) read from shared memory at local offset l, stride
// s, with the Dirichlet / odd-reflection closure
template <int ORDER, typename T>
__device__ __forceinline__ T d2b(const T* __restrict__ a, int l, int gi, int n, int s, T c) {
  const T m1 = gi > 0 ? a[l - s] : T(0);
  const T p1 = gi < n - 1 ? a[l + s] : T(0);
  if (ORDER == 2) return fma(T(-2), c, m1 + p1);
  const T m2 = gi > 1 ? a[l - 2 * s] : (gi == 1 ? T(0) : -c);
  const T p2 = gi < n - 2 ? a[l + 2 * s] : (gi == n - 2 ? T(0) : -c);
  return fma(T(-30), c, fma(T(16), m1 + p1, -(m2 + p2)));
}

// Sweep j of problem p covers steps n0 = j K .. n0 + kk - 1 (W^{n0} -> W^{n0+kk}), kk = min(K,
// nt - n0).  Sweep 0 starts from W^0 = v with the Taylor step; the last sweep writes the FP64
// epilogue instead of the state.  Thread (warp w, lane) owns column 32 (w & 1) + lane and rows
// (w >> 1) + 16 r, r < 4, of the staged region for the whole sweep.
// FP32, 5-point, c = 1, f = 0: the sub-steps run in the four-cells-per-thread mapping of quad2d.cuh
template <typename T, int ORDER, bool VARC, bool FORCED>
constexpr bool kBQuad = sizeof(T) == 4 && ORDER == 2 && !VARC && !FORCED;

template <typename T, int ORDER, bool VARC, bool FORCED>
__global__ void __launch_bounds__(kBThreads, 1) k_batch_block2d(const BTile<T>* __restrict__ P,
                                                                const int* __restrict__ nact, int J, int K,
                                                                const T* __restrict__ wtab,
                                                                const T* __restrict__ ptab, unsigned* bar_count,
                                                                unsigned* bar_gen, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const S0 = reinterpret_cast<T*>(smem_raw);
  T* const S1 = S0 + kBReg * kBReg;
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  __shared__ BTile<T> sB;
  __shared__ T sw[16];      // filter weights of the current sweep (four-cell kernels; k <= 16)
  constexpr int R = ORDER == 2 ? 1 : 2;
  const int np = nact[0];
  for (int p = threadIdx.x; p <= np; p += blockDim.x)
    s_tile0[p] = p < np ? P[p].tile0 : P[np - 1].tile0 + P[np - 1].ntiles;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 1) + lane;
  const int jb = warp >> 1;
  const int H = K * R, TW = kBReg - 2 * H;
  for (int j = 0; j < J; ++j) {
    const int A = nact[j];
    const int64_t total = s_tile0[A];
    int cur_p = -1;
    // four-cell kernels: the column data of this CTA's next item (same sweep, same problem),
    // loaded while the current item's sub-steps run
    T ncur[kBRows], nprv[kBRows], nacr[kBRows];
    int64_t pitem = -1;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
      int p = cur_p < 0 ? 0 : cur_p;
      while (s_tile0[p + 1] <= item) ++p;
      if (p != cur_p) {
        __syncthreads();
        if (threadIdx.x == 0) sB = P[p];
        __syncthreads();
        cur_p = p;
      }
      const BTile<T>& B = sB;
      if (B.halt && *B.halt != 0.0) {
        item = skip_to(item, s_tile0[p + 1]);
        continue;
      }
      const int t = (int)(item - B.tile0);
      const int x0 = (t % B.tiles_x) * TW - H, y0 = (t / B.tiles_x) * TW - H;
      const int gx = x0 + i;
      const int nx = B.nx, ny = B.ny;
      const bool colin = gx >= 0 && gx < nx;
      const int n0 = j * K;
      const int kk = min(K, B.nt - n0);
      const bool first = j == 0, last = n0 + kk == B.nt;
      const T* wtb = wtab + B.wofs;
      const T* ptb = ptab + B.wofs;
      const int qi = (j + 1) & 1, qo = j & 1;   // input pair (written by sweep j - 1), output pair
      T cur[kBRows], prv[kBRows], acr[kBRows];
      T cc[VARC ? kBRows : 1];
      T ff[FORCED ? kBRows : 1];
      const T w0 = first ? wtb[0] : T(0);
      if (kBQuad<T, ORDER, VARC, FORCED> && item == pitem) {
#pragma unroll
        for (int r = 0; r < kBRows; ++r) {
          cur[r] = ncur[r];
          prv[r] = nprv[r];
          acr[r] = nacr[r];
        }
      } else
#pragma unroll
      for (int r = 0; r < kBRows; ++r) {
        const int gy = y0 + jb + kBPitch * r;
        const bool in = colin && gy >= 0 && gy < ny;
        const int64_t gi = gx + (int64_t)nx * gy;
        if (first) {
          cur[r] = (in && B.v) ? (T)__ldg(B.v + gi) : T(0);
          prv[r] = T(0);
        } else {   // written by other CTAs in the previous sweep of this launch: coherent loads
          cur[r] = in ? __ldcg(B.w[2 * qi + 1] + gi) : T(0);
          prv[r] = in ? __ldcg(B.w[2 * qi] + gi) : T(0);
        }
        if (VARC) cc[r] = in ? __ldg(B.c2 + gi) : T(0);
        if (FORCED) ff[r] = (in && B.f) ? (T)__ldg(B.f + gi) : T(0);
        // the filter sum so far of the tile cells, loaded with the state (no read-modify-write
        // round trip at the end)
        const int jr = jb + kBPitch * r;
        const bool tile = in && i >= H && i < kBReg - H && jr >= H && jr < kBReg - H;
        acr[r] = (!first && tile) ? __ldcg(B.acc + gi) : w0 * cur[r];
      }
      if constexpr (kBQuad<T, ORDER, VARC, FORCED>) {
        T* const S2 = S1 + kBReg * kBReg;
#pragma unroll
        for (int r = 0; r < kBRows; ++r) {
          const int l = (jb + kBPitch * r) * kBReg + i;
          S0[l] = cur[r];
          S1[l] = prv[r];
          S2[l] = acr[r];
        }
        if (threadIdx.x < kk) sw[threadIdx.x] = wtb[n0 + 1 + threadIdx.x];
        __syncthreads();
        // issue the next item's loads now: its input pair and filter sums are not written in this
        // sweep (outputs go to the other pair, filter sums to this CTA's own tiles)
        pitem = -1;
        const int64_t nitem = item + gridDim.x;
        if (!first && nitem < s_tile0[p + 1]) {
          const int tn = (int)(nitem - B.tile0);
          const int px0 = (tn % B.tiles_x) * TW - H, py0 = (tn / B.tiles_x) * TW - H;
          const int pgx = px0 + i;
          const bool pcol = pgx >= 0 && pgx < nx;
#pragma unroll
          for (int r = 0; r < kBRows; ++r) {
            const int jr = jb + kBPitch * r;
            const int gy = py0 + jr;
            const bool in = pcol && gy >= 0 && gy < ny;
            const int64_t gi = pgx + (int64_t)nx * gy;
            ncur[r] = in ? __ldcg(B.w[2 * qi + 1] + gi) : T(0);
            nprv[r] = in ? __ldcg(B.w[2 * qi] + gi) : T(0);
            const bool tile = in && i >= H && i < kBReg - H && jr >= H && jr < kBReg - H;
            nacr[r] = tile ? __ldcg(B.acc + gi) : T(0);
          }
          pitem = nitem;
        }
        const QuadCoef q{B.ax, B.ay, B.b, B.ih2x, B.ih2y, 0.5f * B.dt2};
        const bool inside = x0 >= 0 && y0 >= 0 && x0 + kBReg <= nx && y0 + kBReg <= ny;
        const unsigned m = inside ? 0xfu : quad_mask(x0, y0, nx, ny);
        if (first) {
          if (inside) quad_sweep<false, true>(S0, S1, S2, kk, sw, q, m);
          else quad_sweep<true, true>(S0, S1, S2, kk, sw, q, m);
        } else {
          if (inside) quad_sweep<false, false>(S0, S1, S2, kk, sw, q, m);
          else quad_sweep<true, false>(S0, S1, S2, kk, sw, q, m);
        }
#pragma unroll
        for (int r = 0; r < kBRows; ++r) {
          const int l = (jb + kBPitch * r) * kBReg + i;
          cur[r] = S0[l];
          prv[r] = S1[l];
          acr[r] = S2[l];
        }
      } else {
#pragma unroll
      for (int r = 0; r < kBRows; ++r) S0[(jb + kBPitch * r) * kBReg + i] = cur[r];
      __syncthreads();
      T* Ain = S0;
      T* Bout = S1;
      for (int s = 1; s <= kk; ++s) {
        const int n = n0 + s - 1;   // W^n -> W^{n+1}
        const int lo = s * R, hi = kBReg - s * R;
        const bool colact = colin && i >= lo && i < hi;
        const T ws = wtb[n + 1];
        // forcing term dt^2 f cos(omega_hat t^n) (half of it in the Taylor step)
        const T fph = FORCED ? (n > 0 ? B.dt2 : T(0.5) * B.dt2) * ptb[n] : T(0);
#pragma unroll
        for (int r = 0; r < kBRows; ++r) {
          const int jr = jb + kBPitch * r;
          const int gy = y0 + jr;
          if (colact && jr >= lo && jr < hi && gy >= 0 && gy < ny) {
            const int l = jr * kBReg + i;
            const T c = cur[r];
            T wn;
            if (ORDER == 2 && !VARC && n > 0) {
              T u = fma(B.b, c, -prv[r]);
              u = fma(B.ax, (gx > 0 ? Ain[l - 1] : T(0)) + (gx < nx - 1 ? Ain[l + 1] : T(0)), u);
              wn = fma(B.ay, (gy > 0 ? Ain[l - kBReg] : T(0)) + (gy < ny - 1 ? Ain[l + kBReg] : T(0)), u);
            } else {
              T L = d2b<ORDER>(Ain, l, gx, nx, 1, c) * B.ih2x;
              L = fma(d2b<ORDER>(Ain, l, gy, ny, kBReg, c), B.ih2y, L);
              if (VARC) L *= cc[r];
              wn = n > 0 ? fma(B.dt2, L, fma(T(2), c, -prv[r]))
                         : fma(T(0.5) * B.dt2, L, c);   // Taylor start: W^1 = W^0 + dt^2/2 L W^0
            }
            if (FORCED) wn = fma(-fph, ff[r], wn);
            prv[r] = c;
            cur[r] = wn;
            Bout[l] = wn;
            acr[r] = fma(ws, wn, acr[r]);
          }
        }
        __syncthreads();
        T* tmp = Ain;
        Ain = Bout;
        Bout = tmp;
      }
      }
      double part = 0.0;
      const bool coltile = colin && i >= H && i < kBReg - H;
#pragma unroll
      for (int r = 0; r < kBRows; ++r) {
        const int jr = jb + kBPitch * r;
        const int gy = y0 + jr;
        if (!(coltile && jr >= H && jr < kBReg - H && gy >= 0 && gy < ny)) continue;
        const int64_t gi = gx + (int64_t)nx * gy;
        const T a = acr[r];
        if (!last) {
          B.w[2 * qo + 1][gi] = cur[r];
          B.w[2 * qo][gi] = prv[r];
          B.acc[gi] = a;
        } else if (B.epi == 0) {
          B.out[gi] = (double)a;
        } else {
          const double vi = __ldg(B.v + gi);
          const double o = vi - (double)a;
          B.out[gi] = o;
          part = fma(B.mw ? vi * __ldg(B.mw + gi) : vi, o, part);
        }
      }
      if (last && B.epi == 1) {
        part = block_sum(part);
        if (threadIdx.x == 0) B.partials[t] = part;
      }
    }
    if (!grid_barrier(bar_count, bar_gen, err, gridDim.x)) return;
  }
}

// Double-float roles (2-D, second order, c = 1): the b and residual wave solves of the FP64
// residual correction in pairs of FP32 numbers (df64.cuh) instead of FP64 arithmetic, which runs
// at 1/64 of the FP32 rate on this GPU.  Same work items, sweeps and grid barriers as
// k_batch_block2d; each CTA stages a 64 x 64 region of 8-byte hi/lo pairs, thread (warp, lane)
// owns column 32 (w & 1) + lane and rows (w >> 1) + 16 r, and sub-step s advances the window
// [s, 64 - s)^2 (with ~150 FP32 instructions per update the shrinking window pays).  The updates
// are the double-float operations of the single-grid kernels k_first_df / k_step_df:
//   Taylor start  W^1 = W^0 + (dt^2 / 2) (sum_m ih2_m ((W_- + W_+) - 2 W^0) - f)
//   step          W^{n+1} = ((b W^n - W^{n-1}) + a_x (W_l + W_r)) + a_y (W_d + W_u) - fph_n f
//   filter        acc = w_0 W^0 + w_1 W^1, then acc + w_{n+1} W^{n+1}
// with fph_n = dt^2 cos(omega_hat t^n) from the role's table.
template <bool FORCED>
__global__ void __launch_bounds__(kBThreads, 1) k_batch_block2d_df(const BTile<dfl>* __restrict__ P,
                                                                   const int* __restrict__ nact, int J, int K,
                                                                   const dfl* __restrict__ wtab,
                                                                   const dfl* __restrict__ ptab, unsigned* bar_count,
                                                                   unsigned* bar_gen, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dfl* const S0 = reinterpret_cast<dfl*>(smem_raw);
  dfl* const S1 = S0 + kBReg * kBReg;
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  __shared__ BTile<dfl> sB;
  const int np = nact[0];
  for (int p = threadIdx.x; p <= np; p += blockDim.x)
    s_tile0[p] = p < np ? P[p].tile0 : P[np - 1].tile0 + P[np - 1].ntiles;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 1) + lane;
  const int jb = warp >> 1;
  const int H = K, TW = kBReg - 2 * H;
  for (int j = 0; j < J; ++j) {
    const int A = nact[j];
    const int64_t total = s_tile0[A];
    int cur_p = -1;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
      int p = cur_p < 0 ? 0 : cur_p;
      while (s_tile0[p + 1] <= item) ++p;
      if (p != cur_p) {
        __syncthreads();
        if (threadIdx.x == 0) sB = P[p];
        __syncthreads();
        cur_p = p;
      }
      const BTile<dfl>& B = sB;
      if (B.halt && *B.halt != 0.0) {
        item = skip_to(item, s_tile0[p + 1]);
        continue;
      }
      const int t = (int)(item - B.tile0);
      const int x0 = (t % B.tiles_x) * TW - H, y0 = (t / B.tiles_x) * TW - H;
      const int gx = x0 + i;
      const int nx = B.nx, ny = B.ny;
      const bool colin = gx >= 0 && gx < nx;
      const int n0 = j * K;
      const int kk = min(K, B.nt - n0);
      const bool first = j == 0, last = n0 + kk == B.nt;
      const dfl* wtb = wtab + B.wofs;
      const dfl* ptb = ptab + B.wofs;
      const int qi = (j + 1) & 1, qo = j & 1;
      dfl cur[kBRows], prv[kBRows], acr[kBRows];
      dfl ff[FORCED ? kBRows : 1];
#pragma unroll
      for (int r = 0; r < kBRows; ++r) {
        const int jr = jb + kBPitch * r;
        const int gy = y0 + jr;
        const bool in = colin && gy >= 0 && gy < ny;
        const int64_t gi = gx + (int64_t)nx * gy;
        const bool tile = in && i >= H && i < kBReg - H && jr >= H && jr < kBReg - H;
        if (first) {
          cur[r] = (in && B.v) ? df_from(__ldg(B.v + gi)) : df_zero();
          prv[r] = df_zero();
          acr[r] = df_mul(wtb[0], cur[r]);
        } else {   // written by other CTAs in the previous sweep: coherent loads
          const float2 c2v = in ? __ldcg(reinterpret_cast<const float2*>(B.w[2 * qi + 1] + gi)) : make_float2(0.f, 0.f);
          const float2 p2v = in ? __ldcg(reinterpret_cast<const float2*>(B.w[2 * qi] + gi)) : make_float2(0.f, 0.f);
          const float2 a2v = tile ? __ldcg(reinterpret_cast<const float2*>(B.acc + gi)) : make_float2(0.f, 0.f);
          cur[r] = dfl{c2v.x, c2v.y};
          prv[r] = dfl{p2v.x, p2v.y};
          acr[r] = dfl{a2v.x, a2v.y};
        }
        if (FORCED) ff[r] = (in && B.f) ? df_from(__ldg(B.f + gi)) : df_zero();
      }
      // both stages hold 0 at the nodes outside the domain (the Dirichlet values), so that the
      // neighbour reads below need no tests; the other nodes of S1 are written by the first
      // sub-step before any read
#pragma unroll
      for (int r = 0; r < kBRows; ++r) {
        const int jr = jb + kBPitch * r;
        const int gy = y0 + jr;
        S0[jr * kBReg + i] = cur[r];
        if (!(colin && gy >= 0 && gy < ny)) S1[jr * kBReg + i] = df_zero();
      }
      __syncthreads();
      const dfl* Ain = S0;
      dfl* Bout = S1;
      const dfl coef[2] = {B.ax, B.ay};
      for (int s = 1; s <= kk; ++s) {
        const int n = n0 + s - 1;   // W^n -> W^{n+1}
        const int lo = s, hi = kBReg - s;
        const bool colact = colin && i >= lo && i < hi;
        const dfl ws = wtb[n + 1];
        const dfl fph = FORCED ? ptb[n] : df_zero();
#pragma unroll
        for (int r = 0; r < kBRows; ++r) {
          const int jr = jb + kBPitch * r;
          const int gy = y0 + jr;
          if (colact && jr >= lo && jr < hi && gy >= 0 && gy < ny) {
            const int l = jr * kBReg + i;
            const dfl c = cur[r];
            dfl wn;
            if (n == 0) {   // Taylor start
              const dfl sx = df_add(Ain[l - 1], Ain[l + 1]);
              const dfl sy = df_add(Ain[l - kBReg], Ain[l + kBReg]);
              const dfl c2x = {2.0f * c.hi, 2.0f * c.lo};
              dfl L = df_add(df_zero(), df_mul(B.ih2x, df_sub(sx, c2x)));
              L = df_add(L, df_mul(B.ih2y, df_sub(sy, c2x)));
              if (FORCED) L = df_sub(L, ff[r]);
              wn = df_add(c, df_mul(dfl{0.5f * B.dt2.hi, 0.5f * B.dt2.lo}, L));
            } else {
              const dfs sm[2] = {df_pair_sum(Ain[l - 1], Ain[l + 1]), df_pair_sum(Ain[l - kBReg], Ain[l + kBReg])};
              wn = df_leapfrog<2, FORCED>(B.b, c, prv[r], coef, sm, fph, FORCED ? ff[r] : df_zero());
            }
            prv[r] = c;
            cur[r] = wn;
            Bout[l] = wn;
            acr[r] = df_fma_acc(acr[r], ws, wn);
          }
        }
        __syncthreads();
        dfl* tmp = const_cast<dfl*>(Ain);
        Ain = Bout;
        Bout = tmp;
      }
      double part = 0.0;
      const bool coltile = colin && i >= H && i < kBReg - H;
#pragma unroll
      for (int r = 0; r < kBRows; ++r) {
        const int jr = jb + kBPitch * r;
        const int gy = y0 + jr;
        if (!(coltile && jr >= H && jr < kBReg - H && gy >= 0 && gy < ny)) continue;
        const int64_t gi = gx + (int64_t)nx * gy;
        if (!last) {
          B.w[2 * qo + 1][gi] = cur[r];
          B.w[2 * qo][gi] = prv[r];
          B.acc[gi] = acr[r];
        } else if (B.epi == 0) {
          B.out[gi] = df_to(acr[r]);
        } else {
          const double vi = __ldg(B.v + gi);
          const double o = vi - df_to(acr[r]);
          B.out[gi] = o;
          part = fma(B.mw ? vi * __ldg(B.mw + gi) : vi, o, part);
        }
      }
      if (last && B.epi == 1) {
        part = block_sum(part);
        if (threadIdx.x == 0) B.partials[t] = part;
      }
    }
    if (!grid_barrier(bar_count, bar_gen, err, gridDim.x)) return;
  }
}

// ------------------------------------------------------------------ 2-D, FP32, TMA-fed
// The f = 0 FP32 wave solve of the 5-point stencil with c = 1 -- every A p of the batched CG
// loop -- with the state in row-padded buffers (pitch a multiple of 4 floats), so that the copy
// engine can move it: for every work item after the first sweep, one thread issues three tiled
// TMA copies (the 64 x 64 region of W^n and of W^{n-1} with a k-wide halo, out-of-domain cells
// read as 0, and the (64 - 2k)^2 tile of filter sums) into one of two shared-memory stages while
// the CTA steps the previous item in the other stage; the sub-steps run in the four-cell mapping
// of quad2d.cuh on the staged buffers; the tile's new state goes from registers straight to
// global memory as 16-byte stores.  The first sweep reads v (FP64) directly, the last writes the
// FP64 output (and p^T M q partials).  k is a multiple of 4 (the region's x origin tile*TW - k
// must be 16-byte aligned for the copy engine).  Same operations in the same order as
// k_batch_block2d's four-cell path.
struct BTileT {
  float* w[4];           // pitched (W^{n-1}, W^n) pairs: sweep j writes pair j & 1
  float* acc;            // pitched filter sums
  const double* v;       // W^0 (nullptr: 0)
  double* out;           // epi 0: Pi_h v;  epi 1: v - Pi_h v
  const double* mw;      // M weights (nullptr: 1)
  double* partials;      // epi 1: per-tile partial sums of <v, out>_M
  const double* halt;    // problem stopped when *halt != 0 (nullptr: never)
  int64_t tile0;
  int nx, ny, nt, tiles_x, ntiles, epi, wofs, pitch;
  float ax, ay, b, ih2x, ih2y, dt2;
  int64_t tile0b;        // wavefront kernel, work items of 2 kFS rows: first item, count
  int ntilesb;
};

struct BMaps {           // tensor maps of one problem's pitched buffers
  CUtensorMap w[4];      // 64 x 64 boxes
  CUtensorMap acc;       // (64 - 2k)^2 boxes
};

constexpr uint32_t kMbarPolls = 1u << 22;   // bound on the polls of one stage's mbarrier

template <int K>
struct TmaLayout {
  static constexpr int TW = kBReg - 2 * K;
  static constexpr int kRegion = kBReg * kBReg * 4;             // bytes of one 64 x 64 FP32 box
  static constexpr int kAcc = TW * TW * 4;
  static constexpr int kStage = ((2 * kRegion + kAcc) + 1023) / 1024 * 1024;
  static constexpr int kSmem = 2 * kStage + 1024;               // + alignment slack
  static constexpr uint32_t kTx = 2 * kRegion + kAcc;          // bytes one item's copies deliver
};

// next work item of this CTA at or after `item` (stepping by gridDim.x) whose problem is running;
// p is advanced to that item's problem
__device__ __forceinline__ int64_t tma_live_item(int64_t item, int& p, int64_t total, const int64_t* s_tile0,
                                                 const BTileT* __restrict__ P) {
  while (item < total) {
    while (s_tile0[p + 1] <= item) ++p;
    const double* h = P[p].halt;
    if (!h || *h == 0.0) return item;
    item = skip_to(item, s_tile0[p + 1]) + gridDim.x;
  }
  return item;
}

template <int K>
__device__ __forceinline__ void tma_issue(const BMaps* __restrict__ M, const BTileT* __restrict__ P, int p,
                                          int64_t item, int qi, unsigned char* stage, uint64_t* bar) {
  using L = TmaLayout<K>;
  const int t = (int)(item - P[p].tile0);
  const int tx = t % P[p].tiles_x, ty = t / P[p].tiles_x;
  mbar_arrive_expect_tx(bar, L::kTx);
  tma_load_2d(stage, &M[p].w[2 * qi + 1], tx * L::TW - K, ty * L::TW - K, bar);             // W^n
  tma_load_2d(stage + L::kRegion, &M[p].w[2 * qi], tx * L::TW - K, ty * L::TW - K, bar);    // W^{n-1}
  tma_load_2d(stage + 2 * L::kRegion, &M[p].acc, tx * L::TW, ty * L::TW, bar);             // filter sums
}

// R rows of four cells per thread: R = 1, 1024 threads (quad2d.cuh quad_steps), one CTA per SM;
// R = 2, 512 threads (duo_steps), two CTAs per SM, each with its own two stages.
template <int K, int R>
__global__ void __launch_bounds__(kBThreads / R, R) k_batch_tma(const BTileT* __restrict__ P,
                                                                 const BMaps* __restrict__ M,
                                                                 const int* __restrict__ nact, int J,
                                                                 const float* __restrict__ wtab,
                                                                 unsigned* bar_count, unsigned* bar_gen, int* err) {
  using L = TmaLayout<K>;
  constexpr int TW = L::TW;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* const base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  __shared__ BTileT sB;
  __shared__ float sw[16];
  __shared__ __align__(8) uint64_t s_bar[2];
  // the CTA's next work item and its problem, written by thread 0 into the slot of the stage it
  // will use and read by all after the barrier that ends the current item (two slots: a slot is
  // rewritten only after every thread has passed the barrier that follows its last read)
  __shared__ int64_t s_item[2];
  __shared__ int s_p[2];
  const int np = nact[0];
  for (int p = threadIdx.x; p <= np; p += blockDim.x)
    s_tile0[p] = p < np ? P[p].tile0 : P[np - 1].tile0 + P[np - 1].ntiles;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  const int row = (threadIdx.x >> 4) * R, col = (threadIdx.x & 15) * 4;
  const int off = row * kBReg + col;
  // K and row are even: the R = 2 rows of a thread are both in the tile or both in the halo
  const bool trow = row >= K && row < kBReg - K, tcol = col >= K && col < kBReg - K;
  const int aoff = (row - K) * TW + (col - K);   // filter-sum box offset (tile cells only)
  for (int j = 0; j < J; ++j) {
    const int A = nact[j];
    const int64_t total = s_tile0[A];
    const int qi = (j + 1) & 1, qo = j & 1;   // input pair (written by sweep j - 1), output pair
    int stage = 0;
    if (threadIdx.x == 0) {
      if (j > 0) fence_proxy_async_global();   // the previous sweep's stores (all CTAs) before the copies
      int p = 0;
      const int64_t it = tma_live_item(blockIdx.x, p, total, s_tile0, P);
      s_item[0] = it;
      s_p[0] = p;
      if (j > 0 && it < total) tma_issue<K>(M, P, p, it, qi, base, &s_bar[0]);
    }
    __syncthreads();
    int64_t item = s_item[0];
    int p = s_p[0], cur_p = -1;
    while (item < total) {
      if (p != cur_p) {
        if (threadIdx.x == 0) sB = P[p];
        __syncthreads();
        cur_p = p;
      }
      const BTileT& B = sB;
      unsigned char* const st = base + stage * L::kStage;
      float* const SA = reinterpret_cast<float*>(st);
      float* const SB = reinterpret_cast<float*>(st + L::kRegion);
      const float* const SC = reinterpret_cast<const float*>(st + 2 * L::kRegion);
      // the next item's copies into the other stage (free: its item ended with a barrier)
      if (threadIdx.x == 0) {
        int pn = p;
        const int64_t nit = tma_live_item(item + gridDim.x, pn, total, s_tile0, P);
        s_item[stage ^ 1] = nit;
        s_p[stage ^ 1] = pn;
        if (j > 0 && nit < total) tma_issue<K>(M, P, pn, nit, qi, base + (stage ^ 1) * L::kStage, &s_bar[stage ^ 1]);
      }
      const int t = (int)(item - B.tile0);
      const int x0 = (t % B.tiles_x) * TW - K, y0 = (t / B.tiles_x) * TW - K;
      const int nx = B.nx, ny = B.ny;
      const int n0 = j * K;
      const int kk = min(K, B.nt - n0);
      const bool first = j == 0, last = n0 + kk == B.nt;
      const float* wtb = wtab + B.wofs;
      if (threadIdx.x < kk) sw[threadIdx.x] = wtb[n0 + 1 + threadIdx.x];
      const int gx = x0 + col;
      float4 c[R], w[R], a[R];
      if (first) {   // W^0 = v (FP64, unpadded rows), W^{-1} unused (Taylor start), sums w_0 W^0
        const float w0 = wtb[0];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          const int gy = y0 + row + rr;
          float cv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const bool in = gy >= 0 && gy < ny && gx + e >= 0 && gx + e < nx && B.v;
            cv[e] = in ? (float)__ldg(B.v + (gx + e) + (int64_t)nx * gy) : 0.0f;
          }
          c[rr] = make_float4(cv[0], cv[1], cv[2], cv[3]);
          w[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
          a[rr] = make_float4(w0 * c[rr].x, w0 * c[rr].y, w0 * c[rr].z, w0 * c[rr].w);
          q_sts(SA, off + rr * kBReg, c[rr]);
        }
      } else {
        const bool ok = mbar_wait(&s_bar[stage], parity[stage], kMbarPolls);
        if (__syncthreads_or(!ok)) {   // the copies did not arrive: give up (bounded)
          if (threadIdx.x == 0) {
            atomicExch(err, 1);
            mbar_wait(&s_bar[stage ^ 1], parity[stage ^ 1], kMbarPolls);   // drain what may be in flight
          }
          __syncthreads();
          return;
        }
        parity[stage] ^= 1u;
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          c[rr] = q_lds(SA, off + rr * kBReg);
          w[rr] = q_lds(SB, off + rr * kBReg);
          a[rr] = (trow && tcol) ? *reinterpret_cast<const float4*>(SC + aoff + rr * TW)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      const QuadCoef q{B.ax, B.ay, B.b, B.ih2x, B.ih2y, 0.5f * B.dt2};
      const bool inside = x0 >= 0 && y0 >= 0 && x0 + kBReg <= nx && y0 + kBReg <= ny;
      if constexpr (R == 1) {
        const unsigned m = inside ? 0xfu : quad_mask(x0, y0, nx, ny);
        if (first) {
          if (inside) quad_steps<false, true>(c[0], w[0], a[0], SA, SB, kk, sw, q, m);
          else quad_steps<true, true>(c[0], w[0], a[0], SA, SB, kk, sw, q, m);
        } else {
          if (inside) quad_steps<false, false>(c[0], w[0], a[0], SA, SB, kk, sw, q, m);
          else quad_steps<true, false>(c[0], w[0], a[0], SA, SB, kk, sw, q, m);
        }
      } else {
        const unsigned m = inside ? 0xffu : duo_mask(x0, y0, nx, ny);
        if (first) {
          if (inside) duo_steps<false, true>(c[0], c[1], w[0], w[1], a[0], a[1], SA, SB, kk, sw, q, m);
          else duo_steps<true, true>(c[0], c[1], w[0], w[1], a[0], a[1], SA, SB, kk, sw, q, m);
        } else {
          if (inside) duo_steps<false, false>(c[0], c[1], w[0], w[1], a[0], a[1], SA, SB, kk, sw, q, m);
          else duo_steps<true, false>(c[0], c[1], w[0], w[1], a[0], a[1], SA, SB, kk, sw, q, m);
        }
      }
      double part = 0.0;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int gy = y0 + row + rr;
        if (!(trow && tcol && gy < ny && gx < nx)) continue;
        if (!last) {   // 16-byte stores of the tile's new state (padding columns take zeros)
          const int64_t gi = gx + (int64_t)B.pitch * gy;
          *reinterpret_cast<float4*>(B.w[2 * qo + 1] + gi) = c[rr];
          *reinterpret_cast<float4*>(B.w[2 * qo] + gi) = w[rr];
          *reinterpret_cast<float4*>(B.acc + gi) = a[rr];
        } else {
          const float av[4] = {a[rr].x, a[rr].y, a[rr].z, a[rr].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (gx + e >= nx) break;
            const int64_t gi = gx + e + (int64_t)nx * gy;
            if (B.epi == 0) {
              B.out[gi] = (double)av[e];
            } else {
              const double vi = __ldg(B.v + gi);
              const double o = vi - (double)av[e];
              B.out[gi] = o;
              part = fma(B.mw ? vi * __ldg(B.mw + gi) : vi, o, part);
            }
          }
        }
      }
      if (last && B.epi == 1) {   // uniform per CTA (one problem per item)
        part = block_sum(part);
        if (threadIdx.x == 0) B.partials[t] = part;
      }
      __syncthreads();   // this stage is free again; the other slot holds the next item
      stage ^= 1;
      item = s_item[stage];
      p = s_p[stage];
    }
    fence_proxy_async_global();   // this sweep's stores before other CTAs' copies of the next sweep
    if (!grid_barrier(bar_count, bar_gen, err, gridDim.x)) return;
  }
}

// ------------------------------------------------------------------ 2-D, FP32, wavefront
// The f = 0 FP32 wave solve of the 5-point stencil with c = 1 (every A p of the batched CG loop)
// as a wavefront in registers: a work item is a strip of W = 32 C columns (the W - 2K middle ones
// are its output, K on each side are halo) and S rows of one problem (S = kFS or 2 kFS, chosen per
// launch from its parallel work), and ONE WARP advances it K
// time levels in a single pass down the rows.  Lane l holds columns C l .. C l + C - 1; at clock
// c the warp takes input row c (W^n, W^{n-1} and the filter sums, copied by the copy engine into
// the warp's own shared-memory blocks of FRB rows, two blocks in flight) and computes level t of
// row c - t for t = 1 .. K: level t needs rows c - t - 1 .. c - t + 1 of level t - 1 (a ring of
// three rows per level in registers) and row c - t of level t - 2; the x neighbours of a lane's
// outer columns come from the adjacent lanes (shuffles), the others from its own registers.  There is no shared-memory exchange and no block-wide barrier: each
// warp runs on its own.  The filter sum of row y collects w_{n+t} W^{n+t}(y) in a ring of K + 1
// rows; at clock c, row c - K is complete and W^{n+K}, W^{n+K-1} and its filter sum go to global
// memory (vector stores of the output columns).  Rows above and below the strip's S rows are
// input halo: a level-t value is exact at distance >= t from the rows and columns the strip did
// not load, so the K-wide halos leave the output exact.  Cells outside the domain are held at 0.
// The first sweep reads W^0 = v (FP64) directly and takes the Taylor start as level 1; the last
// sweep of a problem writes only the FP64 output (its levels beyond the problem's last step carry
// zero filter weights).  Same operations in the same order as the four-cell kernels: bitwise
// equal results.
constexpr int kFK = 8;                 // time levels per sweep
constexpr int kFC = 4;                 // columns per lane
constexpr int kFW = 32 * kFC;          // strip width
constexpr int kFTW = kFW - 2 * kFK;    // output columns of a strip
constexpr int kFS = 128;               // output rows of a work item (or 2 kFS, see k_batch_front)
// a launch takes items of 2 kFS rows (fewer halo rows per output row) when its work, in item
// sweeps of that height, is at least this many times the number of warps times its longest chain
// of sweeps (the sweeps of one problem run one after another); else kFS rows, for parallelism
constexpr double kFBigRatio = 2.0;
constexpr int kFRB = 8;                // rows per copied block
constexpr int kFWarps = 4;             // warps per CTA
constexpr int kFBlockBytes = (kFW + kFW + kFTW) * kFRB * 4;   // W^n, W^{n-1}, filter sums of FRB rows
constexpr int kFWarpBytes = 2 * kFBlockBytes;                 // two blocks in flight
constexpr int kFSmem = kFWarps * kFWarpBytes + 128;
static_assert(kFC == 2 || kFC == 4, "two or four columns per lane");
static_assert(kFK % 4 == 0 && kFK % kFC == 0, "strip origins x0 = sx (W - 2K) - K stay 16-byte aligned; "
                                               "the output columns are whole lane groups");
static_assert(kFBlockBytes % 128 == 0, "copy destinations stay 128-byte aligned");

struct BMapsF {          // tensor maps of one problem for the wavefront kernel
  CUtensorMap w[4];      // W x FRB boxes of the pitched state buffers
  CUtensorMap acc;       // (W - 2K) x FRB boxes of the filter sums
};

struct FV {              // the values of a lane's C columns
  float v[kFC];
};
__device__ __forceinline__ FV fv_zero() {
  FV r;
#pragma unroll
  for (int e = 0; e < kFC; ++e) r.v[e] = 0.0f;
  return r;
}
__device__ __forceinline__ FV fv_load(const void* p) {   // 8- or 16-byte aligned
  FV r;
  if constexpr (kFC == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
  } else {
    const float2 q = *reinterpret_cast<const float2*>(p);
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}
__device__ __forceinline__ void fv_store(float* p, const FV& a) {
  if constexpr (kFC == 4) *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  else *reinterpret_cast<float2*>(p) = make_float2(a.v[0], a.v[1]);
}

struct FrontState {      // the registers of one lane
  float L[kFK + 1][3][kFC];  // level t - 1 at index t: L[0] = W^{n-1}, L[1] = W^n, L[t + 1] = level t
  float A[kFK + 1][kFC];     // filter sums of the rows in flight: A[t] is row c - t at clock c
};

__device__ __forceinline__ float fr_mask(float v, bool in) { return in ? v : 0.0f; }

// One clock of the wavefront at phase PH = c mod 3 (the level rings).  Input row c: wn, wp (W^n,
// W^{n-1}), an = its filter sum so far (into A[0]).  Levels 1 .. K of rows c - 1 .. c - K.
// Returns in o level K of row c - K (W^{n+K}) and in pv level K - 1 of that row (W^{n+K-1}); the
// complete filter sum of row c - K is then A[K] (front_shift moves the filter sums one row on
// after the clock).
template <int PH, bool FIRST>
__device__ __forceinline__ void front_clock(FrontState& st, int c, const FV& wn, const FV& wp, const FV& an,
                                            const float* wt, float ax, float ay, float b, float ih2x, float ih2y,
                                            float hdt2, const bool* cin, int ny, FV& o, FV& pv) {
  constexpr int r3 = PH % 3;
#pragma unroll
  for (int e = 0; e < kFC; ++e) {
    st.L[0][r3][e] = wp.v[e];
    st.L[1][r3][e] = wn.v[e];
    st.A[0][e] = an.v[e];
  }
#pragma unroll
  for (int t = 1; t <= kFK; ++t) {
    const int y = c - t;
    const int im = (PH - t - 1 + 30) % 3, i0 = (PH - t + 30) % 3, ip = (PH - t + 1 + 30) % 3;
    const float* up = st.L[t][im];
    const float* mid = st.L[t][i0];
    const float* dn = st.L[t][ip];
    const float l = __shfl_up_sync(0xffffffffu, mid[kFC - 1], 1);
    const float r = __shfl_down_sync(0xffffffffu, mid[0], 1);
    const bool rin = (unsigned)y < (unsigned)ny;
    float n[kFC];
#pragma unroll
    for (int e = 0; e < kFC; ++e) {
      const float xl = e == 0 ? l : mid[e - 1];
      const float xr = e == kFC - 1 ? r : mid[e + 1];
      if (FIRST && t == 1) {   // Taylor start W^1 = W^0 + dt^2/2 L W^0
        float L0 = fmaf(-2.0f, mid[e], xl + xr) * ih2x;
        L0 = fmaf(fmaf(-2.0f, mid[e], up[e] + dn[e]), ih2y, L0);
        n[e] = fmaf(hdt2, L0, mid[e]);
      } else {
        const float* pvv = st.L[t - 1][i0];   // level t - 2 at row y
        n[e] = fmaf(ay, up[e] + dn[e], fmaf(ax, xl + xr, fmaf(b, mid[e], -pvv[e])));
      }
      n[e] = fr_mask(n[e], rin && cin[e]);
      st.A[t][e] = fmaf(wt[t - 1], n[e], st.A[t][e]);
    }
    if (t < kFK) {
#pragma unroll
      for (int e = 0; e < kFC; ++e) st.L[t + 1][i0][e] = n[e];
    } else {
#pragma unroll
      for (int e = 0; e < kFC; ++e) {
        o.v[e] = n[e];
        pv.v[e] = st.L[kFK][i0][e];
      }
    }
  }
}

__device__ __forceinline__ FV front_acc(const FrontState& st) {
  FV a;
#pragma unroll
  for (int e = 0; e < kFC; ++e) a.v[e] = st.A[kFK][e];
  return a;
}

// end of a clock: the filter sum of row c - t becomes that of row (c + 1) - (t + 1)
__device__ __forceinline__ void front_shift(FrontState& st) {
#pragma unroll
  for (int t = kFK; t >= 1; --t)
#pragma unroll
    for (int e = 0; e < kFC; ++e) st.A[t][e] = st.A[t - 1][e];
}

__device__ __forceinline__ void front_issue(const BMapsF* __restrict__ M, int p, int qi, int x0, int row,
                                            unsigned char* blk, uint64_t* bar) {
  mbar_arrive_expect_tx(bar, kFBlockBytes);
  tma_load_2d(blk, &M[p].w[2 * qi + 1], x0, row, bar);                       // W^n
  tma_load_2d(blk + kFW * kFRB * 4, &M[p].w[2 * qi], x0, row, bar);          // W^{n-1}
  tma_load_2d(blk + 2 * kFW * kFRB * 4, &M[p].acc, x0 + kFK, row, bar);      // filter sums
}

// bounded wait (one lane) until *cnt >= target; false after the limit (the error flag is raised)
// or once another warp has raised it
__device__ __forceinline__ bool wait_count(const unsigned* cnt, unsigned target, int* err) {
  unsigned long long spins = 0;
  while (*(const volatile unsigned*)cnt < target) {
    if (++spins > kBarrierSpins) {
      atomicExch(err, 1);
      return false;
    }
    if ((spins & 1023ull) == 0 && *(volatile int*)err) return false;
    __nanosleep(64);
  }
  __threadfence();
  return true;
}

__global__ void __launch_bounds__(kFWarps * 32, kFC == 4 ? 2 : 3) k_batch_front(const BTileT* __restrict__ P,
                                                              const BMapsF* __restrict__ M,
                                                              const int* __restrict__ nact, int J,
                                                              const int64_t* __restrict__ joff,
                                                              const int64_t* __restrict__ joffb, int rows_mode,
                                                              unsigned* pcnt, const float* __restrict__ wtab,
                                                              int* err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* const base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  __shared__ __align__(8) uint64_t s_bar[kFWarps][2];
  __shared__ int s_big;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np = nact[0];
  // item height of this launch (rows_mode 0: by the rule at kFBigRatio; 1: kFS; 2: 2 kFS), the
  // same in every CTA: the active problems' item sweeps at 2 kFS rows against the longest chain
  if (warp == 0) {
    bool big = rows_mode == 2;
    if (rows_mode == 0) {
      double work = 0.0;
      int longest = 0;
      for (int p = lane; p < np; p += 32) {
        const BTileT& B = P[p];
        if (B.halt && *B.halt != 0.0) continue;
        const int sw = (B.nt + kFK - 1) / kFK;
        work += (double)B.ntilesb * sw;
        longest = max(longest, sw);
      }
      work = warp_sum(work);
      longest = __reduce_max_sync(0xffffffffu, longest);
      big = work >= kFBigRatio * (double)longest * (double)gridDim.x * kFWarps;
    }
    if (lane == 0) s_big = big ? 1 : 0;
  }
  __syncthreads();
  const bool big = s_big != 0;
  const int64_t* const jo = big ? joffb : joff;
  const int rows = big ? 2 * kFS : kFS;
  for (int p = threadIdx.x; p <= np; p += blockDim.x)
    s_tile0[p] = p < np ? (big ? P[p].tile0b : P[p].tile0)
                        : (big ? P[np - 1].tile0b + P[np - 1].ntilesb : P[np - 1].tile0 + P[np - 1].ntiles);
  if (lane == 0) {
    mbar_init(&s_bar[warp][0], 1);
    mbar_init(&s_bar[warp][1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  unsigned char* const wbase = base + warp * kFWarpBytes;
  uint32_t parity[2] = {0u, 0u};
  const int64_t G = (int64_t)gridDim.x * kFWarps;
  const int64_t gw = (int64_t)blockIdx.x * kFWarps + warp;
  bool failed = false;
  // work items of all sweeps in one sequence (sweep by sweep, the active problems' strips in
  // order), taken round-robin by the warps; a strip of sweep j waits only for the strips of its
  // own problem's sweep j - 1 (per-problem completion counters), not for the whole grid
  const int64_t nitems = jo[J];
  int j = 0, p = 0;
  for (int64_t it = gw; it < nitems && !failed; it += G) {
    while (jo[j + 1] <= it) {
      ++j;
      p = 0;
    }
    const int64_t item = it - jo[j];
    while (s_tile0[p + 1] <= item) ++p;
    const int qi = (j + 1) & 1, qo = j & 1;
    {
      const BTileT& B = P[p];
      if (B.halt && *B.halt != 0.0) continue;
      const int t = (int)(item - (big ? B.tile0b : B.tile0));
      const int ntl = big ? B.ntilesb : B.ntiles;
      const int sx = t % B.tiles_x, sy = t / B.tiles_x;
      const int nx = B.nx, ny = B.ny;
      const int x0 = sx * kFTW - kFK;
      const int Y0 = sy * rows, Y1 = min(Y0 + rows, ny);
      const int c0 = Y0 - kFK, c1 = Y1 - 1 + kFK;       // clocks (input rows) of this item
      const int n0 = j * kFK;
      const int kk = min(kFK, B.nt - n0);
      const bool first = j == 0, last = n0 + kk == B.nt;
      float wt[kFK];
#pragma unroll
      for (int s = 0; s < kFK; ++s) wt[s] = s < kk ? __ldg(wtab + B.wofs + n0 + 1 + s) : 0.0f;
      const float w0 = first ? __ldg(wtab + B.wofs) : 0.0f;
      const int gx0 = x0 + kFC * lane;
      bool cin[kFC];
#pragma unroll
      for (int e = 0; e < kFC; ++e) cin[e] = gx0 + e >= 0 && gx0 + e < nx;
      // output columns: the lane's whole group lies inside [K, W - K) (K is a multiple of C)
      const bool outl = kFC * lane >= kFK && kFC * lane < kFW - kFK;
      const bool outc = outl && gx0 < nx;
      const float ax = B.ax, ay = B.ay, bb = B.b, ih2x = B.ih2x, ih2y = B.ih2y, hdt2 = 0.5f * B.dt2;
      // the descriptor's fields in registers (the stores below could otherwise alias it)
      float* const wout1 = B.w[2 * qo + 1];
      float* const wout0 = B.w[2 * qo];
      float* const accp = B.acc;
      const double* const vv = B.v;
      const double* const mwp = B.mw;
      double* const outp = B.out;
      const int pitch = B.pitch, epi = B.epi;
      FrontState st;
#pragma unroll
      for (int a = 0; a < kFK + 1; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int e = 0; e < kFC; ++e) st.L[a][r][e] = 0.0f;
#pragma unroll
      for (int a = 0; a < kFK + 1; ++a)
#pragma unroll
        for (int e = 0; e < kFC; ++e) st.A[a][e] = 0.0f;
      const int nblk = (c1 - c0 + 1 + kFRB - 1) / kFRB;
      if (!first) {   // every strip of this problem's previous sweep is done: its stores, then the copies
        bool ok = true;
        if (lane == 0) {
          ok = wait_count(pcnt + p, (unsigned)(j * ntl), err);
          if (ok) fence_proxy_async_global();
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          failed = true;
          break;
        }
        if (lane == 0) {
          front_issue(M, p, qi, x0, c0, wbase, &s_bar[warp][0]);
          if (nblk > 1) front_issue(M, p, qi, x0, c0 + kFRB, wbase + kFBlockBytes, &s_bar[warp][1]);
        }
      }
      __syncwarp();
      double part = 0.0;
      int c = c0;
      // FP64 values read one clock ahead and converted or used only at the next clock: the initial
      // state of input row c (first sweep), v of output row c - K (last sweep, A p epilogue)
      double nv[kFC];
      auto fetch_v = [&](auto fst, auto lst, int cc) {
        constexpr bool FIRST = decltype(fst)::value, LAST = decltype(lst)::value;
        if (FIRST) {
          const bool rin = (unsigned)cc < (unsigned)ny;
#pragma unroll
          for (int e = 0; e < kFC; ++e) nv[e] = (rin && cin[e] && vv) ? __ldg(vv + gx0 + e + (int64_t)nx * cc) : 0.0;
        } else if (LAST) {
          const int y = cc - kFK;
          const bool ok = epi != 0 && y >= Y0 && y < Y1 && outc;
#pragma unroll
          for (int e = 0; e < kFC; ++e) nv[e] = (ok && gx0 + e < nx) ? __ldg(vv + gx0 + e + (int64_t)nx * y) : 0.0;
        }
      };
      // clocks in groups of three (the phase of the level rings is c - c0 mod 3)
      // (the first and the last sweep are separate instances, so that the loop of the other
      // sweeps carries neither the Taylor start nor the FP64 epilogue)
      auto clock = [&](auto ph, auto fst, auto lst) {
        constexpr int PH = decltype(ph)::value;
        constexpr bool FIRST = decltype(fst)::value, LAST = decltype(lst)::value;
        const int rel = c - c0, blk = rel / kFRB, row = rel % kFRB, slot = blk & 1;
        double vc[kFC];
#pragma unroll
        for (int e = 0; e < kFC; ++e) vc[e] = nv[e];
        if ((FIRST || LAST) && c + 1 <= c1) fetch_v(fst, lst, c + 1);
        FV wn = fv_zero(), wp = fv_zero(), an = fv_zero();
        if (FIRST) {
#pragma unroll
          for (int e = 0; e < kFC; ++e) {
            wn.v[e] = (float)vc[e];
            an.v[e] = w0 * wn.v[e];
          }
        } else {
          if (row == 0) {   // a new block: wait for its copies
            if (!mbar_wait(&s_bar[warp][slot], parity[slot], kMbarPolls)) failed = true;
            parity[slot] ^= 1u;
          }
          const unsigned char* bp = wbase + slot * kFBlockBytes;
          wn = fv_load(bp + (row * 32 + lane) * kFC * 4);
          wp = fv_load(bp + kFW * kFRB * 4 + (row * 32 + lane) * kFC * 4);
          if (outl) an = fv_load(bp + 2 * kFW * kFRB * 4 + (row * (kFTW / kFC) + lane - kFK / kFC) * kFC * 4);
          if (row == kFRB - 1) {   // block done: refill its slot two blocks ahead
            __syncwarp();
            if (lane == 0 && blk + 2 < nblk)
              front_issue(M, p, qi, x0, c0 + (blk + 2) * kFRB, wbase + slot * kFBlockBytes, &s_bar[warp][slot]);
          }
        }
        FV o, pv;
        front_clock<PH, FIRST>(st, c, wn, wp, an, wt, ax, ay, bb, ih2x, ih2y, hdt2, cin, ny, o, pv);
        const int y = c - kFK;
        if (y >= Y0 && y < Y1 && outc) {
          const FV a = front_acc(st);
          if (!LAST) {
            // rows are padded to a multiple of 4 floats: a group's columns past nx are padding
            const int64_t gi = gx0 + (int64_t)pitch * y;
            fv_store(wout1 + gi, o);
            fv_store(wout0 + gi, pv);
            fv_store(accp + gi, a);
          } else {
            const int64_t gi = gx0 + (int64_t)nx * y;
#pragma unroll
            for (int e = 0; e < kFC; ++e) {
              if (gx0 + e >= nx) break;
              if (epi == 0) {
                outp[gi + e] = (double)a.v[e];
              } else {
                const double vi = vc[e];
                const double ov = vi - (double)a.v[e];
                outp[gi + e] = ov;
                part = fma(mwp ? vi * __ldg(mwp + gi + e) : vi, ov, part);
              }
            }
          }
        }
        front_shift(st);
        ++c;
      };
      auto run = [&](auto fst, auto lst) {
        fetch_v(fst, lst, c0);
        while (c <= c1) {
          clock(std::integral_constant<int, 0>(), fst, lst);
          if (c > c1) break;
          clock(std::integral_constant<int, 1>(), fst, lst);
          if (c > c1) break;
          clock(std::integral_constant<int, 2>(), fst, lst);
        }
      };
      using T_ = std::true_type;
      using F_ = std::false_type;
      if (first) {
        if (last) run(T_(), T_());
        else run(T_(), F_());
      } else {
        if (last) run(F_(), T_());
        else run(F_(), F_());
      }
      if (last && B.epi == 1) {
        part = warp_sum(part);
        if (lane == 0) {
          B.partials[t] = part;
          // the finishing kernel sums B.ntiles partials: taller items leave the rest at zero
          if (big && B.ntilesb + t < B.ntiles) B.partials[B.ntilesb + t] = 0.0;
        }
      }
      // publish this strip: its stores to every thread and to the copy engine, then the count
      fence_proxy_async_global();
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(pcnt + p, 1u);
    }
  }
  if (__syncthreads_or(failed)) {   // a wait or copies that did not complete: give up, after a bounded drain
    if (threadIdx.x == 0) atomicExch(err, 1);
    if (lane == 0) {
      mbar_wait(&s_bar[warp][0], parity[0], kMbarPolls);
      mbar_wait(&s_bar[warp][1], parity[1], kMbarPolls);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ 2-D wavefront, two columns per lane
// The double-float residual wave solves of the FP64 correction (2-D, second order, c = 1; forced
// or not), and the forced FP32 wave solve of b, in the wavefront form of k_batch_front: a work item
// is a strip of 64 columns (64 - 2K output columns, K on each side halo) and kDS rows, ONE WARP
// advances it K time levels in a single pass down the rows with the levels' rows in register
// rings; lane l holds columns 2l, 2l + 1 (T = dfl: hi/lo pairs), x neighbours of its outer columns
// by shuffles.  Input rows (W^n, W^{n-1}, the filter sums; W^0 = v in the first sweep) and the
// forcing rows are read straight from global memory one clock ahead (FP64 values raw, converted
// when used); the forcing of the rows in flight is kept in a register ring.  No shared memory and
// no block-wide barrier; a strip of sweep j waits only for its problem's sweep j - 1 (per-problem
// completion counters).  The updates are those of the staged kernels in the same order (bitwise
// equal results): T = dfl the double-float operations of k_batch_block2d_df,
//   Taylor start  W^1 = W^0 + (dt^2 / 2) (sum_m ih2_m ((W_- + W_+) - 2 W^0) - f)
//   step          df_leapfrog: b W^n - W^{n-1} + a_x (W_l + W_r) + a_y (W_d + W_u) - fph_n f
//   filter        acc = w_0 W^0, then df_fma_acc(acc, w_{n+1}, W^{n+1})
// T = float the FP32 operations of k_batch_block2d,
//   Taylor start  W^1 = fma(dt^2 / 2, L W^0, W^0), then fma(-(dt^2 / 2) cos(omega_hat t^0), f, .)
//   step          fma(a_y, W_d + W_u, fma(a_x, W_l + W_r, fma(b, W^n, -W^{n-1}))),
//                 then fma(-dt^2 cos(omega_hat t^n), f, .)
//   filter        acc = w_0 W^0, then fma(w_{n+1}, W^{n+1}, acc)
constexpr int kDK = 4;                 // time levels per sweep of the double-float roles
constexpr int kDS = 128;               // output rows of a work item
constexpr int kDWarps = 4;             // warps per CTA
template <int K>
__host__ __device__ constexpr int wf_tw() { return 64 - 2 * K; }   // output columns of a strip

template <typename T, int K>
struct WFront {          // the registers of one lane (two columns)
  T L[K + 1][3][2];      // level t - 1 at index t: L[0] = W^{n-1}, L[1] = W^n, L[t + 1] = level t
  T A[K + 1][2];         // filter sums of the rows in flight: A[t] is row c - t at clock c
  T F[K + 1][2];         // forcing of the rows in flight: F[t] is row c - t
};

__device__ __forceinline__ dfl wf_shfl_up(dfl a) {
  return {__shfl_up_sync(0xffffffffu, a.hi, 1), __shfl_up_sync(0xffffffffu, a.lo, 1)};
}
__device__ __forceinline__ dfl wf_shfl_down(dfl a) {
  return {__shfl_down_sync(0xffffffffu, a.hi, 1), __shfl_down_sync(0xffffffffu, a.lo, 1)};
}
__device__ __forceinline__ float wf_shfl_up(float a) { return __shfl_up_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ float wf_shfl_down(float a) { return __shfl_down_sync(0xffffffffu, a, 1); }
template <typename T>
__device__ __forceinline__ T wf_zero() {
  if constexpr (std::is_same<T, dfl>::value) return dfl{0.0f, 0.0f};
  else return 0.0f;
}
template <typename T>
__device__ __forceinline__ T wf_from(double x) {
  if constexpr (std::is_same<T, dfl>::value) return df_from(x);
  else return (float)x;
}
__device__ __forceinline__ double wf_to(dfl a) { return df_to(a); }
__device__ __forceinline__ double wf_to(float a) { return (double)a; }

template <typename T>
struct WfCoef {          // per-item constants of the level updates
  T ax, ay, b, ih2x, ih2y, hdt2;
};

template <typename T, int K, int PH, bool FIRST, bool FORCED>
__device__ __forceinline__ void wf_clock(WFront<T, K>& st, int c, const T* wn, const T* wp, const T* an, const T* fr,
                                         const T* wt, const T* fph, const WfCoef<T>& q, const bool* cin, int ny,
                                         T* o, T* pv) {
  constexpr bool DF = std::is_same<T, dfl>::value;
  constexpr int r3 = PH % 3;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    st.L[0][r3][e] = wp[e];
    st.L[1][r3][e] = wn[e];
    st.A[0][e] = an[e];
    if (FORCED) st.F[0][e] = fr[e];
  }
#pragma unroll
  for (int t = 1; t <= K; ++t) {
    const int y = c - t;
    const int im = (PH - t - 1 + 30) % 3, i0 = (PH - t + 30) % 3, ip = (PH - t + 1 + 30) % 3;
    const T* up = st.L[t][im];
    const T* mid = st.L[t][i0];
    const T* dn = st.L[t][ip];
    const T l = wf_shfl_up(mid[1]);
    const T r = wf_shfl_down(mid[0]);
    const bool rin = (unsigned)y < (unsigned)ny;
    T n[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const T xl = e == 0 ? l : mid[0];
      const T xr = e == 1 ? r : mid[1];
      if constexpr (DF) {
        if (FIRST && t == 1) {   // Taylor start
          const dfl sx = df_add(xl, xr);
          const dfl sy = df_add(up[e], dn[e]);
          const dfl c2x = {2.0f * mid[e].hi, 2.0f * mid[e].lo};
          dfl Lp = df_add(df_zero(), df_mul(q.ih2x, df_sub(sx, c2x)));
          Lp = df_add(Lp, df_mul(q.ih2y, df_sub(sy, c2x)));
          if (FORCED) Lp = df_sub(Lp, st.F[t][e]);
          n[e] = df_add(mid[e], df_mul(q.hdt2, Lp));
        } else {
          const dfl coef[2] = {q.ax, q.ay};
          const dfs sm[2] = {df_pair_sum(xl, xr), df_pair_sum(up[e], dn[e])};
          n[e] = df_leapfrog<2, FORCED>(q.b, mid[e], st.L[t - 1][i0][e], coef, sm, fph[t - 1],
                                        FORCED ? st.F[t][e] : df_zero());
        }
        if (!(rin && cin[e])) n[e] = df_zero();
        st.A[t][e] = df_fma_acc(st.A[t][e], wt[t - 1], n[e]);
      } else {
        if (FIRST && t == 1) {   // Taylor start
          float L0 = fmaf(-2.0f, mid[e], xl + xr) * q.ih2x;
          L0 = fmaf(fmaf(-2.0f, mid[e], up[e] + dn[e]), q.ih2y, L0);
          n[e] = fmaf(q.hdt2, L0, mid[e]);
        } else {
          n[e] = fmaf(q.ay, up[e] + dn[e], fmaf(q.ax, xl + xr, fmaf(q.b, mid[e], -st.L[t - 1][i0][e])));
        }
        if (FORCED) n[e] = fmaf(-fph[t - 1], st.F[t][e], n[e]);
        n[e] = (rin && cin[e]) ? n[e] : 0.0f;
        st.A[t][e] = fmaf(wt[t - 1], n[e], st.A[t][e]);
      }
    }
    if (t < K) {
#pragma unroll
      for (int e = 0; e < 2; ++e) st.L[t + 1][i0][e] = n[e];
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        o[e] = n[e];
        pv[e] = st.L[K][i0][e];
      }
    }
  }
}

// end of a clock: the rows in flight move on by one
template <typename T, int K, bool FORCED>
__device__ __forceinline__ void wf_shift(WFront<T, K>& st) {
#pragma unroll
  for (int t = K; t >= 1; --t)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      st.A[t][e] = st.A[t - 1][e];
      if (FORCED) st.F[t][e] = st.F[t - 1][e];
    }
}

// ptab: the double-float roles take the forcing factor dt^2 cos(omega_hat t^n) whole; the FP32
// role takes cos(omega_hat t^n) and forms the factor as k_batch_block2d does
template <typename T, int K, bool FORCED>
__global__ void __launch_bounds__(kDWarps * 32, std::is_same<T, dfl>::value ? 2 : 3)
    k_batch_front2(const BTile<T>* __restrict__ P, const int* __restrict__ nact, int J,
                   const int64_t* __restrict__ joff, unsigned* pcnt, const T* __restrict__ wtab,
                   const T* __restrict__ ptab, int* err) {
  constexpr bool DF = std::is_same<T, dfl>::value;
  constexpr int TW = wf_tw<K>();
  __shared__ int64_t s_tile0[kBatchMaxProblems + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np = nact[0];
  for (int p = threadIdx.x; p <= np; p += blockDim.x)
    s_tile0[p] = p < np ? P[p].tile0 : P[np - 1].tile0 + P[np - 1].ntiles;
  __syncthreads();
  const int64_t G = (int64_t)gridDim.x * kDWarps;
  const int64_t gw = (int64_t)blockIdx.x * kDWarps + warp;
  const int64_t nitems = joff[J];
  int j = 0, p = 0;
  for (int64_t it = gw; it < nitems; it += G) {
    while (joff[j + 1] <= it) {
      ++j;
      p = 0;
    }
    const int64_t item = it - joff[j];
    while (s_tile0[p + 1] <= item) ++p;
    const int qi = (j + 1) & 1, qo = j & 1;
    const BTile<T>& B = P[p];
    if (B.halt && *B.halt != 0.0) continue;
    const int t = (int)(item - B.tile0);
    const int sx = t % B.tiles_x, sy = t / B.tiles_x;
    const int nx = B.nx, ny = B.ny;
    const int x0 = sx * TW - K;
    const int Y0 = sy * kDS, Y1 = min(Y0 + kDS, ny);
    const int c0 = Y0 - K, c1 = Y1 - 1 + K;   // clocks (input rows) of this item
    const int n0 = j * K;
    const int kk = min(K, B.nt - n0);
    const bool first = j == 0, last = n0 + kk == B.nt;
    if (!first) {   // every strip of this problem's previous sweep is done
      bool ok = true;
      if (lane == 0) ok = wait_count(pcnt + p, (unsigned)(j * B.ntiles), err);
      if (!__shfl_sync(0xffffffffu, ok, 0)) return;
    }
    T wt[K], fph[K];
#pragma unroll
    for (int s = 0; s < K; ++s) {   // the tables carry K zero entries past every problem's nt
      wt[s] = wtab[B.wofs + n0 + 1 + s];
      if constexpr (DF) fph[s] = FORCED ? ptab[B.wofs + n0 + s] : df_zero();
      else fph[s] = FORCED ? (n0 + s > 0 ? B.dt2 : 0.5f * B.dt2) * ptab[B.wofs + n0 + s] : 0.0f;
    }
    const T w0 = first ? wtab[B.wofs] : wf_zero<T>();
    const int gx0 = x0 + 2 * lane;
    const bool cin[2] = {gx0 >= 0 && gx0 < nx, gx0 + 1 >= 0 && gx0 + 1 < nx};
    const bool outc = 2 * lane >= K && 2 * lane < 64 - K && gx0 < nx;   // output columns
    WfCoef<T> q;
    q.ax = B.ax; q.ay = B.ay; q.b = B.b; q.ih2x = B.ih2x; q.ih2y = B.ih2y;
    if constexpr (DF) q.hdt2 = dfl{0.5f * B.dt2.hi, 0.5f * B.dt2.lo};
    else q.hdt2 = 0.5f * B.dt2;
    // the descriptor's fields in registers (the stores below could otherwise alias it)
    const T* const wcur = B.w[2 * qi + 1];
    const T* const wprv = B.w[2 * qi];
    T* const wout1 = B.w[2 * qo + 1];
    T* const wout0 = B.w[2 * qo];
    T* const accp = B.acc;
    const double* const vv = B.v;
    const double* const fv = B.f;
    const double* const mwp = B.mw;
    double* const outp = B.out;
    const int epi = B.epi;
    WFront<T, K> st;
#pragma unroll
    for (int a = 0; a < K + 1; ++a)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int r = 0; r < 3; ++r) st.L[a][r][e] = wf_zero<T>();
        st.A[a][e] = wf_zero<T>();
        st.F[a][e] = wf_zero<T>();
      }
    // input row c, loaded one clock ahead (its filter sum is read only at the output columns, the
    // others are discarded); the FP64 initial state and forcing stay raw here and are converted
    // when the clock uses them, so that no load is waited for one clock early
    auto fetch = [&](auto fst, int c, T* wn, T* wp, T* an, double* vr, double* fr) {
      constexpr bool FIRST = decltype(fst)::value;
      const bool rin = (unsigned)c < (unsigned)ny;
      const int64_t gi = gx0 + (int64_t)nx * c;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const bool in = rin && cin[e];
        if (FIRST) {
          vr[e] = (in && vv) ? __ldg(vv + gi + e) : 0.0;
        } else {   // written by other warps in the previous sweep: coherent loads
          if constexpr (DF) {
            if (in) {
              const float2 a = __ldcg(reinterpret_cast<const float2*>(wcur + gi + e));
              const float2 b2 = __ldcg(reinterpret_cast<const float2*>(wprv + gi + e));
              wn[e] = dfl{a.x, a.y};
              wp[e] = dfl{b2.x, b2.y};
            } else {
              wn[e] = wp[e] = df_zero();
            }
            if (in && outc) {
              const float2 a = __ldcg(reinterpret_cast<const float2*>(accp + gi + e));
              an[e] = dfl{a.x, a.y};
            } else {
              an[e] = df_zero();
            }
          } else {
            wn[e] = in ? __ldcg(wcur + gi + e) : 0.0f;
            wp[e] = in ? __ldcg(wprv + gi + e) : 0.0f;
            an[e] = (in && outc) ? __ldcg(accp + gi + e) : 0.0f;
          }
        }
        if (FORCED) fr[e] = (in && fv) ? __ldg(fv + gi + e) : 0.0;
      }
    };
    T nwn[2], nwp[2], nan[2];
    double nvr[2], nfr[2];
    double part = 0.0;
    int c = c0;
    auto clock = [&](auto ph, auto fst, auto lst) {
      constexpr int PH = decltype(ph)::value;
      constexpr bool FIRST = decltype(fst)::value, LAST = decltype(lst)::value;
      T wn[2], wp[2], an[2], fr[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (FIRST) {
          wn[e] = wf_from<T>(nvr[e]);
          wp[e] = wf_zero<T>();
          if constexpr (DF) an[e] = df_mul(w0, wn[e]);
          else an[e] = w0 * wn[e];
        } else {
          wn[e] = nwn[e];
          wp[e] = nwp[e];
          an[e] = nan[e];
        }
        fr[e] = FORCED ? wf_from<T>(nfr[e]) : wf_zero<T>();
      }
      if (c + 1 <= c1) fetch(fst, c + 1, nwn, nwp, nan, nvr, nfr);   // one clock ahead
      T o[2], pv[2];
      wf_clock<T, K, PH, FIRST, FORCED>(st, c, wn, wp, an, fr, wt, fph, q, cin, ny, o, pv);
      const int y = c - K;
      if (y >= Y0 && y < Y1 && outc) {
        const int64_t gi = gx0 + (int64_t)nx * y;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (gx0 + e >= nx) break;
          const T a = st.A[K][e];
          if (!LAST) {
            wout1[gi + e] = o[e];
            wout0[gi + e] = pv[e];
            accp[gi + e] = a;
          } else if (epi == 0) {
            outp[gi + e] = wf_to(a);
          } else {
            const double vi = __ldg(vv + gi + e);
            const double ov = vi - wf_to(a);
            outp[gi + e] = ov;
            part = fma(mwp ? vi * __ldg(mwp + gi + e) : vi, ov, part);
          }
        }
      }
      wf_shift<T, K, FORCED>(st);
      ++c;
    };
    auto run = [&](auto fst, auto lst) {
      fetch(fst, c0, nwn, nwp, nan, nvr, nfr);
      while (c <= c1) {
        clock(std::integral_constant<int, 0>(), fst, lst);
        if (c > c1) break;
        clock(std::integral_constant<int, 1>(), fst, lst);
        if (c > c1) break;
        clock(std::integral_constant<int, 2>(), fst, lst);
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    if (first) {
      if (last) run(T_(), T_());
      else run(T_(), F_());
    } else {
      if (last) run(F_(), T_());
      else run(F_(), F_());
    }
    if (last && epi == 1) {
      part = warp_sum(part);
      if (lane == 0) B.partials[t] = part;
    }
    __threadfence();   // publish this strip's stores, then count it
    __syncwarp();
    if (lane == 0) atomicAdd(pcnt + p, 1u);
  }
}

// ------------------------------------------------------------------ per-problem small kernels
struct BFin {
  const double* partials;
  const double* halt;
  double* scal;
  int ntiles;
};

// p^T M q of every problem from its per-tile partial sums (one block per problem, fixed order)
__global__ void k_batch_finish(const BFin* __restrict__ F) {
  const BFin& B = F[blockIdx.x];
  if (B.halt && *B.halt != 0.0) return;
  double s = 0.0;
  for (int t = threadIdx.x; t < B.ntiles; t += blockDim.x) s += B.partials[t];
  s = block_sum(s);
  if (threadIdx.x == 0) B.scal[S_PQ] = s;
}

// per-problem convergence test of the batched CG loop (one thread per problem)
__global__ void k_batch_check(double* const* __restrict__ scal, int np) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double* sc = scal[p];
  if (sc[S_HALT] != 0.0) return;
  const double it = sc[S_ITER] + 1.0;
  sc[S_ITER] = it;
  if (!(sc[S_FLAG] == 0.0 && sc[S_RR] > sc[S_STOP] && it < sc[S_MAXIT])) sc[S_HALT] = 1.0;
}

// The CG vector updates of every problem in two launches (instead of two per problem): problem p
// owns blocks [block0, block0 + blocks) with blocks = the grid of the single-grid update (so each
// problem's block partition, and its reduction order, is the single-grid one).  The x / r update
// reduces r^T M r per problem (last block of the problem adds its partials in index order).
struct BCg {
  double *x, *r, *p;
  const double *q, *mw;
  int64_t n;
  double* scal;
  double* partials;
  unsigned* counter;
  int block0, blocks;
};

__device__ __forceinline__ int cg_problem(const BCg* __restrict__ D, int np, int b) {
  int lo = 0, hi = np - 1;   // last problem with block0 <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D[mid].block0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_batch_cg_update(const BCg* __restrict__ D, int np) {
  const BCg& B = D[cg_problem(D, np, blockIdx.x)];
  double* scal = B.scal;
  if (scal[S_HALT] != 0.0) return;   // a stopped problem
  const int lb = blockIdx.x - B.block0;
  const double rr = scal[S_RR];
  const double pq = scal[S_PQ];
  const double alpha = rr / pq;
  const bool ok = (pq != 0.0) && isfinite(alpha);
  const double a = ok ? alpha : 0.0;
  double s = 0.0;
  const int64_t stride = (int64_t)B.blocks * blockDim.x;
  for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += stride) {
    B.x[i] = fma(a, B.p[i], B.x[i]);
    const double ri = fma(-a, B.q[i], B.r[i]);
    B.r[i] = ri;
    s = fma(B.mw ? ri * B.mw[i] : ri, ri, s);
  }
  s = block_sum(s);
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    B.partials[lb] = s;
    __threadfence();
    s_last = atomicAdd(B.counter, 1u) == (unsigned)(B.blocks - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < B.blocks; i += blockDim.x) t += __ldcg(B.partials + i);
  t = block_sum(t);
  if (threadIdx.x == 0) {
    *B.counter = 0u;
    scal[S_ALPHA] = a;
    scal[S_BETA] = t / rr;
    scal[S_RR] = t;
    if (!ok || !isfinite(t)) scal[S_FLAG] = 1.0;
  }
}

__global__ void __launch_bounds__(256) k_batch_cg_direction(const BCg* __restrict__ D, int np) {
  const BCg& B = D[cg_problem(D, np, blockIdx.x)];
  if (B.scal[S_HALT] != 0.0) return;
  const double beta = B.scal[S_BETA];
  const int lb = blockIdx.x - B.block0;
  const int64_t stride = (int64_t)B.blocks * blockDim.x;
  for (int64_t i = lb * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += stride) B.p[i] = fma(beta, B.p[i], B.r[i]);
}

// keep the WHILE loop running while any problem is active
__global__ void k_batch_any(cudaGraphConditionalHandle h, double* const* __restrict__ scal, int np,
                            const int* __restrict__ err) {
  int any = 0;
  for (int p = 0; p < np; ++p) any |= scal[p][S_HALT] == 0.0;
  if (*err) any = 0;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

// ------------------------------------------------------------------ host side
// One role of batched wave solve (e.g. q = A p of every problem in FP32, or b in FP64): its
// device descriptor table and the launcher of the kernel variant it needs.
struct Wave {
  void* desc = nullptr;
  void* maps = nullptr;        // tensor maps (TMA-fed role)
  int* nact = nullptr;
  void* wtab = nullptr;
  void* ptab = nullptr;
  BFin* fin = nullptr;
  int J = 0, K = 1, nblocks = 1;
  int64_t* joff = nullptr;     // wavefront role: first work item of each sweep (J + 1 entries)
  int64_t* joffb = nullptr;    // ... with work items of 2 kFS rows (k_batch_front)
  int rows_mode = 0;           // k_batch_front item height: 0 by launch, 1 kFS, 2 2 kFS
  unsigned* pcnt = nullptr;    // ... and per-problem completion counters
  int np = 0;
  size_t smem = 0;
  cudaError_t (*launch)(cudaStream_t, const Wave&, unsigned*, int*) = nullptr;
};

// per-problem inputs of one role
struct RoleIO {
  std::vector<const double*> v, f;   // v: initial state (nullptr: 0); f: forcing (nullptr: none)
  std::vector<double*> out;
  int epi = 0;
  bool halt = false;                 // skip stopped problems
};

struct BatchCtx {
  int np = 0;
  const whv_grid* grids = nullptr;
  const whv_params* params = nullptr;
  std::vector<TimeGridH> tgs;
  whv_grid g0 = nullptr;
  cudaStream_t st = nullptr;
  int sms = 148;
  unsigned* bar = nullptr;     // count, generation
  int* err = nullptr;
  double** scal = nullptr;     // device array of the problems' scalar blocks
  std::vector<void*> allocs;
  int64_t launches = 0;
  // WHV_LOG=1: host wall time per phase of the batched solve (the phases end with a stream
  // synchronisation, so the host clock brackets the device work), printed at the end
  double t_mark = 0.0;
  double t_phase[5] = {0, 0, 0, 0, 0};   // b wave solve, CG loops, residual wave solves, deflation, other
  void mark(int ph) {
    const double t = now_s();
    if (t_mark > 0.0) t_phase[ph] += t - t_mark;
    t_mark = t;
  }
  ~BatchCtx() {
    if (st) cudaStreamSynchronize(st);
    for (void* p : allocs) cudaFree(p);
  }
  template <typename X>
  cudaError_t alloc(X** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) allocs.push_back((void*)*p);
    return e;
  }
  template <typename F>
  auto each(F fn) const -> std::vector<decltype(fn(grids[0]))> {
    std::vector<decltype(fn(grids[0]))> v(np);
    for (int p = 0; p < np; ++p) v[p] = fn(grids[p]);
    return v;
  }
};

#define B_CUDA(g, call) \
  do { cudaError_t _e = (call); if (_e != cudaSuccess) return cuda_fail((g), _e, #call); } while (0)

// steps per sweep of the blocked 2-D kernel: the grid's setting (whv_set_steps_per_sweep) if
// any, else 8 (FP32) / 4 (FP64) steps of the 5-point stencil, half that for the 9-point one
static int batch_k(whv_grid g, bool fp64) {
  const int R = g->order == 2 ? 1 : 2;
  int k = g->kblock > 0 ? g->kblock : (fp64 ? 4 : 8) / R;
  k = std::min(std::max(k, 1), 16);
  while (k > 1 && kBReg - 2 * k * R < 16) --k;
  return k;
}

template <typename T, int ORDER, bool VARC, bool FORCED>
static cudaError_t launch_block2d(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  const BTile<T>* P = (const BTile<T>*)w.desc;
  const T* wt = (const T*)w.wtab;
  const T* ph = (const T*)w.ptab;
  unsigned* bc = bar;
  unsigned* bg = bar + 1;
  int J = w.J, K = w.K;
  const int* na = w.nact;
  void* args[] = {(void*)&P, (void*)&na, (void*)&J, (void*)&K, (void*)&wt, (void*)&ph,
                  (void*)&bc, (void*)&bg, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_block2d<T, ORDER, VARC, FORCED>, dim3(w.nblocks),
                                     dim3(kBThreads), args, w.smem, st);
}

template <typename T, int DIM, int ORDER, bool VARC>
static cudaError_t launch_wave3(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  const BProb<T>* P = (const BProb<T>*)w.desc;
  const T* wt = (const T*)w.wtab;
  const T* ph = (const T*)w.ptab;
  unsigned* bc = bar;
  unsigned* bg = bar + 1;
  int S = w.J;
  const int* na = w.nact;
  void* args[] = {(void*)&P, (void*)&na, (void*)&S, (void*)&wt, (void*)&ph, (void*)&bc, (void*)&bg, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_wave<T, DIM, ORDER, VARC>, dim3(w.nblocks), dim3(32, 8),
                                     args, 0, st);
}

// opt the blocked kernels into their dynamic shared memory (FP64: 64 KB) once per process,
// outside any stream capture
// dynamic shared memory of the blocked batched kernel: two state buffers, plus W^{n-1} and the
// filter sums for the four-cell kernels
template <typename T, int ORDER, bool VARC, bool FORCED>
static size_t batch_smem() {
  return (kBQuad<T, ORDER, VARC, FORCED> ? 3 : 2) * (size_t)kBReg * kBReg * sizeof(T);
}

template <typename T, int ORDER, bool VARC>
static void block2d_attrs() {
  cudaFuncSetAttribute(k_batch_block2d<T, ORDER, VARC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)batch_smem<T, ORDER, VARC, false>());
  cudaFuncSetAttribute(k_batch_block2d<T, ORDER, VARC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)batch_smem<T, ORDER, VARC, true>());
}
static void batch_init() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_batch_block2d_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       2 * kBReg * kBReg * (int)sizeof(dfl));
  cudaFuncSetAttribute(k_batch_block2d_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       2 * kBReg * kBReg * (int)sizeof(dfl));
  block2d_attrs<float, 2, false>(); block2d_attrs<float, 2, true>();
  block2d_attrs<float, 4, false>(); block2d_attrs<float, 4, true>();
  block2d_attrs<double, 2, false>(); block2d_attrs<double, 2, true>();
  block2d_attrs<double, 4, false>(); block2d_attrs<double, 4, true>();
}

template <typename T>
static T cvt(double x) {
  if constexpr (std::is_same<T, dfl>::value) return df_from(x);
  else return (T)x;
}

template <bool FORCED>
static cudaError_t launch_block2d_df(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  const BTile<dfl>* P = (const BTile<dfl>*)w.desc;
  const dfl* wt = (const dfl*)w.wtab;
  const dfl* ph = (const dfl*)w.ptab;
  unsigned* bc = bar;
  unsigned* bg = bar + 1;
  int J = w.J, K = w.K;
  const int* na = w.nact;
  void* args[] = {(void*)&P, (void*)&na, (void*)&J, (void*)&K, (void*)&wt, (void*)&ph,
                  (void*)&bc, (void*)&bg, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_block2d_df<FORCED>, dim3(w.nblocks), dim3(kBThreads), args,
                                     w.smem, st);
}

// ------------------------------------------------------------------ TMA-fed role (host)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, fetched once through the runtime (no link to libcuda)
static EncodeTiledFn encode_tiled() { return (EncodeTiledFn)tensor_map_encoder(); }

// The FP32 f = 0 roles of 2-D second-order c = 1 batches: k = 8 runs the wavefront kernel
// (k_batch_front), k = 4 and 12 the TMA-fed staged kernel with two rows of cells per thread, other
// k k_batch_block2d; the forced FP32 role at k = 8 and the double-float roles run the two-column
// wavefront kernel (k_batch_front2).  WHV_BATCH_TMA in the environment is a diagnostic switch (0:
// k_batch_block2d / k_batch_block2d_df for every role; 1 or 2: the staged TMA-fed kernel with one
// or two rows per thread for the f = 0 FP32 roles at k = 4, 8, 12, the staged kernels otherwise):
// all of them give the same results bit for bit.
static int tma_env() {
  static const int env = [] { const char* e = getenv("WHV_BATCH_TMA"); return e ? atoi(e) : 3; }();
  return env;
}
static bool tma_role(int K, bool forced) {
  return tma_env() != 0 && !forced && K >= 4 && K <= 12 && K % 4 == 0 && encode_tiled() != nullptr;
}
static int tma_rows() { return tma_env() == 1 ? 1 : 2; }
// k = 8 takes the wavefront kernel (k_batch_front) unless WHV_BATCH_TMA is 0, 1 or 2
static bool front_role(int K, bool forced) { return tma_role(K, forced) && K == kFK && tma_env() >= 3; }

template <int K, int R>
static cudaError_t launch_tma(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  const BTileT* P = (const BTileT*)w.desc;
  const BMaps* M = (const BMaps*)w.maps;
  const float* wt = (const float*)w.wtab;
  unsigned* bc = bar;
  unsigned* bg = bar + 1;
  int J = w.J;
  const int* na = w.nact;
  void* args[] = {(void*)&P, (void*)&M, (void*)&na, (void*)&J, (void*)&wt, (void*)&bc, (void*)&bg, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_tma<K, R>, dim3(w.nblocks), dim3(kBThreads / R), args,
                                     w.smem, st);
}

template <int K, int R>
static cudaError_t tma_prepare(int* per_sm) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_batch_tma<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               TmaLayout<K>::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_tma<K, R>, kBThreads / R,
                                                       TmaLayout<K>::kSmem);
}

// pitched FP32 state buffers of a 2-D grid (rows padded to a multiple of 4 floats), on first use
static whv_status ensure_tma_buffers(whv_grid g) {
  if (g->tacc) return WHV_OK;
  const int pitch = (g->n[0] + 3) / 4 * 4;
  const size_t bytes = (size_t)pitch * g->n[1] * sizeof(float);
  for (int m = 0; m < 4; ++m) {
    WHV_CUDA(g, cudaMalloc(&g->tw[m], bytes));
    WHV_CUDA(g, cudaMemsetAsync(g->tw[m], 0, bytes, g->stream));
  }
  WHV_CUDA(g, cudaMalloc(&g->tacc, bytes));
  WHV_CUDA(g, cudaMemsetAsync(g->tacc, 0, bytes, g->stream));
  g->tpitch = pitch;
  return WHV_OK;
}

static bool encode_box(CUtensorMap* map, float* base, int nx, int ny, int pitch, int box) {
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  const cuuint32_t boxd[2] = {(cuuint32_t)box, (cuuint32_t)box};
  const cuuint32_t es[2] = {1, 1};
  return encode_tiled()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, boxd, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// descriptor and tensor-map tables of the TMA-fed role; problems ordered by sweeps (descending)
static whv_status make_wave_tma(BatchCtx& c, const RoleIO& io, int K, Wave* out) {
  const int np = c.np;
  Wave w;
  w.K = K;
  std::vector<int> order(np), nsw(np);
  for (int p = 0; p < np; ++p) nsw[p] = (c.tgs[p].nt + K - 1) / K;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nsw[a] > nsw[b]; });
  w.J = nsw[order[0]];
  const int TW = kBReg - 2 * K;
  std::vector<float> wtab;
  std::vector<BFin> fin(np);
  std::vector<BTileT> d(np);
  std::vector<BMaps> maps(np);
  int64_t tile0 = 0;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = c.grids[p];
    const TimeGridH& tg = c.tgs[p];
    TRY(ensure_tma_buffers(g));
    const int wofs = (int)wtab.size();
    for (int n = 0; n <= tg.nt; ++n) wtab.push_back((float)tg.weight[n]);
    const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
    BTileT B{};
    for (int m = 0; m < 4; ++m) B.w[m] = g->tw[m];
    B.acc = g->tacc;
    B.v = io.v[p]; B.out = io.out[p];
    B.mw = g->mw; B.partials = chan(g, CH_STEP);
    B.halt = io.halt ? g->scal + S_HALT : nullptr;
    B.nx = g->n[0]; B.ny = g->n[1]; B.nt = tg.nt; B.pitch = g->tpitch;
    B.tiles_x = (g->n[0] + TW - 1) / TW;
    B.ntiles = B.tiles_x * ((g->n[1] + TW - 1) / TW);
    B.epi = io.epi; B.wofs = wofs;
    B.ih2x = (float)(1.0 / h2x);
    B.ih2y = (float)(1.0 / h2y);
    B.dt2 = (float)(tg.dt * tg.dt);
    const double ax = tg.dt * tg.dt / h2x, ay = tg.dt * tg.dt / h2y;
    B.ax = (float)ax; B.ay = (float)ay; B.b = (float)(2.0 - 2.0 * (ax + ay));
    B.tile0 = tile0;
    for (int m = 0; m < 4; ++m)
      if (!encode_box(&maps[k].w[m], g->tw[m], g->n[0], g->n[1], g->tpitch, kBReg))
        return fail(c.g0, WHV_ERR_CUDA, "batched: cuTensorMapEncodeTiled failed (state buffers)");
    if (!encode_box(&maps[k].acc, g->tacc, g->n[0], g->n[1], g->tpitch, TW))
      return fail(c.g0, WHV_ERR_CUDA, "batched: cuTensorMapEncodeTiled failed (filter sums)");
    if (io.epi == 1 && B.ntiles > chan_cap(g, CH_STEP))
      return fail(c.g0, WHV_ERR_INVALID, "batched: grid too large for its reduction channel");
    fin[k] = BFin{chan(g, CH_STEP), io.halt ? g->scal + S_HALT : nullptr, g->scal, B.ntiles};
    d[k] = B;
    tile0 += B.ntiles;
  }
  std::vector<int> nact(w.J);
  for (int j = 0; j < w.J; ++j) {
    int a = 0;
    while (a < np && nsw[order[a]] > j) ++a;
    nact[j] = a;
  }
  B_CUDA(c.g0, c.alloc(&w.desc, np * sizeof(BTileT)));
  B_CUDA(c.g0, c.alloc(&w.maps, np * sizeof(BMaps)));
  B_CUDA(c.g0, c.alloc(&w.nact, w.J * sizeof(int)));
  B_CUDA(c.g0, c.alloc(&w.wtab, wtab.size() * sizeof(float)));
  B_CUDA(c.g0, c.alloc(&w.fin, np * sizeof(BFin)));
  B_CUDA(c.g0, cudaMemcpy(w.desc, d.data(), np * sizeof(BTileT), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.maps, maps.data(), np * sizeof(BMaps), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.nact, nact.data(), w.J * sizeof(int), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.wtab, wtab.data(), wtab.size() * sizeof(float), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.fin, fin.data(), np * sizeof(BFin), cudaMemcpyHostToDevice));
  int per_sm = 0;
  // rows of four cells per thread: 2 (512 threads, two CTAs per SM) unless WHV_BATCH_TMA=1
  const bool duo = tma_rows() == 2;
#define TMA_CASE(KK)                                                                                \
  if (duo) { B_CUDA(c.g0, (tma_prepare<KK, 2>(&per_sm))); w.launch = &launch_tma<KK, 2>; }          \
  else { B_CUDA(c.g0, (tma_prepare<KK, 1>(&per_sm))); w.launch = &launch_tma<KK, 1>; }              \
  w.smem = TmaLayout<KK>::kSmem;
  switch (K) {
    case 4: { TMA_CASE(4) break; }
    case 8: { TMA_CASE(8) break; }
    default: { TMA_CASE(12) break; }
  }
#undef TMA_CASE
  if (per_sm < 1) return fail(c.g0, WHV_ERR_INVALID, "batched: kernel cannot be resident on an SM");
  w.nblocks = (int)std::min<int64_t>((int64_t)per_sm * c.sms, std::max<int64_t>(tile0, 1));
  *out = w;
  return WHV_OK;
}

// ------------------------------------------------------------------ wavefront role (host)
static cudaError_t launch_front(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  (void)bar;   // no grid barrier: per-problem completion counters, zeroed before every launch
  const BTileT* P = (const BTileT*)w.desc;
  const BMapsF* M = (const BMapsF*)w.maps;
  const float* wt = (const float*)w.wtab;
  int J = w.J;
  const int* na = w.nact;
  const int64_t* jo = w.joff;
  const int64_t* job = w.joffb;
  int rm = w.rows_mode;
  unsigned* pc = w.pcnt;
  const cudaError_t e = cudaMemsetAsync(w.pcnt, 0, w.np * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&P,   (void*)&M,  (void*)&na, (void*)&J,  (void*)&jo,
                  (void*)&job, (void*)&rm, (void*)&pc, (void*)&wt, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_front, dim3(w.nblocks), dim3(kFWarps * 32), args, w.smem,
                                     st);
}

static bool encode_rows(CUtensorMap* map, float* base, int nx, int ny, int pitch, int boxw) {
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  const cuuint32_t boxd[2] = {(cuuint32_t)boxw, (cuuint32_t)kFRB};
  const cuuint32_t es[2] = {1, 1};
  return encode_tiled()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, boxd, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// descriptor and tensor-map tables of the wavefront role (k = kFK); problems ordered by sweeps
static whv_status make_wave_front(BatchCtx& c, const RoleIO& io, Wave* out) {
  const int np = c.np;
  const int K = kFK;
  Wave w;
  w.K = K;
  std::vector<int> order(np), nsw(np);
  for (int p = 0; p < np; ++p) nsw[p] = (c.tgs[p].nt + K - 1) / K;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nsw[a] > nsw[b]; });
  w.J = nsw[order[0]];
  std::vector<float> wtab;
  std::vector<BFin> fin(np);
  std::vector<BTileT> d(np);
  std::vector<BMapsF> maps(np);
  int64_t tile0 = 0, tile0b = 0;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = c.grids[p];
    const TimeGridH& tg = c.tgs[p];
    TRY(ensure_tma_buffers(g));
    const int wofs = (int)wtab.size();
    for (int n = 0; n <= tg.nt; ++n) wtab.push_back((float)tg.weight[n]);
    // K extra zero weights: the last sweep may read beyond the problem's nt
    for (int n = 0; n < K; ++n) wtab.push_back(0.0f);
    const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
    BTileT B{};
    for (int m = 0; m < 4; ++m) B.w[m] = g->tw[m];
    B.acc = g->tacc;
    B.v = io.v[p]; B.out = io.out[p];
    B.mw = g->mw; B.partials = chan(g, CH_STEP);
    B.halt = io.halt ? g->scal + S_HALT : nullptr;
    B.nx = g->n[0]; B.ny = g->n[1]; B.nt = tg.nt; B.pitch = g->tpitch;
    B.tiles_x = (g->n[0] + kFTW - 1) / kFTW;
    B.ntiles = B.tiles_x * ((g->n[1] + kFS - 1) / kFS);
    B.ntilesb = B.tiles_x * ((g->n[1] + 2 * kFS - 1) / (2 * kFS));
    B.epi = io.epi; B.wofs = wofs;
    B.ih2x = (float)(1.0 / h2x);
    B.ih2y = (float)(1.0 / h2y);
    B.dt2 = (float)(tg.dt * tg.dt);
    const double ax = tg.dt * tg.dt / h2x, ay = tg.dt * tg.dt / h2y;
    B.ax = (float)ax; B.ay = (float)ay; B.b = (float)(2.0 - 2.0 * (ax + ay));
    B.tile0 = tile0;
    B.tile0b = tile0b;
    for (int m = 0; m < 4; ++m)
      if (!encode_rows(&maps[k].w[m], g->tw[m], g->n[0], g->n[1], g->tpitch, kFW))
        return fail(c.g0, WHV_ERR_CUDA, "batched: cuTensorMapEncodeTiled failed (state buffers)");
    if (!encode_rows(&maps[k].acc, g->tacc, g->n[0], g->n[1], g->tpitch, kFTW))
      return fail(c.g0, WHV_ERR_CUDA, "batched: cuTensorMapEncodeTiled failed (filter sums)");
    if (io.epi == 1 && B.ntiles > chan_cap(g, CH_STEP))
      return fail(c.g0, WHV_ERR_INVALID, "batched: grid too large for its reduction channel");
    fin[k] = BFin{chan(g, CH_STEP), io.halt ? g->scal + S_HALT : nullptr, g->scal, B.ntiles};
    d[k] = B;
    tile0 += B.ntiles;
    tile0b += B.ntilesb;
  }
  std::vector<int> nact(w.J);
  for (int j = 0; j < w.J; ++j) {
    int a = 0;
    while (a < np && nsw[order[a]] > j) ++a;
    nact[j] = a;
  }
  // strips of sweep j: those of its active problems (work items of kFS and of 2 kFS rows)
  std::vector<int64_t> joff(w.J + 1, 0), joffb(w.J + 1, 0);
  for (int j = 0; j < w.J; ++j) {
    joff[j + 1] = joff[j] + (nact[j] < np ? d[nact[j]].tile0 : tile0);
    joffb[j + 1] = joffb[j] + (nact[j] < np ? d[nact[j]].tile0b : tile0b);
  }
  B_CUDA(c.g0, c.alloc(&w.joff, (w.J + 1) * sizeof(int64_t)));
  B_CUDA(c.g0, c.alloc(&w.joffb, (w.J + 1) * sizeof(int64_t)));
  B_CUDA(c.g0, c.alloc(&w.pcnt, np * sizeof(unsigned)));
  B_CUDA(c.g0, cudaMemcpy(w.joff, joff.data(), (w.J + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.joffb, joffb.data(), (w.J + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  w.np = np;
  // WHV_FRONT_ROWS in the environment fixes the item height (128 or 256 rows; a diagnostic and
  // test switch: both give the same wave-solve outputs bit for bit)
  {
    const char* e = getenv("WHV_FRONT_ROWS");
    const int r = e ? atoi(e) : 0;
    w.rows_mode = r == kFS ? 1 : (r == 2 * kFS ? 2 : 0);
  }
  B_CUDA(c.g0, c.alloc(&w.desc, np * sizeof(BTileT)));
  B_CUDA(c.g0, c.alloc(&w.maps, np * sizeof(BMapsF)));
  B_CUDA(c.g0, c.alloc(&w.nact, w.J * sizeof(int)));
  B_CUDA(c.g0, c.alloc(&w.wtab, wtab.size() * sizeof(float)));
  B_CUDA(c.g0, c.alloc(&w.fin, np * sizeof(BFin)));
  B_CUDA(c.g0, cudaMemcpy(w.desc, d.data(), np * sizeof(BTileT), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.maps, maps.data(), np * sizeof(BMapsF), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.nact, nact.data(), w.J * sizeof(int), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.wtab, wtab.data(), wtab.size() * sizeof(float), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.fin, fin.data(), np * sizeof(BFin), cudaMemcpyHostToDevice));
  static bool attr = false;
  if (!attr) {
    B_CUDA(c.g0, cudaFuncSetAttribute(k_batch_front, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmem));
    attr = true;
  }
  int per_sm = 0;
  B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_front, kFWarps * 32, kFSmem));
  if (per_sm < 1) return fail(c.g0, WHV_ERR_INVALID, "batched: kernel cannot be resident on an SM");
  w.smem = kFSmem;
  w.launch = &launch_front;
  w.nblocks = (int)std::min<int64_t>((int64_t)per_sm * c.sms, std::max<int64_t>((tile0 + kFWarps - 1) / kFWarps, 1));
  *out = w;
  return WHV_OK;
}

constexpr int kBDfK = 4;   // sub-steps per sweep of the double-float roles

// Device tables of one role, stepping in T (double on an FP32 grid: its FP64 buffer set; dfl:
// double-float pairs in the same 8-byte buffers, 2-D second order with c = 1 only).
// Problems are ordered by their number of sweeps (descending), so the active problems of sweep j
// are a prefix.
// ------------------------------------------------------------------ two-column wavefront roles (host)
template <typename T, int K, bool FORCED>
static cudaError_t launch_front2(cudaStream_t st, const Wave& w, unsigned* bar, int* err) {
  (void)bar;   // no grid barrier: per-problem completion counters, zeroed before every launch
  const BTile<T>* P = (const BTile<T>*)w.desc;
  const T* wt = (const T*)w.wtab;
  const T* ph = (const T*)w.ptab;
  int J = w.J;
  const int* na = w.nact;
  const int64_t* jo = w.joff;
  unsigned* pc = w.pcnt;
  const cudaError_t e = cudaMemsetAsync(w.pcnt, 0, w.np * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&P, (void*)&na, (void*)&J, (void*)&jo, (void*)&pc, (void*)&wt, (void*)&ph, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_front2<T, K, FORCED>, dim3(w.nblocks), dim3(kDWarps * 32),
                                     args, 0, st);
}

// descriptor tables of a two-column wavefront role (strips of 64 columns x kDS rows, K levels per
// sweep): T = dfl the double-float roles in the grids' 8-byte buffers, T = float the FP32 roles in
// their FP32 buffers
template <typename T, int K>
static whv_status make_wave_front2(BatchCtx& c, const RoleIO& io, bool forced, Wave* out) {
  constexpr bool DF = std::is_same<T, dfl>::value;
  constexpr int TW = wf_tw<K>();
  const int np = c.np;
  Wave w;
  w.K = K;
  std::vector<int> order(np), nsw(np);
  for (int p = 0; p < np; ++p) nsw[p] = (c.tgs[p].nt + K - 1) / K;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nsw[a] > nsw[b]; });
  w.J = nsw[order[0]];
  std::vector<T> wtab, ptab;
  std::vector<BFin> fin(np);
  std::vector<BTile<T>> d(np);
  int64_t tile0 = 0;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = c.grids[p];
    const TimeGridH& tg = c.tgs[p];
    void* const* bufs = DF ? g->wbuf64 : g->wbuf;
    void* const accb = DF ? g->acc64 : g->acc;
    if (!accb || !bufs[0]) return fail(c.g0, WHV_ERR_INVALID, "batched: stepping buffers missing");
    const int wofs = (int)wtab.size();
    for (int n = 0; n <= tg.nt; ++n) {
      wtab.push_back(cvt<T>(tg.weight[n]));
      ptab.push_back(cvt<T>(DF ? tg.dt * tg.dt * tg.phase[n] : tg.phase[n]));
    }
    for (int n = 0; n < K; ++n) {   // the last sweep may read past the problem's nt
      wtab.push_back(cvt<T>(0.0));
      ptab.push_back(cvt<T>(0.0));
    }
    const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
    BTile<T> B{};
    for (int m = 0; m < 4; ++m) B.w[m] = (T*)bufs[m];
    B.acc = (T*)accb;
    B.v = io.v[p]; B.f = io.f[p]; B.out = io.out[p];
    B.c2 = nullptr; B.mw = g->mw; B.partials = chan(g, CH_STEP);
    B.halt = io.halt ? g->scal + S_HALT : nullptr;
    B.nx = g->n[0]; B.ny = g->n[1]; B.nt = tg.nt;
    B.tiles_x = (g->n[0] + TW - 1) / TW;
    B.ntiles = B.tiles_x * ((g->n[1] + kDS - 1) / kDS);
    B.epi = io.epi; B.wofs = wofs;
    B.ih2x = cvt<T>(1.0 / h2x);
    B.ih2y = cvt<T>(1.0 / h2y);
    B.dt2 = cvt<T>(tg.dt * tg.dt);
    const double ax = tg.dt * tg.dt / h2x, ay = tg.dt * tg.dt / h2y;
    B.ax = cvt<T>(ax); B.ay = cvt<T>(ay); B.b = cvt<T>(2.0 - 2.0 * (ax + ay));
    B.tile0 = tile0;
    if (io.epi == 1 && B.ntiles > chan_cap(g, CH_STEP))
      return fail(c.g0, WHV_ERR_INVALID, "batched: grid too large for its reduction channel");
    fin[k] = BFin{chan(g, CH_STEP), io.halt ? g->scal + S_HALT : nullptr, g->scal, B.ntiles};
    d[k] = B;
    tile0 += B.ntiles;
  }
  std::vector<int> nact(w.J);
  for (int j = 0; j < w.J; ++j) {
    int a = 0;
    while (a < np && nsw[order[a]] > j) ++a;
    nact[j] = a;
  }
  std::vector<int64_t> joff(w.J + 1, 0);   // strips of sweep j: those of its active problems
  for (int j = 0; j < w.J; ++j) joff[j + 1] = joff[j] + (nact[j] < np ? d[nact[j]].tile0 : tile0);
  B_CUDA(c.g0, c.alloc(&w.desc, np * sizeof(BTile<T>)));
  B_CUDA(c.g0, c.alloc(&w.nact, w.J * sizeof(int)));
  B_CUDA(c.g0, c.alloc(&w.joff, (w.J + 1) * sizeof(int64_t)));
  B_CUDA(c.g0, c.alloc(&w.pcnt, np * sizeof(unsigned)));
  B_CUDA(c.g0, c.alloc(&w.wtab, wtab.size() * sizeof(T)));
  B_CUDA(c.g0, c.alloc(&w.ptab, ptab.size() * sizeof(T)));
  B_CUDA(c.g0, c.alloc(&w.fin, np * sizeof(BFin)));
  B_CUDA(c.g0, cudaMemcpy(w.desc, d.data(), np * sizeof(BTile<T>), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.nact, nact.data(), w.J * sizeof(int), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.joff, joff.data(), (w.J + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.wtab, wtab.data(), wtab.size() * sizeof(T), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.ptab, ptab.data(), ptab.size() * sizeof(T), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.fin, fin.data(), np * sizeof(BFin), cudaMemcpyHostToDevice));
  w.np = np;
  int per_sm = 0;
  if (forced) {
    w.launch = &launch_front2<T, K, true>;
    B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_front2<T, K, true>, kDWarps * 32, 0));
  } else {
    w.launch = &launch_front2<T, K, false>;
    B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_front2<T, K, false>, kDWarps * 32, 0));
  }
  if (per_sm < 1) return fail(c.g0, WHV_ERR_INVALID, "batched: kernel cannot be resident on an SM");
  w.smem = 0;
  w.nblocks = (int)std::min<int64_t>((int64_t)per_sm * c.sms, std::max<int64_t>((tile0 + kDWarps - 1) / kDWarps, 1));
  *out = w;
  return WHV_OK;
}

template <typename T, int DIM, int ORDER, bool VARC>
static whv_status make_wave(BatchCtx& c, const RoleIO& io, Wave* out) {
  const int np = c.np;
  const bool fp64 = sizeof(T) == 8;
  const bool blocked = DIM == 2;
  bool forced = false;
  for (const double* f : io.f) forced = forced || f != nullptr;
  constexpr bool DF = std::is_same<T, dfl>::value;
  static_assert(!DF || (DIM == 2 && ORDER == 2 && !VARC), "double-float roles: 2-D, second order, c = 1");
  Wave w;
  w.K = DF ? kBDfK : (blocked ? batch_k(c.g0, fp64) : 1);
  if constexpr (std::is_same<T, float>::value && DIM == 2 && ORDER == 2 && !VARC) {
    if (front_role(w.K, forced)) return make_wave_front(c, io, out);
    else if (tma_role(w.K, forced)) return make_wave_tma(c, io, w.K, out);
    else if (forced && w.K == kFK && tma_env() >= 3) return make_wave_front2<float, kFK>(c, io, true, out);
  }
  if constexpr (DF)
    if (tma_env() >= 3) return make_wave_front2<dfl, kDK>(c, io, forced, out);
  std::vector<int> order(np), nsw(np);
  for (int p = 0; p < np; ++p) nsw[p] = (c.tgs[p].nt + w.K - 1) / w.K;
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nsw[a] > nsw[b]; });
  w.J = nsw[order[0]];
  std::vector<T> wtab, ptab;
  std::vector<BFin> fin(np);
  std::vector<BTile<T>> d2(blocked ? np : 0);
  std::vector<BProb<T>> d3(blocked ? 0 : np);
  int64_t tile0 = 0;
  const int R = ORDER == 2 ? 1 : 2;
  const int TW = kBReg - 2 * w.K * R;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = c.grids[p];
    const TimeGridH& tg = c.tgs[p];
    const bool other = fp64 && g->precision != WHV_FP64;
    void* const* bufs = other ? g->wbuf64 : g->wbuf;
    void* accb = other ? g->acc64 : g->acc;
    if (!accb || !bufs[0]) return fail(c.g0, WHV_ERR_INVALID, "batched: stepping buffers missing");
    const T* c2 = VARC ? (const T*)(fp64 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
    const int wofs = (int)wtab.size();
    for (int n = 0; n <= tg.nt; ++n) {
      wtab.push_back(cvt<T>(tg.weight[n]));
      // double-float steps take the forcing factor dt^2 cos(omega_hat t^n) whole
      ptab.push_back(cvt<T>(DF ? tg.dt * tg.dt * tg.phase[n] : tg.phase[n]));
    }
    const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
    int ntiles = 0;
    if constexpr (DIM == 2) {
      BTile<T> B{};
      for (int m = 0; m < 4; ++m) B.w[m] = (T*)bufs[m];
      B.acc = (T*)accb;
      B.v = io.v[p]; B.f = io.f[p]; B.out = io.out[p];
      B.c2 = c2; B.mw = g->mw; B.partials = chan(g, CH_STEP);
      B.halt = io.halt ? g->scal + S_HALT : nullptr;
      B.nx = g->n[0]; B.ny = g->n[1]; B.nt = tg.nt;
      B.tiles_x = (g->n[0] + TW - 1) / TW;
      B.ntiles = B.tiles_x * ((g->n[1] + TW - 1) / TW);
      B.epi = io.epi; B.wofs = wofs;
      B.ih2x = cvt<T>(ORDER == 2 ? 1.0 / h2x : 1.0 / (12.0 * h2x));
      B.ih2y = cvt<T>(ORDER == 2 ? 1.0 / h2y : 1.0 / (12.0 * h2y));
      B.dt2 = cvt<T>(tg.dt * tg.dt);
      const double ax = tg.dt * tg.dt / h2x, ay = tg.dt * tg.dt / h2y;
      B.ax = cvt<T>(ax); B.ay = cvt<T>(ay); B.b = cvt<T>(2.0 - 2.0 * (ax + ay));
      B.tile0 = tile0;
      ntiles = B.ntiles;
      d2[k] = B;
    } else {
      if (!bufs[1]) return fail(c.g0, WHV_ERR_INVALID, "batched: stepping buffers missing");
      BProb<T> B{};
      B.w0 = (T*)bufs[0]; B.w1 = (T*)bufs[1]; B.acc = (T*)accb;
      B.v = io.v[p]; B.f = io.f[p]; B.out = io.out[p];
      B.c2 = c2; B.mw = g->mw; B.partials = chan(g, CH_STEP);
      B.halt = io.halt ? g->scal + S_HALT : nullptr;
      B.nx = g->n[0]; B.ny = g->n[1]; B.nz = g->n[2]; B.nt = tg.nt;
      B.tx = (g->n[0] + 31) / 32; B.ty = (g->n[1] + 7) / 8;
      B.ntiles = B.tx * B.ty * g->n[2];
      B.epi = io.epi; B.wofs = wofs;
      for (int m = 0; m < 3; ++m) {
        const double h2 = g->h[m] * g->h[m];
        B.cf.ih2[m] = (T)(ORDER == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2));
      }
      B.cf.dt2 = (T)(tg.dt * tg.dt);
      B.tile0 = tile0;
      ntiles = B.ntiles;
      d3[k] = B;
    }
    if (io.epi == 1 && ntiles > chan_cap(g, CH_STEP))
      return fail(c.g0, WHV_ERR_INVALID, "batched: grid too large for its reduction channel");
    fin[k] = BFin{chan(g, CH_STEP), io.halt ? g->scal + S_HALT : nullptr, g->scal, ntiles};
    tile0 += ntiles;
  }
  std::vector<int> nact(w.J);
  for (int j = 0; j < w.J; ++j) {
    int a = 0;
    while (a < np && nsw[order[a]] > j) ++a;
    nact[j] = a;
  }
  const size_t dbytes = blocked ? np * sizeof(BTile<T>) : np * sizeof(BProb<T>);
  B_CUDA(c.g0, c.alloc(&w.desc, dbytes));
  B_CUDA(c.g0, c.alloc(&w.nact, w.J * sizeof(int)));
  B_CUDA(c.g0, c.alloc(&w.wtab, wtab.size() * sizeof(T)));
  B_CUDA(c.g0, c.alloc(&w.ptab, ptab.size() * sizeof(T)));
  B_CUDA(c.g0, c.alloc(&w.fin, np * sizeof(BFin)));
  B_CUDA(c.g0, cudaMemcpy(w.desc, blocked ? (const void*)d2.data() : (const void*)d3.data(), dbytes,
                          cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.nact, nact.data(), w.J * sizeof(int), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.wtab, wtab.data(), wtab.size() * sizeof(T), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.ptab, ptab.data(), ptab.size() * sizeof(T), cudaMemcpyHostToDevice));
  B_CUDA(c.g0, cudaMemcpy(w.fin, fin.data(), np * sizeof(BFin), cudaMemcpyHostToDevice));
  int per_sm = 0;
  if constexpr (DF) {
    w.smem = 2 * (size_t)kBReg * kBReg * sizeof(dfl);
    if (forced) {
      w.launch = &launch_block2d_df<true>;
      B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_block2d_df<true>, kBThreads, w.smem));
    } else {
      w.launch = &launch_block2d_df<false>;
      B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_block2d_df<false>, kBThreads, w.smem));
    }
  } else if (blocked) {
    w.smem = forced ? batch_smem<T, ORDER, VARC, true>() : batch_smem<T, ORDER, VARC, false>();
    if (forced) {
      w.launch = &launch_block2d<T, ORDER, VARC, true>;
      B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_block2d<T, ORDER, VARC, true>,
                                                                 kBThreads, w.smem));
    } else {
      w.launch = &launch_block2d<T, ORDER, VARC, false>;
      B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_block2d<T, ORDER, VARC, false>,
                                                                 kBThreads, w.smem));
    }
  } else {
    w.launch = &launch_wave3<T, DIM, ORDER, VARC>;
    B_CUDA(c.g0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_wave<T, DIM, ORDER, VARC>, 256, 0));
  }
  if (per_sm < 1) return fail(c.g0, WHV_ERR_INVALID, "batched: kernel cannot be resident on an SM");
  w.nblocks = (int)std::min<int64_t>((int64_t)per_sm * c.sms, std::max<int64_t>(tile0, 1));
  *out = w;
  return WHV_OK;
}

static whv_status run_wave(BatchCtx& c, const Wave& w) {
  const cudaError_t e = w.launch(c.st, w, c.bar, c.err);
  if (e != cudaSuccess) return cuda_fail(c.g0, e, "batched wave solve launch");
  ++c.launches;
  return WHV_OK;
}

// The barrier error flag starts at zero, or raised (any nonzero value) when whv_inject_barrier_error
// marked one of the grids: then every CTA of the first batched wave solve leaves at its first grid
// barrier exactly as after a wait that gave up, and the call reports WHV_ERR_TIMEOUT.
static cudaError_t clear_err(BatchCtx& c) {
  bool fault = false;
  for (int p = 0; p < c.np; ++p) {
    fault = fault || c.grids[p]->barrier_fault;
    c.grids[p]->barrier_fault = false;
  }
  return cudaMemsetAsync(c.err, fault ? 0x01 : 0, sizeof(int), c.st);
}

static whv_status check_barrier(BatchCtx& c) {
  int herr = 0;
  B_CUDA(c.g0, cudaMemcpyAsync(&herr, c.err, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  B_CUDA(c.g0, cudaStreamSynchronize(c.st));
  if (herr) return fail(c.g0, WHV_ERR_TIMEOUT, "batched wave solve: a grid barrier timed out");
  return WHV_OK;
}

// all problems' scalar blocks -> host (one synchronisation)
static whv_status fetch_all(BatchCtx& c) {
  for (int p = 0; p < c.np; ++p) {
    whv_grid g = c.grids[p];
    B_CUDA(c.g0, cudaMemcpyAsync(g->scal_host, g->scal, S_NSLOTS * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  }
  B_CUDA(c.g0, cudaStreamSynchronize(c.st));
  return WHV_OK;
}

// Problems whose grids share one dense basis (whv_share_basis) form a group: its deflation
// projections and expansions are single contractions over the group's right-hand sides, reading
// the basis once (project_many / expand_many).  A grid with its own basis is a group of one;
// SVD-compressed bases take the per-problem contractions.
struct BasisGroup {
  const double* V = nullptr;
  int nd = 0;
  int64_t N = 0;
  const double* mw = nullptr;
  std::vector<int> members;
  double* C = nullptr;          // nd x k coefficients (column j = member j of the call)
  double* s_inf = nullptr;      // 1 / (omega_eff^2 - lambda^2): DEVD inflation
  double* s_mu = nullptr;       // 1 / mu: modal correction of the FP64 residual
};

struct Groups {
  std::vector<BasisGroup> g;
  std::vector<int> loose;       // problems with a compressed basis (per-problem contractions)
  double* partials = nullptr;
  const double** ptrs = nullptr;   // device: 2 np pointer slots
  std::vector<const double*> hptrs;
};

static whv_status make_groups(BatchCtx& c, Groups* G) {
  for (int p = 0; p < c.np; ++p) {
    const Basis& B = c.grids[p]->basis;
    if (B.nd == 0) continue;
    if (!B.V) { G->loose.push_back(p); continue; }
    BasisGroup* bg = nullptr;
    for (auto& x : G->g)
      if (x.V == B.V) bg = &x;
    if (!bg) {
      G->g.emplace_back();
      bg = &G->g.back();
      bg->V = B.V; bg->nd = B.nd; bg->N = c.grids[p]->N; bg->mw = c.grids[p]->mw;
    }
    bg->members.push_back(p);
  }
  int64_t scratch = 0;
  for (auto& bg : G->g) {
    const int k = (int)bg.members.size();
    const whv_grid g = c.grids[bg.members[0]];
    const Basis& B = g->basis;
    const TimeGridH& tg = c.tgs[bg.members[0]];
    scratch = std::max(scratch, project_many_scratch(bg.N, bg.nd, k));
    B_CUDA(c.g0, c.alloc(&bg.C, (size_t)bg.nd * k * sizeof(double)));
    B_CUDA(c.g0, c.alloc(&bg.s_inf, bg.nd * sizeof(double)));
    B_CUDA(c.g0, c.alloc(&bg.s_mu, bg.nd * sizeof(double)));
    std::vector<double> si(bg.nd), sm(bg.nd);
    const double om2 = tg.omega_eff * tg.omega_eff;
    for (int m = 0; m < bg.nd; ++m) {
      si[m] = 1.0 / (om2 - B.lambda2[m]);
      sm[m] = 1.0 / B.mu[m];
    }
    B_CUDA(c.g0, cudaMemcpy(bg.s_inf, si.data(), bg.nd * sizeof(double), cudaMemcpyHostToDevice));
    B_CUDA(c.g0, cudaMemcpy(bg.s_mu, sm.data(), bg.nd * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (!G->g.empty()) {
    B_CUDA(c.g0, c.alloc(&G->partials, (size_t)scratch * sizeof(double)));
    B_CUDA(c.g0, c.alloc(&G->ptrs, 2 * (size_t)c.np * sizeof(double*)));
  }
  return WHV_OK;
}

// the pointer slots as the output list of expand_many
static double* const* out_ptrs(Groups& G) { return (double* const*)(void*)G.ptrs; }

// upload the group's pointer lists a (slot 0) and b (slot 1): k entries each
static whv_status group_ptrs(BatchCtx& c, Groups& G, const std::vector<const double*>& a,
                             const std::vector<const double*>& b) {
  G.hptrs.assign(2 * (size_t)c.np, nullptr);
  std::copy(a.begin(), a.end(), G.hptrs.begin());
  std::copy(b.begin(), b.end(), G.hptrs.begin() + c.np);
  B_CUDA(c.g0, cudaMemcpyAsync(G.ptrs, G.hptrs.data(), 2 * (size_t)c.np * sizeof(double*), cudaMemcpyHostToDevice,
                               c.st));
  // pageable source: keep the copy ordered before the host reuses the vector
  B_CUDA(c.g0, cudaStreamSynchronize(c.st));
  return WHV_OK;
}

// For the members `who` of group bg: C = W^T M [in_j], then for each (alpha, scale, out) pass
// out_j += alpha W diag(scale) C_j -- one read of W per contraction for all members.
struct ExpandPass {
  double alpha;
  const double* scale;
  std::vector<double*> out;
};
static whv_status group_contract(BatchCtx& c, Groups& G, const BasisGroup& bg, const std::vector<const double*>& in,
                                 const std::vector<ExpandPass>& passes) {
  const int k = (int)in.size();
  if (k == 0) return WHV_OK;
  TRY(group_ptrs(c, G, in, {}));
  B_CUDA(c.g0, project_many(c.st, bg.V, bg.N, bg.nd, k, G.ptrs, bg.mw, G.partials, bg.C));
  for (const ExpandPass& ps : passes) {
    TRY(group_ptrs(c, G, std::vector<const double*>(ps.out.begin(), ps.out.end()), {}));
    B_CUDA(c.g0, expand_many(c.st, bg.V, bg.N, bg.nd, k, bg.C, ps.scale, ps.alpha, out_ptrs(G)));
  }
  return WHV_OK;
}

// The batched CG loop, built for the A p role `ap`: one graph with a WHILE node (device-resident
// loop), or -- with check_every > 1 -- a graph of one iteration that the host launches, testing
// convergence every check_every iterations.
struct CgGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t body_launches = 0;
  int check_every = 1;         // 1: device-resident loop
  ~CgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

static whv_status build_cg_graph(BatchCtx& c, const Wave& ap, int check_every, CgGraph* G) {
  G->check_every = std::max(1, check_every);
  const bool device_loop = G->check_every == 1;
  B_CUDA(c.g0, cudaGraphCreate(&G->graph, 0));
  cudaGraphConditionalHandle h = 0;
  cudaGraph_t body = G->graph;
  if (device_loop) {
    B_CUDA(c.g0, cudaGraphConditionalHandleCreate(&h, G->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    B_CUDA(c.g0, cudaGraphAddNode(&node, G->graph, nullptr, nullptr, 0, &prm));
    body = prm.conditional.phGraph_out[0];
  }
  // descriptor table of the batched CG updates (before the capture: no allocation inside it)
  int cg_blocks = 0;
  BCg* cgd = nullptr;
  {
    std::vector<BCg> d(c.np);
    for (int p = 0; p < c.np; ++p) {
      whv_grid g = c.grids[p];
      const int nb = (int)std::min<int64_t>(std::max<int64_t>((g->N + 255) / 256, 1), kRedBlocks);
      d[p] = BCg{g->x, g->r, g->p, g->q, g->mw, g->N, g->scal, chan(g, CH_UPDATE), g->counters + CH_UPDATE,
                 cg_blocks, nb};
      cg_blocks += nb;
    }
    B_CUDA(c.g0, c.alloc(&cgd, c.np * sizeof(BCg)));
    B_CUDA(c.g0, cudaMemcpy(cgd, d.data(), c.np * sizeof(BCg), cudaMemcpyHostToDevice));
  }
  B_CUDA(c.g0, cudaStreamBeginCaptureToGraph(c.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = whv_kernel_launches();
  whv_status s = WHV_OK;
  cudaError_t e = ap.launch(c.st, ap, c.bar, c.err);
  if (e == cudaSuccess) {
    k_batch_finish<<<c.np, 256, 0, c.st>>>(ap.fin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {   // the CG updates of all problems: one launch each
    k_batch_cg_update<<<cg_blocks, 256, 0, c.st>>>(cgd, c.np);
    k_batch_cg_direction<<<cg_blocks, 256, 0, c.st>>>(cgd, c.np);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && s == WHV_OK) {
    k_batch_check<<<(c.np + 127) / 128, 128, 0, c.st>>>(c.scal, c.np);
    if (device_loop) k_batch_any<<<1, 1, 0, c.st>>>(h, c.scal, c.np, c.err);
    e = cudaGetLastError();
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c.st, &captured);
  G->body_launches = (whv_kernel_launches() - l0) + (device_loop ? 6 : 5);   // wave, finish, 2 updates, check(, any)
  count_launches(-(whv_kernel_launches() - l0));
  if (s != WHV_OK) return s;
  if (e != cudaSuccess) return cuda_fail(c.g0, e, "batched loop body");
  if (e2 != cudaSuccess) return cuda_fail(c.g0, e2, "cudaStreamEndCapture (batched loop)");
  B_CUDA(c.g0, cudaGraphInstantiate(&G->exec, G->graph, 0));
  return WHV_OK;
}

// The batched CG loop on A x = rhs_p for the problems with active[p]: x = 0, r = p = rhs, stop
// once r^T M r <= stop[p] or after maxit[p] iterations.  iters[p] receives the iterations; the
// final r^T M r and the breakdown flag stay in the grids' scalar blocks (host mirrors fetched).
static whv_status run_cg(BatchCtx& c, CgGraph& G, const std::vector<const double*>& rhs,
                         const std::vector<double>& rr, const std::vector<double>& stop,
                         const std::vector<int>& maxit, const std::vector<char>& active, std::vector<int>* iters) {
  for (int p = 0; p < c.np; ++p) {
    whv_grid g = c.grids[p];
    double* sc = g->scal_host;
    sc[S_RR] = rr[p];
    sc[S_RR0] = rr[p];
    sc[S_FLAG] = 0.0;
    sc[S_ITER] = 0.0;
    sc[S_STOP] = stop[p];
    sc[S_MAXIT] = (double)maxit[p];
    sc[S_HALT] = (!active[p] || rr[p] == 0.0 || maxit[p] <= 0 || rr[p] <= stop[p]) ? 1.0 : 0.0;
    B_CUDA(c.g0, cudaMemsetAsync(g->x, 0, g->N * sizeof(double), c.st));
    if (active[p]) {
      B_CUDA(c.g0, cudaMemcpyAsync(g->r, rhs[p], g->N * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
      B_CUDA(c.g0, cudaMemcpyAsync(g->p, rhs[p], g->N * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    }
    B_CUDA(c.g0, cudaMemcpyAsync(g->scal, sc, S_NSLOTS * sizeof(double), cudaMemcpyHostToDevice, c.st));
  }
  int64_t body_runs = -1;
  if (G.check_every == 1) {
    B_CUDA(c.g0, cudaGraphLaunch(G.exec, c.st));
    TRY(check_barrier(c));
    TRY(fetch_all(c));
  } else {   // host-driven: stopped problems skip their work, so extra iterations are no-ops
    int mx = 0;
    for (int p = 0; p < c.np; ++p) mx = std::max(mx, active[p] ? maxit[p] : 0);
    body_runs = 0;
    bool any = false;
    for (int p = 0; p < c.np; ++p) any = any || c.grids[p]->scal_host[S_HALT] == 0.0;
    while (any && body_runs < mx) {
      for (int q = 0; q < G.check_every && body_runs < mx; ++q, ++body_runs)
        B_CUDA(c.g0, cudaGraphLaunch(G.exec, c.st));
      TRY(check_barrier(c));
      TRY(fetch_all(c));
      any = false;
      for (int p = 0; p < c.np; ++p) any = any || c.grids[p]->scal_host[S_HALT] == 0.0;
    }
  }
  int max_it = 0;
  for (int p = 0; p < c.np; ++p) {
    const int it = (int)c.grids[p]->scal_host[S_ITER];
    (*iters)[p] = it;
    max_it = std::max(max_it, it);
  }
  c.launches += G.body_launches * (body_runs >= 0 ? body_runs : max_it);
  return WHV_OK;
}

template <int DIM, int ORDER, bool VARC>
static whv_status batched_solve(BatchCtx& c, const double* const* f_dev, double* const* u_dev, bool refine,
                                whv_info* infos) {
  const int np = c.np;
  const bool g64 = c.g0->precision == WHV_FP64;
  std::vector<int> iters(np, 0), total_its(np, 0), outer(np, 0), ws(np, 0), ws64(np, 0);
  std::vector<double> rel(np, 0.0), true_rel(np, -1.0);
  std::vector<char> conv(np, 0), active(np, 1), flag(np, 0);

  // the A p role of the CG loop, in the grids' stepping precision
  RoleIO io_ap;
  io_ap.v = c.each([](whv_grid g) { return (const double*)g->p; });
  io_ap.f.assign(np, nullptr);
  io_ap.out = c.each([](whv_grid g) { return g->q; });
  io_ap.epi = 1;
  io_ap.halt = true;
  Wave ap;
  TRY(g64 ? (make_wave<double, DIM, ORDER, VARC>(c, io_ap, &ap)) : (make_wave<float, DIM, ORDER, VARC>(c, io_ap, &ap)));
  CgGraph CG;
  TRY(build_cg_graph(c, ap, c.params[0].check_every, &CG));
  Groups G;
  TRY(make_groups(c, &G));
  std::vector<int> maxit(np);
  for (int p = 0; p < np; ++p) maxit[p] = c.params[p].maxit;

  if (!refine) {
    // DEVD (Algorithm 2): deflate each forcing, b = Pi_h(0; f_d) of all problems in one launch
    std::vector<const double*> fd(f_dev, f_dev + np);
    for (const BasisGroup& bg : G.g) {   // f_d = f - W W^T M f, W read once per contraction
      std::vector<const double*> in;
      ExpandPass ps{-1.0, nullptr, {}};
      for (int p : bg.members) {
        whv_grid g = c.grids[p];
        TRY(copy_dev(g, g->fd, f_dev[p], g->N));
        in.push_back(f_dev[p]);
        ps.out.push_back(g->fd);
        fd[p] = g->fd;
      }
      TRY(group_contract(c, G, bg, in, {ps}));
    }
    for (int p : G.loose) {
      whv_grid g = c.grids[p];
      const Basis& B = g->basis;
      TRY(basis_project(g, f_dev[p], B.d_coef));
      TRY(copy_dev(g, g->fd, f_dev[p], g->N));
      TRY(basis_expand(g, B.d_coef, -1.0, g->fd));
      fd[p] = g->fd;
    }
    RoleIO io_b;
    io_b.v.assign(np, nullptr);
    io_b.f = fd;
    io_b.out = c.each([](whv_grid g) { return g->t; });
    Wave wb;
    TRY(g64 ? (make_wave<double, DIM, ORDER, VARC>(c, io_b, &wb)) : (make_wave<float, DIM, ORDER, VARC>(c, io_b, &wb)));
    c.mark(4);
    TRY(run_wave(c, wb));
    TRY(check_barrier(c));
    c.mark(0);
    for (int p = 0; p < np; ++p) TRY(dot_async(c.grids[p], c.grids[p]->t, c.grids[p]->t, S_TMP));
    TRY(fetch_all(c));
    std::vector<double> bb(np), stop(np);
    for (int p = 0; p < np; ++p) {
      bb[p] = c.grids[p]->scal_host[S_TMP];
      if (!isfinite(bb[p])) return fail(c.g0, WHV_ERR_BREAKDOWN, "batched: non-finite right-hand side");
      stop[p] = c.params[p].tol * c.params[p].tol * bb[p];
    }
    const std::vector<const double*> rhs = c.each([](whv_grid g) { return (const double*)g->t; });
    c.mark(4);
    TRY(run_cg(c, CG, rhs, bb, stop, maxit, active, &iters));
    c.mark(1);
    for (int p = 0; p < np; ++p) {
      whv_grid g = c.grids[p];
      total_its[p] = iters[p];
      ws[p] = iters[p] + 1;
      rel[p] = bb[p] > 0 ? sqrt(g->scal_host[S_RR] / bb[p]) : 0.0;
      flag[p] = g->scal_host[S_FLAG] != 0.0;
      conv[p] = !flag[p] && rel[p] <= c.params[p].tol;
    }
    // inflate: u = x + W diag(1/(omega_eff^2 - lambda^2)) W^T M f (the group's C still holds
    // W^T M f: the CG loop does not touch it)
    for (const BasisGroup& bg : G.g) {
      std::vector<double*> xs;
      for (int p : bg.members) xs.push_back(c.grids[p]->x);
      TRY(group_ptrs(c, G, std::vector<const double*>(xs.begin(), xs.end()), {}));
      B_CUDA(c.g0, expand_many(c.st, bg.V, bg.N, bg.nd, (int)xs.size(), bg.C, bg.s_inf, 1.0,
                               out_ptrs(G)));
    }
    for (int p : G.loose) {
      whv_grid g = c.grids[p];
      const Basis& B = g->basis;
      std::vector<double> cf(B.nd);
      TRY(to_host(g, cf.data(), B.d_coef, B.nd));
      const double om2 = c.tgs[p].omega_eff * c.tgs[p].omega_eff;
      for (int m = 0; m < B.nd; ++m) cf[m] /= (om2 - B.lambda2[m]);
      TRY(to_dev(g, g->small, cf.data(), B.nd));
      TRY(basis_expand(g, g->small, 1.0, g->x));
    }
    for (int p = 0; p < np; ++p) TRY(copy_dev(c.grids[p], u_dev[p], c.grids[p]->x, c.grids[p]->N));
  } else {
    // FP64 residual correction on the full system A u = b, b = Pi_h(0; f) in the stepping
    // precision, r = Pi_h(u; f) - u in FP64 (or double-float)
    for (int p = 0; p < np; ++p) TRY(ensure_fp64_buffers(c.grids[p]));
    RoleIO io_b;
    io_b.v.assign(np, nullptr);
    io_b.f.assign(f_dev, f_dev + np);
    io_b.out = c.each([](whv_grid g) { return g->bo; });
    RoleIO io_ax;   // q = u - Pi_h(u; f) = -r in FP64 (or double-float)
    io_ax.v = c.each([](whv_grid g) { return (const double*)g->xo; });
    io_ax.f.assign(f_dev, f_dev + np);
    io_ax.out = c.each([](whv_grid g) { return g->q; });
    io_ax.epi = 1;
    io_ax.halt = true;
    Wave wb, wax;
    bool dfr = false;   // double-float residual wave solves (WHV_RESIDUAL_DF64)
    if constexpr (DIM == 2 && ORDER == 2 && !VARC) dfr = (c.params[0].flags & WHV_RESIDUAL_DF64) != 0;
    if (g64) TRY((make_wave<double, DIM, ORDER, VARC>(c, io_b, &wb)));
    else TRY((make_wave<float, DIM, ORDER, VARC>(c, io_b, &wb)));
    if (dfr) {
      if constexpr (DIM == 2 && ORDER == 2 && !VARC) TRY((make_wave<dfl, 2, 2, false>(c, io_ax, &wax)));
    } else {
      TRY((make_wave<double, DIM, ORDER, VARC>(c, io_ax, &wax)));
    }
    c.mark(4);
    TRY(run_wave(c, wb));
    TRY(check_barrier(c));
    c.mark(0);
    for (int p = 0; p < np; ++p) {
      whv_grid g = c.grids[p];
      if (g64) ws64[p] = 1;
      else ws[p] = 1;
      TRY(dot_async(g, g->bo, g->bo, S_TMP2));
      B_CUDA(c.g0, cudaMemsetAsync(g->xo, 0, g->N * sizeof(double), c.st));
      TRY(copy_dev(g, g->ro, g->bo, g->N));
    }
    TRY(fetch_all(c));
    std::vector<double> bb(np), rr(np, 0.0), stop(np, 0.0);
    for (int p = 0; p < np; ++p) {
      bb[p] = c.grids[p]->scal_host[S_TMP2];
      if (!isfinite(bb[p])) return fail(c.g0, WHV_ERR_BREAKDOWN, "batched: non-finite right-hand side");
    }
    const std::vector<const double*> rhs = c.each([](whv_grid g) { return (const double*)g->ro; });
    for (int pass = 0;; ++pass) {
      if (pass > 0) {   // r = b - A x in FP64 for the problems still running
        for (int p = 0; p < np; ++p) {
          whv_grid g = c.grids[p];
          g->scal_host[S_HALT] = active[p] ? 0.0 : 1.0;
          B_CUDA(c.g0, cudaMemcpyAsync(g->scal + S_HALT, g->scal_host + S_HALT, sizeof(double),
                                       cudaMemcpyHostToDevice, c.st));
        }
        c.mark(4);
        TRY(run_wave(c, wax));
        TRY(check_barrier(c));
        c.mark(2);
        for (int p = 0; p < np; ++p) {
          if (!active[p]) continue;
          whv_grid g = c.grids[p];
          ++ws64[p];
          TRY(axpby(g, g->N, -1.0, g->q, 0.0, g->ro));   // r = Pi_h(x; f) - x
        }
      }
      for (int p = 0; p < np; ++p)
        if (active[p]) TRY(dot_async(c.grids[p], c.grids[p]->ro, c.grids[p]->ro, S_TMP2));
      TRY(fetch_all(c));
      bool any = false;
      for (int p = 0; p < np; ++p) {
        if (!active[p]) continue;
        const double r2 = c.grids[p]->scal_host[S_TMP2];
        rel[p] = bb[p] > 0 ? sqrt(r2 / bb[p]) : 0.0;
        true_rel[p] = rel[p];
        if (!isfinite(rel[p])) { flag[p] = 1; active[p] = 0; continue; }
        if (rel[p] <= c.params[p].tol) { conv[p] = 1; active[p] = 0; continue; }
        if (total_its[p] >= c.params[p].maxit || pass >= 50) { active[p] = 0; continue; }
        any = true;
      }
      if (!any) break;
      // deflated components (exact eigenvectors): x += W diag(1/mu) c, r -= W c, c = W^T M r
      c.mark(4);
      for (const BasisGroup& bg : G.g) {
        std::vector<const double*> in;
        ExpandPass px{1.0, bg.s_mu, {}}, pr{-1.0, nullptr, {}};
        for (int p : bg.members) {
          if (!active[p]) continue;
          whv_grid g = c.grids[p];
          in.push_back(g->ro);
          px.out.push_back(g->xo);
          pr.out.push_back(g->ro);
        }
        TRY(group_contract(c, G, bg, in, {px, pr}));
      }
      for (int p : G.loose) {
        whv_grid g = c.grids[p];
        const Basis& B = g->basis;
        if (!active[p] || B.nd == 0) continue;
        std::vector<double> cf(B.nd), y(B.nd);
        TRY(basis_project(g, g->ro, g->small));
        TRY(to_host(g, cf.data(), g->small, B.nd));
        for (int m = 0; m < B.nd; ++m) y[m] = cf[m] / B.mu[m];
        TRY(to_dev(g, g->small, y.data(), B.nd));
        TRY(basis_expand(g, g->small, 1.0, g->xo));
        TRY(to_dev(g, g->small, cf.data(), B.nd));
        TRY(basis_expand(g, g->small, -1.0, g->ro));
      }
      for (int p = 0; p < np; ++p)
        if (active[p]) TRY(dot_async(c.grids[p], c.grids[p]->ro, c.grids[p]->ro, S_TMP2));
      TRY(fetch_all(c));
      std::vector<int> mx(np, 0);
      for (int p = 0; p < np; ++p) {
        if (!active[p]) continue;
        const whv_params& P = c.params[p];
        rr[p] = c.grids[p]->scal_host[S_TMP2];
        const double itol = correction_tol(P.inner_tol > 0.0 ? P.inner_tol : 1e-3, P.tol, rel[p], pass);
        stop[p] = itol * itol * rr[p];
        mx[p] = P.maxit - total_its[p];
      }
      c.mark(3);
      TRY(run_cg(c, CG, rhs, rr, stop, mx, active, &iters));
      c.mark(1);
      for (int p = 0; p < np; ++p) {
        if (!active[p]) continue;
        whv_grid g = c.grids[p];
        total_its[p] += iters[p];
        ws[p] += iters[p];
        ++outer[p];
        TRY(axpby(g, g->N, 1.0, g->x, 1.0, g->xo));
        if (g->scal_host[S_FLAG] != 0.0) { flag[p] = 1; active[p] = 0; }
      }
    }
    for (int p = 0; p < np; ++p) TRY(copy_dev(c.grids[p], u_dev[p], c.grids[p]->xo, c.grids[p]->N));
  }
  c.mark(4);
  if (getenv("WHV_LOG") && getenv("WHV_LOG")[0] == '1')
    fprintf(stderr, "[whv] batched solve phases (s): b %.3f  CG loops %.3f  residual wave solves %.3f  "
                    "deflation %.3f  other %.3f\n", c.t_phase[0], c.t_phase[1], c.t_phase[2], c.t_phase[3],
            c.t_phase[4]);
  // leave the grids usable by non-batched calls
  for (int p = 0; p < np; ++p) {
    whv_grid g = c.grids[p];
    g->scal_host[S_HALT] = 0.0;
    B_CUDA(c.g0, cudaMemcpyAsync(g->scal + S_HALT, g->scal_host + S_HALT, sizeof(double), cudaMemcpyHostToDevice, c.st));
  }
  B_CUDA(c.g0, cudaStreamSynchronize(c.st));
  count_launches(c.launches);
  bool all = true;
  for (int p = 0; p < np; ++p) {
    all = all && conv[p];
    if (!infos) continue;
    whv_info& I = infos[p];
    I.iterations = total_its[p];
    I.wave_solves = ws[p] + ws64[p];
    I.wave_solves_fp64 = g64 ? ws[p] + ws64[p] : ws64[p];
    I.outer_iterations = outer[p];
    I.rel_residual = rel[p];
    I.true_rel_residual = true_rel[p];
    I.nt = c.tgs[p].nt;
    I.dt = c.tgs[p].dt;
    I.omega_hat = c.tgs[p].omega_hat;
    I.omega_eff = c.tgs[p].omega_eff;
    I.seconds = 0.0;
  }
  for (int p = 0; p < np; ++p)
    if (flag[p]) return fail(c.g0, WHV_ERR_BREAKDOWN, "whv_solve_batched: Krylov breakdown in a problem");
  if (!all) return fail(c.g0, WHV_ERR_NOT_CONVERGED, "whv_solve_batched: some problems did not reach tol");
  return WHV_OK;
}

template <int DIM, int ORDER>
static whv_status batched_vc(BatchCtx& c, const double* const* f, double* const* u, bool refine, whv_info* infos,
                             bool varc) {
  return varc ? batched_solve<DIM, ORDER, true>(c, f, u, refine, infos)
              : batched_solve<DIM, ORDER, false>(c, f, u, refine, infos);
}

}  // namespace whv

using namespace whv;

// Autotuner of the batched steps per sweep (2-D): one batched f = 0 wave solve of every problem
// (v = 0, into the grids' scratch) per candidate k, timed with CUDA events after a warm-up launch;
// the fastest k is stored in grids[0] (whv_set_steps_per_sweep), which the batched solve reads.
extern "C" whv_status whv_autotune_batched(int nprob, const whv_grid* grids, const whv_params* params, int* best) {
  if (nprob < 1 || nprob > kBatchMaxProblems || !grids || !params || !grids[0])
    return fail(nullptr, WHV_ERR_INVALID, "whv_autotune_batched: bad arguments (1 <= nprob <= 1024)");
  whv_grid g0 = grids[0];
  if (g0->dim != 2) {   // 3-D batches step once per sweep: nothing to tune
    if (best) *best = 1;
    return WHV_OK;
  }
  const bool varc = g0->c2 != nullptr;
  BatchCtx c;
  c.np = nprob;
  c.grids = grids;
  c.params = params;
  c.g0 = g0;
  c.tgs.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    whv_grid g = grids[p];
    if (!g || g->stream != g0->stream || g->precision != g0->precision || g->dim != 2 || g->order != g0->order ||
        (g->c2 != nullptr) != varc || g->cons)
      return fail(g0, WHV_ERR_INVALID, "whv_autotune_batched: grids must match as for whv_solve_batched");
    whv_status s = make_time_grid(g, &params[p], &c.tgs[p]);
    if (s != WHV_OK) return fail(g0, s, std::string("whv_autotune_batched: ") + g->err);
  }
  batch_init();
  c.st = g0->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
  B_CUDA(g0, c.alloc(&c.bar, 2 * sizeof(unsigned)));
  B_CUDA(g0, c.alloc(&c.err, sizeof(int)));
  B_CUDA(g0, cudaMemsetAsync(c.bar, 0, 2 * sizeof(unsigned), c.st));
  B_CUDA(g0, clear_err(c));
  RoleIO io;
  io.v.assign(nprob, nullptr);
  io.f.assign(nprob, nullptr);
  io.out = c.each([](whv_grid g) { return g->t; });
  const int saved = g0->kblock;
  cudaEvent_t e0, e1;
  B_CUDA(g0, cudaEventCreate(&e0));
  B_CUDA(g0, cudaEventCreate(&e1));
  const int R = g0->order == 2 ? 1 : 2;
  int kbest = batch_k(g0, g0->precision == WHV_FP64);
  float tbest = 1e30f;
  whv_status s = WHV_OK;
  for (int k : {2, 4, 6, 8, 10, 12}) {
    if (kBReg - 2 * k * R < 16) continue;
    g0->kblock = k;
    Wave w;
    const bool f64 = g0->precision == WHV_FP64;
    if (g0->order == 2)
      s = f64 ? (varc ? make_wave<double, 2, 2, true>(c, io, &w) : make_wave<double, 2, 2, false>(c, io, &w))
              : (varc ? make_wave<float, 2, 2, true>(c, io, &w) : make_wave<float, 2, 2, false>(c, io, &w));
    else
      s = f64 ? (varc ? make_wave<double, 2, 4, true>(c, io, &w) : make_wave<double, 2, 4, false>(c, io, &w))
              : (varc ? make_wave<float, 2, 4, true>(c, io, &w) : make_wave<float, 2, 4, false>(c, io, &w));
    if (s != WHV_OK) break;
    if ((s = run_wave(c, w)) != WHV_OK) break;   // warm-up
    cudaEventRecord(e0, c.st);
    if ((s = run_wave(c, w)) != WHV_OK) break;
    cudaEventRecord(e1, c.st);
    if ((s = check_barrier(c)) != WHV_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < tbest) { tbest = ms; kbest = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  count_launches(c.launches);
  g0->kblock = s == WHV_OK ? kbest : saved;
  if (s != WHV_OK) return s;
  if (best) *best = kbest;
  return WHV_OK;
}

template <int DIM, int ORDER, bool VARC>
static whv_status batched_apply(BatchCtx& c, const RoleIO& io, bool fp64) {
  Wave w;
  TRY(fp64 ? (make_wave<double, DIM, ORDER, VARC>(c, io, &w)) : (make_wave<float, DIM, ORDER, VARC>(c, io, &w)));
  TRY(run_wave(c, w));
  return check_barrier(c);
}

// out_p = Pi_h(v_p; f_p) of every problem in one persistent launch (the batched form of
// whv_apply_pi): the wave solve that each batched CG iteration runs, exposed on its own.
extern "C" whv_status whv_apply_pi_batched(int nprob, const whv_grid* grids, const whv_params* params,
                                           const double* const* v_dev, const double* const* f_dev,
                                           double* const* out_dev) {
  if (nprob < 1 || nprob > kBatchMaxProblems || !grids || !params || !out_dev || !grids[0])
    return fail(nullptr, WHV_ERR_INVALID, "whv_apply_pi_batched: bad arguments (1 <= nprob <= 1024)");
  whv_grid g0 = grids[0];
  const bool varc = g0->c2 != nullptr;
  BatchCtx c;
  c.np = nprob;
  c.grids = grids;
  c.params = params;
  c.g0 = g0;
  c.tgs.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    whv_grid g = grids[p];
    if (!g || !out_dev[p]) return fail(g0, WHV_ERR_INVALID, "whv_apply_pi_batched: NULL grid or output");
    for (int q = 0; q < p; ++q)
      if (grids[q] == g) return fail(g0, WHV_ERR_INVALID, "whv_apply_pi_batched: every problem needs its own grid");
    if (g->stream != g0->stream || g->precision != g0->precision || g->dim != g0->dim || g->order != g0->order ||
        (g->c2 != nullptr) != varc || g->cons)
      return fail(g0, WHV_ERR_INVALID, "whv_apply_pi_batched: grids must match as for whv_solve_batched");
    whv_status s = make_time_grid(g, &params[p], &c.tgs[p]);
    if (s != WHV_OK) return fail(g0, s, std::string("whv_apply_pi_batched: ") + g->err);
  }
  if (g0->dim < 2) return fail(g0, WHV_ERR_INVALID, "whv_apply_pi_batched: batched solves need 2-D or 3-D grids");
  batch_init();
  c.st = g0->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
  B_CUDA(g0, c.alloc(&c.bar, 2 * sizeof(unsigned)));
  B_CUDA(g0, c.alloc(&c.err, sizeof(int)));
  B_CUDA(g0, cudaMemsetAsync(c.bar, 0, 2 * sizeof(unsigned), c.st));
  B_CUDA(g0, clear_err(c));
  RoleIO io;
  io.v.assign(nprob, nullptr);
  io.f.assign(nprob, nullptr);
  for (int p = 0; p < nprob; ++p) {
    if (v_dev) io.v[p] = v_dev[p];
    if (f_dev) io.f[p] = f_dev[p];
  }
  io.out.assign(out_dev, out_dev + nprob);
  io.epi = 0;
  const bool fp64 = g0->precision == WHV_FP64;
  whv_status s;
  switch (g0->dim * 10 + g0->order) {
    case 22: s = varc ? batched_apply<2, 2, true>(c, io, fp64) : batched_apply<2, 2, false>(c, io, fp64); break;
    case 24: s = varc ? batched_apply<2, 4, true>(c, io, fp64) : batched_apply<2, 4, false>(c, io, fp64); break;
    case 32: s = varc ? batched_apply<3, 2, true>(c, io, fp64) : batched_apply<3, 2, false>(c, io, fp64); break;
    default: s = varc ? batched_apply<3, 4, true>(c, io, fp64) : batched_apply<3, 4, false>(c, io, fp64); break;
  }
  count_launches(c.launches);
  return s;
}

extern "C" whv_status whv_solve_batched(int nprob, const whv_grid* grids, const whv_params* params,
                                        const double* const* f_dev, double* const* u_dev, whv_info* infos) {
  const double t0 = now_s();
  if (nprob < 1 || nprob > kBatchMaxProblems || !grids || !params || !f_dev || !u_dev)
    return fail(nullptr, WHV_ERR_INVALID, "whv_solve_batched: bad arguments (1 <= nprob <= 1024)");
  whv_grid g0 = grids[0];
  if (!g0) return fail(nullptr, WHV_ERR_INVALID, "whv_solve_batched: NULL grid");
  const bool varc = g0->c2 != nullptr;
  const bool refine = (params[0].flags & WHV_REFINE_FP64) != 0;
  BatchCtx c;
  c.np = nprob;
  c.grids = grids;
  c.params = params;
  c.g0 = g0;
  c.tgs.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    whv_grid g = grids[p];
    if (!g || !f_dev[p] || !u_dev[p]) return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: NULL grid or buffer");
    for (int q = 0; q < p; ++q)
      if (grids[q] == g) return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: every problem needs its own grid");
    if (g->stream != g0->stream || g->precision != g0->precision || g->dim != g0->dim || g->order != g0->order ||
        (g->c2 != nullptr) != varc)
      return fail(g0, WHV_ERR_INVALID,
                  "whv_solve_batched: grids must share stream, precision, dimension, order and speed kind");
    if (params[p].method != WHV_CG) return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: method must be WHV_CG");
    if (g->cons) return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: the conservative operator is not batched");
    if (((params[p].flags & WHV_RESIDUAL_DF64) != 0) != ((params[0].flags & WHV_RESIDUAL_DF64) != 0))
      return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: WHV_RESIDUAL_DF64 must be set for all problems or none");
    if (((params[p].flags & WHV_REFINE_FP64) != 0) != refine)
      return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: WHV_REFINE_FP64 must be set for all problems or none");
    if (!(params[p].tol >= 0.0) || params[p].maxit < 0)
      return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: tol must be >= 0, maxit >= 0");
    whv_status s = make_time_grid(g, &params[p], &c.tgs[p]);
    if (s != WHV_OK) return fail(g0, s, std::string("whv_solve_batched: ") + g->err);
    const Basis& B = g->basis;
    if (B.nd > 0) {
      if (!(B.flags & WHV_BASIS_EXACT) || (B.flags & WHV_BASIS_REDEFLATE))
        return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: bases must be exact eigenvectors (DEVD)");
      if (B.omega != params[p].omega || B.periods != params[p].periods || B.cfl != c.tgs[p].cfl ||
          B.adjust != (params[p].adjust_omega ? 1 : 0))
        return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: a basis was set for another frequency / time grid");
    }
  }
  if (g0->dim < 2) return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: batched solves need 2-D or 3-D grids");
  batch_init();
  c.st = g0->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
  B_CUDA(g0, c.alloc(&c.bar, 2 * sizeof(unsigned)));
  B_CUDA(g0, c.alloc(&c.err, sizeof(int)));
  B_CUDA(g0, c.alloc(&c.scal, nprob * sizeof(double*)));
  {
    std::vector<double*> sc(nprob);
    for (int p = 0; p < nprob; ++p) sc[p] = grids[p]->scal;
    B_CUDA(g0, cudaMemcpy(c.scal, sc.data(), nprob * sizeof(double*), cudaMemcpyHostToDevice));
  }
  B_CUDA(g0, cudaMemsetAsync(c.bar, 0, 2 * sizeof(unsigned), c.st));
  B_CUDA(g0, clear_err(c));
  whv_status s;
  switch (g0->dim * 10 + g0->order) {
    case 22: s = batched_vc<2, 2>(c, f_dev, u_dev, refine, infos, varc); break;
    case 24: s = batched_vc<2, 4>(c, f_dev, u_dev, refine, infos, varc); break;
    case 32: s = batched_vc<3, 2>(c, f_dev, u_dev, refine, infos, varc); break;
    default: s = batched_vc<3, 4>(c, f_dev, u_dev, refine, infos, varc); break;
  }
  if (infos) {
    const double secs = now_s() - t0;
    for (int p = 0; p < nprob; ++p) infos[p].seconds = secs;
  }
  return s;
}
