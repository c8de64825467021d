// Temporally blocked 2-D leapfrog + trapezoid filter: k time steps per launch (the f = 0 wave
// solves that make up A p in every Krylov iteration).
//
// Each CTA stages a REG x REG region (a tile of (REG - 2H)^2 nodes plus a halo of width
// H = k r; r = 1 for the 5-point, 2 for the 9-point-wide 4th-order stencil) and advances it k
// leapfrog steps; at sub-step s only the window [s r, REG - s r)^2 is updated, which is exactly
// what the next sub-step needs.  Thread (warp w, lane) owns column 32 (w & 1) + lane and rows
// (w >> 1) + 16 t, t < 4, of the region for the whole launch: W^n, W^{n-1} and the filter sum of
// its cells stay in registers, and only W^n goes through shared memory (double-buffered) for the
// neighbours' reads.  All global loads of a thread are issued before the first use.  The tile's
// W^{n+k-1}, W^{n+k} go to the other buffer pair (neighbouring CTAs still read the old pair),
// the filter sums are added to acc -- or, on the last sweep, the FP64 epilogue (Pi_h v, or A v
// with the p^T M A p reduction) is written like the single-step kernel does.
//
// Global traffic per k steps and tile node: 3 reads + 3 writes (+ c^2), plus the halo re-reads
// (REG^2 / tile^2), instead of 5 accesses per step; the price is the redundant halo updates.
#include <math.h>

#include <algorithm>
#include <vector>

#include "quad2d.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

constexpr int kBlkMaxK = 16;
constexpr int kReg = 64;            // staged region edge
constexpr int kBlkThreads = 1024;   // 32 warps
constexpr int kRowPitch = kBlkThreads / 64;   // rows between a thread's cells (16)
constexpr int kRowsPerThread = kReg / kRowPitch;

template <typename T>
struct BlockCoef {
  T ih2x, ih2y, dt2;
  T ax, ay, b;     // 2nd order, c = 1: W^{n+1} = ax s_x + ay s_y + b W^n - W^{n-1}
  T w[kBlkMaxK];   // filter weights w_{n0+1} .. w_{n0+k}
  int k;
};

enum BlkKind { B_STEP = 0, B_LAST_OUT = 1, B_LAST_AV = 2 };

// second difference at global index gi (of n) read from shared memory at local offset l,
// stride s; same Dirichlet / odd-reflection closure as the single-step kernel
template <int ORDER, typename T>
__device__ __forceinline__ T d2s(const T* __restrict__ a, int l, int gi, int n, int s, T c) {
  const T m1 = gi > 0 ? a[l - s] : T(0);
  const T p1 = gi < n - 1 ? a[l + s] : T(0);
  if (ORDER == 2) return fma(T(-2), c, m1 + p1);
  const T m2 = gi > 1 ? a[l - 2 * s] : (gi == 1 ? T(0) : -c);
  const T p2 = gi < n - 2 ? a[l + 2 * s] : (gi == n - 2 ? T(0) : -c);
  return fma(T(-30), c, fma(T(16), m1 + p1, -(m2 + p2)));
}

// FP32: the sub-steps run in the four-cells-per-thread mapping of quad2d.cuh
template <typename T, int ORDER, bool VARC>
constexpr bool kQuad = sizeof(T) == 4;

template <typename T, int ORDER, bool VARC, int KIND>
__global__ void __launch_bounds__(kBlkThreads) k_block2d(const T* __restrict__ gprev,
                                                         const T* __restrict__ gcur,
                                                         T* __restrict__ oprev, T* __restrict__ ocur,
                                                         T* __restrict__ acc,
                                                         const T* __restrict__ c2,
                                                         const double* __restrict__ v,
                                                         const double* __restrict__ mw,
                                                         double* __restrict__ out, int nx, int ny,
                                                         BlockCoef<T> cf, double* partials,
                                                         unsigned* counter, double* scal_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* S1 = S0 + kReg * kReg;
  __shared__ T sw[kBlkMaxK];
  // launched as a programmatic dependent of the previous sweep: wait for its results (returns at
  // once when there is no such dependency)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int R = ORDER == 2 ? 1 : 2;
  const int H = cf.k * R;
  const int TW = kReg - 2 * H;
  const int x0 = blockIdx.x * TW - H, y0 = blockIdx.y * TW - H;   // region origin (global)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 1) + lane;
  const int jb = warp >> 1;
  const int gx = x0 + i;
  const bool colin = gx >= 0 && gx < nx;
  if (threadIdx.x < kBlkMaxK) sw[threadIdx.x] = cf.w[threadIdx.x];
  T cur[kRowsPerThread], prv[kRowsPerThread], acr[kRowsPerThread];
  T cc[VARC ? kRowsPerThread : 1];
  // all global loads up front, the filter accumulator of the tile cells included (its
  // read-modify-write at the end would otherwise be one more L2 round trip on the critical path)
  const bool coltile0 = colin && i >= H && i < kReg - H;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int j = jb + kRowPitch * t;
    const int gy = y0 + j;
    const bool in = colin && gy >= 0 && gy < ny;
    const int64_t gi = gx + (int64_t)nx * gy;
    cur[t] = in ? gcur[gi] : T(0);
    prv[t] = in ? gprev[gi] : T(0);
    if (VARC) cc[t] = in ? c2[gi] : T(0);
    acr[t] = (coltile0 && j >= H && j < kReg - H && in) ? acc[gi] : T(0);
  }
  if constexpr (kQuad<T, ORDER, VARC>) {
    T* const S2 = S1 + kReg * kReg;
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int l = (jb + kRowPitch * t) * kReg + i;
      S0[l] = cur[t];
      S1[l] = prv[t];
      S2[l] = acr[t];
    }
    __syncthreads();
    const bool inside = x0 >= 0 && y0 >= 0 && x0 + kReg <= nx && y0 + kReg <= ny;
    if constexpr (ORDER == 2 && !VARC) {
      const QuadCoef q{cf.ax, cf.ay, cf.b, cf.ih2x, cf.ih2y, 0.5f * cf.dt2};
      if (inside)
        quad_sweep<false, false>(S0, S1, S2, cf.k, sw, q, 0xfu);
      else
        quad_sweep<true, false>(S0, S1, S2, cf.k, sw, q, quad_mask(x0, y0, nx, ny));
    } else {
      const QuadCoefV q{cf.ih2x, cf.ih2y, cf.dt2};
      const QuadBnd bd = inside ? QuadBnd{0xfu, 0u} : quad_bnd(x0, y0, nx, ny);
      float4 cq = make_float4(1.f, 1.f, 1.f, 1.f);
      if constexpr (VARC) {   // c^2 of the thread's four cells (read-only: through L1)
        const int qy = y0 + (int)(threadIdx.x >> 4), qx = x0 + (int)(threadIdx.x & 15) * 4;
        const T* row = c2 + (int64_t)nx * qy + qx;
        cq.x = (bd.in & 1u) ? __ldg(row) : 0.f;
        cq.y = (bd.in & 2u) ? __ldg(row + 1) : 0.f;
        cq.z = (bd.in & 4u) ? __ldg(row + 2) : 0.f;
        cq.w = (bd.in & 8u) ? __ldg(row + 3) : 0.f;
      }
      if (inside)
        quadv_sweep<ORDER, VARC, false>(S0, S1, S2, cf.k, sw, q, bd, cq);
      else
        quadv_sweep<ORDER, VARC, true>(S0, S1, S2, cf.k, sw, q, bd, cq);
    }
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int l = (jb + kRowPitch * t) * kReg + i;
      cur[t] = S0[l];
      prv[t] = S1[l];
      acr[t] = S2[l];
    }
  } else {
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) S0[(jb + kRowPitch * t) * kReg + i] = cur[t];
  __syncthreads();
  T* A = S0;
  T* B = S1;
  for (int s = 1; s <= cf.k; ++s) {
    const int lo = s * R, hi = kReg - s * R;
    const bool colact = colin && i >= lo && i < hi;
    const T ws = sw[s - 1];
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int j = jb + kRowPitch * t;
      const int gy = y0 + j;
      if (colact && j >= lo && j < hi && gy >= 0 && gy < ny) {
        const int l = j * kReg + i;
        const T c = cur[t];
        T wn;
        if constexpr (ORDER == 2 && !VARC) {
          T u = fma(cf.b, c, -prv[t]);
          u = fma(cf.ax, (gx > 0 ? A[l - 1] : T(0)) + (gx < nx - 1 ? A[l + 1] : T(0)), u);
          wn = fma(cf.ay, (gy > 0 ? A[l - kReg] : T(0)) + (gy < ny - 1 ? A[l + kReg] : T(0)), u);
        } else {
          T L = d2s<ORDER>(A, l, gx, nx, 1, c) * cf.ih2x;
          L = fma(d2s<ORDER>(A, l, gy, ny, kReg, c), cf.ih2y, L);
          if (VARC) L *= cc[t];
          wn = fma(cf.dt2, L, fma(T(2), c, -prv[t]));
        }
        prv[t] = c;
        cur[t] = wn;
        B[l] = wn;
        acr[t] = fma(ws, wn, acr[t]);
      }
    }
    __syncthreads();
    T* tmp = A; A = B; B = tmp;
  }
  }
  double part = 0.0;
  const bool coltile = colin && i >= H && i < kReg - H;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int j = jb + kRowPitch * t;
    const int gy = y0 + j;
    if (!(coltile && j >= H && j < kReg - H && gy >= 0 && gy < ny)) continue;
    const int64_t gi = gx + (int64_t)nx * gy;
    if (KIND == B_STEP) {
      ocur[gi] = cur[t];
      oprev[gi] = prv[t];
      acc[gi] = acr[t];
    } else {
      const T a = acr[t];
      if (KIND == B_LAST_OUT) {
        out[gi] = (double)a;
      } else {
        const double vi = v[gi];
        const double o = vi - (double)a;
        out[gi] = o;
        part = fma(mw ? vi * mw[gi] : vi, o, part);
      }
    }
  }
  if (KIND == B_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

// two state buffers; the FP32 four-cell sweep stages W^{n-1} and the filter sums in a third
static size_t blk_smem(size_t esz, bool quad) { return (quad ? 3 : 2) * (size_t)kReg * kReg * esz; }

// largest k <= want that leaves a tile of at least 16 nodes per edge
int blocked_steps(int want, int order) {
  const int R = order == 2 ? 1 : 2;
  int k = std::min(std::max(want, 1), kBlkMaxK);
  while (k > 1 && kReg - 2 * k * R < 16) --k;
  return k;
}

constexpr int kBlkSmemCap = 2 * kReg * kReg * 8;   // FP64 double buffer: 64 KB

template <typename T, int ORDER, bool VARC>
static void set_attrs() {
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_LAST_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_LAST_AV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
}

// opt the blocked kernels into large dynamic shared memory once per process (outside any
// stream capture)
void small_init();

void blocked_init() {
  static bool done = false;
  if (done) return;
  done = true;
  small_init();
  set_attrs<float, 2, false>(); set_attrs<float, 2, true>(); set_attrs<float, 4, false>(); set_attrs<float, 4, true>();
  set_attrs<double, 2, false>(); set_attrs<double, 2, true>(); set_attrs<double, 4, false>(); set_attrs<double, 4, true>();
}

template <typename T, int ORDER, bool VARC, int KIND>
static cudaError_t launch_block(whv_grid g, const T* gp, const T* gc, T* op, T* oc, T* acc,
                                const T* c2, const double* v, double* out, const BlockCoef<T>& cf,
                                double* partials, unsigned* counter, double* scal_out) {
  const size_t smem = blk_smem(sizeof(T), kQuad<T, ORDER, VARC>);
  const int R = ORDER == 2 ? 1 : 2;
  const int TW = kReg - 2 * cf.k * R;
  dim3 grid((g->n[0] + TW - 1) / TW, (g->n[1] + TW - 1) / TW, 1);
  // programmatic dependent launch: the sweep may be scheduled as the previous kernel's CTAs exit;
  // it waits (griddepcontrol.wait) for that kernel's completion before reading anything
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = dim3(kBlkThreads, 1, 1);
  lc.dynamicSmemBytes = smem;
  lc.stream = g->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const double* mw = g->mw;
  const int nx = g->n[0], ny = g->n[1];
  return cudaLaunchKernelEx(&lc, k_block2d<T, ORDER, VARC, KIND>, gp, gc, op, oc, acc, c2, v, mw, out, nx, ny, cf,
                            partials, counter, scal_out);
}

// Steps n = 1 .. nt-1 of a 2-D f = 0 wave solve in sweeps of k steps; the first step (Taylor
// start) has already written W^0 -> wbuf[0], W^1 -> wbuf[1] and acc.
template <typename T, int ORDER, bool VARC>
whv_status blocked_steps_2d(whv_grid g, const TimeGridH& tg, const double* v, double* out, int epi,
                            int k_want, int* launches, void* const* bufs, void* accbuf) {
  T* buf[4] = {(T*)bufs[0], (T*)bufs[1], (T*)bufs[2], (T*)bufs[3]};
  T* acc = (T*)accbuf;
  const T* c2 = VARC ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  const int kmax = blocked_steps(k_want, ORDER);
  BlockCoef<T> cf;
  const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
  cf.ih2x = (T)(ORDER == 2 ? 1.0 / h2x : 1.0 / (12.0 * h2x));
  cf.ih2y = (T)(ORDER == 2 ? 1.0 / h2y : 1.0 / (12.0 * h2y));
  cf.dt2 = (T)(tg.dt * tg.dt);
  const double ax = tg.dt * tg.dt / h2x, ay = tg.dt * tg.dt / h2y;
  cf.ax = (T)ax;
  cf.ay = (T)ay;
  cf.b = (T)(2.0 - 2.0 * (ax + ay));
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  int pair = 0;   // input pair: (buf[2 pair], buf[2 pair + 1]) = (W^{n-1}, W^n)
  int n = 1;      // next step computes W^{n+1}
  int nl = 0;
  while (n < tg.nt) {
    const int k = std::min(kmax, tg.nt - n);
    cf.k = k;
    for (int s = 0; s < k; ++s) cf.w[s] = (T)tg.weight[n + 1 + s];
    const bool last = (n + k == tg.nt);
    T *gp = buf[2 * pair], *gc = buf[2 * pair + 1], *op = buf[2 * (1 - pair)], *oc = buf[2 * (1 - pair) + 1];
    cudaError_t e;
    if (!last)
      e = launch_block<T, ORDER, VARC, B_STEP>(g, gp, gc, op, oc, acc, c2, nullptr, nullptr, cf, nullptr, nullptr, nullptr);
    else if (epi == 0)
      e = launch_block<T, ORDER, VARC, B_LAST_OUT>(g, gp, gc, op, oc, acc, c2, nullptr, out, cf, nullptr, nullptr, nullptr);
    else
      e = launch_block<T, ORDER, VARC, B_LAST_AV>(g, gp, gc, op, oc, acc, c2, v, out, cf, part, cnt, g->scal + S_PQ);
    if (e != cudaSuccess) return cuda_fail(g, e, "k_block2d launch");
    ++nl;
    pair = 1 - pair;
    n += k;
  }
  *launches = nl;
  return WHV_OK;
}

template whv_status blocked_steps_2d<float, 2, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<float, 2, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<float, 4, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<float, 4, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<double, 2, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<double, 2, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<double, 4, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);
template whv_status blocked_steps_2d<double, 4, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*, void* const*, void*);

}  // namespace whv

// ------------------------------------------------------------------ whole wave solve in one CTA
// Small grids (N <= kSmallMaxN unknowns, e.g. the 1-D workload's 199) are bound by launch
// latency when every time step is a kernel.  One CTA runs the whole wave solve instead: thread
// t owns cells t + kBlkThreads c (c < kSmallCells) with their W^n, W^{n-1} and filter sum in
// registers; W^n is double-buffered in shared memory for the neighbours; one barrier per step.
// The FP64 epilogue (out = acc, or out = v - acc with p^T M out) is reduced inside the block.
namespace whv {

constexpr int kSmallCells = 4;
constexpr int kSmallMaxN = kBlkThreads * kSmallCells;   // 4096

template <typename T>
struct SmallArgs {
  const double* v;        // initial state (nullptr: 0)
  const double* f;        // forcing (nullptr: 0)
  double* out;
  const T* c2;            // nullptr: c = 1
  const double* mw;
  double* scal_pq;        // epi 1: <v, out>_M
  const double* wtab;     // w_n, n = 0..nt
  const double* ptab;     // cos(omega_hat t^n), n = 0..nt
  int nx, ny, nz, nt, epi;
  T ih2x, ih2y, ih2z, dt2;
};

template <typename T, int DIM, int ORDER>
__device__ __forceinline__ T lap_small(const T* __restrict__ A, int i, int nx, int ny, int nz,
                                       const SmallArgs<T>& a, T c) {
  const int x = i % nx;
  T L = d2s<ORDER>(A, i, x, nx, 1, c) * a.ih2x;
  if (DIM > 1) {
    const int y = (i / nx) % ny;
    L = fma(d2s<ORDER>(A, i, y, ny, nx, c), a.ih2y, L);
  }
  if (DIM > 2) {
    const int z = i / (nx * ny);
    L = fma(d2s<ORDER>(A, i, z, nz, nx * ny, c), a.ih2z, L);
  }
  return L;
}

template <typename T, int DIM, int ORDER, bool VARC>
__global__ void __launch_bounds__(kBlkThreads) k_wave_small(SmallArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.nx * a.ny * a.nz;
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + N;
  const int tid = threadIdx.x;
  T cur[kSmallCells], prv[kSmallCells], acc[kSmallCells], cc[kSmallCells], ff[kSmallCells];
#pragma unroll
  for (int c = 0; c < kSmallCells; ++c) {
    const int i = tid + kBlkThreads * c;
    cur[c] = (i < N && a.v) ? (T)a.v[i] : T(0);
    cc[c] = (VARC && i < N) ? a.c2[i] : T(1);
    ff[c] = (i < N && a.f) ? (T)a.f[i] : T(0);
    if (i < N) A[i] = cur[c];
  }
  __syncthreads();
  // first step from D0t W^0 = 0
  {
    const T w0 = (T)a.wtab[0], w1 = (T)a.wtab[1];
#pragma unroll
    for (int c = 0; c < kSmallCells; ++c) {
      const int i = tid + kBlkThreads * c;
      if (i >= N) continue;
      T L = lap_small<T, DIM, ORDER>(A, i, a.nx, a.ny, a.nz, a, cur[c]);
      if (VARC) L *= cc[c];
      L -= ff[c];   // cos(0) = 1
      const T W1 = fma(T(0.5) * a.dt2, L, cur[c]);
      acc[c] = fma(w1, W1, w0 * cur[c]);
      prv[c] = cur[c];
      cur[c] = W1;
      B[i] = W1;
    }
  }
  __syncthreads();
  T* X = B;
  T* Y = A;
  for (int n = 1; n < a.nt; ++n) {
    const T wn1 = (T)a.wtab[n + 1];
    const T ph = (T)a.ptab[n];
#pragma unroll
    for (int c = 0; c < kSmallCells; ++c) {
      const int i = tid + kBlkThreads * c;
      if (i >= N) continue;
      T L = lap_small<T, DIM, ORDER>(X, i, a.nx, a.ny, a.nz, a, cur[c]);
      if (VARC) L *= cc[c];
      L = fma(-ff[c], ph, L);
      const T wn = fma(a.dt2, L, fma(T(2), cur[c], -prv[c]));
      acc[c] = fma(wn1, wn, acc[c]);
      prv[c] = cur[c];
      cur[c] = wn;
      Y[i] = wn;
    }
    __syncthreads();
    T* t = X; X = Y; Y = t;
  }
  double part = 0.0;
#pragma unroll
  for (int c = 0; c < kSmallCells; ++c) {
    const int i = tid + kBlkThreads * c;
    if (i >= N) continue;
    if (a.epi == 0) {
      a.out[i] = (double)acc[c];
    } else {
      const double vi = a.v[i];
      const double o = vi - (double)acc[c];
      a.out[i] = o;
      part = fma(a.mw ? vi * a.mw[i] : vi, o, part);
    }
  }
  if (a.epi == 1) {
    part = block_sum(part);
    if (tid == 0) *a.scal_pq = part;
  }
}

template <typename T, int DIM, int ORDER, bool VARC>
static cudaError_t launch_small_t(whv_grid g, const SmallArgs<T>& a) {
  const size_t smem = 2 * (size_t)g->N * sizeof(T);
  k_wave_small<T, DIM, ORDER, VARC><<<1, kBlkThreads, smem, g->stream>>>(a);
  return cudaGetLastError();
}

template <typename T>
static whv_status launch_small(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                               int epi) {
  SmallArgs<T> a{};
  a.v = v; a.f = f; a.out = out;
  a.c2 = g->c2 ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  a.mw = g->mw;
  a.scal_pq = g->scal + S_PQ;
  a.wtab = g->wtab_small;
  a.ptab = g->wtab_small + (tg.nt + 1);
  a.nx = g->n[0]; a.ny = g->n[1]; a.nz = g->n[2]; a.nt = tg.nt; a.epi = epi;
  auto ih = [&](int m) { const double h2 = g->h[m] * g->h[m]; return (T)(g->order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2)); };
  a.ih2x = ih(0); a.ih2y = ih(1); a.ih2z = ih(2);
  a.dt2 = (T)(tg.dt * tg.dt);
  const bool varc = g->c2 != nullptr;
  cudaError_t e = cudaErrorInvalidValue;
  switch (g->dim * 10 + g->order) {
    case 12: e = varc ? launch_small_t<T, 1, 2, true>(g, a) : launch_small_t<T, 1, 2, false>(g, a); break;
    case 14: e = varc ? launch_small_t<T, 1, 4, true>(g, a) : launch_small_t<T, 1, 4, false>(g, a); break;
    case 22: e = varc ? launch_small_t<T, 2, 2, true>(g, a) : launch_small_t<T, 2, 2, false>(g, a); break;
    case 24: e = varc ? launch_small_t<T, 2, 4, true>(g, a) : launch_small_t<T, 2, 4, false>(g, a); break;
    case 32: e = varc ? launch_small_t<T, 3, 2, true>(g, a) : launch_small_t<T, 3, 2, false>(g, a); break;
    case 34: e = varc ? launch_small_t<T, 3, 4, true>(g, a) : launch_small_t<T, 3, 4, false>(g, a); break;
  }
  if (e != cudaSuccess) return cuda_fail(g, e, "k_wave_small launch");
  return WHV_OK;
}

bool small_grid(whv_grid g) { return g->N <= kSmallMaxN; }

// weight / phase table of tg in device memory, uploaded when the time grid changes (outside
// stream captures).  Returns 0 if the table was current, 1 if it was (re)uploaded -- graphs
// captured against the old table must then be dropped -- and -1 if it is stale and cannot be
// uploaded now (the grid's stream is being captured).
int small_tables(whv_grid g, const TimeGridH& tg) {
  if (g->wtab_small && g->tab_nt == tg.nt && g->tab_key[0] == tg.omega && g->tab_key[1] == tg.cfl &&
      g->tab_key[2] == tg.periods && g->tab_key[3] == tg.adjust)
    return 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(g->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
  if (g->wtab_small && g->tab_cap < tg.nt + 1) { cudaFree(g->wtab_small); g->wtab_small = nullptr; }
  if (!g->wtab_small) {
    if (cudaMalloc(&g->wtab_small, 2 * (size_t)(tg.nt + 1) * sizeof(double)) != cudaSuccess) return -1;
    g->tab_cap = tg.nt + 1;
  }
  std::vector<double> tab(2 * (size_t)(tg.nt + 1));
  std::copy(tg.weight.begin(), tg.weight.end(), tab.begin());
  std::copy(tg.phase.begin(), tg.phase.end(), tab.begin() + (tg.nt + 1));
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return -1;
  if (cudaMemcpy(g->wtab_small, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return -1;
  g->tab_nt = tg.nt;
  g->tab_key[0] = tg.omega; g->tab_key[1] = tg.cfl; g->tab_key[2] = tg.periods; g->tab_key[3] = tg.adjust;
  return 1;
}

whv_status small_wave_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                            int epi, int prec) {
  return prec == WHV_FP64 ? launch_small<double>(g, tg, v, f, out, epi) : launch_small<float>(g, tg, v, f, out, epi);
}

template <typename T, int DIM, int ORDER, bool VARC>
static void small_attr() {
  cudaFuncSetAttribute(k_wave_small<T, DIM, ORDER, VARC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * kSmallMaxN * sizeof(T)));
}

void small_init() {
  small_attr<float, 1, 2, false>(); small_attr<float, 1, 2, true>(); small_attr<float, 1, 4, false>(); small_attr<float, 1, 4, true>();
  small_attr<float, 2, 2, false>(); small_attr<float, 2, 2, true>(); small_attr<float, 2, 4, false>(); small_attr<float, 2, 4, true>();
  small_attr<float, 3, 2, false>(); small_attr<float, 3, 2, true>(); small_attr<float, 3, 4, false>(); small_attr<float, 3, 4, true>();
  small_attr<double, 1, 2, false>(); small_attr<double, 1, 2, true>(); small_attr<double, 1, 4, false>(); small_attr<double, 1, 4, true>();
  small_attr<double, 2, 2, false>(); small_attr<double, 2, 2, true>(); small_attr<double, 2, 4, false>(); small_attr<double, 2, 4, true>();
  small_attr<double, 3, 2, false>(); small_attr<double, 3, 2, true>(); small_attr<double, 3, 4, false>(); small_attr<double, 3, 4, true>();
}

}  // namespace whv
