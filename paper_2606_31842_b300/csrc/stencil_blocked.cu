// Temporally blocked 2-D leapfrog + trapezoid filter: k time steps per launch (the f = 0 wave
// solves that make up A p in every Krylov iteration).
//
// Each CTA owns a TX x TY tile.  It stages W^{n-1}, W^n (and c^2) of the tile plus a halo of
// width H = k r (r = 1 for the 5-point, 2 for the 9-point-wide 4th-order stencil) in shared
// memory, advances k leapfrog steps there -- at sub-step s the valid region shrinks by r on
// every side that is not a Dirichlet boundary -- and accumulates the filter terms w_{n+s} W^{n+s}
// of its own tile points in registers.  It then writes W^{n+k-1}, W^{n+k} of the tile to the
// other buffer pair (neighbouring CTAs still read the old pair) and adds the accumulated filter
// sum to acc, or, on the last block of steps, writes the FP64 epilogue (Pi_h v, or A v with the
// p^T M A p reduction) like the single-step kernel.
//
// Global traffic per k steps and node: 3 reads + 3 writes (+ c^2) instead of 5 per step, so the
// sweep count per wave solve drops from Nt to Nt/k; the cost is the redundant halo updates
// ((TX + 2H)(TY + 2H) / (TX TY) on the first sub-step, shrinking to 1).
#include <math.h>

#include <algorithm>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

constexpr int kBlkMaxK = 16;
constexpr int kBlkTX = 32, kBlkTY = 32;   // tile per CTA; block of 32 x 8 threads

template <typename T>
struct BlockCoef {
  T ih2x, ih2y, dt2;
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

template <typename T, int ORDER, bool VARC, int KIND>
__global__ void __launch_bounds__(256) k_block2d(const T* __restrict__ gprev, const T* __restrict__ gcur,
                                                 T* __restrict__ oprev, T* __restrict__ ocur,
                                                 T* __restrict__ acc, const T* __restrict__ c2,
                                                 const double* __restrict__ v,
                                                 const double* __restrict__ mw,
                                                 double* __restrict__ out, int nx, int ny,
                                                 BlockCoef<T> cf, double* partials,
                                                 unsigned* counter, double* scal_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = ORDER == 2 ? 1 : 2;
  constexpr int NB = kBlkTY / 8;   // owned tile rows per thread
  const int H = cf.k * R;
  const int x0 = blockIdx.x * kBlkTX, y0 = blockIdx.y * kBlkTY;
  const int rx0 = max(x0 - H, 0), rx1 = min(x0 + kBlkTX + H, nx);
  const int ry0 = max(y0 - H, 0), ry1 = min(y0 + kBlkTY + H, ny);
  const int RW = rx1 - rx0, RH = ry1 - ry0;
  const bool physL = rx0 == 0, physR = rx1 == nx, physB = ry0 == 0, physT = ry1 == ny;
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Y = X + RW * RH;
  T* C = Y + RW * RH;
  const int tx = threadIdx.x, ty = threadIdx.y;
  __shared__ T sw[kBlkMaxK];   // filter weights, indexed by sub-step
  if (ty == 0 && tx < kBlkMaxK) sw[tx] = cf.w[tx];
  for (int j = ty; j < RH; j += 8) {
    const int64_t grow = (int64_t)nx * (ry0 + j) + rx0;
    for (int i = tx; i < RW; i += 32) {
      X[j * RW + i] = gprev[grow + i];
      Y[j * RW + i] = gcur[grow + i];
      if (VARC) C[j * RW + i] = c2[grow + i];
    }
  }
  __syncthreads();
  T accr[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) accr[b] = T(0);
  const int ox = x0 + tx;                    // owned column
  T* cur = Y;
  T* prv = X;
  for (int s = 1; s <= cf.k; ++s) {
    const int vx0 = physL ? 0 : s * R, vx1 = physR ? RW : RW - s * R;
    const int vy0 = physB ? 0 : s * R, vy1 = physT ? RH : RH - s * R;
    for (int j = vy0 + ty; j < vy1; j += 8) {
      const int gy = ry0 + j;
      for (int i = vx0 + tx; i < vx1; i += 32) {
        const int l = j * RW + i;
        const T c = cur[l];
        T L = d2s<ORDER>(cur, l, rx0 + i, nx, 1, c) * cf.ih2x;
        L = fma(d2s<ORDER>(cur, l, gy, ny, RW, c), cf.ih2y, L);
        if (VARC) L *= C[l];
        prv[l] = fma(cf.dt2, L, fma(T(2), c, -prv[l]));
      }
    }
    __syncthreads();
    T* t = cur; cur = prv; prv = t;          // cur = W^{n0+s}
    const T ws = sw[s - 1];
    if (ox < nx) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int oy = y0 + ty + 8 * b;
        if (oy < ny) accr[b] = fma(ws, cur[(oy - ry0) * RW + (ox - rx0)], accr[b]);
      }
    }
  }
  double part = 0.0;
  if (ox < nx) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int oy = y0 + ty + 8 * b;
      if (oy >= ny) continue;
      const int l = (oy - ry0) * RW + (ox - rx0);
      const int64_t gi = ox + (int64_t)nx * oy;
      if (KIND == B_STEP) {
        ocur[gi] = cur[l];
        oprev[gi] = prv[l];
        acc[gi] += accr[b];
      } else {
        const T a = acc[gi] + accr[b];
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
  }
  if (KIND == B_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

static size_t blk_smem(int k, int order, bool varc, size_t esz) {
  const int R = order == 2 ? 1 : 2;
  const size_t w = kBlkTX + 2 * k * R, h = kBlkTY + 2 * k * R;
  return (varc ? 3 : 2) * w * h * esz;
}

// largest k <= want whose staged region fits the shared-memory budget
int blocked_steps(int want, int order, bool varc, size_t esz) {
  int k = std::min(std::max(want, 1), kBlkMaxK);
  while (k > 1 && blk_smem(k, order, varc, esz) > 160u * 1024u) --k;
  return k;
}

constexpr int kBlkSmemCap = 160 * 1024;

template <typename T, int ORDER, bool VARC>
static void set_attrs() {
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_LAST_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
  cudaFuncSetAttribute(k_block2d<T, ORDER, VARC, B_LAST_AV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlkSmemCap);
}

// opt the blocked kernels into large dynamic shared memory once per process (outside any
// stream capture)
void blocked_init() {
  static bool done = false;
  if (done) return;
  done = true;
  set_attrs<float, 2, false>(); set_attrs<float, 2, true>(); set_attrs<float, 4, false>(); set_attrs<float, 4, true>();
  set_attrs<double, 2, false>(); set_attrs<double, 2, true>(); set_attrs<double, 4, false>(); set_attrs<double, 4, true>();
}

template <typename T, int ORDER, bool VARC, int KIND>
static cudaError_t launch_block(whv_grid g, const T* gp, const T* gc, T* op, T* oc, T* acc,
                                const T* c2, const double* v, double* out, const BlockCoef<T>& cf,
                                double* partials, unsigned* counter, double* scal_out) {
  const size_t smem = blk_smem(cf.k, ORDER, VARC, sizeof(T));
  auto kern = k_block2d<T, ORDER, VARC, KIND>;
  dim3 grid((g->n[0] + kBlkTX - 1) / kBlkTX, (g->n[1] + kBlkTY - 1) / kBlkTY, 1);
  kern<<<grid, dim3(32, 8, 1), smem, g->stream>>>(gp, gc, op, oc, acc, c2, v, g->mw, out, g->n[0],
                                                  g->n[1], cf, partials, counter, scal_out);
  return cudaGetLastError();
}

// Steps n = 1 .. nt-1 of a 2-D f = 0 wave solve in sweeps of k steps; the first step (Taylor
// start) has already written W^0 -> wbuf[0], W^1 -> wbuf[1] and acc.
template <typename T, int ORDER, bool VARC>
whv_status blocked_steps_2d(whv_grid g, const TimeGridH& tg, const double* v, double* out, int epi,
                            int k_want, int* launches) {
  T* buf[4] = {(T*)g->wbuf[0], (T*)g->wbuf[1], (T*)g->wbuf[2], (T*)g->wbuf[3]};
  T* acc = (T*)g->acc;
  const T* c2 = VARC ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  const int kmax = blocked_steps(k_want, ORDER, VARC, sizeof(T));
  BlockCoef<T> cf;
  const double h2x = g->h[0] * g->h[0], h2y = g->h[1] * g->h[1];
  cf.ih2x = (T)(ORDER == 2 ? 1.0 / h2x : 1.0 / (12.0 * h2x));
  cf.ih2y = (T)(ORDER == 2 ? 1.0 / h2y : 1.0 / (12.0 * h2y));
  cf.dt2 = (T)(tg.dt * tg.dt);
  double* part = g->partials + CH_STEP * kMaxStepBlocks;
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

template whv_status blocked_steps_2d<float, 2, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<float, 2, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<float, 4, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<float, 4, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<double, 2, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<double, 2, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<double, 4, false>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);
template whv_status blocked_steps_2d<double, 4, true>(whv_grid, const TimeGridH&, const double*, double*, int, int, int*);

}  // namespace whv
