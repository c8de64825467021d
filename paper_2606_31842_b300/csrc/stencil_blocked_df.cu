// Temporally blocked double-float wave solves (2-D, second order, c = 1): the b and residual wave
// solves of the FP64 residual correction with double-float residuals, k_df sub-steps per launch
// instead of one.
//
// Same staging as the scalar FP32/FP64 blocked sweeps: a CTA stages a 64 x 64 region (tile of
// (64 - 2k)^2 nodes plus a halo of k), thread (warp w, lane) owns column 32 (w & 1) + lane and
// rows (w >> 1) + 16 t, t < 4, keeping W^n, W^{n-1} and the filter sum of its cells in registers,
// and W^n goes through shared memory (double-buffered, 8-byte hi/lo pairs) for the neighbours'
// reads.  At sub-step s only the window [s, 64 - s)^2 is advanced: with ~150 FP32 instructions
// per double-float update the shrinking window saves more than it costs.  Every update is the
// sequence of double-float operations of the single-step kernel k_step_df in its order,
//   W^{n+1} = ((b W^n - W^{n-1}) + a_x (W_l + W_r)) + a_y (W_d + W_u)  [- dt^2 cos(w t^n) f]
//   acc     = acc + w_{n+1} W^{n+1}
// so the result is bitwise that of single steps.  Global traffic per node and k steps: 3 reads
// and 3 writes of 8 bytes (+ f), against 5 per step.
#include <math.h>

#include "df64.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

constexpr int kDfReg = 64;
constexpr int kDfThreads = 1024;
constexpr int kDfPitch = kDfThreads / 64;    // rows between a thread's cells (16)
constexpr int kDfRows = kDfReg / kDfPitch;   // cells per thread (4)
constexpr int kDfMaxK = 8;
constexpr int kDfK = 4;                      // sub-steps per launch

struct BlockDfCoef {
  dfl a[2], b;
  dfl w[kDfMaxK];     // w_{n0+1} .. w_{n0+k}
  dfl fph[kDfMaxK];   // dt^2 cos(omega_hat t^n), n = n0 .. n0+k-1 (FORCE)
  int k;
};

enum DfBlkKind { DB_STEP = 0, DB_LAST_OUT = 1, DB_LAST_AV = 2 };

template <bool FORCE, int KIND>
__global__ void __launch_bounds__(kDfThreads) k_block2d_df(const dfl* __restrict__ gprev, const dfl* __restrict__ gcur,
                                                           dfl* __restrict__ oprev, dfl* __restrict__ ocur,
                                                           dfl* __restrict__ acc, const double* __restrict__ f,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ mw, double* __restrict__ out,
                                                           int nx, int ny, BlockDfCoef cf, double* partials,
                                                           unsigned* counter, double* scal_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dfl* const S0 = reinterpret_cast<dfl*>(smem_raw);
  dfl* const S1 = S0 + kDfReg * kDfReg;
  __shared__ dfl sw[kDfMaxK], sf[kDfMaxK];
  const int H = cf.k;
  const int TW = kDfReg - 2 * H;
  const int x0 = blockIdx.x * TW - H, y0 = blockIdx.y * TW - H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = 32 * (warp & 1) + lane;
  const int jb = warp >> 1;
  const int gx = x0 + i;
  const bool colin = gx >= 0 && gx < nx;
  if (threadIdx.x < kDfMaxK) {
    sw[threadIdx.x] = cf.w[threadIdx.x];
    sf[threadIdx.x] = cf.fph[threadIdx.x];
  }
  dfl cur[kDfRows], prv[kDfRows], acr[kDfRows];
  dfl ff[FORCE ? kDfRows : 1];
  const bool coltile0 = colin && i >= H && i < kDfReg - H;
#pragma unroll
  for (int t = 0; t < kDfRows; ++t) {
    const int j = jb + kDfPitch * t;
    const int gy = y0 + j;
    const bool in = colin && gy >= 0 && gy < ny;
    const int64_t gi = gx + (int64_t)nx * gy;
    cur[t] = in ? gcur[gi] : df_zero();
    prv[t] = in ? gprev[gi] : df_zero();
    if (FORCE) ff[t] = in ? df_from(f[gi]) : df_zero();
    acr[t] = (coltile0 && j >= H && j < kDfReg - H && in) ? acc[gi] : df_zero();
  }
#pragma unroll
  for (int t = 0; t < kDfRows; ++t) S0[(jb + kDfPitch * t) * kDfReg + i] = cur[t];
  __syncthreads();
  const dfl* A = S0;
  dfl* B = S1;
  for (int s = 1; s <= cf.k; ++s) {
    const int lo = s, hi = kDfReg - s;
    const bool colact = colin && i >= lo && i < hi;
    const dfl ws = sw[s - 1];
    const dfl fph = sf[s - 1];
#pragma unroll
    for (int t = 0; t < kDfRows; ++t) {
      const int j = jb + kDfPitch * t;
      const int gy = y0 + j;
      if (colact && j >= lo && j < hi && gy >= 0 && gy < ny) {
        const int l = j * kDfReg + i;
        const dfl c = cur[t];
        dfl wn = df_sub(df_mul(cf.b, c), prv[t]);
        const dfl sx = df_add(gx > 0 ? A[l - 1] : df_zero(), gx < nx - 1 ? A[l + 1] : df_zero());
        wn = df_add(wn, df_mul(cf.a[0], sx));
        const dfl sy = df_add(gy > 0 ? A[l - kDfReg] : df_zero(), gy < ny - 1 ? A[l + kDfReg] : df_zero());
        wn = df_add(wn, df_mul(cf.a[1], sy));
        if (FORCE) wn = df_sub(wn, df_mul(fph, ff[t]));
        prv[t] = c;
        cur[t] = wn;
        B[l] = wn;
        acr[t] = df_add(acr[t], df_mul(ws, wn));
      }
    }
    __syncthreads();
    dfl* tmp = const_cast<dfl*>(A);
    A = B;
    B = tmp;
  }
  double part = 0.0;
  const bool coltile = colin && i >= H && i < kDfReg - H;
#pragma unroll
  for (int t = 0; t < kDfRows; ++t) {
    const int j = jb + kDfPitch * t;
    const int gy = y0 + j;
    if (!(coltile && j >= H && j < kDfReg - H && gy >= 0 && gy < ny)) continue;
    const int64_t gi = gx + (int64_t)nx * gy;
    if (KIND == DB_STEP) {
      ocur[gi] = cur[t];
      oprev[gi] = prv[t];
      acc[gi] = acr[t];
    } else if (KIND == DB_LAST_OUT) {
      out[gi] = df_to(acr[t]);
    } else {
      const double vi = v[gi];
      const double o = vi - df_to(acr[t]);
      out[gi] = o;
      part = fma(mw ? vi * mw[gi] : vi, o, part);
    }
  }
  if (KIND == DB_LAST_AV) {
    part = block_sum(part);
    double total;
    if (grid_reduce(part, partials, counter, &total) && flat_tid() == 0) *scal_out = total;
  }
}

static constexpr int kDfSmem = 2 * kDfReg * kDfReg * (int)sizeof(dfl);   // 64 KB

template <bool FORCE>
static void df_attrs() {
  cudaFuncSetAttribute(k_block2d_df<FORCE, DB_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDfSmem);
  cudaFuncSetAttribute(k_block2d_df<FORCE, DB_LAST_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDfSmem);
  cudaFuncSetAttribute(k_block2d_df<FORCE, DB_LAST_AV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDfSmem);
}

// opt the double-float blocked kernels into 64 KB of dynamic shared memory once per process
// (outside any stream capture)
void blocked_df_init() {
  static bool done = false;
  if (done) return;
  done = true;
  df_attrs<false>();
  df_attrs<true>();
}

template <bool FORCE, int KIND>
static cudaError_t launch_df(whv_grid g, const dfl* gp, const dfl* gc, dfl* op, dfl* oc, dfl* acc, const double* f,
                             const double* v, double* out, const BlockDfCoef& cf, double* partials, unsigned* counter,
                             double* scal_out) {
  const int TW = kDfReg - 2 * cf.k;
  dim3 grid((g->n[0] + TW - 1) / TW, (g->n[1] + TW - 1) / TW, 1);
  k_block2d_df<FORCE, KIND><<<grid, kDfThreads, kDfSmem, g->stream>>>(gp, gc, op, oc, acc, f, v, g->mw, out, g->n[0],
                                                                     g->n[1], cf, partials, counter, scal_out);
  return cudaGetLastError();
}

// Steps n = 1 .. nt-1 of a 2-D double-float wave solve (c = 1) in sweeps of kDfK steps; the
// Taylor start has written W^0 -> bufs[0], W^1 -> bufs[1] and acc.
template <bool FORCE>
whv_status blocked_steps_2d_df(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                               int epi, int* launches, void* const* bufs, void* accbuf) {
  dfl* buf[4] = {(dfl*)bufs[0], (dfl*)bufs[1], (dfl*)bufs[2], (dfl*)bufs[3]};
  dfl* acc = (dfl*)accbuf;
  BlockDfCoef cf{};
  double asum = 0.0;
  for (int m = 0; m < 2; ++m) {
    const double am = tg.dt * tg.dt / (g->h[m] * g->h[m]);
    cf.a[m] = df_from(am);
    asum += am;
  }
  cf.b = df_from(2.0 - 2.0 * asum);
  double* part = chan(g, CH_STEP);
  unsigned* cnt = g->counters + CH_STEP;
  int pair = 0;   // input pair (buf[2 pair], buf[2 pair + 1]) = (W^{n-1}, W^n)
  int n = 1;
  int nl = 0;
  while (n < tg.nt) {
    const int k = std::min(kDfK, tg.nt - n);
    cf.k = k;
    for (int s = 0; s < k; ++s) {
      cf.w[s] = df_from(tg.weight[n + 1 + s]);
      cf.fph[s] = df_from(tg.dt * tg.dt * tg.phase[n + s]);
    }
    const bool last = (n + k == tg.nt);
    dfl *gp = buf[2 * pair], *gc = buf[2 * pair + 1], *op = buf[2 * (1 - pair)], *oc = buf[2 * (1 - pair) + 1];
    cudaError_t e;
    if (!last)
      e = launch_df<FORCE, DB_STEP>(g, gp, gc, op, oc, acc, f, nullptr, nullptr, cf, nullptr, nullptr, nullptr);
    else if (epi == 0)
      e = launch_df<FORCE, DB_LAST_OUT>(g, gp, gc, op, oc, acc, f, nullptr, out, cf, nullptr, nullptr, nullptr);
    else
      e = launch_df<FORCE, DB_LAST_AV>(g, gp, gc, op, oc, acc, f, v, out, cf, part, cnt, g->scal + S_PQ);
    if (e != cudaSuccess) return cuda_fail(g, e, "k_block2d_df launch");
    ++nl;
    pair = 1 - pair;
    n += k;
  }
  *launches = nl;
  return WHV_OK;
}

template whv_status blocked_steps_2d_df<false>(whv_grid, const TimeGridH&, const double*, const double*, double*, int,
                                               int*, void* const*, void*);
template whv_status blocked_steps_2d_df<true>(whv_grid, const TimeGridH&, const double*, const double*, double*, int,
                                              int*, void* const*, void*);

}  // namespace whv
