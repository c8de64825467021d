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

#include <vector>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

template <typename T>
struct StepCoef {
  T ih2[3];   // 1/h^2 per direction (order 4: 1/(12 h^2))
  T dt2;      // dt^2
  T fph;      // cos(omega_hat t^n) of the step (first step: 1)
  T w0, w1;   // first step: w_0, w_1; other steps: w1 = w_{n+1}
};

enum Kind { K_STEP = 0, K_LAST_OUT = 1, K_LAST_AV = 2 };

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

template <int DIM, int ORDER, typename T, typename S>
__device__ __forceinline__ T lap(const S* __restrict__ w, int64_t idx, int x, int y, int z, int nx,
                                 int ny, int nz, const StepCoef<T>& cf, T c) {
  T l = d2<ORDER, T>(w, idx, x, nx, 1, c) * cf.ih2[0];
  if (DIM > 1) l = fma(d2<ORDER, T>(w, idx, y, ny, (int64_t)nx, c), cf.ih2[1], l);
  if (DIM > 2) l = fma(d2<ORDER, T>(w, idx, z, nz, (int64_t)nx * ny, c), cf.ih2[2], l);
  return l;
}

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
    T L = lap<DIM, ORDER, T>(wc, idx, x, y, z, nx, ny, nz, cf, c);
    if (VARC) L *= c2[idx];
    if (FORCE) L = fma(-(T)f[idx], cf.fph, L);
    const T wn = fma(cf.dt2, L, fma(T(2), c, -wp[idx]));
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

// --------------------------------------------------------------------------- host side
struct LaunchShape {
  dim3 grid, block;
};

static LaunchShape shape_of(whv_grid g) {
  LaunchShape s;
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
  return cf;
}

template <typename T, int DIM, int ORDER, bool VARC, bool FORCE>
static whv_status launch_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                               double* out, int epi, int* nlaunch) {
  const LaunchShape ls = shape_of(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  T* b0 = (T*)g->wbuf[0];
  T* b1 = (T*)g->wbuf[1];
  T* acc = (T*)g->acc;
  const T* c2 = VARC ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
  StepCoef<T> cf = coef_of<T>(g, tg);
  if (v)
    k_first<T, DIM, ORDER, VARC, FORCE, false><<<ls.grid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf);
  else
    k_first<T, DIM, ORDER, VARC, FORCE, true><<<ls.grid, ls.block, 0, g->stream>>>(v, b0, b1, acc, c2, f, nx, ny, nz, cf);
  WHV_CUDA(g, cudaGetLastError());
  *nlaunch = 1;
  if constexpr (DIM == 2 && !FORCE) {
    const int kb = g->kblock > 0 ? g->kblock : default_kblock(g);
    if (kb > 1) {
      int nl = 0;
      whv_status s = blocked_steps_2d<T, ORDER, VARC>(g, tg, v, out, epi, kb, &nl);
      *nlaunch += nl;
      return s;
    }
  }
  *nlaunch += tg.nt - 1;
  // after the first step: W^{n-1} in b0, W^n in b1
  T* wprev = b0;
  T* wcur = b1;
  double* part = g->partials + CH_STEP * kMaxStepBlocks;
  unsigned* cnt = g->counters + CH_STEP;
  for (int n = 1; n < tg.nt; ++n) {
    cf.fph = (T)tg.phase[n];
    cf.w1 = (T)tg.weight[n + 1];
    const bool last = (n == tg.nt - 1);
    if (!last) {
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

template <typename T, int DIM, int ORDER>
static whv_status dispatch_vf(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                              double* out, int epi, int* nl) {
  const bool varc = g->c2 != nullptr;
  if (varc) {
    return f ? launch_solve<T, DIM, ORDER, true, true>(g, tg, v, f, out, epi, nl)
             : launch_solve<T, DIM, ORDER, true, false>(g, tg, v, f, out, epi, nl);
  }
  return f ? launch_solve<T, DIM, ORDER, false, true>(g, tg, v, f, out, epi, nl)
           : launch_solve<T, DIM, ORDER, false, false>(g, tg, v, f, out, epi, nl);
}

template <typename T>
static whv_status dispatch(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                           double* out, int epi, int* nl) {
  switch (g->dim * 10 + g->order) {
    case 12: return dispatch_vf<T, 1, 2>(g, tg, v, f, out, epi, nl);
    case 14: return dispatch_vf<T, 1, 4>(g, tg, v, f, out, epi, nl);
    case 22: return dispatch_vf<T, 2, 2>(g, tg, v, f, out, epi, nl);
    case 24: return dispatch_vf<T, 2, 4>(g, tg, v, f, out, epi, nl);
    case 32: return dispatch_vf<T, 3, 2>(g, tg, v, f, out, epi, nl);
    case 34: return dispatch_vf<T, 3, 4>(g, tg, v, f, out, epi, nl);
  }
  return fail(g, WHV_ERR_INVALID, "unsupported dim/order");
}

// default steps per sweep of the blocked 2-D kernel: FP32 stepping is bound by launches and
// L2 traffic (block 8 steps); FP64 stepping is bound by the FP64 pipe, where the redundant halo
// updates of a blocked sweep cost more than the launches they save (one step per launch)
int default_kblock(whv_grid g) { return g->precision == WHV_FP32_STEP ? 8 : 1; }

static whv_status launch_wave_solve(whv_grid g, const TimeGridH& tg, const double* v,
                                    const double* f, double* out, int epi, int* nl) {
  const LaunchShape ls = shape_of(g);
  if ((int64_t)ls.grid.x * ls.grid.y * ls.grid.z > kMaxStepBlocks)
    return fail(g, WHV_ERR_INVALID, "grid too large for the fused reduction");
  return g->precision == WHV_FP64 ? dispatch<double>(g, tg, v, f, out, epi, nl)
                                  : dispatch<float>(g, tg, v, f, out, epi, nl);
}

// ------------------------------------------------------------------ CUDA graph cache
// A wave solve is Nt kernel launches; the solvers replay it many times with the same pointers,
// so each (pointers, time grid) combination is captured once into a CUDA graph.
struct PlanEntry {
  const double *v, *f;
  double* out;
  int epi;
  double omega, cfl;
  int periods, adjust, nt, kblock;
  int launches;   // kernels in the graph
  cudaGraphExec_t exec;
  unsigned long long last_use;
};

struct StepPlan {
  std::vector<PlanEntry> entries;
  unsigned long long tick = 0;
};

void free_plan(whv_grid g) {
  if (!g->plan) return;
  for (auto& e : g->plan->entries) cudaGraphExecDestroy(e.exec);
  delete g->plan;
  g->plan = nullptr;
}

whv_status wave_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                      double* out, int epi) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  WHV_CUDA(g, cudaStreamIsCapturing(g->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // caller is capturing: record the launches into its graph
    int nl = 0;
    whv_status s = launch_wave_solve(g, tg, v, f, out, epi, &nl);
    count_launches(nl);
    return s;
  }
  if (!g->plan) g->plan = new StepPlan();
  StepPlan* P = g->plan;
  P->tick++;
  for (auto& e : P->entries) {
    if (e.v == v && e.f == f && e.out == out && e.epi == epi && e.omega == tg.omega &&
        e.cfl == tg.cfl && e.periods == tg.periods && e.adjust == tg.adjust && e.nt == tg.nt &&
        e.kblock == g->kblock) {
      e.last_use = P->tick;
      WHV_CUDA(g, cudaGraphLaunch(e.exec, g->stream));
      count_launches(e.launches);
      return WHV_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  WHV_CUDA(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  int nl = 0;
  whv_status s = launch_wave_solve(g, tg, v, f, out, epi, &nl);
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
                                g->kblock, nl, exec, P->tick});
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
  *k = g->kblock > 0 ? g->kblock : default_kblock(g);
  return WHV_OK;
}

// Autotuner of the steps per sweep: times two f = 0 wave solves per candidate (graph replay,
// CUDA events on the grid's stream, after one warm-up replay) and keeps the fastest.
extern "C" whv_status whv_autotune(whv_grid g, const whv_params* p, int* best) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  const int cands2d[] = {1, 2, 4, 6, 8, 10, 12, 16};
  const int cands_other[] = {1};
  const int* cands = g->dim == 2 ? cands2d : cands_other;
  const int nc = g->dim == 2 ? 8 : 1;
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
