// Grid lifetime, time grid, speed, basis bookkeeping and the small C-ABI entry points.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

static thread_local std::string t_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

whv_status fail(whv_grid g, whv_status s, const std::string& msg) {
  if (g) g->err = msg; else t_last_error = msg;
  return s;
}

void hold_vectors(Basis& b) {
  b.vhold = std::shared_ptr<void>(b.V, [](void* p) { if (p) cudaFree(p); });
}

void free_basis(whv_grid g) {
  Basis& b = g->basis;
  b.vhold.reset();   // the vectors go with the last grid that uses them
  for (void* p : {(void*)b.d_coef, (void*)b.AW, (void*)b.Einv, (void*)b.QAW, (void*)b.cU, (void*)b.cV,
                  (void*)b.cs, (void*)b.cT, (void*)b.cc, (void*)b.cR, (void*)b.coff, (void*)b.cowner})
    if (p) cudaFree(p);
  g->basis = Basis();
  free_cgloop(g);
}

whv_status cuda_fail(whv_grid g, cudaError_t e, const char* what) {
  std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                  ") in " + what;
  return fail(g, e == cudaErrorMemoryAllocation ? WHV_ERR_OOM : WHV_ERR_CUDA, m);
}

// Time grid of Sec. 2.2 (reading): dt0 = cfl h_min / c_max, Tbar = Np 2 pi / omega,
// Nt = ceil(Tbar/dt0), dt = Tbar/Nt; with adjust_omega the smallest Nt with
// dt = 2 sin(pi Np / Nt)/omega <= dt0 and omega_hat = 2 pi Np/(Nt dt), so that
// (2/dt) sin(omega_hat dt / 2) = omega.  Trapezoid weights of eq. quadrature.
whv_status make_time_grid(whv_grid g, const whv_params* p, TimeGridH* tg) {
  if (!p) return fail(g, WHV_ERR_INVALID, "params is NULL");
  if (!(p->omega > 0.0) || !isfinite(p->omega)) return fail(g, WHV_ERR_INVALID, "omega must be > 0");
  if (p->periods < 1) return fail(g, WHV_ERR_INVALID, "periods must be >= 1");
  const double cfl = p->cfl > 0.0 ? p->cfl : (g->order == 2 ? 0.5 : 0.4);
  double hmin = g->h[0];
  for (int m = 1; m < g->dim; ++m) hmin = std::min(hmin, g->h[m]);
  const double cmax = sqrt(g->c2max);
  const double dt0 = cfl * hmin / cmax;
  const double pi = 3.14159265358979323846;
  TimeGridH t;
  t.omega = p->omega; t.periods = p->periods; t.adjust = p->adjust_omega ? 1 : 0; t.cfl = cfl;
  if (!t.adjust) {
    t.tbar = p->periods * 2.0 * pi / p->omega;
    double q = ceil(t.tbar / dt0);
    if (q > 1e7) return fail(g, WHV_ERR_INVALID, "more than 1e7 time steps per wave solve");
    t.nt = (int)q;
    t.dt = t.tbar / t.nt;
    t.omega_hat = p->omega;
  } else {
    int nt = 2 * p->periods + 1;
    while (2.0 * sin(pi * p->periods / nt) / p->omega > dt0) {
      if (++nt > 10000000) return fail(g, WHV_ERR_INVALID, "more than 1e7 time steps per wave solve");
    }
    t.nt = nt;
    t.dt = 2.0 * sin(pi * p->periods / nt) / p->omega;
    t.omega_hat = 2.0 * pi * p->periods / (nt * t.dt);
    t.tbar = nt * t.dt;
  }
  if (t.nt < 2) return fail(g, WHV_ERR_INVALID, "fewer than 2 time steps per wave solve");
  t.omega_eff = 2.0 / t.dt * sin(t.omega_hat * t.dt / 2.0);
  // explicit leapfrog stability: dt^2 lambda_max^2 / 4 <= 1 (Fourier bound of -L_h)
  const double per = g->order == 2 ? 4.0 : 16.0 / 3.0;
  double lmax = 0.0;
  for (int m = 0; m < g->dim; ++m) lmax += per / (g->h[m] * g->h[m]);
  lmax *= g->c2max;
  if (t.dt * t.dt * lmax / 4.0 > 1.0)
    return fail(g, WHV_ERR_INVALID, "time step above the explicit leapfrog stability limit (lower cfl)");
  t.phase.resize(t.nt + 1);
  t.weight.resize(t.nt + 1);
  for (int n = 0; n <= t.nt; ++n) {
    const double ph = cos(t.omega_hat * (n * t.dt));
    const double eta = (n == 0 || n == t.nt) ? 0.5 : 1.0;
    t.phase[n] = ph;
    t.weight[n] = (2.0 / t.tbar) * eta * (ph - 0.25) * t.dt;
  }
  *tg = std::move(t);
  return WHV_OK;
}

// ---------------------------------------------------------------------------- kernels
__global__ void k_speed_setup(const double* __restrict__ c2in, double* __restrict__ c2,
                              float* __restrict__ c2f, double* __restrict__ mw, int64_t n,
                              double* partials, unsigned* counter, double* scal) {
  double bad = 0.0, mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = c2in[i];
    if (!(v > 0.0) || !isfinite(v)) bad += 1.0;
    c2[i] = v;
    c2f[i] = (float)v;
    mw[i] = 1.0 / v;
    mx = fmax(mx, v);
  }
  // max via a second shared pass: reuse the sum reduction on "bad" and keep max in S_TMP2
  __shared__ double smx[32];
  mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, 16));
  mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, 8));
  mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, 4));
  mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, 2));
  mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, 1));
  if ((threadIdx.x & 31) == 0) smx[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, smx[w]);
    partials[kRedBlocks + blockIdx.x] = m;  // second half of the channel: block maxima
  }
  __syncthreads();
  double total;
  if (grid_reduce(bad, partials, counter, &total) && threadIdx.x == 0) {
    double m = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) m = fmax(m, __ldcg(partials + kRedBlocks + b));
    scal[S_TMP] = total;
    scal[S_TMP2] = m;
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
void* tensor_map_encoder() {
  static void* fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = p;
  }
  return fn;
}

}  // namespace whv

using namespace whv;

// ============================================================================ C ABI
extern "C" {

const char* whv_version(void) { return "whv 0.1 (sm_103a)"; }

int64_t whv_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* whv_last_error(whv_grid g) { return g ? g->err.c_str() : t_last_error.c_str(); }

int64_t whv_num_unknowns(whv_grid g) { return g ? g->N : 0; }

static void free_all(whv_grid g) {
  if (!g) return;
  free_plan(g);
  void* ptrs[] = {g->c2, g->c2f, g->mw, g->wbuf[0], g->wbuf[1], g->wbuf[2], g->wbuf[3], g->acc, g->x, g->r, g->p, g->q,
                  g->t, g->fd, g->krylov, g->small, g->small2, g->partials, g->counters, g->scal,
                  g->basis.d_coef, g->basis.AW, g->basis.Einv, g->basis.QAW, g->basis.cU, g->basis.cV,
                  g->basis.cs, g->basis.cT, g->basis.cc, g->basis.cR, g->basis.coff, g->basis.cowner, g->wbuf64[0], g->wbuf64[1], g->wbuf64[2],
                  g->wbuf64[3], g->acc64, g->tw[0], g->tw[1], g->tw[2], g->tw[3], g->tacc, g->pw3[0], g->pw3[1], g->pw3[2], g->pw3[3], g->pacc3, g->maps3, g->xo, g->ro, g->bo, g->wtab_small, g->face64[0], g->face64[1],
                  g->face64[2], g->face32[0], g->face32[1], g->face32[2]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->scal_host) cudaFreeHost(g->scal_host);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
}

whv_status whv_create_grid(int dim, const int64_t npts[3], const double lo[3], const double hi[3],
                           int order, int precision, void* cuda_stream, whv_grid* out) {
  if (!out) return fail(nullptr, WHV_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (dim < 1 || dim > 3) return fail(nullptr, WHV_ERR_INVALID, "dim must be 1, 2 or 3");
  if (order != 2 && order != 4) return fail(nullptr, WHV_ERR_INVALID, "order must be 2 or 4");
  if (precision != WHV_FP64 && precision != WHV_FP32_STEP)
    return fail(nullptr, WHV_ERR_INVALID, "precision must be WHV_FP64 or WHV_FP32_STEP");
  if (!npts) return fail(nullptr, WHV_ERR_INVALID, "npts is NULL");
  blocked_init();
  step3d2_init();
  whv_grid g = new whv_grid_s();
  g->dim = dim; g->order = order; g->precision = precision;
  int64_t N = 1;
  for (int m = 0; m < 3; ++m) {
    if (m < dim) {
      const int64_t minpts = order == 4 ? 4 : 3;
      if (npts[m] < minpts || npts[m] > (int64_t)1 << 30) {
        delete g;
        return fail(nullptr, WHV_ERR_INVALID, "npts out of range (>= 3, >= 4 for order 4)");
      }
      g->npts[m] = npts[m];
      g->n[m] = (int)(npts[m] - 2);
      g->lo[m] = lo ? lo[m] : 0.0;
      g->hi[m] = hi ? hi[m] : 1.0;
      if (!(g->hi[m] > g->lo[m])) {
        delete g;
        return fail(nullptr, WHV_ERR_INVALID, "hi must exceed lo");
      }
      g->h[m] = (g->hi[m] - g->lo[m]) / (double)(npts[m] - 1);
      N *= g->n[m];
    } else {
      g->npts[m] = 3; g->n[m] = 1; g->h[m] = 1.0;
    }
  }
  if (N > ((int64_t)1 << 31)) {
    delete g;
    return fail(nullptr, WHV_ERR_INVALID, "more than 2^31 unknowns");
  }
  g->N = N;
  cudaError_t e;
  if (cuda_stream) {
    g->stream = (cudaStream_t)cuda_stream;
  } else {
    // legacy default stream cannot be captured into graphs: use a blocking stream, which
    // still orders itself with the legacy default stream
    e = cudaStreamCreate(&g->stream);
    if (e != cudaSuccess) { whv_status s = cuda_fail(nullptr, e, "cudaStreamCreate"); delete g; return s; }
    g->own_stream = true;
  }
  const size_t esz = precision == WHV_FP64 ? sizeof(double) : sizeof(float);
  const size_t nb = (size_t)N;
  struct A { void** p; size_t bytes; } allocs[] = {
      {&g->wbuf[0], nb * esz}, {&g->wbuf[1], nb * esz}, {&g->wbuf[2], nb * esz},
      {&g->wbuf[3], nb * esz}, {&g->acc, nb * esz},
      {(void**)&g->x, nb * 8}, {(void**)&g->r, nb * 8}, {(void**)&g->p, nb * 8},
      {(void**)&g->q, nb * 8}, {(void**)&g->t, nb * 8}, {(void**)&g->fd, nb * 8},
      {(void**)&g->small, (size_t)kMaxND * 8}, {(void**)&g->small2, (size_t)kMaxND * 8},
      {(void**)&g->partials, 0},   // sized below
      {(void**)&g->counters, (size_t)CH_NCH * sizeof(unsigned)},
      {(void**)&g->scal, (size_t)S_NSLOTS * 8}};
  // reduction channels: step kernels (<= N/256 blocks + slack), grid-stride reductions
  // (2 x kRedBlocks: the speed set-up keeps block maxima after the sums), projections
  // (ceil(N/2048) blocks x up to kMaxND columns)
  g->chan_cap[CH_STEP] = N / 32 + 4096;
  g->chan_cap[CH_UPDATE] = 2 * kRedBlocks;
  g->chan_cap[CH_DOT] = 2 * kRedBlocks;
  g->chan_cap[CH_PROJ] = ((N + 2047) / 2048) * kMaxND;
  int64_t off = 0;
  for (int ch = 0; ch < CH_NCH; ++ch) { g->chan_off[ch] = off; off += g->chan_cap[ch]; }
  for (auto& a : allocs)
    if (a.p == (void**)&g->partials) a.bytes = (size_t)off * sizeof(double);
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      whv_status s = cuda_fail(nullptr, e, "cudaMalloc (grid scratch)");
      free_all(g);
      delete g;
      return s;
    }
  }
  e = cudaMallocHost((void**)&g->scal_host, S_NSLOTS * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->counters, 0, CH_NCH * sizeof(unsigned), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->scal, 0, S_NSLOTS * 8, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    whv_status s = cuda_fail(nullptr, e, "grid setup");
    free_all(g);
    delete g;
    return s;
  }
  *out = g;
  return WHV_OK;
}

whv_status whv_destroy_grid(whv_grid g) {
  if (!g) return WHV_OK;
  cudaStreamSynchronize(g->stream);
  free_all(g);
  delete g;
  return WHV_OK;
}

// face values of the conservative operator: face[m][idx] between node idx and its + neighbour
// along axis m (mean of the two c^2), or the node's own c^2 on the face to the boundary node
__global__ void k_faces(const double* __restrict__ c2, int nx, int ny, int nz, int dim, double* __restrict__ f0,
                        double* __restrict__ f1, double* __restrict__ f2, float* __restrict__ g0,
                        float* __restrict__ g1, float* __restrict__ g2) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((int64_t)nx * ny));
    const double c = c2[idx];
    const double fx = x < nx - 1 ? 0.5 * (c + c2[idx + 1]) : c;
    f0[idx] = fx; g0[idx] = (float)fx;
    if (dim > 1) {
      const double fy = y < ny - 1 ? 0.5 * (c + c2[idx + nx]) : c;
      f1[idx] = fy; g1[idx] = (float)fy;
    }
    if (dim > 2) {
      const double fz = z < nz - 1 ? 0.5 * (c + c2[idx + (int64_t)nx * ny]) : c;
      f2[idx] = fz; g2[idx] = (float)fz;
    }
  }
}

// *flag = 1 if a and b differ anywhere (bitwise comparison of two c^2 arrays)
__global__ void k_differ(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                         double* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) *flag = 1.0;
}

static void free_faces(whv_grid g) {
  for (int m = 0; m < 3; ++m) {
    if (g->face64[m]) cudaFree(g->face64[m]);
    if (g->face32[m]) cudaFree(g->face32[m]);
    g->face64[m] = nullptr;
    g->face32[m] = nullptr;
  }
  g->cons = 0;
}

whv_status whv_set_speed(whv_grid g, const double* c2_dev) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  // any basis was built for the old operator
  free_basis(g);
  free_plan(g);
  free_faces(g);
  if (!c2_dev) {
    if (g->c2) cudaFree(g->c2);
    if (g->c2f) cudaFree(g->c2f);
    if (g->mw) cudaFree(g->mw);
    g->c2 = nullptr; g->c2f = nullptr; g->mw = nullptr;
    g->c2max = 1.0;
    return WHV_OK;
  }
  if (!g->c2) WHV_CUDA(g, cudaMalloc(&g->c2, g->N * 8));
  if (!g->c2f) WHV_CUDA(g, cudaMalloc(&g->c2f, g->N * 4));
  if (!g->mw) WHV_CUDA(g, cudaMalloc(&g->mw, g->N * 8));
  k_speed_setup<<<kRedBlocks, 256, 0, g->stream>>>(c2_dev, g->c2, g->c2f, g->mw, g->N,
                                                   chan(g, CH_DOT),
                                                   g->counters + CH_DOT, g->scal);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  whv_status st = fetch_scalars(g);
  if (st != WHV_OK) return st;
  if (g->scal_host[S_TMP] != 0.0) {
    cudaFree(g->c2); cudaFree(g->c2f); cudaFree(g->mw);
    g->c2 = nullptr; g->c2f = nullptr; g->mw = nullptr; g->c2max = 1.0;
    return fail(g, WHV_ERR_INVALID, "c^2 must be finite and > 0 at every interior node");
  }
  g->c2max = g->scal_host[S_TMP2];
  return WHV_OK;
}

whv_status whv_set_speed_form(whv_grid g, const double* c2_dev, int form) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (form != WHV_SPEED_NONCONSERVATIVE && form != WHV_SPEED_CONSERVATIVE)
    return fail(g, WHV_ERR_INVALID, "unknown speed form");
  if (form == WHV_SPEED_CONSERVATIVE && (!c2_dev || g->order != 2))
    return fail(g, WHV_ERR_INVALID, "the conservative form needs c^2 and a second-order grid");
  whv_status s = whv_set_speed(g, c2_dev);
  if (s != WHV_OK || form == WHV_SPEED_NONCONSERVATIVE) return s;
  // div_h(c^2 grad_h) is symmetric in the Euclidean inner product: no M weights
  cudaFree(g->mw);
  g->mw = nullptr;
  for (int m = 0; m < g->dim; ++m) {
    WHV_CUDA(g, cudaMalloc(&g->face64[m], g->N * 8));
    WHV_CUDA(g, cudaMalloc(&g->face32[m], g->N * 4));
  }
  k_faces<<<kRedBlocks, 256, 0, g->stream>>>(g->c2, g->n[0], g->n[1], g->n[2], g->dim, g->face64[0], g->face64[1],
                                             g->face64[2], g->face32[0], g->face32[1], g->face32[2]);
  count_launches(1);
  WHV_CUDA(g, cudaGetLastError());
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  g->cons = 1;
  return WHV_OK;
}

whv_status whv_time_grid(whv_grid g, const whv_params* p, int* nt, double* dt, double* omega_hat,
                         double* omega_eff) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  if (nt) *nt = tg.nt;
  if (dt) *dt = tg.dt;
  if (omega_hat) *omega_hat = tg.omega_hat;
  if (omega_eff) *omega_eff = tg.omega_eff;
  return WHV_OK;
}

whv_status whv_set_deflation_basis(whv_grid g, const whv_params* p, int nd, const double* V_dev,
                                   const double* lambda2_host, int mode, int flags) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (mode == WHV_BASIS_NONE) {
    free_basis(g);
    return WHV_OK;
  }
  TimeGridH tg;
  whv_status s = make_time_grid(g, p, &tg);
  if (s != WHV_OK) return s;
  if (nd < 1 || nd > kMaxND || nd > g->N)
    return fail(g, WHV_ERR_INVALID, "nd must be in [1, min(N, 1024)]");
  Basis b;
  b.nd = nd; b.mode = mode; b.flags = flags;
  b.omega = p->omega; b.periods = p->periods; b.adjust = p->adjust_omega ? 1 : 0; b.cfl = tg.cfl;
  if (mode == WHV_BASIS_USER) {
    if (!V_dev || !lambda2_host) return fail(g, WHV_ERR_INVALID, "USER basis needs V_dev and lambda2_host");
    WHV_CUDA(g, cudaMalloc(&b.V, (size_t)g->N * nd * 8));
    WHV_CUDA(g, cudaMemcpyAsync(b.V, V_dev, (size_t)g->N * nd * 8, cudaMemcpyDeviceToDevice, g->stream));
    b.lambda2.assign(lambda2_host, lambda2_host + nd);
    b.mu.resize(nd);
    // mu = 1 - beta_h(lambda), the eigenvalue of A on a true eigenvector
    for (int m = 0; m < nd; ++m) {
      const double x = 1.0 - 0.5 * tg.dt * tg.dt * b.lambda2[m];
      if (!(fabs(x) <= 1.0)) { cudaFree(b.V); return fail(g, WHV_ERR_INVALID, "lambda^2 outside the stable range"); }
      const double th = acos(x);
      double be = 0.0;
      for (int n = 0; n <= tg.nt; ++n) be += tg.weight[n] * cos(n * th);
      b.mu[m] = 1.0 - be;
    }
    b.modes.assign((size_t)nd * g->dim, 0);
  } else if (mode == WHV_BASIS_CLOSED_FORM) {
    if (g->c2) return fail(g, WHV_ERR_INVALID, "closed-form basis needs c = 1");
    b.flags |= WHV_BASIS_EXACT;
    s = closed_form_basis(g, tg, nd, &b);
    if (s != WHV_OK) { if (b.V) cudaFree(b.V); return s; }
  } else if (mode == WHV_BASIS_LANCZOS) {
    const int64_t mm = std::min<int64_t>(std::min<int64_t>(g->N, kMaxND), std::max(4 * nd, nd + 40));
    return whv_lanczos(g, p, nd, (int)mm, V_dev, 1, flags | WHV_BASIS_REDEFLATE, nullptr, nullptr);
  } else {
    return fail(g, WHV_ERR_INVALID, "unknown basis mode");
  }
  {
    const cudaError_t e = cudaMalloc(&b.d_coef, (size_t)kMaxND * 8);
    if (e != cudaSuccess) { if (b.V) cudaFree(b.V); return cuda_fail(g, e, "cudaMalloc (basis scratch)"); }
  }
  hold_vectors(b);
  free_basis(g);
  g->basis = std::move(b);
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}

whv_status whv_share_basis(whv_grid dst, whv_grid src) {
  if (!dst || !src) return fail(dst, WHV_ERR_INVALID, "whv_share_basis: grid is NULL");
  if (dst == src) return WHV_OK;
  const Basis& s = src->basis;
  if (s.nd == 0 || !s.V) return fail(dst, WHV_ERR_INVALID, "whv_share_basis: the source grid has no dense basis");
  bool same = dst->dim == src->dim && dst->order == src->order && dst->cons == 0 && src->cons == 0 &&
              (dst->c2 == nullptr) == (src->c2 == nullptr);
  for (int m = 0; m < 3 && same; ++m)
    same = dst->n[m] == src->n[m] && dst->lo[m] == src->lo[m] && dst->hi[m] == src->hi[m];
  if (!same)
    return fail(dst, WHV_ERR_INVALID,
                "whv_share_basis: grids differ in shape, box, order or speed kind (conservative grids cannot share)");
  if (dst->c2) {   // the basis is M-orthonormal for src's c^2: dst must have the same field
    WHV_CUDA(dst, cudaStreamSynchronize(src->stream));
    dst->scal_host[S_TMP] = 0.0;
    WHV_CUDA(dst, cudaMemcpyAsync(dst->scal + S_TMP, dst->scal_host + S_TMP, sizeof(double), cudaMemcpyHostToDevice,
                                  dst->stream));
    k_differ<<<kRedBlocks, 256, 0, dst->stream>>>(dst->c2, src->c2, dst->N, dst->scal + S_TMP);
    count_launches(1);
    WHV_CUDA(dst, cudaGetLastError());
    TRY(fetch_scalars(dst));
    if (dst->scal_host[S_TMP] != 0.0) return fail(dst, WHV_ERR_INVALID, "whv_share_basis: the grids' c^2 differ");
  }
  Basis b;
  b.nd = s.nd; b.mode = s.mode; b.flags = s.flags;
  b.V = s.V; b.vhold = s.vhold;
  b.lambda2 = s.lambda2; b.mu = s.mu; b.modes = s.modes;
  b.omega = s.omega; b.periods = s.periods; b.adjust = s.adjust; b.cfl = s.cfl;
  WHV_CUDA(dst, cudaMalloc(&b.d_coef, (size_t)kMaxND * 8));
  // src's pending writes of the vectors must land before dst's stream reads them
  WHV_CUDA(dst, cudaStreamSynchronize(src->stream));
  free_basis(dst);
  dst->basis = std::move(b);
  return WHV_OK;
}

whv_status whv_get_basis(whv_grid g, int* nd, int* modes_host, double* lambda2_host, double* V_dev) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  const Basis& b = g->basis;
  if (nd) *nd = b.nd;
  if (b.nd == 0) return WHV_OK;
  if (modes_host) std::memcpy(modes_host, b.modes.data(), b.modes.size() * sizeof(int));
  if (lambda2_host) std::memcpy(lambda2_host, b.lambda2.data(), b.nd * sizeof(double));
  if (V_dev) {   // the compressed vectors are written out dense
    for (int m = 0; m < b.nd; ++m) {
      whv_status s = basis_column(g, m, V_dev + (size_t)m * g->N);
      if (s != WHV_OK) return s;
    }
    WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  }
  return WHV_OK;
}

whv_status whv_project(whv_grid g, const double* r_dev, double* coeff_dev) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (g->basis.nd == 0) return fail(g, WHV_ERR_INVALID, "no deflation basis set");
  if (!r_dev || !coeff_dev) return fail(g, WHV_ERR_INVALID, "NULL pointer");
  return basis_project(g, r_dev, coeff_dev);
}

whv_status whv_expand(whv_grid g, const double* y_dev, double alpha, double* out_dev) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (g->basis.nd == 0) return fail(g, WHV_ERR_INVALID, "no deflation basis set");
  if (!y_dev || !out_dev) return fail(g, WHV_ERR_INVALID, "NULL pointer");
  return basis_expand(g, y_dev, alpha, out_dev);
}

whv_status whv_dot(whv_grid g, const double* x_dev, const double* y_dev, double* out_host) {
  if (!g) return fail(nullptr, WHV_ERR_INVALID, "grid is NULL");
  if (!x_dev || !y_dev || !out_host) return fail(g, WHV_ERR_INVALID, "NULL pointer");
  whv_status s = dot_async(g, x_dev, y_dev, S_TMP);
  if (s != WHV_OK) return s;
  s = fetch_scalars(g);
  if (s != WHV_OK) return s;
  *out_host = g->scal_host[S_TMP];
  return WHV_OK;
}

}  // extern "C"
