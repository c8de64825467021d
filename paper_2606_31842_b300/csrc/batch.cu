// Batched solves: many independent problems -- right-hand sides, frequencies and grids of uneven
// size -- advanced together.
//
// One persistent cooperative kernel (k_batch_wave) performs a wave solve of every active problem:
// at global step s it sweeps the tiles of all problems whose Nt exceeds s (problems sorted by Nt,
// so they are a prefix of the list), then all CTAs meet at a grid barrier before step s + 1.
// Problems with fewer steps drop out early; converged problems are skipped.  The barrier spins
// with an iteration limit: a CTA that gives up raises an error flag and every CTA returns.
//
// The batched CG loop is one CUDA graph: a conditional WHILE node whose body is the persistent
// wave solve (q_p = A p_p for all p, with the per-tile partial sums of p^T M q), a finishing
// kernel (p^T M q per problem, deterministic order), each problem's fused CG update and direction
// update (which return at once for stopped problems), a per-problem convergence check and a
// one-thread kernel that keeps the loop running while any problem is active.  DEVD (Algorithm 2)
// deflation / inflation per problem happens before and after, with each grid's basis.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "stencil_ops.cuh"
#include "whv_device.cuh"
#include "whv_internal.cuh"

namespace whv {

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

constexpr unsigned long long kBarrierSpins = 1ull << 26;   // x 64 ns sleeps: ~4 s

// Grid-wide barrier of a cooperative launch with a bounded wait.  Returns false (and raises
// *err) if a CTA waited past the limit or another CTA raised *err.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, int* err, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned* vgen = gen;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    int ok = 1;
    if (arrived == nblocks) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == g0) {
        if (++spins > kBarrierSpins) { atomicExch(err, 1); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kBatchMaxProblems = 1024;

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
      if (B.halt && *B.halt != 0.0) continue;   // uniform per block
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

// p^T M q of every problem from its per-tile partial sums (one block per problem, fixed order)
template <typename T>
__global__ void k_batch_finish(const BProb<T>* __restrict__ P, double* const* __restrict__ scal) {
  const BProb<T>& B = P[blockIdx.x];
  if (B.epi != 1 || (B.halt && *B.halt != 0.0)) return;
  double s = 0.0;
  for (int t = threadIdx.x; t < B.ntiles; t += blockDim.x) s += B.partials[t];
  s = block_sum(s);
  if (threadIdx.x == 0) scal[blockIdx.x][S_PQ] = s;
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

// keep the WHILE loop running while any problem is active
__global__ void k_batch_any(cudaGraphConditionalHandle h, double* const* __restrict__ scal, int np,
                            const int* __restrict__ err) {
  int any = 0;
  for (int p = 0; p < np; ++p) any |= scal[p][S_HALT] == 0.0;
  if (*err) any = 0;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

struct BatchScratch {
  void* desc = nullptr;       // BProb<T>[np] for the A p solves
  void* desc_b = nullptr;     // BProb<T>[np] for the b solves
  int* nact = nullptr;
  void* wtab = nullptr;
  void* ptab = nullptr;
  double** scal = nullptr;
  unsigned* bar = nullptr;    // count, generation
  int* err = nullptr;
  void free_all() {
    for (void* p : {desc, desc_b, (void*)nact, wtab, ptab, (void*)scal, (void*)bar, (void*)err})
      if (p) cudaFree(p);
  }
};

template <typename T, int DIM, int ORDER, bool VARC>
static cudaError_t launch_batch_wave(cudaStream_t st, const void* desc, const int* nact, int S, const void* wtab,
                                     const void* ptab, unsigned* bar, int* err, int nblocks) {
  const BProb<T>* P = (const BProb<T>*)desc;
  const T* w = (const T*)wtab;
  const T* ph = (const T*)ptab;
  unsigned* bc = bar;
  unsigned* bg = bar + 1;
  void* args[] = {(void*)&P, (void*)&nact, (void*)&S, (void*)&w, (void*)&ph, (void*)&bc, (void*)&bg, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_batch_wave<T, DIM, ORDER, VARC>, dim3(nblocks), dim3(32, 8),
                                     args, 0, st);
}

template <typename T, int DIM, int ORDER, bool VARC>
static int max_coresident(int sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_wave<T, DIM, ORDER, VARC>, 256, 0);
  return std::max(1, per_sm) * sms;
}

template <typename T, int DIM, int ORDER, bool VARC>
static whv_status batched_cg(int np, const whv_grid* grids, const whv_params* params,
                             const std::vector<TimeGridH>& tgs, const std::vector<const double*>& rhs_force,
                             whv_info* infos, int* iters_out, BatchScratch& bs) {
  whv_grid g0 = grids[0];
  cudaStream_t st = g0->stream;
  // problems sorted by Nt descending: the active ones at step s are a prefix
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tgs[a].nt > tgs[b].nt; });
  const int S = tgs[order[0]].nt;
  std::vector<BProb<T>> desc(np), desc_b(np);
  std::vector<T> wtab, ptab;
  std::vector<double*> scal(np);
  int64_t tile0 = 0;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = grids[p];
    const TimeGridH& tg = tgs[p];
    BProb<T> B{};
    B.w0 = (T*)g->wbuf[0];
    B.w1 = (T*)g->wbuf[1];
    B.acc = (T*)g->acc;
    B.c2 = VARC ? (const T*)(sizeof(T) == 8 ? (const void*)g->c2 : (const void*)g->c2f) : nullptr;
    B.mw = g->mw;
    B.partials = chan(g, CH_STEP);
    B.halt = g->scal + S_HALT;
    B.nx = g->n[0]; B.ny = g->n[1]; B.nz = g->n[2];
    B.nt = tg.nt;
    B.tx = (g->n[0] + 31) / 32;
    B.ty = (g->n[1] + 7) / 8;
    B.ntiles = B.tx * B.ty * (DIM > 2 ? g->n[2] : 1);
    if (B.ntiles > chan_cap(g, CH_STEP)) return fail(g0, WHV_ERR_INVALID, "batched: grid too large for its reduction channel");
    B.tile0 = tile0;
    tile0 += B.ntiles;
    B.wofs = (int)wtab.size();
    for (int n = 0; n <= tg.nt; ++n) { wtab.push_back((T)tg.weight[n]); ptab.push_back((T)tg.phase[n]); }
    for (int m = 0; m < 3; ++m) {
      const double h2 = g->h[m] * g->h[m];
      B.cf.ih2[m] = (T)(g->order == 2 ? 1.0 / h2 : 1.0 / (12.0 * h2));
    }
    B.cf.dt2 = (T)(tg.dt * tg.dt);
    // A p solves: v = p, out = q, epi 1
    B.v = g->p; B.f = nullptr; B.out = g->q; B.epi = 1;
    desc[k] = B;
    // b solves: v = 0, forcing, out = t (b), epi 0, never halted
    BProb<T> Bb = B;
    Bb.v = nullptr; Bb.f = rhs_force[p]; Bb.out = g->t; Bb.epi = 0; Bb.halt = nullptr;
    desc_b[k] = Bb;
    scal[k] = g->scal;
  }
  std::vector<int> nact(S);
  for (int s = 0; s < S; ++s) {
    int a = 0;
    while (a < np && tgs[order[a]].nt > s) ++a;
    nact[s] = a;
  }
  // device tables
#define B_CUDA(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) return cuda_fail(g0, _e, #call); } while (0)
  B_CUDA(cudaMalloc(&bs.desc, np * sizeof(BProb<T>)));
  B_CUDA(cudaMalloc(&bs.desc_b, np * sizeof(BProb<T>)));
  B_CUDA(cudaMalloc(&bs.nact, S * sizeof(int)));
  B_CUDA(cudaMalloc(&bs.wtab, wtab.size() * sizeof(T)));
  B_CUDA(cudaMalloc(&bs.ptab, ptab.size() * sizeof(T)));
  B_CUDA(cudaMalloc(&bs.scal, np * sizeof(double*)));
  B_CUDA(cudaMalloc(&bs.bar, 2 * sizeof(unsigned)));
  B_CUDA(cudaMalloc(&bs.err, sizeof(int)));
  B_CUDA(cudaMemcpyAsync(bs.desc, desc.data(), np * sizeof(BProb<T>), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemcpyAsync(bs.desc_b, desc_b.data(), np * sizeof(BProb<T>), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemcpyAsync(bs.nact, nact.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemcpyAsync(bs.wtab, wtab.data(), wtab.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemcpyAsync(bs.ptab, ptab.data(), ptab.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemcpyAsync(bs.scal, scal.data(), np * sizeof(double*), cudaMemcpyHostToDevice, st));
  B_CUDA(cudaMemsetAsync(bs.bar, 0, 2 * sizeof(unsigned), st));
  B_CUDA(cudaMemsetAsync(bs.err, 0, sizeof(int), st));
  B_CUDA(cudaStreamSynchronize(st));   // host tables above are pageable
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nblocks = (int)std::min<int64_t>(max_coresident<T, DIM, ORDER, VARC>(sms), std::max<int64_t>(tile0, 1));
  int64_t launches = 0;

  // ---- b = Pi_h(0; f_p) of every problem: one persistent launch
  B_CUDA((launch_batch_wave<T, DIM, ORDER, VARC>(st, bs.desc_b, bs.nact, S, bs.wtab, bs.ptab, bs.bar, bs.err, nblocks)));
  ++launches;
  // per-problem start: rr0 = <b, b>, x = 0, r = p = b, loop scalars
  for (int k = 0; k < np; ++k) {
    whv_grid g = grids[order[k]];
    const whv_params* pp = &params[order[k]];
    whv_status s = dot_async(g, g->t, g->t, S_RR0);
    if (s != WHV_OK) return s;
    s = fetch_scalars(g);
    if (s != WHV_OK) return s;
    const double bb = g->scal_host[S_RR0];
    if (!isfinite(bb)) return fail(g0, WHV_ERR_BREAKDOWN, "batched: non-finite right-hand side");
    B_CUDA(cudaMemsetAsync(g->x, 0, g->N * sizeof(double), st));
    B_CUDA(cudaMemcpyAsync(g->r, g->t, g->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    B_CUDA(cudaMemcpyAsync(g->p, g->t, g->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // S_RR, S_FLAG, S_ITER, S_STOP, S_MAXIT, S_HALT
    double init[S_NSLOTS];
    for (int i = 0; i < S_NSLOTS; ++i) init[i] = g->scal_host[i];
    init[S_RR] = bb;
    init[S_FLAG] = 0.0;
    init[S_ITER] = 0.0;
    init[S_STOP] = pp->tol * pp->tol * bb;
    init[S_MAXIT] = (double)pp->maxit;
    init[S_HALT] = (bb == 0.0 || pp->maxit == 0 || bb <= init[S_STOP]) ? 1.0 : 0.0;
    B_CUDA(cudaMemcpyAsync(g->scal, init, S_NSLOTS * sizeof(double), cudaMemcpyHostToDevice, st));
    B_CUDA(cudaStreamSynchronize(st));
  }
  launches += 3 * np;
  // ---- the batched CG loop: one graph with a WHILE node
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto gfree = [&]() { if (exec) cudaGraphExecDestroy(exec); if (graph) cudaGraphDestroy(graph); };
  B_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { gfree(); return cuda_fail(g0, e, "cudaGraphConditionalHandleCreate"); }
  cudaGraphNodeParams np_ = {};
  np_.type = cudaGraphNodeTypeConditional;
  np_.conditional.handle = h;
  np_.conditional.type = cudaGraphCondTypeWhile;
  np_.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np_);
  if (e != cudaSuccess) { gfree(); return cuda_fail(g0, e, "cudaGraphAddNode (batched loop)"); }
  cudaGraph_t body = np_.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { gfree(); return cuda_fail(g0, e, "cudaStreamBeginCaptureToGraph (batched loop)"); }
  const int64_t l0 = whv_kernel_launches();
  whv_status s = WHV_OK;
  e = launch_batch_wave<T, DIM, ORDER, VARC>(st, bs.desc, bs.nact, S, bs.wtab, bs.ptab, bs.bar, bs.err, nblocks);
  if (e == cudaSuccess) {
    k_batch_finish<T><<<np, 256, 0, st>>>((const BProb<T>*)bs.desc, bs.scal);
    e = cudaGetLastError();
  }
  for (int k = 0; k < np && e == cudaSuccess && s == WHV_OK; ++k) {
    whv_grid g = grids[order[k]];
    s = cg_update(g);
    if (s == WHV_OK) s = cg_direction(g);
  }
  if (e == cudaSuccess && s == WHV_OK) {
    k_batch_check<<<(np + 127) / 128, 128, 0, st>>>(bs.scal, np);
    k_batch_any<<<1, 1, 0, st>>>(h, bs.scal, np, bs.err);
    e = cudaGetLastError();
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &captured);
  const int64_t body_launches = (whv_kernel_launches() - l0) + 4;   // + wave, finish, check, any
  count_launches(-(whv_kernel_launches() - l0));
  if (s != WHV_OK) { gfree(); return s; }
  if (e != cudaSuccess) { gfree(); return cuda_fail(g0, e, "batched loop body"); }
  if (e2 != cudaSuccess) { gfree(); return cuda_fail(g0, e2, "cudaStreamEndCapture (batched loop)"); }
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) { gfree(); return cuda_fail(g0, e, "cudaGraphInstantiate (batched loop)"); }
  e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  gfree();
  if (e != cudaSuccess) return cuda_fail(g0, e, "batched loop");
  int herr = 0;
  B_CUDA(cudaMemcpy(&herr, bs.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return fail(g0, WHV_ERR_TIMEOUT, "batched wave solve: a grid barrier timed out");
  int max_it = 0;
  for (int k = 0; k < np; ++k) {
    const int p = order[k];
    whv_grid g = grids[p];
    s = fetch_scalars(g);
    if (s != WHV_OK) return s;
    const int it = (int)g->scal_host[S_ITER];
    max_it = std::max(max_it, it);
    iters_out[p] = it;
    if (infos) {
      infos[p].iterations = it;
      infos[p].wave_solves = it + 1;
      infos[p].rel_residual = g->scal_host[S_RR0] > 0 ? sqrt(g->scal_host[S_RR] / g->scal_host[S_RR0]) : 0.0;
    }
  }
  count_launches(launches + body_launches * max_it);
#undef B_CUDA
  return WHV_OK;
}

template <typename T, int DIM, int ORDER>
static whv_status batched_vc(int np, const whv_grid* grids, const whv_params* params,
                             const std::vector<TimeGridH>& tgs, const std::vector<const double*>& rf,
                             whv_info* infos, int* iters, BatchScratch& bs, bool varc) {
  return varc ? batched_cg<T, DIM, ORDER, true>(np, grids, params, tgs, rf, infos, iters, bs)
              : batched_cg<T, DIM, ORDER, false>(np, grids, params, tgs, rf, infos, iters, bs);
}

template <typename T>
static whv_status batched_dispatch(int np, const whv_grid* grids, const whv_params* params,
                                   const std::vector<TimeGridH>& tgs, const std::vector<const double*>& rf,
                                   whv_info* infos, int* iters, BatchScratch& bs, bool varc) {
  switch (grids[0]->dim * 10 + grids[0]->order) {
    case 22: return batched_vc<T, 2, 2>(np, grids, params, tgs, rf, infos, iters, bs, varc);
    case 24: return batched_vc<T, 2, 4>(np, grids, params, tgs, rf, infos, iters, bs, varc);
    case 32: return batched_vc<T, 3, 2>(np, grids, params, tgs, rf, infos, iters, bs, varc);
    case 34: return batched_vc<T, 3, 4>(np, grids, params, tgs, rf, infos, iters, bs, varc);
  }
  return fail(grids[0], WHV_ERR_INVALID, "batched solves need 2-D or 3-D grids");
}

}  // namespace whv

using namespace whv;

extern "C" whv_status whv_solve_batched(int nprob, const whv_grid* grids, const whv_params* params,
                                        const double* const* f_dev, double* const* u_dev, whv_info* infos) {
  if (nprob < 1 || nprob > kBatchMaxProblems || !grids || !params || !f_dev || !u_dev)
    return fail(nullptr, WHV_ERR_INVALID, "whv_solve_batched: bad arguments (1 <= nprob <= 1024)");
  whv_grid g0 = grids[0];
  if (!g0) return fail(nullptr, WHV_ERR_INVALID, "whv_solve_batched: NULL grid");
  const bool varc = g0->c2 != nullptr;
  std::vector<TimeGridH> tgs(nprob);
  std::vector<const double*> rf(nprob);
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
    whv_status s = make_time_grid(g, &params[p], &tgs[p]);
    if (s != WHV_OK) return fail(g0, s, std::string("whv_solve_batched: ") + g->err);
    const Basis& B = g->basis;
    if (B.nd > 0) {
      if (!(B.flags & WHV_BASIS_EXACT) || (B.flags & WHV_BASIS_REDEFLATE))
        return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: bases must be exact eigenvectors (DEVD)");
      if (B.omega != params[p].omega || B.periods != params[p].periods || B.cfl != tgs[p].cfl ||
          B.adjust != (params[p].adjust_omega ? 1 : 0))
        return fail(g0, WHV_ERR_INVALID, "whv_solve_batched: a basis was set for another frequency / time grid");
    }
  }
  // DEVD (Algorithm 2): deflate each forcing
  for (int p = 0; p < nprob; ++p) {
    whv_grid g = grids[p];
    const Basis& B = g->basis;
    rf[p] = f_dev[p];
    if (B.nd > 0) {
      whv_status s = project(g, B.V, B.nd, f_dev[p], B.d_coef);
      if (s == WHV_OK && cudaMemcpyAsync(g->fd, f_dev[p], g->N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
        s = fail(g0, WHV_ERR_CUDA, "copy");
      if (s == WHV_OK) s = expand(g, B.V, B.nd, B.d_coef, -1.0, g->fd);
      if (s != WHV_OK) return s;
      rf[p] = g->fd;
    }
  }
  std::vector<int> iters(nprob, 0);
  BatchScratch bs;
  whv_status s = g0->precision == WHV_FP64 ? batched_dispatch<double>(nprob, grids, params, tgs, rf, infos, iters.data(), bs, varc)
                                           : batched_dispatch<float>(nprob, grids, params, tgs, rf, infos, iters.data(), bs, varc);
  cudaStreamSynchronize(g0->stream);
  bs.free_all();
  if (s != WHV_OK) return s;
  // inflate and write the solutions
  bool all_conv = true;
  for (int p = 0; p < nprob; ++p) {
    whv_grid g = grids[p];
    const Basis& B = g->basis;
    if (B.nd > 0) {
      std::vector<double> cf(B.nd);
      if (cudaMemcpy(cf.data(), B.d_coef, B.nd * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(g0, WHV_ERR_CUDA, "copy");
      const double om2 = tgs[p].omega_eff * tgs[p].omega_eff;
      for (int m = 0; m < B.nd; ++m) cf[m] /= (om2 - B.lambda2[m]);
      if (cudaMemcpy(g->small, cf.data(), B.nd * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(g0, WHV_ERR_CUDA, "copy");
      s = expand(g, B.V, B.nd, g->small, 1.0, g->x);
      if (s != WHV_OK) return s;
    }
    if (cudaMemcpyAsync(u_dev[p], g->x, g->N * sizeof(double), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
      return fail(g0, WHV_ERR_CUDA, "copy");
    s = fetch_scalars(g);
    if (s != WHV_OK) return s;
    const double rel = g->scal_host[S_RR0] > 0 ? sqrt(g->scal_host[S_RR] / g->scal_host[S_RR0]) : 0.0;
    if (!(rel <= params[p].tol)) all_conv = false;
    if (g->scal_host[S_FLAG] != 0.0) all_conv = false;
    if (infos) {
      infos[p].nt = tgs[p].nt;
      infos[p].dt = tgs[p].dt;
      infos[p].omega_hat = tgs[p].omega_hat;
      infos[p].omega_eff = tgs[p].omega_eff;
      infos[p].true_rel_residual = -1.0;
      infos[p].seconds = 0.0;
      infos[p].outer_iterations = 0;
      infos[p].wave_solves_fp64 = g->precision == WHV_FP64 ? iters[p] + 1 : 0;
    }
    // leave the grid usable by non-batched calls
    double zero = 0.0;
    cudaMemcpy(g->scal + S_HALT, &zero, sizeof(double), cudaMemcpyHostToDevice);
  }
  cudaStreamSynchronize(g0->stream);
  if (!all_conv) return fail(g0, WHV_ERR_NOT_CONVERGED, "whv_solve_batched: some problems did not reach tol");
  return WHV_OK;
}
