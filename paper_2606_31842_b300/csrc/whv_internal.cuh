// Internal declarations of the B300 WaveHoltz library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <memory>
#include <string>
#include <vector>

#include "whv.h"

namespace whv {

// ---------------------------------------------------------------- device scalar slots
// Krylov scalars live in device memory so that iterations run without host round trips.
enum Slot {
  S_RR = 0,     // r^T M r of the current residual
  S_PQ = 1,     // p^T M (A p)
  S_ALPHA = 2,
  S_BETA = 3,
  S_RR0 = 4,    // residual norm^2 at the start (stopping reference)
  S_FLAG = 5,   // breakdown flag (nonzero: non-finite or non-positive scalar seen)
  S_TMP = 6,    // scratch result of whv_dot and friends
  S_TMP2 = 7,
  S_ITER = 8,   // iteration counter of the device-resident CG loop
  S_STOP = 9,   // tol^2 rr0: the loop runs while r^T M r > S_STOP
  S_MAXIT = 10, // iteration limit of the device-resident CG loop
  S_HALT = 11,  // batched solves: nonzero once this problem has stopped (its kernels return)
  S_NSLOTS = 16
};

// reduction "channels": each kernel that reduces uses its own partials/counter pair so that
// reductions of consecutive kernels never share a counter.
enum Channel { CH_STEP = 0, CH_UPDATE = 1, CH_DOT = 2, CH_PROJ = 3, CH_NCH = 4 };

constexpr int kRedBlocks = 592;          // 4 x 148 SMs: grid of the grid-stride reduction kernels
constexpr int kMaxStepBlocks = 1 << 20;  // upper bound on blocks of a fused step+reduction kernel
constexpr int kMaxND = 1024;             // deflation / Krylov basis columns per contraction

struct TimeGridH {
  double omega = 0, omega_hat = 0, dt = 0, tbar = 0, omega_eff = 0, cfl = 0;
  int periods = 0, adjust = 0, nt = 0;
  std::vector<double> phase;   // cos(omega_hat t^n), n = 0..nt
  std::vector<double> weight;  // (2/Tbar) eta_n (cos(omega_hat t^n) - 1/4) dt
};

struct Basis {
  int nd = 0, mode = WHV_BASIS_NONE, flags = 0;
  double* V = nullptr;                // N x nd, column-major, FP64
  // owner of V: grids that share one basis (whv_share_basis) hold references to the same
  // storage, which is freed with the last of them
  std::shared_ptr<void> vhold;
  double* d_coef = nullptr;           // nd scratch
  std::vector<double> lambda2, mu;    // lambda^2 and mu = 1 - beta_h
  std::vector<int> modes;             // nd * dim (closed form)
  double omega = 0; int periods = 0, adjust = 0; double cfl = 0;  // time grid it was built for
  // general (non-eigenvector) deflation for Algorithm 4: A W and (W^T M A W)^{-1}, built on the
  // first DCG solve with a basis that is not WHV_BASIS_EXACT
  double* AW = nullptr;               // N x nd
  double* Einv = nullptr;             // nd x nd, row-major
  // Algorithm 5: A W = QAW Raw (thin QR in <.,.>_M), built on the first AGMRES solve
  double* QAW = nullptr;              // N x nd, M-orthonormal columns
  std::vector<double> Raw;            // nd x nd upper triangular, column-major
  // SVD-compressed vectors (whv_compress_basis; V is then freed): vector m = sum over its
  // columns k of s_k u_k v_k^T, u_k (ny) and v_k (nx) the columns off[m] .. off[m+1]-1 of cU, cV
  int comp_R = 0;                     // total rank (0: dense basis)
  double comp_tau = 0.0;
  double *cU = nullptr, *cV = nullptr, *cs = nullptr;   // ny x R, nx x R (column-major), R
  double *cT = nullptr, *cc = nullptr, *cR = nullptr;   // scratch: ny x R, R, N
  int *coff = nullptr, *cowner = nullptr;               // nd + 1 offsets, owner vector of each column
};

struct StepPlan;  // cached CUDA graphs of wave solves (stencil.cu)
struct CgLoop;    // cached device-resident CG loop graph (solve.cu)

}  // namespace whv

struct whv_grid_s {
  int dim = 1, order = 2, precision = WHV_FP64;
  int64_t npts[3] = {3, 3, 3};
  int n[3] = {1, 1, 1};        // interior counts nx, ny, nz
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  int64_t N = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;     // created by the grid (caller passed the legacy default stream)

  // speed
  double* c2 = nullptr;        // FP64 c^2 (nullptr: c = 1)
  float* c2f = nullptr;        // FP32 copy for FP32 stepping
  double* mw = nullptr;        // M weights 1/c^2 (nullptr: ones)
  double c2max = 1.0;

  // stepping buffers (element type double or float by precision): two (W^{n-1}, W^n) pairs so
  // that temporally blocked sweeps read one pair and write the other
  void* wbuf[4] = {nullptr, nullptr, nullptr, nullptr};
  void* acc = nullptr;
  int cons = 0;                // 1: L_h = div_h(c^2 grad_h) (whv_set_speed_form), Euclidean inner products
  double* face64[3] = {nullptr, nullptr, nullptr};   // its face values per axis (FP64, FP32)
  float* face32[3] = {nullptr, nullptr, nullptr};
  int kblock = 0;              // steps per sweep of the blocked 2-D kernel (0: default, 1: off)
  // FP64 stepping buffers of an FP32-stepping grid (FP64 residual correction), allocated on
  // first use, with the outer solution / residual / right-hand side of the refinement loop
  void* wbuf64[4] = {nullptr, nullptr, nullptr, nullptr};
  void* acc64 = nullptr;
  // FP32 state of the TMA-fed batched 2-D kernel (k_batch_tma): two (W^{n-1}, W^n) pairs and the
  // filter sums with rows padded to tpitch floats (a multiple of 4: the copy engine needs 16-byte
  // row strides), allocated on first use
  float* tw[4] = {nullptr, nullptr, nullptr, nullptr};
  float* tacc = nullptr;
  int tpitch = 0;
  // FP32 state of the two-step 3-D kernel (k_step3d2), rows padded to pitch3 floats, and the
  // device copy of its tensor maps; allocated outside any stream capture, on first use
  float* pw3[4] = {nullptr, nullptr, nullptr, nullptr};
  float* pacc3 = nullptr;
  void* maps3 = nullptr;
  int pitch3 = 0;
  double *xo = nullptr, *ro = nullptr, *bo = nullptr;

  // FP64 Krylov work vectors
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *t = nullptr, *fd = nullptr;
  double* krylov = nullptr;    // GMRES basis, (restart+1) * N
  int krylov_cols = 0;
  double* small = nullptr;     // device small-vector scratch (kMaxND)
  double* small2 = nullptr;    // second small-vector scratch (kMaxND)
  // weight / phase table of the single-CTA wave solve (small grids)
  double* wtab_small = nullptr;
  int tab_nt = 0, tab_cap = 0;
  double tab_key[4] = {0, 0, 0, 0};

  // reductions
  double* partials = nullptr;  // reduction scratch, one region per channel
  int64_t chan_off[4] = {0, 0, 0, 0}, chan_cap[4] = {0, 0, 0, 0};
  unsigned* counters = nullptr;// CH_NCH
  bool barrier_fault = false;  // whv_inject_barrier_error: the next batched solve starts with its
                               // barrier error flag raised
  double* scal = nullptr;      // S_NSLOTS device scalars
  double* scal_host = nullptr; // pinned mirror

  whv::Basis basis;
  whv::StepPlan* plan = nullptr;
  whv::CgLoop* cgloop = nullptr;
  std::string err;
};

namespace whv {

// per-block partial sums of reduction channel ch, and how many blocks it can hold
inline double* chan(whv_grid g, int ch) { return g->partials + g->chan_off[ch]; }

// Relative tolerance of correction solve number `pass` (0: the first) of the FP64 residual
// correction, at outer residual rel: the first takes the requested fraction `inner` (a loose pass:
// its accuracy is limited by the stepping precision, which the later passes correct); later ones
// aim at half the remaining gap to tol, no tighter than inner / 10.
inline double correction_tol(double inner, double tol, double rel, int pass) {
  const double need = 0.5 * tol / (rel > 1e-300 ? rel : 1e-300);
  const double floor_ = pass == 0 ? inner : 0.1 * inner;
  return need > floor_ ? need : floor_;
}
inline int64_t chan_cap(whv_grid g, int ch) { return g->chan_cap[ch]; }

// ------------------------------------------------------------------ host helpers (core.cu)
whv_status fail(whv_grid g, whv_status s, const std::string& msg);
whv_status cuda_fail(whv_grid g, cudaError_t e, const char* what);
#define WHV_CUDA(g, call)                                   \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return whv::cuda_fail(g, _e, #call); \
  } while (0)

#define TRY(expr)                          \
  do {                                     \
    whv_status _s = (expr);                \
    if (_s != WHV_OK) return _s;           \
  } while (0)

// stream-ordered copies on the grid's stream; the host ones synchronise (pageable host memory)
inline whv_status copy_dev(whv_grid g, double* dst, const double* src, int64_t n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  return WHV_OK;
}
inline whv_status to_host(whv_grid g, double* dst, const double* src, int n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}
inline whv_status to_dev(whv_grid g, double* dst, const double* src, int n) {
  WHV_CUDA(g, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  // src is pageable host memory that may be reused right after: wait for the copy
  WHV_CUDA(g, cudaStreamSynchronize(g->stream));
  return WHV_OK;
}
inline double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

whv_status make_time_grid(whv_grid g, const whv_params* p, TimeGridH* tg);
void free_basis(whv_grid g);   // frees the deflation basis (and what depends on it)
// make b.vhold the owner of b.V (a cudaMalloc'ed buffer)
void hold_vectors(Basis& b);

// launch accounting (whv_kernel_launches)
void count_launches(int64_t n);

// ---------------------------------------------------------------- kernels launchers
// stencil.cu: one wave solve.  v (FP64, nullable => 0), f (FP64, nullable => 0).
//   epi = 0: out = Pi_h(v; f)                  (out FP64)
//   epi = 1: out = v - Pi_h(v; f) = A v (f=0), and scal[S_PQ] = <v, out>_M
//   prec = -1: the grid's stepping precision; WHV_FP64 on an FP32-stepping grid uses the
//   grid's FP64 buffer set (ensure_fp64_buffers first).
//   prec = kPrecDF64: double-float stepping (pairs of FP32, second-order grids) in the FP64
//   buffer set -- the residual wave solves of WHV_RESIDUAL_DF64.
constexpr int kPrecDF64 = 2;
whv_status wave_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f,
                      double* out, int epi, int prec = -1);
void free_plan(whv_grid g);
void free_cgloop(whv_grid g);
int default_kblock(whv_grid g);
whv_status ensure_fp64_buffers(whv_grid g);

// stencil_blocked.cu: steps 1..nt-1 of a 2-D f = 0 wave solve in sweeps of k steps, on the
// stepping buffers bufs[0..3] (two (W^{n-1}, W^n) pairs) and accumulator acc
template <typename T, int ORDER, bool VARC>
whv_status blocked_steps_2d(whv_grid g, const TimeGridH& tg, const double* v, double* out, int epi,
                            int k_want, int* launches, void* const* bufs, void* acc);
void blocked_init();
void step3d2_init();   // stencil.cu: resident CTA slots of the persistent two-step 3-D kernel
whv_status ensure_pitched3(whv_grid g);   // stencil.cu: buffers and tensor maps of the two-step 3-D kernel
void* tensor_map_encoder();               // core.cu: cuTensorMapEncodeTiled (driver entry point) or nullptr

// single-CTA wave solve for small grids (stencil_blocked.cu)
bool small_grid(whv_grid g);
int small_tables(whv_grid g, const TimeGridH& tg);   // 0 current, 1 uploaded, -1 stale
whv_status small_wave_solve(whv_grid g, const TimeGridH& tg, const double* v, const double* f, double* out,
                            int epi, int prec);

// reduce.cu
whv_status dot_async(whv_grid g, const double* x, const double* y, int slot);   // scal[slot] = <x,y>_M
whv_status cg_update(whv_grid g);        // alpha = rr/pq; x += a p; r -= a q; rr' ; beta
whv_status cg_direction(whv_grid g);     // p = r + beta p
whv_status axpby(whv_grid g, int64_t n, double a, const double* x, double b, double* y);  // y = a x + b y
whv_status fetch_scalars(whv_grid g);    // scal -> scal_host (synchronises the stream)

// deflate.cu: contractions with a column-major N x nd matrix (basis or Krylov basis)
//   project:  coef[m] = sum_i W[i + m N] M_i r_i            (m < nd)
//   expand:   out_i  += alpha sum_m W[i + m N] coef[m]
whv_status project(whv_grid g, const double* W, int nd, const double* r, double* coef);
whv_status expand(whv_grid g, const double* W, int nd, const double* coef, double alpha,
                  double* out);
whv_status closed_form_basis(whv_grid g, const TimeGridH& tg, int nd, Basis* b);
// k right-hand sides sharing one basis W (W read once for all of them):
//   project_many: C[j nd + m] = sum_i W[i + m N] mw_i R[j][i]   (mw NULL: 1); R a DEVICE array of k
//                 pointers; partials needs project_many_scratch(N, nd, k) doubles
//   expand_many:  out[j][i] += alpha sum_m W[i + m N] s_m C[j nd + m]   (scale NULL: s = 1); out a
//                 DEVICE array of k pointers
int64_t project_many_scratch(int64_t N, int nd, int k);
cudaError_t project_many(cudaStream_t st, const double* W, int64_t N, int nd, int k, const double* const* R,
                         const double* mw, double* partials, double* C);
cudaError_t expand_many(cudaStream_t st, const double* W, int64_t N, int nd, int k, const double* C,
                        const double* scale, double alpha, double* const* out);

// compress.cu: contractions with the grid's basis, dense or SVD-compressed
whv_status basis_project(whv_grid g, const double* r, double* coef);                  // W^T M r
whv_status basis_expand(whv_grid g, const double* coef, double alpha, double* out);   // out += a W c
whv_status basis_column(whv_grid g, int m, double* dst);                             // dst = W e_m
const void* basis_key(const Basis& B);   // identity of the basis storage (graph cache keys)
// lanczos.cu: the kw largest eigenpairs of a dense symmetric n x n matrix (row-major) by
// Householder reduction, bisection and inverse iteration; S is n x kw, column-major
void host_sym_top_eigenpairs(const std::vector<double>& A, int n, int kw, std::vector<double>& theta,
                             std::vector<double>& S);

}  // namespace whv
