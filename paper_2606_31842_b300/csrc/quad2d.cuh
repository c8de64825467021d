// Sub-steps of a staged 64 x 64 region for the FP32 2-D stencils -- the f = 0 wave solves, i.e.
// every A p of the Krylov iterations: quad_sweep for the 5-point stencil with c = 1 (with the
// Taylor start for the batched kernel), quadv_sweep for c^2 Delta_h and the 9-point-wide
// 4th-order stencil -- in a thread mapping chosen for the issue rate rather than for the global
// loads.
//
// Thread t of the 1024 owns the four consecutive cells 4 (t mod 16) .. 4 (t mod 16) + 3 of region
// row t / 16 for the whole sweep, their W^n, W^{n-1} and filter sums in registers.  Per sub-step a
// thread stores its four new values with one 16-byte shared store and reads its y neighbours with
// two 16-byte shared loads; its x neighbours are its own registers and, for the two end cells,
// the adjacent lanes' registers (one shuffle each).  Every region cell is advanced at every
// sub-step: a cell at distance d from the region edge is exact up to sub-step d (what the edge
// cells read instead of their missing neighbours -- their own row, another row's lane -- only
// spoils cells that are already out of date), and the tile the caller writes back lies at
// distance >= k.  This removes the per-cell window tests of the scalar kernels.  Cells outside
// the domain are loaded as 0 and, when the region crosses the boundary (MASK), held at 0, so the
// neighbour sums see the homogeneous Dirichlet values without tests either.
//
// The update and the filter sum use the operations of the scalar kernels in the same order
//   W^{n+1} = fma(ay, up + down, fma(ax, left + right, fma(b, W^n, -W^{n-1})))
//   Taylor start W^1 = fma(dt^2 / 2, L W^0, W^0),  L = ih2x (l + r - 2c) + ih2y (u + d - 2c)
//   acc = fma(w_{n+1}, W^{n+1}, acc)
// so the results are bitwise those of the scalar kernels.
#pragma once

#include <cuda_runtime.h>

namespace whv {

constexpr int kQReg = 64;   // region edge; 1024 threads x 4 cells

struct QuadCoef {
  float ax, ay, b;          // dt^2 / h_x^2, dt^2 / h_y^2, 2 - 2 (ax + ay)
  float ih2x, ih2y, hdt2;   // 1 / h_x^2, 1 / h_y^2, dt^2 / 2 (Taylor start)
};

__device__ __forceinline__ float4 q_lds(const float* S, int off) {
  return *reinterpret_cast<const float4*>(S + off);
}
__device__ __forceinline__ void q_sts(float* S, int off, float4 v) { *reinterpret_cast<float4*>(S + off) = v; }
__device__ __forceinline__ void q_swap(float4& a, float4& b) {
  const float4 t = a;
  a = b;
  b = t;
}

// in-domain bits of the thread's four cells (bit e: cell 4 (t mod 16) + e of its row)
__device__ __forceinline__ unsigned quad_mask(int x0, int y0, int nx, int ny) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int gy = y0 + row;
  if (gy < 0 || gy >= ny) return 0u;
  unsigned m = 0u;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int gx = x0 + col + e;
    if (gx >= 0 && gx < nx) m |= 1u << e;
  }
  return m;
}

// one leapfrog sub-step: w <- W^{n+1} from c = W^n and w = W^{n-1}; stored to Bout, added to a
template <bool MASK>
__device__ __forceinline__ void quad_step(const float4& c, float4& w, float4& a, const float* Ain, float* Bout,
                                          int off, int up, int dn, float ws, const QuadCoef& q, unsigned m) {
  const float4 U = q_lds(Ain, up), D = q_lds(Ain, dn);
  const float l = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float r = __shfl_down_sync(0xffffffffu, c.x, 1);
  float4 n;
  n.x = fmaf(q.ay, U.x + D.x, fmaf(q.ax, l + c.y, fmaf(q.b, c.x, -w.x)));
  n.y = fmaf(q.ay, U.y + D.y, fmaf(q.ax, c.x + c.z, fmaf(q.b, c.y, -w.y)));
  n.z = fmaf(q.ay, U.z + D.z, fmaf(q.ax, c.y + c.w, fmaf(q.b, c.z, -w.z)));
  n.w = fmaf(q.ay, U.w + D.w, fmaf(q.ax, c.z + r, fmaf(q.b, c.w, -w.w)));
  if (MASK) {
    n.x = (m & 1u) ? n.x : 0.0f;
    n.y = (m & 2u) ? n.y : 0.0f;
    n.z = (m & 4u) ? n.z : 0.0f;
    n.w = (m & 8u) ? n.w : 0.0f;
  }
  q_sts(Bout, off, n);
  a.x = fmaf(ws, n.x, a.x);
  a.y = fmaf(ws, n.y, a.y);
  a.z = fmaf(ws, n.z, a.z);
  a.w = fmaf(ws, n.w, a.w);
  w = n;
}

// the Taylor start W^1 = W^0 + dt^2 / 2 L W^0 into w (its old content unused)
template <bool MASK>
__device__ __forceinline__ void quad_taylor(const float4& c, float4& w, float4& a, const float* Ain, float* Bout,
                                            int off, int up, int dn, float ws, const QuadCoef& q, unsigned m) {
  const float4 U = q_lds(Ain, up), D = q_lds(Ain, dn);
  const float l = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float r = __shfl_down_sync(0xffffffffu, c.x, 1);
  auto one = [&](float cm, float cl, float cr, float cu, float cd) {
    float L = fmaf(-2.0f, cm, cl + cr) * q.ih2x;
    L = fmaf(fmaf(-2.0f, cm, cu + cd), q.ih2y, L);
    return fmaf(q.hdt2, L, cm);
  };
  float4 n;
  n.x = one(c.x, l, c.y, U.x, D.x);
  n.y = one(c.y, c.x, c.z, U.y, D.y);
  n.z = one(c.z, c.y, c.w, U.z, D.z);
  n.w = one(c.w, c.z, r, U.w, D.w);
  if (MASK) {
    n.x = (m & 1u) ? n.x : 0.0f;
    n.y = (m & 2u) ? n.y : 0.0f;
    n.z = (m & 4u) ? n.z : 0.0f;
    n.w = (m & 8u) ? n.w : 0.0f;
  }
  q_sts(Bout, off, n);
  a.x = fmaf(ws, n.x, a.x);
  a.y = fmaf(ws, n.y, a.y);
  a.z = fmaf(ws, n.z, a.z);
  a.w = fmaf(ws, n.w, a.w);
  w = n;
}

// Variable speed (c^2 Delta_h) with the 5-point or the 9-point-wide 4th-order stencil: the second
// differences of the scalar kernels, fma(-2, c, m1 + p1) and fma(-30, c, fma(16, m1 + p1,
// -(m2 + p2))), times 1 / h^2 (1 / 12 h^2), W^{n+1} = fma(dt^2, c^2 L, fma(2, c, -W^{n-1})).  The
// 4th-order closure at the boundary (odd reflection: the value two nodes outside the first or last
// interior node is minus that node) is applied to the cells whose bits are set in e (MASK only):
// bits 0-3 the cells at x = 0, bits 4-7 at x = nx - 1, bit 8 the row y = 0, bit 9 the row y = ny - 1.
struct QuadBnd {
  unsigned in;   // in-domain bits of the four cells
  unsigned e;    // 4th-order boundary bits
};

__device__ __forceinline__ QuadBnd quad_bnd(int x0, int y0, int nx, int ny) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int gy = y0 + row;
  QuadBnd b{quad_mask(x0, y0, nx, ny), 0u};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int gx = x0 + col + e;
    if (gx == 0) b.e |= 1u << e;
    if (gx == nx - 1) b.e |= 16u << e;
  }
  if (gy == 0) b.e |= 256u;
  if (gy == ny - 1) b.e |= 512u;
  return b;
}

template <int ORDER, bool MASK>
__device__ __forceinline__ float q_d2(float c, float m1, float p1, float m2, float p2, bool lo, bool hi) {
  if (ORDER == 2) return fmaf(-2.0f, c, m1 + p1);
  if (MASK) {
    m2 = lo ? -c : m2;
    p2 = hi ? -c : p2;
  }
  return fmaf(-30.0f, c, fmaf(16.0f, m1 + p1, -(m2 + p2)));
}

struct QuadCoefV {
  float ih2x, ih2y, dt2;   // 1 / h^2 (order 2) or 1 / (12 h^2) (order 4); dt^2
};

template <int ORDER, bool VARC, bool MASK>
__device__ __forceinline__ void quadv_step(const float4& c, float4& w, float4& a, const float4& cc, const float* Ain,
                                           float* Bout, int off, int rowoff[4], float ws, const QuadCoefV& q,
                                           const QuadBnd& b) {
  // y neighbours: rows -1, +1 (and -2, +2 for order 4), clamped to the region
  const float4 U1 = q_lds(Ain, rowoff[1]), D1 = q_lds(Ain, rowoff[2]);
  float4 U2 = make_float4(0.f, 0.f, 0.f, 0.f), D2 = U2;
  if (ORDER == 4) {
    U2 = q_lds(Ain, rowoff[0]);
    D2 = q_lds(Ain, rowoff[3]);
  }
  const float lw = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float rx = __shfl_down_sync(0xffffffffu, c.x, 1);
  float lz = 0.f, ry = 0.f;
  if (ORDER == 4) {
    lz = __shfl_up_sync(0xffffffffu, c.z, 1);
    ry = __shfl_down_sync(0xffffffffu, c.y, 1);
  }
  const bool ylo = MASK && (b.e & 256u), yhi = MASK && (b.e & 512u);
  auto upd = [&](float cm, float m1, float p1, float m2, float p2, float um1, float dp1, float um2, float dp2,
                 float wp, float c2, int e) {
    float L = q_d2<ORDER, MASK>(cm, m1, p1, m2, p2, MASK && (b.e & (1u << e)), MASK && (b.e & (16u << e))) * q.ih2x;
    L = fmaf(q_d2<ORDER, MASK>(cm, um1, dp1, um2, dp2, ylo, yhi), q.ih2y, L);
    if (VARC) L *= c2;
    return fmaf(q.dt2, L, fmaf(2.0f, cm, -wp));
  };
  float4 n;
  n.x = upd(c.x, lw, c.y, lz, c.z, U1.x, D1.x, U2.x, D2.x, w.x, cc.x, 0);
  n.y = upd(c.y, c.x, c.z, lw, c.w, U1.y, D1.y, U2.y, D2.y, w.y, cc.y, 1);
  n.z = upd(c.z, c.y, c.w, c.x, rx, U1.z, D1.z, U2.z, D2.z, w.z, cc.z, 2);
  n.w = upd(c.w, c.z, rx, c.y, ry, U1.w, D1.w, U2.w, D2.w, w.w, cc.w, 3);
  if (MASK) {
    n.x = (b.in & 1u) ? n.x : 0.0f;
    n.y = (b.in & 2u) ? n.y : 0.0f;
    n.z = (b.in & 4u) ? n.z : 0.0f;
    n.w = (b.in & 8u) ? n.w : 0.0f;
  }
  q_sts(Bout, off, n);
  a.x = fmaf(ws, n.x, a.x);
  a.y = fmaf(ws, n.y, a.y);
  a.z = fmaf(ws, n.z, a.z);
  a.w = fmaf(ws, n.w, a.w);
  w = n;
}

// quad_sweep for the variable-speed and 4th-order kernels (no Taylor start: the single-grid path
// takes its first step separately); cc holds c^2 of the thread's four cells (VARC)
template <int ORDER, bool VARC, bool MASK>
__device__ __forceinline__ void quadv_sweep(float* S0, float* S1, float* S2, int kk, const float* sw,
                                            const QuadCoefV& q, const QuadBnd& b, const float4 cc) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int off = row * kQReg + col;
  int rowoff[4];
  rowoff[0] = max(row - 2, 0) * kQReg + col;
  rowoff[1] = max(row - 1, 0) * kQReg + col;
  rowoff[2] = min(row + 1, kQReg - 1) * kQReg + col;
  rowoff[3] = min(row + 2, kQReg - 1) * kQReg + col;
  float4 c = q_lds(S0, off), w = q_lds(S1, off), a = q_lds(S2, off);
  __syncthreads();
  float* A = S0;
  float* B = S1;
  int s = 0;
  for (; s + 2 <= kk; s += 2) {
    quadv_step<ORDER, VARC, MASK>(c, w, a, cc, A, B, off, rowoff, sw[s], q, b);
    __syncthreads();
    quadv_step<ORDER, VARC, MASK>(w, c, a, cc, B, A, off, rowoff, sw[s + 1], q, b);
    __syncthreads();
  }
  if (s < kk) {
    quadv_step<ORDER, VARC, MASK>(c, w, a, cc, A, B, off, rowoff, sw[s], q, b);
    __syncthreads();
    q_swap(c, w);
  }
  q_sts(S0, off, c);
  q_sts(S1, off, w);
  q_sts(S2, off, a);
  __syncthreads();
}

// The sub-steps with the thread's four cells in registers: on entry c = W^n, w = W^{n-1} and a =
// the filter sums of its cells, and A holds W^n of the whole region (written and synchronised by
// the caller); on return c = W^{n+kk}, w = W^{n+kk-1}, a the updated sums.  A and B are the two
// exchange buffers (both overwritten); B may hold the W^{n-1} the threads loaded w from, so the
// first barrier comes before the first sub-step writes it.  FIRST: sub-step 1 is the Taylor start.
// All 1024 threads call it (shuffles and barriers); it ends with a barrier.
template <bool MASK, bool FIRST>
__device__ __forceinline__ void quad_steps(float4& c, float4& w, float4& a, float* A, float* B, int kk,
                                           const float* sw, const QuadCoef& q, unsigned m) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int off = row * kQReg + col;
  const int up = max(row - 1, 0) * kQReg + col, dn = min(row + 1, kQReg - 1) * kQReg + col;
  __syncthreads();
  int s = 0;
  if (FIRST && kk > 0) {
    quad_taylor<MASK>(c, w, a, A, B, off, up, dn, sw[0], q, m);
    __syncthreads();
    q_swap(c, w);
    float* t = A; A = B; B = t;
    s = 1;
  }
  for (; s + 2 <= kk; s += 2) {   // two sub-steps with the roles of c and w exchanged: no moves
    quad_step<MASK>(c, w, a, A, B, off, up, dn, sw[s], q, m);
    __syncthreads();
    quad_step<MASK>(w, c, a, B, A, off, up, dn, sw[s + 1], q, m);
    __syncthreads();
  }
  if (s < kk) {
    quad_step<MASK>(c, w, a, A, B, off, up, dn, sw[s], q, m);
    __syncthreads();
    q_swap(c, w);
  }
}

// Advances the region staged in S0 (W^n), S1 (W^{n-1}) and S2 (filter sums) kk sub-steps with the
// weights sw[0 .. kk-1] (FIRST: sub-step 1 is the Taylor start).  The caller has synchronised
// after staging; on return, after a barrier, S0 = W^{n+kk}, S1 = W^{n+kk-1}, S2 = filter sums.
// All 1024 threads call it (shuffles and barriers).
template <bool MASK, bool FIRST>
__device__ __forceinline__ void quad_sweep(float* S0, float* S1, float* S2, int kk, const float* sw,
                                           const QuadCoef& q, unsigned m) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int off = row * kQReg + col;
  float4 c = q_lds(S0, off), w = q_lds(S1, off), a = q_lds(S2, off);
  quad_steps<MASK, FIRST>(c, w, a, S0, S1, kk, sw, q, m);
  q_sts(S0, off, c);
  q_sts(S1, off, w);
  q_sts(S2, off, a);
  __syncthreads();
}

// ------------------------------------------------------------------ two rows per thread
// The same sub-steps with 512 threads per 64 x 64 region: thread t owns the four cells
// 4 (t mod 16) .. + 3 of rows 2 (t / 16) and 2 (t / 16) + 1.  The y neighbours between its two
// rows are its own registers, so per sub-step it stores its two rows (two 16-byte stores) and
// reads the row above the first and below the second (two 16-byte loads): 4 shared accesses per
// 8 cells instead of 6.  Same operations in the same order as quad_step / quad_taylor (bitwise
// equal results).

// in-domain bits of the thread's two rows of four cells (bits 0-3 the first row, 4-7 the second)
__device__ __forceinline__ unsigned duo_mask(int x0, int y0, int nx, int ny) {
  const int row = (threadIdx.x >> 4) * 2, col = (threadIdx.x & 15) * 4;
  unsigned m = 0u;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int gy = y0 + row + rr;
    if (gy < 0 || gy >= ny) continue;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int gx = x0 + col + e;
      if (gx >= 0 && gx < nx) m |= 1u << (4 * rr + e);
    }
  }
  return m;
}

__device__ __forceinline__ float4 q_mask4(float4 n, unsigned m) {
  n.x = (m & 1u) ? n.x : 0.0f;
  n.y = (m & 2u) ? n.y : 0.0f;
  n.z = (m & 4u) ? n.z : 0.0f;
  n.w = (m & 8u) ? n.w : 0.0f;
  return n;
}

__device__ __forceinline__ float4 q_update(const float4& c, const float4& w, float l, float r, const float4& U,
                                           const float4& D, const QuadCoef& q) {
  float4 n;
  n.x = fmaf(q.ay, U.x + D.x, fmaf(q.ax, l + c.y, fmaf(q.b, c.x, -w.x)));
  n.y = fmaf(q.ay, U.y + D.y, fmaf(q.ax, c.x + c.z, fmaf(q.b, c.y, -w.y)));
  n.z = fmaf(q.ay, U.z + D.z, fmaf(q.ax, c.y + c.w, fmaf(q.b, c.z, -w.z)));
  n.w = fmaf(q.ay, U.w + D.w, fmaf(q.ax, c.z + r, fmaf(q.b, c.w, -w.w)));
  return n;
}

__device__ __forceinline__ float4 q_taylor(const float4& c, float l, float r, const float4& U, const float4& D,
                                           const QuadCoef& q) {
  auto one = [&](float cm, float cl, float cr, float cu, float cd) {
    float L = fmaf(-2.0f, cm, cl + cr) * q.ih2x;
    L = fmaf(fmaf(-2.0f, cm, cu + cd), q.ih2y, L);
    return fmaf(q.hdt2, L, cm);
  };
  float4 n;
  n.x = one(c.x, l, c.y, U.x, D.x);
  n.y = one(c.y, c.x, c.z, U.y, D.y);
  n.z = one(c.z, c.y, c.w, U.z, D.z);
  n.w = one(c.w, c.z, r, U.w, D.w);
  return n;
}

__device__ __forceinline__ void q_acc(float4& a, const float4& n, float ws) {
  a.x = fmaf(ws, n.x, a.x);
  a.y = fmaf(ws, n.y, a.y);
  a.z = fmaf(ws, n.z, a.z);
  a.w = fmaf(ws, n.w, a.w);
}

// one sub-step of both rows: (c0, c1) = W^n, (w0, w1) = W^{n-1} <- W^{n+1} (or the Taylor start)
template <bool MASK, bool TAYLOR>
__device__ __forceinline__ void duo_step(const float4& c0, const float4& c1, float4& w0, float4& w1, float4& a0,
                                         float4& a1, const float* Ain, float* Bout, int off, int up, int dn,
                                         float ws, const QuadCoef& q, unsigned m) {
  const float4 U = q_lds(Ain, up), D = q_lds(Ain, dn);
  const float l0 = __shfl_up_sync(0xffffffffu, c0.w, 1);
  const float r0 = __shfl_down_sync(0xffffffffu, c0.x, 1);
  const float l1 = __shfl_up_sync(0xffffffffu, c1.w, 1);
  const float r1 = __shfl_down_sync(0xffffffffu, c1.x, 1);
  float4 n0 = TAYLOR ? q_taylor(c0, l0, r0, U, c1, q) : q_update(c0, w0, l0, r0, U, c1, q);
  float4 n1 = TAYLOR ? q_taylor(c1, l1, r1, c0, D, q) : q_update(c1, w1, l1, r1, c0, D, q);
  if (MASK) {
    n0 = q_mask4(n0, m);
    n1 = q_mask4(n1, m >> 4);
  }
  q_sts(Bout, off, n0);
  q_sts(Bout, off + kQReg, n1);
  q_acc(a0, n0, ws);
  q_acc(a1, n1, ws);
  w0 = n0;
  w1 = n1;
}

// quad_steps for the two-rows mapping (512 threads call it); same contract
template <bool MASK, bool FIRST>
__device__ __forceinline__ void duo_steps(float4& c0, float4& c1, float4& w0, float4& w1, float4& a0, float4& a1,
                                          float* A, float* B, int kk, const float* sw, const QuadCoef& q,
                                          unsigned m) {
  const int row = (threadIdx.x >> 4) * 2, col = (threadIdx.x & 15) * 4;
  const int off = row * kQReg + col;
  const int up = max(row - 1, 0) * kQReg + col, dn = min(row + 2, kQReg - 1) * kQReg + col;
  __syncthreads();
  int s = 0;
  if (FIRST && kk > 0) {
    duo_step<MASK, true>(c0, c1, w0, w1, a0, a1, A, B, off, up, dn, sw[0], q, m);
    __syncthreads();
    q_swap(c0, w0);
    q_swap(c1, w1);
    float* t = A; A = B; B = t;
    s = 1;
  }
  for (; s + 2 <= kk; s += 2) {
    duo_step<MASK, false>(c0, c1, w0, w1, a0, a1, A, B, off, up, dn, sw[s], q, m);
    __syncthreads();
    duo_step<MASK, false>(w0, w1, c0, c1, a0, a1, B, A, off, up, dn, sw[s + 1], q, m);
    __syncthreads();
  }
  if (s < kk) {
    duo_step<MASK, false>(c0, c1, w0, w1, a0, a1, A, B, off, up, dn, sw[s], q, m);
    __syncthreads();
    q_swap(c0, w0);
    q_swap(c1, w1);
  }
}

}  // namespace whv
