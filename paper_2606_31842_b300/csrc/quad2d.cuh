// Sub-steps of a staged 64 x 64 region for the FP32 5-point stencil with c = 1 -- the f = 0 wave
// solves of the constant-speed 2-D grids, i.e. every A p of their Krylov iterations -- in a
// thread mapping chosen for the issue rate rather than for the global loads.
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

// Advances the region staged in S0 (W^n), S1 (W^{n-1}) and S2 (filter sums) kk sub-steps with the
// weights sw[0 .. kk-1] (FIRST: sub-step 1 is the Taylor start).  The caller has synchronised
// after staging; on return, after a barrier, S0 = W^{n+kk}, S1 = W^{n+kk-1}, S2 = filter sums.
// All 1024 threads call it (shuffles and barriers).
template <bool MASK, bool FIRST>
__device__ __forceinline__ void quad_sweep(float* S0, float* S1, float* S2, int kk, const float* sw,
                                           const QuadCoef& q, unsigned m) {
  const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 4;
  const int off = row * kQReg + col;
  const int up = max(row - 1, 0) * kQReg + col, dn = min(row + 1, kQReg - 1) * kQReg + col;
  float4 c = q_lds(S0, off), w = q_lds(S1, off), a = q_lds(S2, off);
  __syncthreads();   // the first sub-step overwrites S1
  float* A = S0;
  float* B = S1;
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
  q_sts(S0, off, c);
  q_sts(S1, off, w);
  q_sts(S2, off, a);
  __syncthreads();
}

}  // namespace whv
