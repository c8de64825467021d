// k leapfrog steps + trapezoid filter on a 64 x 64 region held in registers: the inner loop shared
// by the temporally blocked 2-D kernels (single grid, persistent, batched).
//
// Thread t of the 1024-thread CTA owns column i = t % 64 and the contiguous strip of rows
// 4 s .. 4 s + 3, s = t / 64, of the region: W^n, W^{n-1} and the filter sum of its four cells
// live in registers.  For the 5-point stencil (order 2) the neighbours of a cell come from
//   - the thread's own registers (rows inside the strip),
//   - shared memory for the strip edges (top / bottom cell of the strips above and below),
//   - warp shuffles along x, with shared memory only across the two warps of a row (columns
//     31 | 32),
// so a step costs two shared stores, two shared loads and eight shuffles per thread instead of
// five shared accesses per cell.  The edge arrays are double-buffered: one barrier per step.
// Cells outside the grid are forced to 0 every step (they hold the Dirichlet boundary value the
// in-grid cells read); cells on the region edge read 0 beyond it, so their values go wrong by
// one cell per step inward -- exactly the shrinking valid window of temporal blocking: after k
// steps the cells at distance >= k from the region edge are exact.
#pragma once

#include <cuda_runtime.h>

namespace whv {

constexpr int kTileReg = 64;      // region edge
constexpr int kTileRows = 4;      // rows per thread (strip height)
constexpr int kTileStrips = 16;   // strips per region

// shared-memory edge exchange of one step (per buffer parity)
template <typename T>
struct TileEdges {
  T top[kTileStrips][kTileReg];   // first row of each strip
  T bot[kTileStrips][kTileReg];   // last row of each strip
  T xe[kTileStrips][2][kTileRows];  // columns 31 and 32 (the x neighbours across the two warps)
};

template <typename T>
struct TileCoef {
  T ih2x, ih2y, dt2;
  T ax, ay, b;     // c = 1: W^{n+1} = ax (W_{x-} + W_{x+}) + ay (W_{y-} + W_{y+}) + b W^n - W^{n-1}
};

// Steps n = n0 .. n0 + kk - 1 (W^n -> W^{n+1}).  wt(n) is w_n of the filter, ph(n) the forcing
// phase cos(omega_hat t^n); act[r] says whether the cell is inside the grid.  n = 0 is the
// Taylor start W^1 = W^0 + dt^2/2 (c^2 Delta W^0 - f).
template <typename T, bool VARC, bool FORCED, typename WF, typename PF>
__device__ __forceinline__ void tile_steps_o2(T (&cur)[kTileRows], T (&prv)[kTileRows], T (&acr)[kTileRows],
                                              const T (&cc)[kTileRows], const T (&ff)[kTileRows],
                                              const bool (&act)[kTileRows], int n0, int kk,
                                              const TileCoef<T>& cf, WF wt, PF ph, TileEdges<T>* E) {
  const int tid = threadIdx.x;
  const int i = tid & 63, s = tid >> 6, lane = tid & 31;
  for (int q = 0; q < kk; ++q) {
    const int n = n0 + q;
    TileEdges<T>& e = E[q & 1];
    e.top[s][i] = cur[0];
    e.bot[s][i] = cur[kTileRows - 1];
    if (i == 31 || i == 32) {
#pragma unroll
      for (int r = 0; r < kTileRows; ++r) e.xe[s][i - 31][r] = cur[r];
    }
    __syncthreads();
    const T up0 = s > 0 ? e.bot[s - 1][i] : T(0);
    const T dn3 = s < kTileStrips - 1 ? e.top[s + 1][i] : T(0);
    const T w = wt(n + 1);
    const T fph = FORCED ? (n > 0 ? cf.dt2 : T(0.5) * cf.dt2) * ph(n) : T(0);
    T wn[kTileRows];
#pragma unroll
    for (int r = 0; r < kTileRows; ++r) {
      const T c = cur[r];
      T l = __shfl_up_sync(0xffffffffu, c, 1);
      T rt = __shfl_down_sync(0xffffffffu, c, 1);
      if (lane == 0) l = i == 0 ? T(0) : e.xe[s][0][r];
      if (lane == 31) rt = i == kTileReg - 1 ? T(0) : e.xe[s][1][r];
      const T u = r > 0 ? cur[r - 1] : up0;
      const T d = r < kTileRows - 1 ? cur[r + 1] : dn3;
      T x;
      if (!VARC && n > 0) {
        x = fma(cf.ay, u + d, fma(cf.ax, l + rt, fma(cf.b, c, -prv[r])));
      } else {
        T L = fma(l + rt - T(2) * c, cf.ih2x, (u + d - T(2) * c) * cf.ih2y);
        if (VARC) L *= cc[r];
        x = n > 0 ? fma(cf.dt2, L, fma(T(2), c, -prv[r])) : fma(T(0.5) * cf.dt2, L, c);
      }
      if (FORCED) x = fma(-fph, ff[r], x);
      wn[r] = act[r] ? x : T(0);
    }
#pragma unroll
    for (int r = 0; r < kTileRows; ++r) {
      prv[r] = cur[r];
      cur[r] = wn[r];
      acr[r] = fma(w, wn[r], acr[r]);
    }
  }
  __syncthreads();   // the last step's edge reads are done before a next call writes the edges
}

}  // namespace whv
