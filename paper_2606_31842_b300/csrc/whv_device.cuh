// Device helpers shared by the kernels: warp / block sums and the deterministic grid reduction.
#pragma once

#include <cuda_runtime.h>

namespace whv {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int flat_tid() {
  return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int flat_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }
__device__ __forceinline__ int flat_bid() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int flat_nblocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Block-wide sum (block size a multiple of 32, at most 1024); the result is valid in thread 0.
// Fixed tree order => deterministic.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  const int tid = flat_tid();
  const int lane = tid & 31, wid = tid >> 5, nw = flat_nthreads() >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (tid < nw) ? sh[tid] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Grid reduction without a second launch: every block deposits its sum, the last block to
// arrive adds the deposits in index order (deterministic) and returns true; thread 0 of that
// block receives the total in *total.  The counter is re-armed for the next launch.
__device__ __forceinline__ bool grid_reduce(double bsum, double* partials, unsigned* counter,
                                            double* total) {
  __shared__ bool s_last;
  const int tid = flat_tid();
  const int nb = flat_nblocks();
  if (tid == 0) {
    partials[flat_bid()] = bsum;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned)(nb - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = tid; i < nb; i += flat_nthreads()) s += __ldcg(partials + i);
  s = block_sum(s);
  if (tid == 0) {
    *total = s;
    *counter = 0u;
  }
  return true;
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident) with a bounded wait: count
// and gen are the arrival counter and generation, err an error flag.  Returns false (and raises
// *err) if this CTA waited past the limit (~4 s) or another CTA raised *err; every CTA then
// returns false at its next barrier.
constexpr unsigned long long kBarrierSpins = 1ull << 26;   // x 64 ns sleeps

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* err, unsigned nblocks) {
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
        // another CTA gave up: stop waiting for a barrier that will not complete
        if ((spins & 1023ull) == 0 && *(volatile int*)err) { ok = 0; break; }
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

}  // namespace whv
