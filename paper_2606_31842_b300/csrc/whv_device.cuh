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

}  // namespace whv
