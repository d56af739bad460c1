// Deterministic block reductions (fixed shuffle tree, then warps in order).
#pragma once

namespace bie {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// All threads of the block must call; every thread gets the result.  sh needs
// B/32 doubles and may be reused by the next call.
template <int B>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < B / 32; ++k) r += sh[k];
  return r;
}

template <int B>
__device__ __forceinline__ double block_min(double v, double* sh) {
  v = warp_min(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
#pragma unroll
  for (int k = 1; k < B / 32; ++k) r = fmin(r, sh[k]);
  return r;
}

}  // namespace bie
