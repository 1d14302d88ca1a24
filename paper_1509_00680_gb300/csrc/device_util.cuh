// Device helpers shared by the kernels of the library: complex arithmetic on
// double2/float2 and deterministic block / grid reductions.
#pragma once

#include <cuda_runtime.h>

#include "gps_internal.h"

namespace gps {

template <typename V> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

template <typename V>
__device__ __forceinline__ V mk(typename Real<V>::T x, typename Real<V>::T y) {
  V v; v.x = x; v.y = y; return v;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, typename Real<V>::T s) { return mk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mk<V>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Sum of v over the block (any blockDim.x multiple of 32, <= 1024); result
// valid in every thread.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
  __shared__ double total;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = lane < nw ? warp_part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) total = t;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ unsigned int linear_block() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ unsigned int num_blocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Deterministic grid reduction: every block stores its partial; the last block
// to arrive (atomic ticket) sums all partials in a fixed order and returns
// true in all of its threads with *result set.  The sum order does not depend
// on which block arrives last, so results are bitwise reproducible.
__device__ __forceinline__ bool grid_reduce(double v, double* partials, unsigned int* counter,
                                            double* result) {
  __shared__ bool am_last;
  const double bs = block_sum(v);
  if (threadIdx.x == 0) {
    partials[linear_block()] = bs;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == num_blocks() - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const unsigned int nb = num_blocks();
  double s = 0.0;
  for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *result = s;
    *counter = 0u;
  }
  __syncthreads();
  return true;
}

}  // namespace gps
