// Device helpers shared by the kernels of the library: complex arithmetic on
// double2/float2 and deterministic block / grid reductions.
#pragma once

#include <cuda_runtime.h>

#include "gps_internal.h"

namespace gps {

// Double-float number: the unevaluated sum hi + lo of two floats, about 48
// significant bits.  Arithmetic by error-free transformations (Knuth's
// TwoSum, FMA-based TwoProd; Dekker's renormalizing Fast2Sum where a
// normalized value is wanted) runs on the FP32 pipe, which on this GPU
// issues 64x the FP64 rate.  Neither addition nor multiplication
// renormalizes its result: hi is the rounded result of the hi parts and lo
// collects the exact error terms, so each operation's error stays bounded by
// a small multiple of u^2 (|a| + |b|) or u^2 |a||b| (u = 2^-24), the
// norm-wise bound an FFT's error analysis needs, while |lo| may reach a few
// ulps of hi along a chain of butterflies.
using ::fma;

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit constexpr df(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit constexpr df(int i) : df((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return df(s, b - (s - a));
}
// Addition without the final renormalization: the TwoSum of the hi parts is
// exact for any operands, so hi + lo stays the sum to within the rounding of
// the lo parts.  In the FFT passes an element goes through a few additions
// and at most one product per stage, so lo grows by a few ulps of hi and the
// norm-wise error bound keeps its u^2 order (tested: df64 spectra match the
// FP64 oracle to 1e-12).
__device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum error of hi parts
  return df(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// Product without the final renormalization, like operator+: hi is the
// rounded product of the hi parts, lo its exact TwoProd error plus the cross
// terms, so hi + lo is the product to within u^2 |a||b| while lo may exceed
// half an ulp of hi (by the few ulps that a chain of butterflies adds).
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                     // TwoProd error
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df(p, e);
}
// a b + s c d (s = +1 or -1) as one double-float: the TwoSum of the two hi
// products, their TwoProd errors and the four cross terms accumulated in the
// low part (16 FP32 operations against 22 for two products and a sum).
template <int S>
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
  const float p = a.hi * b.hi;
  const float q = S > 0 ? c.hi * d.hi : -(c.hi * d.hi);
  const float e1 = fmaf(a.hi, b.hi, -p);
  const float e2 = S > 0 ? fmaf(c.hi, d.hi, -q) : fmaf(-c.hi, d.hi, -q);
  const float s = p + q;
  const float bb = s - p;
  float lo = (p - (s - bb)) + (q - bb);                // TwoSum error of p + q
  lo += e1 + e2;
  lo = fmaf(a.hi, b.lo, lo);
  lo = fmaf(a.lo, b.hi, lo);
  lo = S > 0 ? fmaf(c.hi, d.lo, lo) : fmaf(-c.hi, d.lo, lo);
  lo = S > 0 ? fmaf(c.lo, d.hi, lo) : fmaf(-c.lo, d.hi, lo);
  return df(s, lo);
}
__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }

// IEEE 754 conversions on the integer pipe.  On this GPU the FP64 pipe,
// which also carries the double <-> float conversion instructions, issues at
// 1/64 of the FP32 rate, so a pass that converts every point is FP64-bound
// unless the conversion is done with integer operations.  Written from the
// binary64 / binary32 formats: d2f_rn rounds to nearest, ties to even;
// results below the smallest normal float flush to signed zero (f2d flushes
// float subnormals the same way); overflow gives a signed infinity; a NaN
// stays a (quiet) NaN.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned int hi = (unsigned int)(u >> 32), lo = (unsigned int)u;
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned int m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
  const unsigned int rest = lo & 0x1FFFFFFFu;                   // the 29 bits rounded off
  const int ef = e - 1023 + 127;
  unsigned int bits;
  if (e == 0x7FF) {
    bits = 0x7F800000u | ((m | rest) ? 0x400000u | m : 0u);
  } else if (ef >= 0xFF) {
    bits = 0x7F800000u;
  } else if (ef <= 0) {
    bits = 0u;
  } else {
    bits = ((unsigned int)ef << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) bits += 1u;   // may carry to inf
  }
  return __uint_as_float(bits | sign);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int sign = b & 0x80000000u;
  const unsigned int e = (b >> 23) & 0xFFu;
  const unsigned int m = b & 0x7FFFFFu;
  unsigned int hi;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
  if (e == 0xFF) hi = 0x7FF00000u | (m ? 0x80000u : 0u) | (m >> 3);
  else hi = ((e + 896u) << 20) | (m >> 3);
  return __longlong_as_double((long long)(((unsigned long long)(hi | sign) << 32) | (unsigned long long)(m << 29)));
}

// double -> double-float and back with one FP64 operation each.
__device__ __forceinline__ df df_of(double d) {
  const float h = d2f_rn(d);
  return df(h, d2f_rn(d - f2d(h)));
}
__device__ __forceinline__ double dbl_of(df a) { return f2d(a.hi) + f2d(a.lo); }

// Complex double-float (16 bytes, the size of a double2).
struct __align__(16) dfc {
  df x, y;
};

template <typename V> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };
template <> struct Real<dfc> { using T = df; };

template <typename V>
__device__ __forceinline__ V mk(typename Real<V>::T x, typename Real<V>::T y) {
  V v; v.x = x; v.y = y; return v;
}
template <typename V> __device__ __forceinline__ V czero() {
  using T = typename Real<V>::T;
  return mk<V>(T(0), T(0));
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
// double-float complex products: each component one two-product sum
template <> __device__ __forceinline__ dfc cmul<dfc>(dfc a, dfc b) {
  return mk<dfc>(df_dot2<-1>(a.x, b.x, a.y, b.y), df_dot2<+1>(a.x, b.y, a.y, b.x));
}
template <> __device__ __forceinline__ dfc cmulc<dfc>(dfc a, dfc b) {
  return mk<dfc>(df_dot2<+1>(a.x, b.x, a.y, b.y), df_dot2<-1>(a.y, b.x, a.x, b.y));
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

// Blocks of one slot: the x-y plane of the grid (blockIdx.z is the slot).
__device__ __forceinline__ unsigned int linear_block() { return blockIdx.x + gridDim.x * blockIdx.y; }
__device__ __forceinline__ unsigned int num_blocks() { return gridDim.x * gridDim.y; }

// Deterministic grid reduction over the blocks of one slot: every block stores
// its partial; the last block to arrive (atomic ticket) sums all partials in
// a fixed order and returns true in all of its threads with *result set.  The sum order does not depend
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

// Three sums over the blocks of one slot in one pass (one block reduction,
// one atomic ticket, one last-block tail); same fixed-order determinism as
// grid_reduce.
__device__ __forceinline__ bool grid_reduce3(double a, double b, double c, double* pa, double* pb,
                                             double* pc, unsigned int* counter, double* ra,
                                             double* rb, double* rc) {
  __shared__ double part[3][32];
  __shared__ bool am_last;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    part[0][wid] = a;
    part[1][wid] = b;
    part[2][wid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    double x = lane < nw ? part[0][lane] : 0.0;
    double y = lane < nw ? part[1][lane] : 0.0;
    double z = lane < nw ? part[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
      z += __shfl_down_sync(0xffffffffu, z, o);
    }
    if (lane == 0) {
      const unsigned int lb = linear_block();
      pa[lb] = x;
      pb[lb] = y;
      pc[lb] = z;
      __threadfence();
      const unsigned int t = atomicAdd(counter, 1u);
      am_last = (t == num_blocks() - 1);
    }
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const unsigned int nb = num_blocks();
  double x = 0.0, y = 0.0, z = 0.0;
  for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) {
    x += __ldcg(pa + i);
    y += __ldcg(pb + i);
    z += __ldcg(pc + i);
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
    z += __shfl_down_sync(0xffffffffu, z, o);
  }
  __syncthreads();
  if (lane == 0) {
    part[0][wid] = x;
    part[1][wid] = y;
    part[2][wid] = z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int w = 0; w < nw; ++w) {
      sx += part[0][w];
      sy += part[1][w];
      sz += part[2][w];
    }
    *ra = sx;
    *rb = sy;
    *rc = sz;
    *counter = 0u;
  }
  __syncthreads();
  return true;
}

}  // namespace gps
