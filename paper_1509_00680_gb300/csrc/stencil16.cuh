// Order-16 central first derivatives on the grid (the paper's finite-
// difference filters, Sec. "Numerical results"): d/dx u ~ (1/h) sum_j d_j
// (u(x + jh) - u(x - jh)), j = 1..8.  Periodic axes wrap (they must have at
// least 8 points); free axes continue the field by its face value.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace gps {

struct Stencil16 {
  int nx, ny, nz;
  int perx, pery, perz;   // axes that wrap
  double ihx, ihy, ihz;   // 1 / h
  double d[9];            // d_1..d_8 (d[0] unused)
};

__device__ __forceinline__ void point_of16(size_t idx, const Stencil16& s, int* i, int* j, int* k) {
  *i = (int)(idx % s.nx);
  *j = (int)((idx / s.nx) % s.ny);
  *k = (int)(idx / ((size_t)s.nx * s.ny));
}

__device__ __forceinline__ int shift16(int i, int m, int n, int per) {
  if (per) return i + m >= n ? i + m - n : (i + m < 0 ? i + m + n : i + m);
  const int t = i + m;
  return t >= n ? n - 1 : (t < 0 ? 0 : t);
}

// grad u at point idx = (i, j, k).
__device__ __forceinline__ double3 grad16(const double* __restrict__ u, size_t idx, int i, int j, int k,
                                          const Stencil16& s) {
  const double* row = u + (idx - i);
  const size_t sy = s.nx, sz = (size_t)s.nx * s.ny;
  const size_t bxz = (size_t)k * sz + i, bxy = (size_t)j * s.nx + i;
  double dx = 0.0, dy = 0.0, dz = 0.0;
#pragma unroll
  for (int m = 1; m <= 8; ++m) {
    const double c = s.d[m];
    dx = fma(c, row[shift16(i, m, s.nx, s.perx)] - row[shift16(i, -m, s.nx, s.perx)], dx);
    dy = fma(c, u[bxz + (size_t)shift16(j, m, s.ny, s.pery) * sy] - u[bxz + (size_t)shift16(j, -m, s.ny, s.pery) * sy],
             dy);
    dz = fma(c, u[bxy + (size_t)shift16(k, m, s.nz, s.perz) * sz] - u[bxy + (size_t)shift16(k, -m, s.nz, s.perz) * sz],
             dz);
  }
  return make_double3(dx * s.ihx, dy * s.ihy, dz * s.ihz);
}

}  // namespace gps
