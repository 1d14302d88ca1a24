// Test harness: the integer-pipe IEEE conversions of the library's device
// helpers next to the CUDA casts, element by element.
#include "device_util.cuh"

using namespace gps;

__global__ void k_conv(const double* __restrict__ d, const float* __restrict__ f, float* d2f_mine,
                       float* d2f_ref, double* f2d_mine, double* f2d_ref, double* df_back, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  d2f_mine[i] = d2f_rn(d[i]);
  d2f_ref[i] = __double2float_rn(d[i]);
  f2d_mine[i] = f2d(f[i]);
  f2d_ref[i] = (double)f[i];
  df_back[i] = dbl_of(df_of(d[i]));
}

extern "C" int run_conversion_check(const double* d, const float* f, float* a, float* b, double* c,
                                    double* e, double* g, int n) {
  if (n <= 0) return 0;
  k_conv<<<(n + 255) / 256, 256>>>(d, f, a, b, c, e, g, n);
  return (int)cudaDeviceSynchronize();
}
