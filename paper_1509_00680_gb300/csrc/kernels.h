// Host launchers of the pointwise / stencil / table kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "gps_internal.h"

namespace gps {

// Order-16 central second-derivative coefficients c_0..c_8.
struct Fd16 {
  double c[9];
};

// Base pointers (slot 0) of every per-slot vector of a pool; slot k is at
// base + k * Batch::vstride.
struct Fields {
  double *rho, *eps, *phi;               // request inputs / output
  double *s, *sq, *q, *qlam;             // eps^-1/2, sqrt(eps), q, q + lambda
  double *r, *p, *Ap, *v;                // PCG vectors
  double *rions, *rp, *fresh, *lam, *dphi, *src;   // Algorithm 4
  double *tmp;                           // certificate source
  float *s32;                            // eps^-1/2 rounded to float (FP32 spectrum passes)
  const double *wphi, *wd;               // warm start: previous phi and b - r (slot 0 only)
};

int vec_blocks(size_t n, int nslots);
void launch_setup_s(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st);
void launch_fd16_q(const Batch& b, const Fields& f, int nx, int ny, int nz, double hx, double hy,
                   double hz, int perx, int pery, int perz, const Fd16& c, int nslots,
                   cudaStream_t st);
void launch_setup_final(const Batch& b, const Fields& f, size_t n, double inv_p, int periodic,
                        int nslots, cudaStream_t st);
void launch_init(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st);
void launch_update_p(const Batch& b, const Fields& f, size_t n, int periodic, int nslots,
                     cudaStream_t st);
void launch_update_r(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st);
void launch_nl_eval(const Batch& b, const Fields& f, size_t n, double inv_p, int periodic,
                    int nslots, cudaStream_t st);
void launch_nl_step(const Batch& b, const Fields& f, size_t n, int commit, int nslots,
                    cudaStream_t st);
void launch_fp_source(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st);
void launch_fp_residual(const Batch& b, const Fields& f, size_t n, int periodic, int nslots,
                        cudaStream_t st);
void launch_eps_differ(const double* a, const double* b, size_t n, int* flag, cudaStream_t st);
void launch_warm_store(const Batch& b, const Fields& f, double* weps, double* wphi, double* wd,
                       size_t n, cudaStream_t st);
void launch_table_split(const double* t, float* t32, float2* tdf, size_t n, cudaStream_t st);
void launch_ionic_charge(const double* phi, const double* eps, double* out, size_t n,
                         const IonParams& ip, cudaStream_t st);
void launch_table_periodic(double* kern, double* lap, int Hx, int hy, int hz, double dkx, double dky,
                           double dkz, double inv_n, cudaStream_t st);
void launch_table_surface(double* kern, int Hx, int hy, int hz, double dkx, double dky, double dkz,
                          double Lz, double inv_n, cudaStream_t st);
void launch_free_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz,
                      double R, cudaStream_t st);
void launch_axis_matrix(const double* in, double* out, const double* C, int A, int J, int B, int K,
                        cudaStream_t st);

}  // namespace gps
