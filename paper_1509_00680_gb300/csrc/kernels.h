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

void launch_setup_s(const double* eps, double* s, double* sq, size_t n, PcgScalars* sc,
                    cudaStream_t st);
void launch_fd16_q(const double* sq, double* q, int nx, int ny, int nz, double hx, double hy,
                   double hz, int perx, int pery, int perz, const Fd16& c, cudaStream_t st);
void launch_qlam_linear(const double* q, const double* eps, double* qlam, size_t n, double lambda0,
                        double inv_e0m1, double* partials, PcgScalars* sc, cudaStream_t st);
void launch_sum(const double* a, size_t n, double* partials, unsigned int* counter, double* out,
                cudaStream_t st);
void launch_copy_scaled(const double* a, double* b, size_t n, double f, cudaStream_t st);
void launch_mul(const double* a, const double* b, double* c, size_t n, cudaStream_t st);
void launch_init(const double* rho, double* r, double* phi, double* p, double* Ap, size_t n,
                 double tol_abs, double tol_rel, int max_iter, double* partials, PcgScalars* sc,
                 int zero_phi, const double* bg_sum, cudaStream_t st);
void launch_update_p(const double* v, const double* r, const double* qlam, const double* sqrt_eps,
                     const double* s, double* p, double* Ap, size_t n, int periodic, int project,
                     double* partials, PcgScalars* sc, cudaStream_t st);
void launch_update_r(double* phi, double* r, const double* p, const double* Ap, size_t n,
                     double* partials, PcgScalars* sc, cudaStream_t st);
void launch_fp_source(const double* rho, const double* rions, const double* qlam, const double* phi,
                      const double* sq, double* out, size_t n, double bg, double* partials,
                      PcgScalars* sc, cudaStream_t st);
void launch_fp_residual(const double* w, const double* s, const double* phi, size_t n, double c,
                        double* partials, double* partials2, PcgScalars* sc, cudaStream_t st);
void launch_ionic_charge(const double* phi, const double* eps, double* out, size_t n,
                         const IonParams& ip, cudaStream_t st);
void launch_nl_eval(const double* phi, const double* eps, const double* rions, const double* rp,
                    double* fresh, double* lam, size_t n, const IonParams& ip, int newton,
                    double* partials, PcgScalars* sc, cudaStream_t st);
void launch_nl_source(const double* fresh, const double* rions, const double* rp, const double* q,
                      const double* lam, double* src, double* qlam, size_t n, double eta,
                      double* partials, PcgScalars* sc, cudaStream_t st);
void launch_nl_step(double* phi, const double* eps, double* rions, double* rp, const double* fresh,
                    const double* lam, const double* dphi, const double* r, size_t n,
                    const IonParams& ip, double eta, double t, int commit, double* partials,
                    PcgScalars* sc, cudaStream_t st);
void launch_table_periodic(double* kern, double* lap, int Hx, int hy, int hz, double dkx, double dky,
                           double dkz, double inv_n, cudaStream_t st);
void launch_table_surface(double* kern, int Hx, int hy, int hz, double dkx, double dky, double dkz,
                          double Lz, double inv_n, cudaStream_t st);
void launch_free_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz,
                      double R, cudaStream_t st);
void launch_axis_matrix(const double* in, double* out, const double* C, int A, int J, int B, int K,
                        cudaStream_t st);

}  // namespace gps
