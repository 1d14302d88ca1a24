// Host launchers of the pointwise / stencil / table kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "gps_internal.h"
#include "stencil16.cuh"

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
  const double *wphi, *wd;               // warm start: phi_0 and b_prev - r_prev at each slot's offset
                                         // (single solves: the retained arrays, slot 0; engine pools:
                                         // phi and Ap themselves, filled at admission)
  const double* gam;                     // ion-exclusion function given by the caller (slot 0
                                         // only); nullptr: the cavity function (eps-1)/(eps0-1)
};

int vec_blocks(size_t n, int nslots);
void launch_setup_s(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st);
// out = in rounded to float (round to nearest even), n values.
void launch_to_float(const double* in, float* out, size_t n, cudaStream_t st);
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
void launch_warm_store(const Batch& b, const Fields& f, int slot, double* weps, double* wphi, double* wd,
                       size_t n, cudaStream_t st);
void launch_table_split(const double* t, float* t32, float2* tdf, size_t n, cudaStream_t st);
void launch_ionic_charge(const double* phi, const double* eps, const double* gam, double* out, size_t n,
                         const IonParams& ip, cudaStream_t st);
void launch_table_periodic(double* kern, double* lap, int Hx, int hy, int hz, double dkx, double dky,
                           double dkz, double inv_n, cudaStream_t st);
void launch_table_surface(double* kern, int Hx, int hy, int hz, double dkx, double dky, double dkz,
                          double Lz, double inv_n, cudaStream_t st);
void launch_free_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz,
                      double R, cudaStream_t st);
void launch_wire_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz, double R,
                      const double* k0R, const double* k1R, cudaStream_t st);
void launch_axis_matrix(const double* in, double* out, const double* C, int A, int J, int B, int K,
                        cudaStream_t st);

// ---- DFT-facing quantities (dft.cu) --------------------------------------

int dft_blocks(size_t n);
void launch_sccs(const double* rho, double* eps, double* deps, size_t n, double rho_max, double rho_min,
                 double eps0, cudaStream_t st);
// rho_pol; tmp: n doubles of scratch (ln eps)
void launch_polarization(const Stencil16& s, const double* rho, const double* eps, const double* phi,
                         double* tmp, double* out, size_t n, cudaStream_t st);
void launch_veps(const Stencil16& s, const double* deps, const double* phi, double* out, size_t n, cudaStream_t st);
// part: 2 x dft_blocks(n) doubles, per block sum rho phi and sum eps |grad phi|^2
void launch_energy(const Stencil16& s, const double* rho, const double* eps, const double* phi, size_t n,
                   double* part, cudaStream_t st);

// ---- comparison solvers (sc.cu): Algorithm 1 (SC), PSD, PSD + DIIS ------

constexpr int kMaxDiis = 8;   // GPS_MAX_DIIS

// Ring slots of the DIIS history in use, oldest first (the newest last).
struct DiisSlots {
  int cnt;
  int slot[kMaxDiis];
};

// Everything the comparison-solver kernels touch.  Periodic axes must have
// at least 8 points (the order-16 stencil wraps once).
struct ScArgs {
  SlotState* S;                 // slot 0 of the pool: phase, scalars, convergence
  double* part;                 // 4 x pstride reduction partials
  double* dpart;                // kMaxDiis x pstride partials (DIIS dot products)
  int pstride;
  unsigned int* cnt;            // 5 reduction tickets (zero between launches)
  const double *eps, *rho;
  double* phi;                  // SC output (PSD: see the launchers)
  double *gx, *gy, *gz;         // grad ln eps (order 16)
  double* isc;                  // -1 / (4 pi eps)
  double* tmp;                  // ln eps during setup
  double *rho_eps, *rho_iter, *src;   // SC
  double *hist_phi, *hist_r, *hist_v; // DIIS ring, hist_m slots of n each
  double* hist_mr;              // <r/eps> of every ring slot; [kMaxDiis]: of the combination
  double* diis_B;               // kMaxDiis x kMaxDiis Gram matrix (ring-slot indexed)
  double* diis_c;               // coefficients of the current combination
  int hist_m;
  Stencil16 s16;                // grid, wrapping axes, order-16 coefficients
  size_t n;
  int periodic;
  double inv_n;
  double alpha;                 // PSD: fixed step, 0 = steepest descent
  int* acted;                   // optional: set by a launch that did work (profiling)
};

int sc_blocks(size_t n);
// Setup of SC (psd = 0) or PSD (psd = 1; phi0 = 0 and r0 = -4 pi rho are
// written to the given arrays) and g = grad ln eps.
void launch_sc_prep(const ScArgs& a, int psd, double* phi0, double* r0, cudaStream_t st);
// SC step after the vacuum solve phi = S(src).
void launch_sc_step(const ScArgs& a, cudaStream_t st);
// PSD: A v and alpha (diis: the mean <r/eps> of the DIIS combination).
void launch_psd_av(const ScArgs& a, const double* v, const double* r, double* Av, int diis, cudaStream_t st);
// PSD: phi_out = phi + alpha v, r_out = r - alpha A v, convergence; hist_slot
// >= 0 records <r_out/eps> for that DIIS ring slot.
void launch_psd_update(const ScArgs& a, const double* phi, const double* r, const double* v, const double* Av,
                       double* phi_out, double* r_out, int hist_slot, cudaStream_t st);
// DIIS: Gram row of the newest v, coefficients, combination into phi_w, r_w, v_w.
void launch_diis(const ScArgs& a, const DiisSlots& sl, double* phi_w, double* r_w, double* v_w,
                 cudaStream_t st);

}  // namespace gps
