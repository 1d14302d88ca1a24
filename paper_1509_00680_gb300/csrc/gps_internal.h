// Internal declarations of the GB300 solver library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gps.h"

namespace gps {

constexpr int kMaxStages = 16;
constexpr int kMaxLen = 4096;
constexpr double kPi = 3.14159265358979323846;
constexpr double kFourPi = 4.0 * kPi;

// Stockham schedule of one 1D transform length: L = prod radix[s].
struct FftSched {
  int L;
  int nst;
  int radix[kMaxStages];
  int ns[kMaxStages];   // product of the radices of the previous stages
};

// Device scalars of one PCG run (Algorithm 2).  Written by the last block of
// the reducing kernels, read by every block of the following kernels.
struct PcgScalars {
  double vr, vr_prev, pAp, alpha, beta, rr, rr0, tol2;
  double mu_sum;        // periodic: sum of s*r over the grid (FP64, x pass)
  double wsum;          // periodic: sum of w = sqrt(eps) v over the grid (x inverse pass)
  double background;    // periodic GPe: mean of rho removed
  double aux[8];        // scratch results of one-off reductions
  int iter, done, status, max_iter;
  int bad_eps;          // set if an eps value is not positive
  int pad_;
  unsigned int counter[8];
};

enum Counter { CNT_VR = 0, CNT_PAP = 1, CNT_RR = 2, CNT_AUX = 3, CNT_AUX2 = 4, CNT_MU = 5,
               CNT_WSUM = 6 };

// Precomputed factors of the ionic charge (Eqs. rhoions, ionsconcPB).
struct IonParams {
  int nspecies;
  double zq[GPS_MAX_SPECIES];    // valences
  double zn[GPS_MAX_SPECIES];    // z_i * n_i  (bohr^-3)
  double z2n_kt[GPS_MAX_SPECIES];  // z_i^2 n_i / kT
  double inv_kt;
  double inv_eps0m1;             // 1/(eps0 - 1)
  double exp_cap;
};

// One FFT pass configuration shared by the pass kernels.
struct PassGeom {
  int nx, ny, nz;      // real grid
  int Px, Py, Pz;      // padded transform lengths
  int Hx;              // Px/2 + 1
  int nrows;           // ny*nz (rows of the x passes)
  int lines_x;         // lines per CTA in x passes (row pairs)
  int tile_y, tile_z;  // columns per CTA in the y / z passes
};

template <typename V>
struct SpecBuf {
  V* W;                // [nz][Py][Hx] complex
};

// ---- FFT pass launchers (fft.cu) -----------------------------------------
// Forward x pass: rows of in (optionally scaled by scale) -> half spectra.
template <typename V>
void launch_x_fwd(const PassGeom& g, const FftSched& s, const V* tw, const double* in,
                  const double* scale, V* W, const int* done, cudaStream_t st,
                  double* partials = nullptr, PcgScalars* sc = nullptr, double* sum_out = nullptr);
template <typename V>
void launch_y(const PassGeom& g, const FftSched& s, const V* tw, V* W, bool inverse,
              const int* done, cudaStream_t st);
template <typename V>
void launch_z(const PassGeom& g, const FftSched& s, const V* tw, V* W, const double* table,
              double k0_override, int use_k0, double* mu_sum, const int* done, cudaStream_t st);
template <typename V>
void launch_x_inv(const PassGeom& g, const FftSched& s, const V* tw, const V* W, double* out,
                  const double* out_scale, const double* dot_with, double* partials,
                  PcgScalars* sc, int counter_slot, double* dot_out, const int* done,
                  cudaStream_t st, double* partials2 = nullptr, double* wsum_out = nullptr);
size_t x_lines_smem_bytes(int L, int lines, size_t vbytes);

// ---- kernels.cu ------------------------------------------------------------
int grid_blocks(size_t n, int threads);
void count_launch();
unsigned long long launch_count();

}  // namespace gps
