// Internal declarations of the GB300 solver library (not part of the ABI).
//
// Every solve runs in a slot of a pool.  A pool holds the per-shape data
// (FFT schedules, twiddles, Green's table) and `capacity` slots; each slot
// owns strided vectors, a spectrum workspace, reduction partials and a
// SlotState.  Kernels carry a batch dimension: blockIdx.z indexes a
// device-side active list of slots, and each kernel acts only on slots whose
// phase matches the phase it serves.  A single solve is a pool of one slot.
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

// Spectrum precision of a slot: FP64, FP32, or double-float on the FP32 pipe.
enum Spec { SPEC_FP64 = 0, SPEC_FP32 = 1, SPEC_DF64 = 2 };

// Per-slot phases of the device state machine.
enum Phase {
  PH_IDLE = 0,     // free or finished and collected
  PH_SETUP = 1,    // s, sqrt(eps), q, q + lambda
  PH_INIT = 2,     // r_0 of the next PCG
  PH_ITER = 3,     // Algorithm 2 iterations
  PH_NLEVAL = 4,   // nonlinear PB: fresh ionic charge, outer residual, next source
  PH_TRIAL = 5,    // nonlinear PB: residual at a trial step t
  PH_COMMIT = 6,   // nonlinear PB: apply the accepted step
  PH_CERT = 7,     // FP64 certificate of the result
  PH_DONE = 8      // result ready for the host
};

enum Counter {
  CNT_VR = 0, CNT_PAP, CNT_RR, CNT_AUX, CNT_AUX2, CNT_MU, CNT_WSUM, CNT_AUX3, CNT_APSUM, CNT_PSUM,
  CNT_COUNT
};

// Precomputed factors of the ionic charge (Eqs. rhoions, ionsconcPB).
struct IonParams {
  int nspecies;
  double zq[GPS_MAX_SPECIES];      // valences
  double zn[GPS_MAX_SPECIES];      // z_i * n_i  (bohr^-3)
  double z2n_kt[GPS_MAX_SPECIES];  // z_i^2 n_i / kT
  double inv_kt;
  double inv_eps0m1;               // 1/(eps0 - 1)
  double exp_cap;
  double lambda0;                  // 4 pi sum z_i^2 n_i / kT
  int steric;                      // modified PB (Eq. ionsconcMPB)
  double a[GPS_MAX_SPECIES];       // n_i^inf / n_i^max (Eq. maxconc)
};

// Device state of one slot (one request).
struct SlotState {
  IonParams ion;
  // PCG (Algorithm 2)
  double vr, vr_prev, pAp, alpha, beta, rr, rr0, tol2;
  double mu_sum;        // periodic: sum of s*r (FP64, x pass)
  double wsum;          // periodic GPe: sum of w = sqrt(eps) v (x inverse pass)
  double background;    // periodic GPe: mean of rho removed
  double k0;            // periodic linear operator: k = 0 value of the normalized kernel
  double tol_abs, tol_rel, mixed_switch;
  double aux[8];        // results of one-off reductions
  // nonlinear PB (Algorithm 4)
  double F, F0, t, tol_outer, eta, forcing, lam_sum, eps_sum;
  double F_prev, eta_prev;  // Newton: previous outer residual and inner tolerance (forcing rule)
  double cert;          // ||g|| / ||phi||, -1 if not computed
  double rr_min;        // smallest ||r||^2 seen in the FP32 phase
  double rr_switch;     // ||r||^2 below which the FP32 spectrum takes over (mixed)
  double ap_mean;       // periodic GPe: grid mean of A p removed in the r update
  double ap_sum, p_sum;
  int stall;            // FP32 iterations since the last new minimum
  int phase, kind, status;
  int iter, max_iter, iters_total, fp64_iters;
  int use_k0, neutralize, gauge;
  int mixed, spec, spec_hi, restart, certify;   // spec: spectrum precision in use
  int mixed_req;        // the caller asked for a mixed precision (nonlinear PB: each inner solve)
  int newton, outer, max_outer, bad_eps;
  int forcing_ew;       // Newton inner tolerance by Eisenstat-Walker choice 2 (else min(forcing, F/F0))
  // Set by the x inverse pass once v and (v, r) of this iteration exist,
  // and by update_p once p, A p and alpha do; each update kernel acts only
  // on its predecessor's flag (a pipeline of another precision may have
  // been left out of the launch sequence) and clears it.
  int vdone, pdone;
  int warm;             // INIT starts from the previous solve (Fields wphi, wd)
  unsigned int counter[CNT_COUNT];
};

// Geometry of the FFT passes, shared by every slot of a pool.
// Row pitch of a spectrum row of Hx complex values.
inline int spectrum_pitch(int Hx) { return Hx + (Hx & 1); }

struct PassGeom {
  int nx, ny, nz;      // real grid
  int Px, Py, Pz;      // padded transform lengths
  int Hx;              // Px/2 + 1
  int Hp;              // row pitch of the spectrum (elements): Hx rounded up to even, so
                       // that every spectrum row starts on a 16-byte boundary
  int nrows;           // ny*nz (rows of the x passes)
  int lines_x;         // row pairs per CTA in the x passes
  int tile_y, tile_z;  // columns per CTA in the y / z passes
  int x_reg;           // FP32 spectrum: 1 = x passes by the register-resident kernels
  int z_tma;           // FP32 / df64 spectrum: 1 = z pass by the TMA-staged kernel
};

// Slot addressing of one launch.  active == nullptr: slot 0 only, no phase
// test (st may then be nullptr too).
struct Batch {
  const int* active;   // active[0] = count, active[1 + i] = slot id
  SlotState* st;       // per-slot states (array of capacity)
  int phase;           // the phase this launch serves
  int prec;            // FFT passes: serve slots whose spectrum precision is prec, -1 any
  size_t vstride;      // elements between slots in every vector
  double* partials;    // reduction partials, pstride per slot
  double* partials2;
  double* partials3;
  int pstride;
  int* acted;          // optional: set to 1 by a block that served a slot (profiling)
};

// Field roles of one spectrum-pipeline launch (base pointers of slot 0).
struct PipeArgs {
  const double* in;         // x_fwd input
  const double* in_scale;   // optional factor (s)
  const float* in_scale32;  // optional: in_scale rounded to float, for the FP32 spectrum
  const float* out_scale32; // optional: out_scale rounded to float, for the FP32 spectrum
  double* out;              // x_inv output
  const double* out_scale;  // optional factor (s or sqrt(eps))
  const double* dot_with;   // optional: reduce (out, dot_with) into st.vr
  const double* table;      // normalized octant Green's / Laplacian table
  const float* table32;     // optional: the table rounded to float (FP32 spectrum)
  const float2* tabledf;    // optional: the table as double-float (hi, lo) (df64 spectrum)
  void* W;                  // spectrum base (slot 0)
  size_t wstride;           // complex elements between slots
  int slot_k0;              // use st[slot].k0 for k = 0 when st[slot].use_k0
  int red_mu;               // reduce sum(in * in_scale) into st.mu_sum (x_fwd)
  int red_wsum;             // reduce sum of unscaled output into st.wsum (x_inv)
};

// Block prologue: slot served by this block, or -1.
__device__ __forceinline__ int batch_slot(const Batch& b) {
  if (!b.active) return blockIdx.z == 0 ? 0 : -1;
  if ((int)blockIdx.z >= b.active[0]) return -1;
  const int s = b.active[1 + blockIdx.z];
  if (b.st && b.st[s].phase != b.phase) return -1;
  return s;
}

// Records that this launch did work for some slot (profiling only).
__device__ __forceinline__ void mark_acted(const Batch& b) {
  if (b.acted && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) *b.acted = 1;
}

// ---- FFT pass launchers (fft.cu) -----------------------------------------
template <typename V>
void launch_x_fwd(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st);
template <typename V>
void launch_y(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, bool inverse, int nslots, cudaStream_t st);
template <typename V>
void launch_z(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, int nslots, cudaStream_t st);
template <typename V>
void launch_x_inv(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st);
// Register-resident column passes (fft_col.cu) for power-of-two lengths
// 64 .. 1024: mode 0 y forward, 1 y inverse, 2 z.  false: length not covered
// (and always for the FP64 spectrum).  Their twiddle array `tw` must hold
// 3 L entries: the plain table and the two per-stage layouts whose plain
// indices col_stage_twiddle_index(L, idx[2 L]) writes (forward, reversed).
bool col_pass_supported(int L);
// Bounded device waits (TMA-staged passes) that gave up since the last call;
// resets the count.
unsigned int take_wait_timeouts();
bool col_stage_twiddle_index(int L, int* idx);
// Register-resident x passes (same lengths and twiddle requirement; used
// for the df64 spectrum).
template <typename V>
bool launch_xr_pass(bool inverse, int L, const PassGeom& g, const V* tw, const Batch& b,
                    const PipeArgs& a, int nslots, cudaStream_t st);
template <typename V>
bool launch_col_pass(int mode, int L, const PassGeom& g, const V* tw, const Batch& b,
                     const PipeArgs& a, int nslots, cudaStream_t st);
size_t x_lines_smem_bytes(int L, int lines, size_t vbytes);
int x_pass_blocks(const PassGeom& g);
// Lines (x passes) or columns (y, z passes) per CTA that the shared-memory
// kernels support: 1 .. kMaxLinesPerCta, with at most kMaxLinesSmem bytes of
// shared memory (x_lines_smem_bytes).  The tuner tries every count in that
// range; default_lines is the untuned choice for `units` lines of length L:
// about 2048 elements per CTA while that leaves >= ~2 CTAs per SM, clamped to
// the supported range.
constexpr int kMaxLinesPerCta = 16;
constexpr size_t kMaxLinesSmem = 220 * 1024;
int default_lines(int L, int units, size_t vbytes);

// ---- kernels.cu ------------------------------------------------------------
int grid_blocks(size_t n, int threads);
void count_launch();
unsigned long long launch_count();

}  // namespace gps
