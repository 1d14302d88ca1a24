// Pointwise, stencil, reduction and table kernels of the PCG solver, in
// batched slot form (see gps_internal.h), and the device-side phase machine
// of every slot:
//
//   SETUP   s = eps^-1/2, sqrt(eps); q = sqrt(eps) lap sqrt(eps) by the
//           order-16 stencil (free/surface; periodic uses the spectrum
//           pipeline); q + lambda (Eq. corrPB)            -> INIT | NLEVAL
//   INIT    r_0 = -4 pi (source - background)                 -> ITER
//   ITER    Algorithm 2 with the identity of Eq. corr / corrPB
//                                   -> TRIAL | COMMIT (NLPB), CERT | DONE
//   NLEVAL  fresh ionic charge (Eqs. rhoions, ionsconcPB), outer residual,
//           next inner source (Algorithm 4)           -> INIT | CERT | DONE
//   TRIAL   outer residual at the trial step t (Newton line search)
//   COMMIT  apply the step                                   -> NLEVAL
//   CERT    FP64 certificate g = M(src - qlam phi/4pi) [+ c s] - phi -> DONE
//
// Phase changes are made by the last block of a slot's reduction, after every
// block of that slot has finished, so launches later in the same stream see
// them.  Every reduction is deterministic (fixed-order partials).
#include <atomic>
#include <cmath>

#include "device_util.cuh"
#include "gps_internal.h"
#include "kernels.h"

namespace gps {

constexpr int kT = 256;

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int grid_blocks(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  // 4 blocks of 256 threads on each of the 152 SMs: every block is resident
  // at once for any kernel of up to 64 registers, so no second partial wave
  // of blocks runs after the first (each thread loops over its elements).
  const size_t cap = 152 * 4;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Blocks per slot for the vector kernels.  It depends on the grid only, not
// on how many slots share the launch, so every slot reduces in the same order
// alone and in a batch (bitwise identical results).
int vec_blocks(size_t n, int nslots) {
  (void)nslots;
  return grid_blocks(n, kT);
}

#define GRID_STRIDE(i, n) \
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

#define SLOT_PROLOGUE(b)                  \
  const int slot = batch_slot(b);         \
  if (slot < 0) return;                   \
  mark_acted(b);                          \
  SlotState& S = b.st[slot];              \
  const size_t off = (size_t)slot * b.vstride;

__device__ __forceinline__ double* slot_partials(const Batch& b, int slot) {
  return b.partials + (size_t)slot * b.pstride;
}
__device__ __forceinline__ double* slot_partials2(const Batch& b, int slot) {
  return b.partials2 + (size_t)slot * b.pstride;
}
__device__ __forceinline__ double* slot_partials3(const Batch& b, int slot) {
  return b.partials3 + (size_t)slot * b.pstride;
}

// State after a PCG has stopped (converged, failed or out of iterations).
__device__ void after_pcg(SlotState& S) {
  if (S.kind == GPS_NLPB) {
    if (S.status == GPS_ERR_BREAKDOWN) {
      S.phase = PH_DONE;
      return;
    }
    S.status = GPS_OK;          // an inexact inner solve is a valid Newton / mixing step
    S.t = 1.0;
    S.phase = S.newton ? PH_TRIAL : PH_COMMIT;
    return;
  }
  S.phase = (S.status == GPS_OK && S.certify) ? PH_CERT : PH_DONE;
}

// ------------------------------------------------------------------ setup --

__global__ void k_setup_s(Batch b, Fields f, size_t n) {
  SLOT_PROLOGUE(b)
  const double* eps = f.eps + off;
  double* s = f.s + off;
  float* s32 = f.s32 ? f.s32 + off : nullptr;
  double* sq = f.sq + off;
  double acc = 0.0;
  int bad = 0;
  GRID_STRIDE(i, n) {
    const double e = eps[i];
    if (!(e > 0.0)) bad = 1;
    const double r = sqrt(e);
    sq[i] = r;
    const double si = 1.0 / r;
    s[i] = si;
    if (s32) s32[i] = (float)si;
    acc += e;
  }
  if (bad) S.bad_eps = 1;
  grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_AUX], &S.eps_sum);
}

// q = sqrt(eps) * sum_axes (1/h^2) sum_j c_|j| sqrt(eps)(i + j e_axis).
// Free axes continue the field by its face value; periodic axes wrap.
__global__ void k_fd16_q(Batch b, Fields f, int nx, int ny, int nz, double ihx2, double ihy2,
                         double ihz2, int perx, int pery, int perz, Fd16 c) {
  SLOT_PROLOGUE(b)
  (void)S;
  const double* sq = f.sq + off;
  double* q = f.q + off;
  const size_t n = (size_t)nx * ny * nz;
  GRID_STRIDE(idx, n) {
    const int i = (int)(idx % nx);
    const int j = (int)((idx / nx) % ny);
    const int k = (int)(idx / ((size_t)nx * ny));
    const double* rowx = sq + (idx - i);
    double ax = c.c[0] * rowx[i], ay = c.c[0] * sq[idx], az = c.c[0] * sq[idx];
#pragma unroll
    for (int m = 1; m <= 8; ++m) {
      int ip = i + m, im = i - m;
      if (perx) { ip %= nx; im = ((im % nx) + nx) % nx; }
      else { ip = ip >= nx ? nx - 1 : ip; im = im < 0 ? 0 : im; }
      ax += c.c[m] * (rowx[ip] + rowx[im]);
      int jp = j + m, jm = j - m;
      if (pery) { jp %= ny; jm = ((jm % ny) + ny) % ny; }
      else { jp = jp >= ny ? ny - 1 : jp; jm = jm < 0 ? 0 : jm; }
      const size_t bxz = (size_t)k * ny * nx + i;
      ay += c.c[m] * (sq[bxz + (size_t)jp * nx] + sq[bxz + (size_t)jm * nx]);
      int kp = k + m, km = k - m;
      if (perz) { kp %= nz; km = ((km % nz) + nz) % nz; }
      else { kp = kp >= nz ? nz - 1 : kp; km = km < 0 ? 0 : km; }
      const size_t bxy = (size_t)j * nx + i;
      az += c.c[m] * (sq[bxy + (size_t)kp * nx * ny] + sq[bxy + (size_t)km * nx * ny]);
    }
    q[idx] = sq[idx] * (ax * ihx2 + ay * ihy2 + az * ihz2);
  }
}

// Ion-exclusion function at element k of a slot: the caller's array when one
// was given (single-slot pools only, so k is also its index), else the cavity
// function (eps - 1)/(eps0 - 1).
__device__ __forceinline__ double gamma_at(const double* gam, size_t k, double eps_k, const IonParams& ip) {
  return gam ? gam[k] : (eps_k - 1.0) * ip.inv_eps0m1;
}

// Ionic charge gamma sum_i Z_i n_i[phi] and its derivative in phi (Eqs.
// rhoions, ionsconcPB; with ip.steric the Bikerman denominator of Eq.
// ionsconcMPB, 1 + sum_j a_j (e_j - 1), a_j = n_j^inf / n_j^max).  A
// species' exponential counts as constant where its cap is active.
__device__ __forceinline__ void ion_terms(double phi, double gamma, const IonParams& ip,
                                          double* rho_i, double* drho) {
  double a = 0.0, d = 0.0, den = 1.0, dden = 0.0;
  for (int s = 0; s < ip.nspecies; ++s) {
    const double u = -ip.zq[s] * phi * ip.inv_kt;
    const double capped = fmin(u, ip.exp_cap);
    const double e = exp(capped);
    a += ip.zn[s] * e;
    if (u < ip.exp_cap) d -= ip.z2n_kt[s] * e;
    if (ip.steric) {
      den += ip.a[s] * (e - 1.0);
      if (u < ip.exp_cap) dden -= ip.a[s] * ip.zq[s] * ip.inv_kt * e;
    }
  }
  if (ip.steric) {
    d = (d * den - a * dden) / (den * den);
    a /= den;
  }
  *rho_i = gamma * a;
  *drho = gamma * d;
}

// qlam = q (+ lambda0 gamma for linear PB); sums of lambda and rho.
// Nonlinear PB also starts Algorithm 4: phi = 0, rho_ions = rho_ions[0], r' = rho.
__global__ void k_setup_final(Batch b, Fields f, size_t n) {
  SLOT_PROLOGUE(b)
  const double* q = f.q + off;
  const double* eps = f.eps + off;
  const double* rho = f.rho + off;
  double* qlam = f.qlam + off;
  const int kind = S.kind;
  const IonParams ip = S.ion;
  double lam_acc = 0.0, rho_acc = 0.0;
  GRID_STRIDE(i, n) {
    double lam = 0.0;
    if (kind == GPS_LPB) lam = ip.lambda0 * gamma_at(f.gam, off + i, eps[i], ip);
    qlam[i] = q[i] + lam;
    lam_acc += lam;
    rho_acc += rho[i];
    if (kind == GPS_NLPB) {
      double a, d;
      ion_terms(0.0, gamma_at(f.gam, off + i, eps[i], ip), ip, &a, &d);
      f.phi[off + i] = 0.0;
      f.rions[off + i] = a;
      f.rp[off + i] = rho[i];
    }
  }
  grid_reduce(lam_acc, slot_partials(b, slot), &S.counter[CNT_AUX], &S.lam_sum);
  grid_reduce(rho_acc, slot_partials2(b, slot), &S.counter[CNT_AUX2], &S.aux[3]);
}

// Next phase after setup (one block per slot): periodic k = 0 value,
// background and gauge, or the INVALID status for a non-positive eps.
__global__ void k_setup_phase(Batch b, size_t n, double inv_p, int periodic) {
  SLOT_PROLOGUE(b)
  (void)off;
  if (threadIdx.x != 0) return;
  if (S.bad_eps) {
    S.status = GPS_ERR_INVALID;
    S.phase = PH_DONE;
    return;
  }
  S.use_k0 = 0;
  S.k0 = 0.0;
  S.background = 0.0;
  S.gauge = 0;
  if (periodic && S.kind != GPS_NLPB) {
    if (S.kind == GPS_LPB && S.lam_sum > 0) {
      S.use_k0 = 1;
      S.k0 = kFourPi * S.eps_sum / S.lam_sum * inv_p;
    } else {
      // singular operator (GPe, or linear PB without solvent): A 1 = 0 --
      // neutral source, iterates on the gauge subspace
      S.gauge = 1;
      S.background = S.aux[3] / (double)n;
    }
  }
  S.iters_total = 0;
  S.fp64_iters = 0;
  S.outer = 0;
  S.F0 = -1.0;
  S.F_prev = -1.0;
  S.eta_prev = 0.0;
  S.F = 0.0;
  S.cert = -1.0;
  S.phase = S.kind == GPS_NLPB ? PH_NLEVAL : PH_INIT;
}

// ---------------------------------------------------------------- PCG ------

// r_0 = -4 pi (source - background), x = p = A p = 0 (Algorithm 2, x_0 = 0);
// source/x are rho/phi, or the inner source/correction for nonlinear PB.
__global__ void k_init(Batch b, Fields f, size_t n) {
  SLOT_PROLOGUE(b)
  const bool nl = S.kind == GPS_NLPB;
  const double* src = (nl ? f.src : f.rho) + off;
  double* x = (nl ? f.dphi : f.phi) + off;
  double* r = f.r + off;
  double* p = f.p + off;
  double* Ap = f.Ap + off;
  const double bg = S.background;
  // warm start of Algorithm 2 (x_0 = phi_prev): the previous solve's b - r
  // stands in for A phi_prev, so r_0 = b - (b_prev - r_prev)
  const bool warm = S.warm && f.wphi && f.wd && !nl;
  const double* wphi = warm ? f.wphi + off : nullptr;
  const double* wd = warm ? f.wd + off : nullptr;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double ri = -kFourPi * (src[i] - bg) - (warm ? wd[i] : 0.0);
    r[i] = ri;
    x[i] = warm ? wphi[i] : 0.0;
    p[i] = 0.0;
    Ap[i] = 0.0;
    acc += ri * ri;
  }
  if (grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_RR], &S.rr0) && threadIdx.x == 0) {
    const double r0 = sqrt(S.rr0);
    const double tol = fmax(S.tol_abs, S.tol_rel * r0);
    S.tol2 = tol * tol;
    S.rr = S.rr0;
    S.iter = 0;
    S.status = GPS_OK;
    S.vr_prev = 1.0;
    S.restart = 0;
    S.vdone = 0;
    S.pdone = 0;
    S.spec = S.spec_hi;
    // nonlinear PB: an FP32 stall or breakdown returns one inner solve to the
    // high precision, not the later ones (each starts from its own residual)
    if (nl) S.mixed = S.mixed_req;
    if (S.mixed) {
      // FP32 spectrum once ||r|| <= mixed_switch ||r_ref||.  r_ref is r_0 of a
      // linear solve; for nonlinear PB it is the first outer step's residual
      // (4 pi F_0 in the units of r), so the inner solves of later outer
      // steps whose residual is already that small run in FP32 from the
      // start: the drift they add is bounded by the same eps_32 mixed_switch
      // ||r_ref|| per solve as for a linear solve.
      const double ref = nl ? kFourPi * kFourPi * S.F0 * S.F0 : S.rr0;
      S.rr_switch = S.mixed_switch * S.mixed_switch * ref;
      if (nl && S.rr0 <= S.rr_switch) {
        S.spec = SPEC_FP32;
        S.rr_min = S.rr0;
        S.stall = 0;
      }
    }
    if (S.rr0 <= S.tol2) after_pcg(S);
    else S.phase = PH_ITER;
  }
}

// p = v + beta p ; A p = -(q + lambda) v - 4 pi r [+ 4 pi <s r> sqrt(eps)] + beta A p ;
// partial (p, A p).  beta = (v,r)/(v,r)_prev, beta_0 = 0 (Algorithm 2).
// Periodic GPe (gauge): the operator is singular with A 1 = 0, so v is put
// back on the subspace sum sqrt(eps) v = 0 (v -= c s, c = <sqrt(eps) v>, with
// (v, r) corrected by -c (s, r)), and A p on the range of A (its grid mean m
// is removed: alpha uses (p, A p) - m sum p and the r update uses A p - m).
// Both are identities in exact arithmetic that remove the rounding of the
// spectrum passes, which would otherwise leave r a component along the
// constants that no iteration can reduce.  A breakdown while the FP32
// spectrum is in use falls back to the FP64-accurate spectrum and restarts
// the directions (beta = 0) instead of stopping.
__global__ void k_update_p(Batch b, Fields f, size_t n, double inv_n, int periodic) {
  SLOT_PROLOGUE(b)
  if (!S.vdone) return;   // this iteration's preconditioner did not run for the slot
  const double* __restrict__ v = f.v + off;
  const double* __restrict__ r = f.r + off;
  const double* __restrict__ qlam = f.qlam + off;
  const double* __restrict__ sqe = f.sq + off;
  const double* __restrict__ s = f.s + off;
  double* __restrict__ p = f.p + off;
  double* __restrict__ Ap = f.Ap + off;
  const bool project = S.gauge != 0;
  const double c = project ? S.wsum * inv_n : 0.0;
  const double vr = project ? S.vr - c * S.mu_sum : S.vr;
  const double beta = (S.iter == 0 || S.restart) ? 0.0 : vr / S.vr_prev;
  const double mu4pi = periodic ? kFourPi * S.mu_sum * inv_n : 0.0;
  double acc = 0.0, ap_acc = 0.0, p_acc = 0.0;
  if (project) {
#pragma unroll 2
    GRID_STRIDE(i, n) {
      const double vi = v[i] - c * s[i];
      const double av = -qlam[i] * vi - kFourPi * r[i] + mu4pi * sqe[i];
      const double pi_ = vi + beta * p[i];
      const double api = av + beta * Ap[i];
      p[i] = pi_;
      Ap[i] = api;
      acc += pi_ * api;
      ap_acc += api;
      p_acc += pi_;
    }
  } else if (periodic) {
#pragma unroll 2
    GRID_STRIDE(i, n) {
      const double vi = v[i];
      const double av = -qlam[i] * vi - kFourPi * r[i] + mu4pi * sqe[i];
      const double pi_ = vi + beta * p[i];
      const double api = av + beta * Ap[i];
      p[i] = pi_;
      Ap[i] = api;
      acc += pi_ * api;
    }
  } else {
    // free, surface and wire BC: five FP64 operations per point (the FP64
    // pipe, not HBM, is the tighter bound of this kernel on GB300)
#pragma unroll 2
    GRID_STRIDE(i, n) {
      const double vi = v[i];
      const double av = -qlam[i] * vi - kFourPi * r[i];
      const double pi_ = vi + beta * p[i];
      const double api = av + beta * Ap[i];
      p[i] = pi_;
      Ap[i] = api;
      acc += pi_ * api;
    }
  }
  bool last;
  if (project)
    last = grid_reduce3(acc, ap_acc, p_acc, slot_partials(b, slot), slot_partials2(b, slot),
                        slot_partials3(b, slot), &S.counter[CNT_PAP], &S.pAp, &S.ap_sum, &S.p_sum);
  else
    last = grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_PAP], &S.pAp);
  if (last && threadIdx.x == 0) {
    double pap = S.pAp;
    S.ap_mean = 0.0;
    if (project) {
      S.ap_mean = S.ap_sum * inv_n;
      pap -= S.ap_mean * S.p_sum;
      S.pAp = pap;
    }
    S.beta = beta;
    S.vr = vr;
    S.vr_prev = vr;
    S.restart = 0;
    S.vdone = 0;
    S.pdone = 1;
    if (!(pap < 0.0) || !isfinite(pap) || !isfinite(vr)) {
      S.alpha = 0.0;
      if (S.spec == SPEC_FP32) {   // FP32 noise floor reached: continue in FP64 accuracy
        S.spec = S.spec_hi;
        S.mixed = 0;
        S.restart = 1;
      } else {
        S.status = GPS_ERR_BREAKDOWN;
      }
    } else {
      S.alpha = vr / pap;
    }
  }
}

// x += alpha p ; r -= alpha A p ; partial ||r||^2 ; convergence test.
__global__ void k_update_r(Batch b, Fields f, size_t n) {
  SLOT_PROLOGUE(b)
  if (!S.pdone) return;   // update_p did not run for the slot in this iteration
  const bool nl = S.kind == GPS_NLPB;
  double* __restrict__ x = (nl ? f.dphi : f.phi) + off;
  double* __restrict__ r = f.r + off;
  const double* __restrict__ p = f.p + off;
  double* __restrict__ Ap = f.Ap + off;
  const double alpha = S.alpha;
  const double m = S.gauge ? S.ap_mean : 0.0;
  double acc = 0.0;
  if (m != 0.0) {
#pragma unroll 2
    GRID_STRIDE(i, n) {
      x[i] += alpha * p[i];
      const double api = Ap[i] - m;
      Ap[i] = api;   // keep the projected A p for the recurrence
      const double ri = r[i] - alpha * api;
      r[i] = ri;
      acc += ri * ri;
    }
  } else {
#pragma unroll 2
    GRID_STRIDE(i, n) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * Ap[i];
      r[i] = ri;
      acc += ri * ri;
    }
  }
  if (grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_RR], &S.rr) && threadIdx.x == 0) {
    S.pdone = 0;
    S.iter += 1;
    S.iters_total += 1;
    if (S.spec != SPEC_FP32) S.fp64_iters += 1;
    if (S.status == GPS_ERR_BREAKDOWN || !isfinite(S.rr)) {
      S.status = GPS_ERR_BREAKDOWN;
      after_pcg(S);
    } else if (S.rr <= S.tol2) {
      after_pcg(S);
    } else if (S.iter >= S.max_iter) {
      S.status = GPS_ERR_NOT_CONVERGED;
      after_pcg(S);
    } else if (S.mixed && S.spec != SPEC_FP32 && S.rr <= S.rr_switch) {
      S.spec = SPEC_FP32;
      S.rr_min = S.rr;
      S.stall = 0;
    } else if (S.spec == SPEC_FP32) {
      // The FP32 spectrum has a noise floor: once the residual stops reaching
      // new minima, continue in FP64 with restarted directions.
      if (S.rr < S.rr_min) {
        S.rr_min = S.rr;
        S.stall = 0;
      } else if (++S.stall >= 8) {
        S.spec = S.spec_hi;
        S.mixed = 0;
        S.restart = 1;
      }
    }
  }
}

// ------------------------------------------------------------------ ions ---

// Outer step of Algorithm 4: fresh = rho_ions[phi]; lambda (Newton: the
// linear PB term at phi, else 0); source = r' + mix - rho_ions, qlam = q +
// lambda; outer residual ||fresh - rho_ions + r'||.
__global__ void k_nl_eval(Batch b, Fields f, size_t n, double inv_p, int periodic) {
  SLOT_PROLOGUE(b)
  const IonParams ip = S.ion;
  const double eta = S.newton ? 1.0 : S.eta;
  double acc = 0.0, lam_acc = 0.0, src_acc = 0.0;
  GRID_STRIDE(i, n) {
    const size_t k = off + i;
    double a, d;
    ion_terms(f.phi[k], gamma_at(f.gam, k, f.eps[k], ip), ip, &a, &d);
    const double lam = S.newton ? -kFourPi * d : 0.0;
    const double ri = f.rions[k], rp = f.rp[k];
    f.fresh[k] = a;
    f.lam[k] = lam;
    const double mix = eta * a + (1.0 - eta) * ri;
    const double src = rp + mix - ri;
    f.src[k] = src;
    f.qlam[k] = f.q[k] + lam;
    const double fr = a - ri + rp;
    acc += fr * fr;
    lam_acc += lam;
    src_acc += src;
  }
  grid_reduce(lam_acc, slot_partials2(b, slot), &S.counter[CNT_AUX2], &S.lam_sum);
  grid_reduce(src_acc, slot_partials3(b, slot), &S.counter[CNT_PSUM], &S.aux[4]);
  if (grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_AUX], &S.aux[0]) && threadIdx.x == 0) {
    const double F = sqrt(S.aux[0]);
    S.F = F;
    if (S.F0 < 0) S.F0 = F;
    if (!isfinite(F)) {
      S.status = GPS_ERR_BREAKDOWN;
      S.phase = PH_DONE;
    } else if (F <= S.tol_outer) {
      S.status = GPS_OK;
      S.background = 0.0;
      S.phase = S.certify ? PH_CERT : PH_DONE;
    } else if (S.outer >= S.max_outer) {
      S.status = GPS_ERR_NOT_CONVERGED;
      S.phase = PH_DONE;
    } else {
      if (S.newton) {
        S.tol_abs = 0.1 * kFourPi * S.tol_outer;
        double eta = fmin(S.forcing, F / S.F0);
        if (S.forcing_ew) {
          // Eisenstat-Walker choice 2 (gamma 0.9, exponent 2) with its safeguard
          eta = S.forcing;
          if (S.F_prev > 0.0) {
            const double q = F / S.F_prev;
            eta = 0.9 * q * q;
            const double sg = 0.9 * S.eta_prev * S.eta_prev;
            if (sg > 0.1) eta = fmax(eta, sg);
            eta = fmin(eta, S.forcing);
          }
        }
        S.tol_rel = eta;
        S.F_prev = F;
        S.eta_prev = eta;
      } else if (S.outer < 2) {
        S.tol_abs = 0.0;
        S.tol_rel = 1e-4;
      } else {
        S.tol_abs = kFourPi * S.tol_outer;
        S.tol_rel = 0.0;
      }
      S.use_k0 = 0;
      S.k0 = 0.0;
      S.gauge = 0;
      S.background = 0.0;
      if (periodic && S.lam_sum > 0) {
        S.use_k0 = 1;
        S.k0 = kFourPi * S.eps_sum / S.lam_sum * inv_p;
      } else if (periodic) {
        // no screening this step: singular inner operator, neutral source
        S.gauge = 1;
        S.background = S.aux[4] / (double)n;
      }
      S.phase = PH_INIT;
    }
  }
}

// Trial (commit == 0) or accepted (commit == 1) step t of the outer loop:
//   phi_t = phi + t dphi ; rions_t = rions + t (mix - rions - lam dphi / 4pi) ;
//   rp_t = (1-t) rp + t (-r / 4pi) ; F_t = ||rho_ions[phi_t] - rions_t + rp_t||.
__global__ void k_nl_step(Batch b, Fields f, size_t n, int commit) {
  SLOT_PROLOGUE(b)
  const IonParams ip = S.ion;
  const double eta = S.newton ? 1.0 : S.eta;
  const double t = S.t;
  const double inv4pi = 1.0 / kFourPi;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const size_t k = off + i;
    const double ri = f.rions[k];
    const double mix = eta * f.fresh[k] + (1.0 - eta) * ri;
    const double dph = f.dphi[k];
    const double ph = f.phi[k] + t * dph;
    const double rit = ri + t * (mix - ri - f.lam[k] * dph * inv4pi);
    const double rpt = (1.0 - t) * f.rp[k] + t * (-f.r[k] * inv4pi);
    if (commit) {
      f.phi[k] = ph;
      f.rions[k] = rit;
      f.rp[k] = rpt;
    } else {
      double a, d;
      ion_terms(ph, gamma_at(f.gam, k, f.eps[k], ip), ip, &a, &d);
      const double fr = a - rit + rpt;
      acc += fr * fr;
    }
  }
  if (grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_AUX3], &S.aux[2]) && threadIdx.x == 0) {
    if (commit) {
      S.outer += 1;
      S.phase = PH_NLEVAL;
    } else if (sqrt(S.aux[2]) < S.F || S.t < 1e-4) {
      S.phase = PH_COMMIT;
    } else {
      S.t *= 0.5;
    }
  }
}

__global__ void k_ionic_charge(const double* __restrict__ phi, const double* __restrict__ eps,
                               const double* __restrict__ gam, double* __restrict__ out, size_t n,
                               IonParams ip) {
  GRID_STRIDE(i, n) {
    double a, d;
    ion_terms(phi[i], gamma_at(gam, i, eps[i], ip), ip, &a, &d);
    out[i] = a;
  }
}

// ----------------------------------------------------------- certificate --

// tmp = rho - bg [+ rho_ions[phi]] - qop phi / 4 pi, qop = q (NLPB) or
// q + lambda ; partial of sqrt(eps) phi.
__global__ void k_fp_source(Batch b, Fields f, size_t n) {
  SLOT_PROLOGUE(b)
  const bool nl = S.kind == GPS_NLPB;
  const IonParams ip = S.ion;
  const double bg = S.background;
  const double inv4pi = 1.0 / kFourPi;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const size_t k = off + i;
    const double ph = f.phi[k];
    double src = f.rho[k] - bg - (nl ? f.q[k] : f.qlam[k]) * ph * inv4pi;
    if (nl) {
      double a, d;
      ion_terms(ph, gamma_at(f.gam, k, f.eps[k], ip), ip, &a, &d);
      src += a;
    }
    f.tmp[k] = src;
    acc += f.sq[k] * ph;
  }
  grid_reduce(acc, slot_partials(b, slot), &S.counter[CNT_AUX], &S.aux[5]);
}

// g = w + c s - phi (w = M tmp, written into f.Ap) ; ||g|| / ||phi|| -> cert ; DONE.
__global__ void k_fp_residual(Batch b, Fields f, size_t n, int periodic) {
  SLOT_PROLOGUE(b)
  const double c = periodic ? S.aux[5] / (double)n : 0.0;
  double a = 0.0, q2 = 0.0;
  GRID_STRIDE(i, n) {
    const size_t k = off + i;
    const double g = f.Ap[k] + c * f.s[k] - f.phi[k];
    a += g * g;
    q2 += f.phi[k] * f.phi[k];
  }
  grid_reduce(q2, slot_partials2(b, slot), &S.counter[CNT_AUX2], &S.aux[7]);
  if (grid_reduce(a, slot_partials(b, slot), &S.counter[CNT_AUX], &S.aux[6]) && threadIdx.x == 0) {
    const double nphi = sqrt(S.aux[7]);
    S.cert = nphi > 0 ? sqrt(S.aux[6]) / nphi : sqrt(S.aux[6]);
    S.phase = PH_DONE;
  }
}

// ----------------------------------------------------------------- tables --

// Periodic: kernel 4 pi / k^2 / N and Laplacian -k^2 / N on the octant
// [Pz/2+1][Py/2+1][Hx], k = 0 -> 0.
__global__ void k_table_periodic(double* __restrict__ kern, double* __restrict__ lap, int Hx,
                                 int hy, int hz, double dkx, double dky, double dkz, double inv_n) {
  const size_t n = (size_t)Hx * hy * hz;
  GRID_STRIDE(idx, n) {
    const int i = (int)(idx % Hx);
    const int j = (int)((idx / Hx) % hy);
    const int k = (int)(idx / ((size_t)Hx * hy));
    const double kx = i * dkx, ky = j * dky, kz = k * dkz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    kern[idx] = idx == 0 ? 0.0 : kFourPi / k2 * inv_n;
    if (lap) lap[idx] = -k2 * inv_n;   // spectral Laplacian (periodic q); optional
  }
}

// Surface: 4 pi (1 - (-1)^j exp(-k L)) / (k^2 + kz_j^2) / N, 2 pi L^2 / N at 0.
__global__ void k_table_surface(double* __restrict__ kern, int Hx, int hy, int hz, double dkx,
                                double dky, double dkz, double Lz, double inv_n) {
  const size_t n = (size_t)Hx * hy * hz;
  GRID_STRIDE(idx, n) {
    const int i = (int)(idx % Hx);
    const int j = (int)((idx / Hx) % hy);
    const int k = (int)(idx / ((size_t)Hx * hy));
    const double kx = i * dkx, ky = j * dky, kz = k * dkz;
    const double kp = sqrt(kx * kx + ky * ky);
    double v;
    if (idx == 0) {
      v = 2.0 * kPi * Lz * Lz;
    } else {
      const double sgn = (k & 1) ? -1.0 : 1.0;
      v = kFourPi * (1.0 - sgn * exp(-kp * Lz)) / (kp * kp + kz * kz);
    }
    kern[idx] = v * inv_n;
  }
}

// Free, step 1: truncated-Coulomb transform 8 pi sin^2(R k/2)/k^2 (2 pi R^2 at
// k = 0) on the octant of the 4x oversampled frequency grid.
__global__ void k_free_ghat(double* __restrict__ out, int mx, int my, int mz, double dkx, double dky,
                            double dkz, double R) {
  const size_t n = (size_t)mx * my * mz;
  GRID_STRIDE(idx, n) {
    const int i = (int)(idx % mx);
    const int j = (int)((idx / mx) % my);
    const int k = (int)(idx / ((size_t)mx * my));
    const double kx = i * dkx, ky = j * dky, kz = k * dkz;
    const double kk = sqrt(kx * kx + ky * ky + kz * kz);
    double v;
    if (idx == 0) {
      v = 2.0 * kPi * R * R;
    } else {
      const double sn = sin(0.5 * R * kk);
      v = 8.0 * kPi * sn * sn / (kk * kk);
    }
    out[idx] = v;
  }
}

// Wire-BC transform of the transversely truncated Green's function on the
// oversampled (kx, ky) quadrant for every |kz| index jz (cylindrical
// truncation at R): kz != 0, 4 pi / (k^2 + kz^2) [1 + kR J1(kR) K0(kz R) -
// kz R J0(kR) K1(kz R)] with K0(kz R), K1(kz R) given per jz; kz = 0 (gauge
// 2 ln(R / rho)), 4 pi (1 - J0(kR)) / k^2, pi R^2 at k = 0.
__global__ void k_wire_ghat(double* __restrict__ out, int mx, int my, int mz, double dkx, double dky,
                            double dkz, double R, const double* __restrict__ k0R,
                            const double* __restrict__ k1R) {
  const size_t n = (size_t)mx * my * mz;
  GRID_STRIDE(idx, n) {
    const int i = (int)(idx % mx);
    const int j = (int)((idx / mx) % my);
    const int k = (int)(idx / ((size_t)mx * my));
    const double kx = i * dkx, ky = j * dky, kz = k * dkz;
    const double kp2 = kx * kx + ky * ky, x = sqrt(kp2) * R;
    double v;
    if (k == 0) {
      v = (i == 0 && j == 0) ? kPi * R * R : 4.0 * kPi * (1.0 - j0(x)) / kp2;
    } else {
      const double a = kz * R;
      v = 4.0 * kPi / (kp2 + kz * kz) * (1.0 + x * j1(x) * k0R[k] - a * j0(x) * k1R[k]);
    }
    out[idx] = v;
  }
}

// Dense transform along the middle index of in[A][J][B] -> out[A][K][B]:
// out[a][k][b] = sum_j C[k][j] in[a][j][b].  Used for the even (cosine)
// transforms of the free-BC table.
__global__ void k_axis_matrix(const double* __restrict__ in, double* __restrict__ out,
                              const double* __restrict__ C, int A, int J, int B, int K) {
  const size_t n = (size_t)A * K * B;
  GRID_STRIDE(idx, n) {
    const int b = (int)(idx % B);
    const int k = (int)((idx / B) % K);
    const int a = (int)(idx / ((size_t)B * K));
    const double* src = in + (size_t)a * J * B + b;
    const double* crow = C + (size_t)k * J;
    double acc = 0.0;
    for (int j = 0; j < J; ++j) acc = fma(crow[j], src[(size_t)j * B], acc);
    out[idx] = acc;
  }
}

// ------------------------------------------------------------- launchers --

#define VEC_GRID(n, nslots) dim3(vec_blocks(n, nslots), 1, nslots), kT, 0, st

void launch_setup_s(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st) {
  count_launch();
  k_setup_s<<<VEC_GRID(n, nslots)>>>(b, f, n);
}

void launch_fd16_q(const Batch& b, const Fields& f, int nx, int ny, int nz, double hx, double hy,
                   double hz, int perx, int pery, int perz, const Fd16& c, int nslots,
                   cudaStream_t st) {
  const size_t n = (size_t)nx * ny * nz;
  count_launch();
  k_fd16_q<<<VEC_GRID(n, nslots)>>>(b, f, nx, ny, nz, 1.0 / (hx * hx), 1.0 / (hy * hy),
                                     1.0 / (hz * hz), perx, pery, perz, c);
}

void launch_setup_final(const Batch& b, const Fields& f, size_t n, double inv_p, int periodic,
                        int nslots, cudaStream_t st) {
  count_launch();
  k_setup_final<<<VEC_GRID(n, nslots)>>>(b, f, n);
  count_launch();
  k_setup_phase<<<dim3(1, 1, nslots), 32, 0, st>>>(b, n, inv_p, periodic);
}

void launch_init(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st) {
  count_launch();
  k_init<<<VEC_GRID(n, nslots)>>>(b, f, n);
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  GRID_STRIDE(i, n) out[i] = d2f_rn(in[i]);
}

void launch_to_float(const double* in, float* out, size_t n, cudaStream_t st) {
  count_launch();
  k_to_float<<<grid_blocks(n, kT), kT, 0, st>>>(in, out, n);
}

void launch_update_p(const Batch& b, const Fields& f, size_t n, int periodic, int nslots,
                     cudaStream_t st) {
  count_launch();
  k_update_p<<<VEC_GRID(n, nslots)>>>(b, f, n, 1.0 / (double)n, periodic);
}

void launch_update_r(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st) {
  count_launch();
  k_update_r<<<VEC_GRID(n, nslots)>>>(b, f, n);
}

void launch_nl_eval(const Batch& b, const Fields& f, size_t n, double inv_p, int periodic,
                    int nslots, cudaStream_t st) {
  count_launch();
  k_nl_eval<<<VEC_GRID(n, nslots)>>>(b, f, n, inv_p, periodic);
}

void launch_nl_step(const Batch& b, const Fields& f, size_t n, int commit, int nslots,
                    cudaStream_t st) {
  count_launch();
  k_nl_step<<<VEC_GRID(n, nslots)>>>(b, f, n, commit);
}

void launch_fp_source(const Batch& b, const Fields& f, size_t n, int nslots, cudaStream_t st) {
  count_launch();
  k_fp_source<<<VEC_GRID(n, nslots)>>>(b, f, n);
}

void launch_fp_residual(const Batch& b, const Fields& f, size_t n, int periodic, int nslots,
                        cudaStream_t st) {
  count_launch();
  k_fp_residual<<<VEC_GRID(n, nslots)>>>(b, f, n, periodic);
}

// flag = 1 if a and b differ anywhere (the same-eps test of a warm start).
__global__ void k_eps_differ(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                             int* flag) {
  int d = 0;
  GRID_STRIDE(i, n) d |= a[i] != b[i];
  if (__syncthreads_or(d) && threadIdx.x == 0) *flag = 1;
}

void launch_eps_differ(const double* a, const double* b, size_t n, int* flag, cudaStream_t st) {
  count_launch();
  k_eps_differ<<<grid_blocks(n, kT), kT, 0, st>>>(a, b, n, flag);
}

// State kept for the next warm start, from slot `slot`: eps, phi and b - r
// with b = -4 pi (rho - background).
__global__ void k_warm_store(Batch b, Fields f, int slot, double* __restrict__ weps,
                             double* __restrict__ wphi, double* __restrict__ wd, size_t n) {
  const SlotState& S = b.st[slot];
  const double bg = S.background;
  const size_t off = (size_t)slot * b.vstride;
  GRID_STRIDE(i, n) {
    weps[i] = f.eps[off + i];
    wphi[i] = f.phi[off + i];
    wd[i] = -kFourPi * (f.rho[off + i] - bg) - f.r[off + i];
  }
}

void launch_warm_store(const Batch& b, const Fields& f, int slot, double* weps, double* wphi, double* wd,
                       size_t n, cudaStream_t st) {
  count_launch();
  k_warm_store<<<grid_blocks(n, kT), kT, 0, st>>>(b, f, slot, weps, wphi, wd, n);
}

// Float and double-float copies of a Green's table, made once per shape.
__global__ void k_table_split(const double* __restrict__ t, float* __restrict__ t32,
                              float2* __restrict__ tdf, size_t n) {
  GRID_STRIDE(i, n) {
    const double v = t[i];
    const float hi = (float)v;
    t32[i] = hi;
    tdf[i] = make_float2(hi, (float)(v - (double)hi));
  }
}

void launch_table_split(const double* t, float* t32, float2* tdf, size_t n, cudaStream_t st) {
  count_launch();
  k_table_split<<<grid_blocks(n, kT), kT, 0, st>>>(t, t32, tdf, n);
}

void launch_ionic_charge(const double* phi, const double* eps, const double* gam, double* out, size_t n,
                         const IonParams& ip, cudaStream_t st) {
  count_launch();
  k_ionic_charge<<<grid_blocks(n, kT), kT, 0, st>>>(phi, eps, gam, out, n, ip);
}

void launch_table_periodic(double* kern, double* lap, int Hx, int hy, int hz, double dkx, double dky,
                           double dkz, double inv_n, cudaStream_t st) {
  const size_t n = (size_t)Hx * hy * hz;
  count_launch();
  k_table_periodic<<<grid_blocks(n, kT), kT, 0, st>>>(kern, lap, Hx, hy, hz, dkx, dky, dkz, inv_n);
}

void launch_table_surface(double* kern, int Hx, int hy, int hz, double dkx, double dky, double dkz,
                          double Lz, double inv_n, cudaStream_t st) {
  const size_t n = (size_t)Hx * hy * hz;
  count_launch();
  k_table_surface<<<grid_blocks(n, kT), kT, 0, st>>>(kern, Hx, hy, hz, dkx, dky, dkz, Lz, inv_n);
}

void launch_free_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz,
                      double R, cudaStream_t st) {
  const size_t n = (size_t)mx * my * mz;
  count_launch();
  k_free_ghat<<<grid_blocks(n, kT), kT, 0, st>>>(out, mx, my, mz, dkx, dky, dkz, R);
}

void launch_wire_ghat(double* out, int mx, int my, int mz, double dkx, double dky, double dkz, double R,
                      const double* k0R, const double* k1R, cudaStream_t st) {
  const size_t n = (size_t)mx * my * mz;
  count_launch();
  k_wire_ghat<<<grid_blocks(n, kT), kT, 0, st>>>(out, mx, my, mz, dkx, dky, dkz, R, k0R, k1R);
}

void launch_axis_matrix(const double* in, double* out, const double* C, int A, int J, int B, int K,
                        cudaStream_t st) {
  const size_t n = (size_t)A * K * B;
  count_launch();
  k_axis_matrix<<<grid_blocks(n, kT), kT, 0, st>>>(in, out, C, A, J, B, K);
}

}  // namespace gps
