// Pointwise, stencil, reduction and table kernels of the PCG solver.
//
//   setup        s = eps^-1/2, sqrt(eps); q = sqrt(eps) lap sqrt(eps) by the
//                order-16 central stencil (Sec. "Numerical results")
//   PCG updates  Algorithm 2 with the operator identity of Eq. (corr)/(corrPB)
//   ions         Eqs. (rhoions, ionsconcPB) and the outer step of Algorithm 4
//   tables       vacuum Green's-function tables for the three BCs
//
// Every reduction is deterministic (fixed-order per-block partials combined by
// the last block), so repeated solves are bitwise identical.
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
  const size_t cap = 152 * 8;   // SMs x resident blocks of 256 threads
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

#define GRID_STRIDE(i, n) \
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ setup --

__global__ void k_setup_s(const double* __restrict__ eps, double* __restrict__ s,
                          double* __restrict__ sq, size_t n, PcgScalars* sc) {
  GRID_STRIDE(i, n) {
    const double e = eps[i];
    if (!(e > 0.0)) sc->bad_eps = 1;
    const double r = sqrt(e);
    sq[i] = r;
    s[i] = 1.0 / r;
  }
}

// q = sqrt(eps) * sum_axes (1/h^2) sum_j c_|j| sqrt(eps)(i + j e_axis).
// Free axes continue the field by its face value; periodic axes wrap.
__global__ void k_fd16_q(const double* __restrict__ sq, double* __restrict__ q, int nx, int ny,
                         int nz, double ihx2, double ihy2, double ihz2, int perx, int pery,
                         int perz, Fd16 c) {
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

// qlam = q + lambda0 * gamma, gamma = (eps - 1)/(eps0 - 1); partial sums of
// eps and lambda for the periodic k = 0 kernel value.
__global__ void k_qlam_linear(const double* __restrict__ q, const double* __restrict__ eps,
                              double* __restrict__ qlam, size_t n, double lambda0, double inv_e0m1,
                              double* partials, PcgScalars* sc) {
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double lam = lambda0 * (eps[i] - 1.0) * inv_e0m1;
    qlam[i] = q[i] + lam;
    acc += lam;
  }
  grid_reduce(acc, partials, &sc->counter[CNT_AUX], &sc->aux[1]);
}

__global__ void k_sum(const double* __restrict__ a, size_t n, double* partials, unsigned int* counter,
                      double* out) {
  double acc = 0.0;
  GRID_STRIDE(i, n) acc += a[i];
  grid_reduce(acc, partials, counter, out);
}

__global__ void k_copy_scaled(const double* __restrict__ a, double* __restrict__ b, size_t n,
                              double f) {
  GRID_STRIDE(i, n) b[i] = f * a[i];
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ c, size_t n) {
  GRID_STRIDE(i, n) c[i] = a[i] * b[i];
}

// ---------------------------------------------------------------- PCG ------

// r_0 = -4 pi (rho - background), phi = p = A p = 0 (Algorithm 2, phi_0 = 0).
__global__ void k_init(const double* __restrict__ rho, double* __restrict__ r,
                       double* __restrict__ phi, double* __restrict__ p, double* __restrict__ Ap,
                       size_t n, double tol_abs, double tol_rel, int max_iter, double* partials,
                       PcgScalars* sc, int zero_phi, const double* bg_sum) {
  const double bg = bg_sum ? *bg_sum / (double)n : 0.0;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double ri = -kFourPi * (rho[i] - bg);
    r[i] = ri;
    if (zero_phi) phi[i] = 0.0;
    p[i] = 0.0;
    Ap[i] = 0.0;
    acc += ri * ri;
  }
  if (grid_reduce(acc, partials, &sc->counter[CNT_RR], &sc->rr0) && threadIdx.x == 0) {
    const double r0 = sqrt(sc->rr0);
    const double tol = fmax(tol_abs, tol_rel * r0);
    sc->tol2 = tol * tol;
    sc->rr = sc->rr0;
    sc->iter = 0;
    sc->max_iter = max_iter;
    sc->status = 0;
    sc->done = (sc->rr0 <= sc->tol2) ? 1 : 0;
    sc->vr_prev = 1.0;
    sc->background = bg;
  }
}

// p = v + beta p ; A p = -(q + lambda) v - 4 pi r [+ 4 pi <s r> sqrt(eps)] + beta A p ;
// partial (p, A p).  beta = (v,r)/(v,r)_prev, beta_0 = 0 (Algorithm 2).
// Periodic GPe (project != 0): v is first put back on the gauge subspace
// sum sqrt(eps) v = 0 by v -= c s, c = <sqrt(eps) v>, and (v, r) is corrected
// by -c (s, r); in exact arithmetic c = 0 (the vacuum solve drops k = 0), the
// projection only removes the rounding of the spectrum passes.
__global__ void k_update_p(const double* __restrict__ v, const double* __restrict__ r,
                           const double* __restrict__ qlam, const double* __restrict__ sqrt_eps,
                           const double* __restrict__ s, double* __restrict__ p,
                           double* __restrict__ Ap, size_t n, double inv_n, int periodic,
                           int project, double* partials, PcgScalars* sc) {
  if (sc->done) return;
  const double c = project ? sc->wsum * inv_n : 0.0;
  const double vr = project ? sc->vr - c * sc->mu_sum : sc->vr;
  const double beta = sc->iter == 0 ? 0.0 : vr / sc->vr_prev;
  const double mu4pi = periodic ? kFourPi * sc->mu_sum * inv_n : 0.0;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double vi = project ? v[i] - c * s[i] : v[i];
    double av = -qlam[i] * vi - kFourPi * r[i];
    if (periodic) av += mu4pi * sqrt_eps[i];
    const double pi_ = vi + beta * p[i];
    const double api = av + beta * Ap[i];
    p[i] = pi_;
    Ap[i] = api;
    acc += pi_ * api;
  }
  if (grid_reduce(acc, partials, &sc->counter[CNT_PAP], &sc->pAp) && threadIdx.x == 0) {
    const double pap = sc->pAp;
    sc->beta = beta;
    sc->vr = vr;
    sc->vr_prev = vr;
    if (!(pap < 0.0) || !isfinite(pap) || !isfinite(vr)) {
      sc->status = GPS_ERR_BREAKDOWN;
      sc->done = 1;
      sc->alpha = 0.0;
    } else {
      sc->alpha = vr / pap;
    }
  }
}

// phi += alpha p ; r -= alpha A p ; partial ||r||^2 ; convergence test.
__global__ void k_update_r(double* __restrict__ phi, double* __restrict__ r,
                           const double* __restrict__ p, const double* __restrict__ Ap, size_t n,
                           double* partials, PcgScalars* sc) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    phi[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    acc += ri * ri;
  }
  if (grid_reduce(acc, partials, &sc->counter[CNT_RR], &sc->rr) && threadIdx.x == 0) {
    sc->iter += 1;
    if (!isfinite(sc->rr)) {
      sc->status = GPS_ERR_BREAKDOWN;
      sc->done = 1;
    } else if (sc->rr <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = GPS_ERR_NOT_CONVERGED;
      sc->done = 1;
    }
  }
}

// ----------------------------------------------------------- certificate --

// out = rho - bg [+ rions] - qlam phi / 4 pi ; partial of sqrt(eps) phi.
__global__ void k_fp_source(const double* __restrict__ rho, const double* __restrict__ rions,
                            const double* __restrict__ qlam, const double* __restrict__ phi,
                            const double* __restrict__ sq, double* __restrict__ out, size_t n,
                            double bg, double* partials, PcgScalars* sc) {
  double acc = 0.0;
  const double inv4pi = 1.0 / kFourPi;
  GRID_STRIDE(i, n) {
    double src = rho[i] - bg - qlam[i] * phi[i] * inv4pi;
    if (rions) src += rions[i];
    out[i] = src;
    acc += sq[i] * phi[i];
  }
  grid_reduce(acc, partials, &sc->counter[CNT_AUX], &sc->aux[5]);
}

// g = w + c s - phi ; partials of ||g||^2 (aux[6]) and ||phi||^2 (aux[7]).
__global__ void k_fp_residual(const double* __restrict__ w, const double* __restrict__ s,
                              const double* __restrict__ phi, size_t n, double c, double* partials,
                              double* partials2, PcgScalars* sc) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(i, n) {
    const double g = w[i] + c * s[i] - phi[i];
    a += g * g;
    b += phi[i] * phi[i];
  }
  grid_reduce(a, partials, &sc->counter[CNT_AUX], &sc->aux[6]);
  grid_reduce(b, partials2, &sc->counter[CNT_AUX2], &sc->aux[7]);
}

// ------------------------------------------------------------------ ions ---

__device__ __forceinline__ void ion_terms(double phi, double gamma, const IonParams& ip,
                                          double* rho_i, double* drho) {
  double a = 0.0, d = 0.0;
  for (int s = 0; s < ip.nspecies; ++s) {
    const double u = -ip.zq[s] * phi * ip.inv_kt;
    const double capped = fmin(u, ip.exp_cap);
    const double e = exp(capped);
    a += ip.zn[s] * e;
    if (u < ip.exp_cap) d -= ip.z2n_kt[s] * e;
  }
  *rho_i = gamma * a;
  *drho = gamma * d;
}

__global__ void k_ionic_charge(const double* __restrict__ phi, const double* __restrict__ eps,
                               double* __restrict__ out, size_t n, IonParams ip) {
  GRID_STRIDE(i, n) {
    double a, d;
    ion_terms(phi[i], (eps[i] - 1.0) * ip.inv_eps0m1, ip, &a, &d);
    out[i] = a;
  }
}

// fresh = rho_ions[phi]; lam = -4 pi d rho_ions/d phi (newton) ; partial of
// ||fresh - rions + rp||^2 (the outer residual).
__global__ void k_nl_eval(const double* __restrict__ phi, const double* __restrict__ eps,
                          const double* __restrict__ rions, const double* __restrict__ rp,
                          double* __restrict__ fresh, double* __restrict__ lam, size_t n,
                          IonParams ip, int newton, double* partials, PcgScalars* sc) {
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    double a, d;
    ion_terms(phi[i], (eps[i] - 1.0) * ip.inv_eps0m1, ip, &a, &d);
    fresh[i] = a;
    lam[i] = newton ? -kFourPi * d : 0.0;
    const double f = a - rions[i] + rp[i];
    acc += f * f;
  }
  grid_reduce(acc, partials, &sc->counter[CNT_AUX], &sc->aux[0]);
}

// Inner-solve inputs of one outer step: source charge and operator term.
//   mix = eta fresh + (1-eta) rions ; src = rp + mix - rions ; qlam = q + lam.
// Partial sums of lam (periodic k = 0 value).
__global__ void k_nl_source(const double* __restrict__ fresh, const double* __restrict__ rions,
                            const double* __restrict__ rp, const double* __restrict__ q,
                            const double* __restrict__ lam, double* __restrict__ src,
                            double* __restrict__ qlam, size_t n, double eta, double* partials,
                            PcgScalars* sc) {
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double mix = eta * fresh[i] + (1.0 - eta) * rions[i];
    src[i] = rp[i] + mix - rions[i];
    qlam[i] = q[i] + lam[i];
    acc += lam[i];
  }
  grid_reduce(acc, partials, &sc->counter[CNT_AUX], &sc->aux[1]);
}

// Outer residual after a trial step t (Newton line search):
//   phi_t = phi + t dphi ; rions_t = rions + t (mix - rions - lam dphi/4pi) ;
//   rp_t = (1-t) rp + t (-r/4pi) ;  F_t = ||rho_ions[phi_t] - rions_t + rp_t||.
// With commit != 0 the trial state is written back.
__global__ void k_nl_step(double* __restrict__ phi, const double* __restrict__ eps,
                          double* __restrict__ rions, double* __restrict__ rp,
                          const double* __restrict__ fresh, const double* __restrict__ lam,
                          const double* __restrict__ dphi, const double* __restrict__ r, size_t n,
                          IonParams ip, double eta, double t, int commit, double* partials,
                          PcgScalars* sc) {
  double acc = 0.0;
  const double inv4pi = 1.0 / kFourPi;
  GRID_STRIDE(i, n) {
    const double ri = rions[i];
    const double mix = eta * fresh[i] + (1.0 - eta) * ri;
    const double ph = phi[i] + t * dphi[i];
    const double rit = ri + t * (mix - ri - lam[i] * dphi[i] * inv4pi);
    const double rpt = (1.0 - t) * rp[i] + t * (-r[i] * inv4pi);
    double a, d;
    ion_terms(ph, (eps[i] - 1.0) * ip.inv_eps0m1, ip, &a, &d);
    const double f = a - rit + rpt;
    acc += f * f;
    if (commit) {
      phi[i] = ph;
      rions[i] = rit;
      rp[i] = rpt;
    }
  }
  grid_reduce(acc, partials, &sc->counter[CNT_AUX2], &sc->aux[2]);
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
    lap[idx] = -k2 * inv_n;
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

void launch_setup_s(const double* eps, double* s, double* sq, size_t n, PcgScalars* sc,
                    cudaStream_t st) {
  count_launch();
  k_setup_s<<<grid_blocks(n, kT), kT, 0, st>>>(eps, s, sq, n, sc);
}

void launch_fd16_q(const double* sq, double* q, int nx, int ny, int nz, double hx, double hy,
                   double hz, int perx, int pery, int perz, const Fd16& c, cudaStream_t st) {
  const size_t n = (size_t)nx * ny * nz;
  count_launch();
  k_fd16_q<<<grid_blocks(n, kT), kT, 0, st>>>(sq, q, nx, ny, nz, 1.0 / (hx * hx), 1.0 / (hy * hy),
                                              1.0 / (hz * hz), perx, pery, perz, c);
}

void launch_qlam_linear(const double* q, const double* eps, double* qlam, size_t n, double lambda0,
                        double inv_e0m1, double* partials, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_qlam_linear<<<grid_blocks(n, kT), kT, 0, st>>>(q, eps, qlam, n, lambda0, inv_e0m1, partials, sc);
}

void launch_sum(const double* a, size_t n, double* partials, unsigned int* counter, double* out,
                cudaStream_t st) {
  count_launch();
  k_sum<<<grid_blocks(n, kT), kT, 0, st>>>(a, n, partials, counter, out);
}

void launch_copy_scaled(const double* a, double* b, size_t n, double f, cudaStream_t st) {
  count_launch();
  k_copy_scaled<<<grid_blocks(n, kT), kT, 0, st>>>(a, b, n, f);
}

void launch_mul(const double* a, const double* b, double* c, size_t n, cudaStream_t st) {
  count_launch();
  k_mul<<<grid_blocks(n, kT), kT, 0, st>>>(a, b, c, n);
}

void launch_init(const double* rho, double* r, double* phi, double* p, double* Ap, size_t n,
                 double tol_abs, double tol_rel, int max_iter, double* partials, PcgScalars* sc,
                 int zero_phi, const double* bg_sum, cudaStream_t st) {
  count_launch();
  k_init<<<grid_blocks(n, kT), kT, 0, st>>>(rho, r, phi, p, Ap, n, tol_abs, tol_rel, max_iter,
                                            partials, sc, zero_phi, bg_sum);
}

void launch_update_p(const double* v, const double* r, const double* qlam, const double* sqrt_eps,
                     const double* s, double* p, double* Ap, size_t n, int periodic, int project,
                     double* partials, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_update_p<<<grid_blocks(n, kT), kT, 0, st>>>(v, r, qlam, sqrt_eps, s, p, Ap, n, 1.0 / (double)n,
                                                periodic, project, partials, sc);
}

void launch_update_r(double* phi, double* r, const double* p, const double* Ap, size_t n,
                     double* partials, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_update_r<<<grid_blocks(n, kT), kT, 0, st>>>(phi, r, p, Ap, n, partials, sc);
}

void launch_fp_source(const double* rho, const double* rions, const double* qlam, const double* phi,
                      const double* sq, double* out, size_t n, double bg, double* partials,
                      PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_fp_source<<<grid_blocks(n, kT), kT, 0, st>>>(rho, rions, qlam, phi, sq, out, n, bg, partials, sc);
}

void launch_fp_residual(const double* w, const double* s, const double* phi, size_t n, double c,
                        double* partials, double* partials2, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_fp_residual<<<grid_blocks(n, kT), kT, 0, st>>>(w, s, phi, n, c, partials, partials2, sc);
}

void launch_ionic_charge(const double* phi, const double* eps, double* out, size_t n,
                         const IonParams& ip, cudaStream_t st) {
  count_launch();
  k_ionic_charge<<<grid_blocks(n, kT), kT, 0, st>>>(phi, eps, out, n, ip);
}

void launch_nl_eval(const double* phi, const double* eps, const double* rions, const double* rp,
                    double* fresh, double* lam, size_t n, const IonParams& ip, int newton,
                    double* partials, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_nl_eval<<<grid_blocks(n, kT), kT, 0, st>>>(phi, eps, rions, rp, fresh, lam, n, ip, newton,
                                               partials, sc);
}

void launch_nl_source(const double* fresh, const double* rions, const double* rp, const double* q,
                      const double* lam, double* src, double* qlam, size_t n, double eta,
                      double* partials, PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_nl_source<<<grid_blocks(n, kT), kT, 0, st>>>(fresh, rions, rp, q, lam, src, qlam, n, eta,
                                                 partials, sc);
}

void launch_nl_step(double* phi, const double* eps, double* rions, double* rp, const double* fresh,
                    const double* lam, const double* dphi, const double* r, size_t n,
                    const IonParams& ip, double eta, double t, int commit, double* partials,
                    PcgScalars* sc, cudaStream_t st) {
  count_launch();
  k_nl_step<<<grid_blocks(n, kT), kT, 0, st>>>(phi, eps, rions, rp, fresh, lam, dphi, r, n, ip, eta,
                                               t, commit, partials, sc);
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

void launch_axis_matrix(const double* in, double* out, const double* C, int A, int J, int B, int K,
                        cudaStream_t st) {
  const size_t n = (size_t)A * K * B;
  count_launch();
  k_axis_matrix<<<grid_blocks(n, kT), kT, 0, st>>>(in, out, C, A, J, B, K);
}

}  // namespace gps
