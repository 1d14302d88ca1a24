// Quantities a DFT code takes from the generalized Poisson solve:
//
//   sccs dielectric (Eq. sccs): eps = 1 (rho_elec >= rho_max), eps0
//       (rho_elec <= rho_min), eps0^w in between, w = (z - sin z)/(2 pi),
//       z = 2 pi ln(rho_max / rho_elec) / ln(rho_max / rho_min) (the printed
//       middle branch eps0 exp(w) is discontinuous at both thresholds; eps0^w
//       is continuous), and d eps / d rho_elec;
//   polarization charge (Eqs. remap, rhopol): rho_pol = grad ln eps . grad phi
//       / 4 pi - ((eps - 1)/eps) rho (the sign Eq. remap requires);
//   v_eps (Eq. veps) = -(1/8 pi) (d eps / d rho_elec) |grad phi|^2;
//   electrostatic energy: (1/2) sum rho phi and (1/8 pi) sum eps |grad phi|^2
//       (times h^3, by the host).
//
// Gradients by the order-16 central differences of stencil16.cuh.  One-off
// post-processing passes: pointwise or one stencil per point, no iteration.
#include <cmath>

#include "device_util.cuh"
#include "gps_internal.h"
#include "kernels.h"

namespace gps {

constexpr int kTd = 256;

#define DFT_STRIDE(i, n) \
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

__global__ void k_sccs(const double* __restrict__ rho, double* __restrict__ eps, double* __restrict__ deps,
                       size_t n, double rmax, double rmin, double inv_lnr, double lne, double eps0) {
  DFT_STRIDE(i, n) {
    const double x = rho[i];
    double e, d = 0.0;
    if (x >= rmax) {
      e = 1.0;
    } else if (x <= rmin) {
      e = eps0;
    } else {
      const double z = 2.0 * kPi * log(rmax / x) * inv_lnr;
      double sz, cz;
      sincos(z, &sz, &cz);
      e = exp((z - sz) / (2.0 * kPi) * lne);
      d = -e * lne * (1.0 - cz) * inv_lnr / x;
    }
    eps[i] = e;
    if (deps) deps[i] = d;
  }
}

__global__ void k_log(const double* __restrict__ eps, double* __restrict__ out, size_t n) {
  DFT_STRIDE(i, n) out[i] = log(eps[i]);
}

__global__ void k_pol(Stencil16 s, const double* __restrict__ lne, const double* __restrict__ phi,
                      const double* __restrict__ rho, const double* __restrict__ eps, double* __restrict__ out,
                      size_t n) {
  DFT_STRIDE(idx, n) {
    int i, j, k;
    point_of16(idx, s, &i, &j, &k);
    const double3 a = grad16(lne, idx, i, j, k, s);
    const double3 b = grad16(phi, idx, i, j, k, s);
    const double e = eps[idx];
    out[idx] = (a.x * b.x + a.y * b.y + a.z * b.z) / (4.0 * kPi) - (e - 1.0) / e * rho[idx];
  }
}

__global__ void k_veps(Stencil16 s, const double* __restrict__ deps, const double* __restrict__ phi,
                       double* __restrict__ out, size_t n) {
  DFT_STRIDE(idx, n) {
    const double d = deps[idx];
    double v = 0.0;
    if (d != 0.0) {   // outside the sccs transition d eps / d rho = 0
      int i, j, k;
      point_of16(idx, s, &i, &j, &k);
      const double3 g = grad16(phi, idx, i, j, k, s);
      v = -d * (g.x * g.x + g.y * g.y + g.z * g.z) / (8.0 * kPi);
    }
    out[idx] = v;
  }
}

// Per-block partial sums of rho phi and eps |grad phi|^2 into part[2 b], part[2 b + 1].
__global__ void k_energy(Stencil16 s, const double* __restrict__ rho, const double* __restrict__ eps,
                         const double* __restrict__ phi, size_t n, double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  DFT_STRIDE(idx, n) {
    int i, j, k;
    point_of16(idx, s, &i, &j, &k);
    const double3 g = grad16(phi, idx, i, j, k, s);
    a = fma(rho[idx], phi[idx], a);
    b = fma(eps[idx], g.x * g.x + g.y * g.y + g.z * g.z, b);
  }
  const double sa = block_sum(a);
  const double sb = block_sum(b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

int dft_blocks(size_t n) {
  size_t b = (n + kTd - 1) / kTd;
  if (b > 152 * 4) b = 152 * 4;
  return b < 1 ? 1 : (int)b;
}

void launch_sccs(const double* rho, double* eps, double* deps, size_t n, double rho_max, double rho_min,
                 double eps0, cudaStream_t st) {
  count_launch();
  k_sccs<<<dft_blocks(n), kTd, 0, st>>>(rho, eps, deps, n, rho_max, rho_min, 1.0 / std::log(rho_max / rho_min),
                                        std::log(eps0), eps0);
}

void launch_polarization(const Stencil16& s, const double* rho, const double* eps, const double* phi,
                         double* tmp, double* out, size_t n, cudaStream_t st) {
  count_launch();
  k_log<<<dft_blocks(n), kTd, 0, st>>>(eps, tmp, n);
  count_launch();
  k_pol<<<dft_blocks(n), kTd, 0, st>>>(s, tmp, phi, rho, eps, out, n);
}

void launch_veps(const Stencil16& s, const double* deps, const double* phi, double* out, size_t n, cudaStream_t st) {
  count_launch();
  k_veps<<<dft_blocks(n), kTd, 0, st>>>(s, deps, phi, out, n);
}

void launch_energy(const Stencil16& s, const double* rho, const double* eps, const double* phi, size_t n,
                   double* part, cudaStream_t st) {
  count_launch();
  k_energy<<<dft_blocks(n), kTd, 0, st>>>(s, rho, eps, phi, n, part);
}

}  // namespace gps
