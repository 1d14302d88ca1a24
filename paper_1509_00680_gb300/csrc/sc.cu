// Comparison solvers of the generalized Poisson equation: Algorithm 1 (the
// self-consistent iteration, SC, Eqs. remap and rhoiter) and preconditioned
// steepest descent (Algorithm 2 with beta = 0 and the preconditioner of Eq.
// PrePSD), optionally with DIIS (Pulay).  One slot (slot 0 of a direct pool);
// the vacuum solve of every iteration is the pool's FP64 spectrum pipeline,
// gated by the slot's phase so that a finished solve does no more work.
//
// Discretization: g = grad ln eps by the order-16 central first derivative
// (Sec. "Numerical results"; free faces continue the field by its face
// value, periodic axes wrap), the Laplacian the vacuum solve S inverts; the
// operator is A phi = eps (lap_S phi + g . grad phi).  Every solver stops on
// ||r||_2 <= max(tol_abs, tol_rel ||r_0||_2) with r = -4 pi rho - A phi; for
// periodic BC r is measured modulo its component along eps (the vacuum solve
// drops the mean of its source), r - eps <r / eps>.
//
//   SC   per iteration: phi = S(rho/eps + rho_iter); rho~ = g.grad phi / 4pi;
//        r = -4 pi eps (rho~ - rho_iter); rho_iter <- eta rho~ + (1-eta) rho_iter
//   PSD  v = S(-r / (4 pi eps)) (eps lap v = r); A v = r - eps <r/eps> + eps g.grad v;
//        alpha = (v, r') / (v, A v) (r' = r - eps <r/eps>) or fixed;
//        phi += alpha v; r -= alpha A v
//   DIIS the last m triples (phi_i, r_i, v_i); c minimizing ||sum c_i v_i||_2,
//        sum c_i = 1; one PSD step from the combination
//
// The stored r is not projected: <r/eps> of every stored r is carried as a
// scalar and enters A v and (v, r) instead, which gives the same iterates as
// projecting it.
#include <cmath>

#include "device_util.cuh"
#include "gps_internal.h"
#include "kernels.h"

namespace gps {

constexpr int kT = 256;

#define SC_STRIDE(i, n) \
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// ||r'||^2 of r' = r - eps <r/eps> from A = sum r^2, B = sum eps r,
// C = sum r isc (isc = -1/(4 pi eps), so <r/eps> = -4 pi C / n) and
// E = sum eps^2.
__device__ __forceinline__ double proj_norm2(double A, double B, double C, double E, const ScArgs& a) {
  if (!a.periodic) return A;
  const double m = -kFourPi * C * a.inv_n;   // <r / eps>
  return A - 2.0 * m * B + m * m * E;
}

// g . grad u at point idx = (i, j, k), order-16 central differences.
// grad ln eps is exactly zero wherever eps is flat over the stencil (inside
// the cavities, in the bulk solvent): the product is then zero without the
// differences, which are the kernel's FP64 work and its neighbour loads.
__device__ __forceinline__ double g_dot_grad(const double* __restrict__ u, size_t idx, int i, int j, int k,
                                             const ScArgs& a) {
  const double gx = a.gx[idx], gy = a.gy[idx], gz = a.gz[idx];
  if (gx == 0.0 && gy == 0.0 && gz == 0.0) return 0.0;
  const double3 gu = grad16(u, idx, i, j, k, a.s16);
  return gx * gu.x + gy * gu.y + gz * gu.z;
}

__device__ __forceinline__ void point_of(size_t idx, const ScArgs& a, int* i, int* j, int* k) {
  point_of16(idx, a.s16, i, j, k);
}

// Whether the solve is still iterating; marks the launch as having done work.
__device__ __forceinline__ bool active(const ScArgs& a) {
  if (a.S->phase != PH_ITER) return false;
  if (a.acted && threadIdx.x == 0 && blockIdx.x == 0) *a.acted = 1;
  return true;
}

// Convergence test of the last block after a residual reduction.
__device__ __forceinline__ void after_residual(const ScArgs& a, double rr) {
  SlotState& S = *a.S;
  S.rr = rr;
  S.iter += 1;
  S.iters_total += 1;
  S.fp64_iters += 1;
  if (!isfinite(rr)) {
    S.status = GPS_ERR_BREAKDOWN;
    S.phase = PH_DONE;
  } else if (rr <= S.tol2) {
    S.status = GPS_OK;
    S.phase = PH_DONE;
  } else if (S.iter >= S.max_iter) {
    S.status = GPS_ERR_NOT_CONVERGED;
    S.phase = PH_DONE;
  }
}

// Setup: tmp = ln eps, isc = -1/(4 pi eps); SC: rho_eps = rho/eps, rho_iter = 0,
// src = rho/eps, phi = 0; PSD: phi = 0, r = -4 pi rho (into r0 / phi0);
// ||r_0|| (projected), <r_0/eps>, sum eps^2.  Sets tol2 and the phase.
__global__ void k_sc_prep(ScArgs a, int psd, double* __restrict__ phi0, double* __restrict__ r0) {
  SlotState& S = *a.S;
  if (a.acted && threadIdx.x == 0 && blockIdx.x == 0) *a.acted = 1;
  double sa = 0.0, sb = 0.0, sc = 0.0, se = 0.0;
  SC_STRIDE(i, a.n) {
    const double e = a.eps[i], rho = a.rho[i];
    const double isc = -1.0 / (kFourPi * e);
    a.tmp[i] = log(e);
    a.isc[i] = isc;
    const double r = -kFourPi * rho;
    if (psd) {
      phi0[i] = 0.0;
      r0[i] = r;
    } else {
      const double re = rho / e;
      a.rho_eps[i] = re;
      a.rho_iter[i] = 0.0;
      a.src[i] = re;
      a.phi[i] = 0.0;
    }
    sa += r * r;
    sb += e * r;
    sc += r * isc;
    se += e * e;
  }
  grid_reduce(se, a.part + 3 * a.pstride, &a.cnt[3], &S.aux[7]);
  if (grid_reduce3(sa, sb, sc, a.part, a.part + a.pstride, a.part + 2 * a.pstride, &a.cnt[0], &S.aux[0],
                   &S.aux[1], &S.aux[2]) &&
      threadIdx.x == 0) {
    // sum eps^2 comes from the other reduction's last block (an L2 read)
    const double rr0 = proj_norm2(S.aux[0], S.aux[1], S.aux[2], __ldcg(&S.aux[7]), a);
    S.rr0 = rr0;
    S.rr = rr0;
    const double tol = fmax(S.tol_abs, S.tol_rel * sqrt(rr0));
    S.tol2 = tol * tol;
    S.aux[3] = a.periodic ? -kFourPi * S.aux[2] * a.inv_n : 0.0;   // <r_0 / eps>
    if (a.hist_m) a.hist_mr[0] = S.aux[3];
    S.iter = 0;
    S.status = GPS_OK;
    S.phase = rr0 <= S.tol2 ? PH_DONE : PH_ITER;
  }
}

// g = grad(tmp) by order-16 central differences (tmp = ln eps).
__global__ void k_sc_grad(ScArgs a) {
  SC_STRIDE(idx, a.n) {
    int i, j, k;
    point_of(idx, a, &i, &j, &k);
    const double3 g = grad16(a.tmp, idx, i, j, k, a.s16);
    a.gx[idx] = g.x;
    a.gy[idx] = g.y;
    a.gz[idx] = g.z;
  }
}

// SC, after phi = S(src): rho~ = g.grad phi / 4pi; r = -4 pi eps (rho~ - rho_iter);
// rho_iter <- eta rho~ + (1 - eta) rho_iter; src = rho/eps + rho_iter.
__global__ void k_sc_step(ScArgs a) {
  if (!active(a)) return;
  SlotState& S = *a.S;
  const double eta = S.eta, inv4pi = 1.0 / kFourPi;
  double sa = 0.0, sb = 0.0, sc = 0.0;
  SC_STRIDE(idx, a.n) {
    int i, j, k;
    point_of(idx, a, &i, &j, &k);
    const double rt = g_dot_grad(a.phi, idx, i, j, k, a) * inv4pi;
    const double ri = a.rho_iter[idx], e = a.eps[idx];
    const double r = -kFourPi * e * (rt - ri);
    sa += r * r;
    sb += e * r;
    sc += r * a.isc[idx];
    const double rn = eta * rt + (1.0 - eta) * ri;
    a.rho_iter[idx] = rn;
    a.src[idx] = a.rho_eps[idx] + rn;
  }
  if (grid_reduce3(sa, sb, sc, a.part, a.part + a.pstride, a.part + 2 * a.pstride, &a.cnt[0], &S.aux[0],
                   &S.aux[1], &S.aux[2]) &&
      threadIdx.x == 0)
    after_residual(a, proj_norm2(S.aux[0], S.aux[1], S.aux[2], S.aux[7], a));
}

// PSD: A v = r - eps m + eps g.grad v (m = <r/eps> of this r, or of the DIIS
// combination); (v, r') = (v, r) - m (v, eps); alpha.
__global__ void k_psd_av(ScArgs a, const double* __restrict__ v, const double* __restrict__ r,
                         double* __restrict__ Av, int diis) {
  if (!active(a)) return;
  SlotState& S = *a.S;
  const double m = diis ? a.hist_mr[kMaxDiis] : S.aux[3];
  double svr = 0.0, sve = 0.0, svav = 0.0;
  SC_STRIDE(idx, a.n) {
    int i, j, k;
    point_of(idx, a, &i, &j, &k);
    const double e = a.eps[idx], vi = v[idx], ri = r[idx];
    const double av = ri - e * m + e * g_dot_grad(v, idx, i, j, k, a);
    Av[idx] = av;
    svr += vi * ri;
    sve += vi * e;
    svav += vi * av;
  }
  if (grid_reduce3(svr, sve, svav, a.part, a.part + a.pstride, a.part + 2 * a.pstride, &a.cnt[1], &S.aux[4],
                   &S.aux[5], &S.aux[6]) &&
      threadIdx.x == 0) {
    const double vr = S.aux[4] - m * S.aux[5], vav = S.aux[6];
    S.vr = vr;
    S.pAp = vav;
    if (a.alpha > 0.0) {
      S.alpha = a.alpha;
    } else if (!isfinite(vav) || vav >= 0.0) {
      S.status = GPS_ERR_BREAKDOWN;
      S.phase = PH_DONE;
    } else {
      S.alpha = vr / vav;
    }
  }
}

// PSD: phi_out = phi + alpha v; r_out = r - alpha A v; ||r_out'||, <r_out/eps>.
__global__ void k_psd_update(ScArgs a, const double* __restrict__ phi, const double* __restrict__ r,
                             const double* __restrict__ v, const double* __restrict__ Av,
                             double* __restrict__ phi_out, double* __restrict__ r_out, int hist_slot) {
  if (!active(a)) return;
  SlotState& S = *a.S;
  const double al = S.alpha;
  double sa = 0.0, sb = 0.0, sc = 0.0;
  SC_STRIDE(i, a.n) {
    const double rn = r[i] - al * Av[i];
    phi_out[i] = phi[i] + al * v[i];
    r_out[i] = rn;
    sa += rn * rn;
    sb += a.eps[i] * rn;
    sc += rn * a.isc[i];
  }
  if (grid_reduce3(sa, sb, sc, a.part, a.part + a.pstride, a.part + 2 * a.pstride, &a.cnt[2], &S.aux[0],
                   &S.aux[1], &S.aux[2]) &&
      threadIdx.x == 0) {
    const double m = a.periodic ? -kFourPi * S.aux[2] * a.inv_n : 0.0;
    S.aux[3] = m;
    if (hist_slot >= 0) a.hist_mr[hist_slot] = m;
    after_residual(a, proj_norm2(S.aux[0], S.aux[1], S.aux[2], S.aux[7], a));
  }
}

// Pulay coefficients of the bordered system [[B, 1], [1^T, 0]] [c, mu] =
// [0, 1] by Gaussian elimination with partial pivoting (thread 0).
static __device__ void diis_solve(const double* B, int cnt, const int* slots, double* c) {
  double M[kMaxDiis + 1][kMaxDiis + 2];
  const int n = cnt + 1;
  for (int i = 0; i < cnt; ++i) {
    for (int j = 0; j < cnt; ++j) M[i][j] = B[slots[i] * kMaxDiis + slots[j]];
    M[i][cnt] = 1.0;
    M[i][n] = 0.0;
  }
  for (int j = 0; j < cnt; ++j) M[cnt][j] = 1.0;
  M[cnt][cnt] = 0.0;
  M[cnt][n] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
    if (piv != col)
      for (int j = 0; j <= n; ++j) {
        const double t = M[col][j];
        M[col][j] = M[piv][j];
        M[piv][j] = t;
      }
    for (int i = col + 1; i < n; ++i) {
      const double f = M[i][col] / M[col][col];
      for (int j = col; j <= n; ++j) M[i][j] -= f * M[col][j];
    }
  }
  double x[kMaxDiis + 1];
  for (int i = n - 1; i >= 0; --i) {
    double s = M[i][n];
    for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  for (int i = 0; i < cnt; ++i) c[i] = x[i];
}

// DIIS: (v_new, v_i) for the cnt entries of the history (ring slots
// slot[0..cnt-1], oldest first; the newest, slot[cnt-1], holds v_new), the
// matrix row of the new entry, then the coefficients c and the combined
// mean <r/eps>.  One block reduction of up to kMaxDiis sums.
__global__ void k_diis_row(ScArgs a, DiisSlots sl) {
  if (!active(a)) return;
  const int cnt = sl.cnt, jn = sl.slot[cnt - 1];
  const double* vn = a.hist_v + (size_t)jn * a.n;
  double acc[kMaxDiis];
#pragma unroll
  for (int q = 0; q < kMaxDiis; ++q) acc[q] = 0.0;
  SC_STRIDE(i, a.n) {
    const double x = vn[i];
#pragma unroll
    for (int q = 0; q < kMaxDiis; ++q)
      if (q < cnt) acc[q] = fma(x, a.hist_v[(size_t)sl.slot[q] * a.n + i], acc[q]);
  }
  __shared__ double red[kMaxDiis][kT / 32];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxDiis; ++q) {
    double s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][wid] = s;
  }
  __syncthreads();
  const unsigned int nb = gridDim.x;
  if (threadIdx.x == 0) {
    for (int q = 0; q < cnt; ++q) {
      double s = 0.0;
      for (int w = 0; w < kT / 32; ++w) s += red[q][w];
      a.dpart[(size_t)q * a.pstride + blockIdx.x] = s;
    }
    __threadfence();
    const unsigned int t = atomicAdd(&a.cnt[4], 1u);
    am_last = (t == nb - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    for (int q = 0; q < cnt; ++q) {
      double s = 0.0;
      for (unsigned int b = lane; b < nb; b += 32) s += __ldcg(a.dpart + (size_t)q * a.pstride + b);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) {
        a.diis_B[jn * kMaxDiis + sl.slot[q]] = s;
        a.diis_B[sl.slot[q] * kMaxDiis + jn] = s;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.cnt[4] = 0u;
    double c[kMaxDiis];
    if (cnt == 1) c[0] = 1.0;
    else diis_solve(a.diis_B, cnt, sl.slot, c);
    double m = 0.0;
    for (int q = 0; q < cnt; ++q) {
      a.diis_c[q] = c[q];
      m += c[q] * a.hist_mr[sl.slot[q]];
    }
    a.hist_mr[kMaxDiis] = m;
  }
}

// DIIS: phi_w = sum c_q phi_q, r_w = sum c_q r_q, v_w = sum c_q v_q.
__global__ void k_diis_combine(ScArgs a, DiisSlots sl, double* __restrict__ phi_w, double* __restrict__ r_w,
                               double* __restrict__ v_w) {
  if (!active(a)) return;
  const int cnt = sl.cnt;
  double c[kMaxDiis];
#pragma unroll
  for (int q = 0; q < kMaxDiis; ++q) c[q] = q < cnt ? a.diis_c[q] : 0.0;
  SC_STRIDE(i, a.n) {
    double p = 0.0, r = 0.0, v = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxDiis; ++q) {
      if (q < cnt) {
        const size_t o = (size_t)sl.slot[q] * a.n + i;
        p = fma(c[q], a.hist_phi[o], p);
        r = fma(c[q], a.hist_r[o], r);
        v = fma(c[q], a.hist_v[o], v);
      }
    }
    phi_w[i] = p;
    r_w[i] = r;
    v_w[i] = v;
  }
}

int sc_blocks(size_t n) {
  size_t b = (n + kT - 1) / kT;
  const size_t cap = 152 * 4;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_sc_prep(const ScArgs& a, int psd, double* phi0, double* r0, cudaStream_t st) {
  count_launch();
  k_sc_prep<<<sc_blocks(a.n), kT, 0, st>>>(a, psd, phi0, r0);
  count_launch();
  k_sc_grad<<<sc_blocks(a.n), kT, 0, st>>>(a);
}

void launch_sc_step(const ScArgs& a, cudaStream_t st) {
  count_launch();
  k_sc_step<<<sc_blocks(a.n), kT, 0, st>>>(a);
}

void launch_psd_av(const ScArgs& a, const double* v, const double* r, double* Av, int diis, cudaStream_t st) {
  count_launch();
  k_psd_av<<<sc_blocks(a.n), kT, 0, st>>>(a, v, r, Av, diis);
}

void launch_psd_update(const ScArgs& a, const double* phi, const double* r, const double* v, const double* Av,
                       double* phi_out, double* r_out, int hist_slot, cudaStream_t st) {
  count_launch();
  k_psd_update<<<sc_blocks(a.n), kT, 0, st>>>(a, phi, r, v, Av, phi_out, r_out, hist_slot);
}

void launch_diis(const ScArgs& a, const DiisSlots& sl, double* phi_w, double* r_w, double* v_w,
                 cudaStream_t st) {
  count_launch();
  k_diis_row<<<sc_blocks(a.n), kT, 0, st>>>(a, sl);
  count_launch();
  k_diis_combine<<<sc_blocks(a.n), kT, 0, st>>>(a, sl, phi_w, r_w, v_w);
}

}  // namespace gps
