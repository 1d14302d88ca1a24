// C ABI of the solver (include/gps.h) and its host engine.
//
// Shape: everything that depends on (grid, spacing, BC) only -- FFT
//   schedules, twiddles, Green's-function and Laplacian tables.
// Pool: `cap` slots of one shape, each with strided vectors, a spectrum
//   workspace, reduction partials and a SlotState; one round launches every
//   stage of the device phase machine (kernels.cu) once and `m` PCG
//   iterations, each kernel acting on the slots in its phase.
// Engine: pools of one device, a queue of requests, admission into free
//   slots under the HBM budget, rounds on every busy pool (one stream per
//   pool, so pools overlap on the device) and collection of finished slots.
// Single solves run in a one-slot pool per shape, driven on the caller's
// stream; batches and the server run an Engine.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include "device_util.cuh"
#include "gps_internal.h"
#include "kernels.h"

using namespace gps;

namespace {

struct CudaError {};
inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaError{};
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool factorable(int L) {
  int r = L;
  for (int p : {2, 3, 5})
    while (r % p == 0) r /= p;
  return r == 1;
}

// Stockham schedule of length L.  order 0: radix 8 first, then 4/2, 5, 3;
// order 1: the radix-2/4 remainder first, then the 8s; order 2: radix 4
// throughout (then 2), then 5 and 3.
bool make_sched(int L, FftSched* s, int order = 0) {
  if (L < 2 || L > kMaxLen || !factorable(L)) return false;
  std::memset(s, 0, sizeof(*s));
  s->L = L;
  std::vector<int> rad;
  int rem = L;
  int p2 = 0;
  while (rem % 2 == 0) { rem /= 2; ++p2; }
  std::vector<int> twos;
  if (order == 3) {   // radix 16 first (FP64 kernels only); no 16 in L: not a new schedule
    if (p2 < 4) return false;
    while (p2 >= 4) { twos.push_back(16); p2 -= 4; }
    if (p2 == 3) twos.push_back(8);
    if (p2 == 2) twos.push_back(4);
    if (p2 == 1) twos.push_back(2);
  } else if (order == 2) {
    while (p2 >= 2) { twos.push_back(4); p2 -= 2; }
    if (p2) twos.push_back(2);
  } else {
    while (p2 >= 3) { twos.push_back(8); p2 -= 3; }
    if (p2 == 2) twos.push_back(4);
    if (p2 == 1) twos.push_back(2);
    if (order == 1) std::reverse(twos.begin(), twos.end());
  }
  rad = twos;
  while (rem % 5 == 0) { rad.push_back(5); rem /= 5; }
  while (rem % 3 == 0) { rad.push_back(3); rem /= 3; }
  if (rem != 1 || (int)rad.size() > kMaxStages) return false;
  int ns = 1;
  for (size_t k = 0; k < rad.size(); ++k) {
    s->radix[k] = rad[k];
    s->ns[k] = ns;
    ns *= rad[k];
  }
  s->nst = (int)rad.size();
  return true;
}

// Order-16 central second-derivative coefficients (exact formula, long double):
// c_j = 2 (-1)^(j+1) (8!)^2 / (j^2 (8-j)! (8+j)!), c_0 = -2 sum c_j.
Fd16 fd16_coeffs() {
  auto fact = [](int n) {
    long double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  Fd16 c;
  long double sum = 0;
  for (int j = 1; j <= 8; ++j) {
    long double v = 2.0L * fact(8) * fact(8) / ((long double)j * j * fact(8 - j) * fact(8 + j));
    if (j % 2 == 0) v = -v;
    c.c[j] = (double)v;
    sum += v;
  }
  c.c[0] = (double)(-2.0L * sum);
  return c;
}

// Order-16 central first-derivative coefficients (exact formula, long double):
// f'(x) ~ (1/h) sum_j d_j (f(x + jh) - f(x - jh)),
// d_j = (-1)^(j+1) (8!)^2 / (j (8-j)! (8+j)!).
void fd16_first_coeffs(double* d) {
  auto fact = [](int n) {
    long double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  d[0] = 0.0;
  for (int j = 1; j <= 8; ++j) {
    long double v = fact(8) * fact(8) / ((long double)j * fact(8 - j) * fact(8 + j));
    d[j] = (double)(j % 2 == 0 ? -v : v);
  }
}

// Order-16 first-derivative stencil of a grid: wrapping axes per BC.
Stencil16 stencil16_of(const gps_grid& g) {
  Stencil16 s{};
  s.nx = g.nx;
  s.ny = g.ny;
  s.nz = g.nz;
  s.perx = g.bc == GPS_BC_PERIODIC || g.bc == GPS_BC_SURFACE;
  s.pery = s.perx;
  s.perz = g.bc == GPS_BC_PERIODIC || g.bc == GPS_BC_WIRE;
  s.ihx = 1.0 / g.hx;
  s.ihy = 1.0 / g.hy;
  s.ihz = 1.0 / g.hz;
  fd16_first_coeffs(s.d);
  return s;
}

// Even (cosine) transform matrix C[k][j] = w_j cos(2 pi j k / M) * scale,
// j = 0..M/2, k = 0..K-1, w_0 = w_(M/2) = 1, otherwise 2.
std::vector<double> cosine_matrix(int M, int K, double scale) {
  const int J = M / 2 + 1;
  std::vector<double> C((size_t)K * J);
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < J; ++j) {
      const long long t = ((long long)j * k) % M;
      const long double ang = 2.0L * 3.141592653589793238462643383279502884L * t / M;
      const double w = (j == 0 || j == M / 2) ? 1.0 : 2.0;
      C[(size_t)k * J + j] = w * (double)cosl(ang) * scale;
    }
  return C;
}

IonParams ion_params(const gps_electrolyte* el, bool steric = false) {
  const double NA = 6.02214076e23, a0 = 5.29177210903e-11, kB = 3.1668115634556e-6;
  IonParams ip;
  std::memset(&ip, 0, sizeof(ip));
  ip.exp_cap = 40.0;
  ip.inv_eps0m1 = 1.0;
  if (!el) return ip;
  ip.nspecies = el->nspecies;
  const double kt = kB * el->temperature;
  ip.inv_kt = 1.0 / kt;
  ip.inv_eps0m1 = 1.0 / (el->eps0 - 1.0);
  double l = 0.0;
  for (int s = 0; s < el->nspecies; ++s) {
    const double nb = el->c_molar[s] * 1000.0 * NA * a0 * a0 * a0;
    ip.zq[s] = el->z[s];
    ip.zn[s] = el->z[s] * nb;
    ip.z2n_kt[s] = (double)el->z[s] * el->z[s] * nb / kt;
    l += ip.z2n_kt[s];
  }
  ip.lambda0 = kFourPi * l;
  if (steric) {
    // Eq. (maxconc) as a number density: p / ((4/3) pi R^3), R in bohr
    ip.steric = 1;
    for (int s = 0; s < el->nspecies; ++s) {
      const double r = el->radius_angstrom[s] * 1e-10 / a0;
      const double nmax = el->packing / (4.0 / 3.0 * kPi * r * r * r);
      ip.a[s] = el->c_molar[s] * 1000.0 * NA * a0 * a0 * a0 / nmax;
    }
  }
  return ip;
}

// Modified PB needs a packing coefficient and a radius per species.
int validate_steric(const gps_electrolyte* el) {
  if (!el || !(el->packing > 0)) return GPS_ERR_INVALID;
  for (int s = 0; s < el->nspecies; ++s)
    if (!(el->radius_angstrom[s] > 0)) return GPS_ERR_INVALID;
  return GPS_OK;
}

// gps_opts.method: the comparison solvers take GPe, FP64, cold starts, and
// periodic axes of at least 8 points (the order-16 stencil wraps once).
int validate_method(const gps_opts& o, int kind, const gps_grid* g) {
  if (o.forcing_rule != GPS_FORCING_EW2 && o.forcing_rule != GPS_FORCING_RATIO) return GPS_ERR_INVALID;
  if (o.method == GPS_PCG) return GPS_OK;
  if (o.method != GPS_SC && o.method != GPS_PSD) return GPS_ERR_INVALID;
  if (kind != GPS_GPE || o.precision != GPS_FP64 || o.warm_start) return GPS_ERR_INVALID;
  if (o.method == GPS_SC && !(o.eta > 0.0 && o.eta <= 1.0)) return GPS_ERR_INVALID;
  if (o.method == GPS_PSD && (!(o.alpha >= 0.0) || o.diis < 0 || o.diis > GPS_MAX_DIIS)) return GPS_ERR_INVALID;
  const bool pxy = g->bc == GPS_BC_PERIODIC || g->bc == GPS_BC_SURFACE;
  const bool pz = g->bc == GPS_BC_PERIODIC || g->bc == GPS_BC_WIRE;
  if ((pxy && (g->nx < 8 || g->ny < 8)) || (pz && g->nz < 8)) return GPS_ERR_INVALID;
  return GPS_OK;
}

int validate_grid(const gps_grid* g) {
  if (!g) return GPS_ERR_INVALID;
  if (g->nx < 4 || g->ny < 4 || g->nz < 4) return GPS_ERR_INVALID;
  if (!(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) return GPS_ERR_INVALID;
  if (g->bc < GPS_BC_FREE || g->bc > GPS_BC_WIRE) return GPS_ERR_INVALID;
  const bool fx = g->bc == GPS_BC_FREE || g->bc == GPS_BC_WIRE;
  const bool fz = g->bc == GPS_BC_FREE || g->bc == GPS_BC_SURFACE;
  const int Px = fx ? 2 * g->nx : g->nx, Py = fx ? 2 * g->ny : g->ny, Pz = fz ? 2 * g->nz : g->nz;
  for (int P : {Px, Py, Pz})
    if (P % 2 || P > kMaxLen || !factorable(P)) return GPS_ERR_INVALID;
  if (g->bc == GPS_BC_FREE) {
    const double R = std::sqrt(std::pow(g->nx * g->hx, 2) + std::pow(g->ny * g->hy, 2) +
                               std::pow(g->nz * g->hz, 2));
    if (4 * g->nx * g->hx < g->nx * g->hx + R || 4 * g->ny * g->hy < g->ny * g->hy + R ||
        4 * g->nz * g->hz < g->nz * g->hz + R)
      return GPS_ERR_INVALID;   // aspect ratio too large for the 4x oversampled kernel
  }
  if (g->bc == GPS_BC_WIRE) {
    const double R = std::sqrt(std::pow(g->nx * g->hx, 2) + std::pow(g->ny * g->hy, 2));
    if (4 * g->nx * g->hx < g->nx * g->hx + R || 4 * g->ny * g->hy < g->ny * g->hy + R)
      return GPS_ERR_INVALID;   // transverse aspect ratio too large for the oversampled kernel
  }
  return GPS_OK;
}

int validate_el(const gps_electrolyte* el) {
  if (!el || el->nspecies < 0 || el->nspecies > GPS_MAX_SPECIES) return GPS_ERR_INVALID;
  if (!(el->temperature > 0) || !(el->eps0 > 1.0)) return GPS_ERR_INVALID;
  for (int s = 0; s < el->nspecies; ++s)
    if (!(el->c_molar[s] >= 0)) return GPS_ERR_INVALID;
  return GPS_OK;
}

bool same_grid(const gps_grid& a, const gps_grid& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.hx == b.hx && a.hy == b.hy &&
         a.hz == b.hz && a.bc == b.bc;
}

// Device allocations released together.
struct DevMem {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    const size_t b = count * sizeof(T);
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// ------------------------------------------------------------- profiling --

// Opt-in per-kernel timing with CUDA events on the launching stream.  Each
// timed launch gets a device flag that its first serving block sets; launches
// that found no slot to serve (the PCG had already converged) are dropped.
struct Profiler {
  bool on = false;
  int mask = 0;
  struct Rec { int kind; cudaEvent_t a, b; int flag; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  int* flags = nullptr;              // device, kFlags entries
  static constexpr int kFlags = 1 << 15;
  int next_flag = 0;
  long long launches[GPS_PROFILE_KINDS] = {0};
  double ms[GPS_PROFILE_KINDS] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int* flag_for(int* idx) {
    if (!flags) {
      if (cudaMalloc(&flags, sizeof(int) * kFlags) != cudaSuccess) return nullptr;
      cudaMemset(flags, 0, sizeof(int) * kFlags);
    }
    if (next_flag >= kFlags) resolve();
    *idx = next_flag++;
    return flags + *idx;
  }
  void resolve() {
    if (pending.empty()) return;
    cudaEventSynchronize(pending.back().b);
    std::vector<int> acted(next_flag, 0);
    if (flags && next_flag > 0) {
      cudaMemcpy(acted.data(), flags, sizeof(int) * next_flag, cudaMemcpyDeviceToHost);
      cudaMemset(flags, 0, sizeof(int) * next_flag);
    }
    for (auto& r : pending) {
      float t = 0.f;
      const bool did = r.flag < 0 || acted[r.flag];
      if (did && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        launches[r.kind] += 1;
        ms[r.kind] += t;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
    next_flag = 0;
  }
  ~Profiler() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
    if (flags) cudaFree(flags);
  }
};

thread_local Profiler* t_prof = nullptr;

// Runs launch(b') with b' = b plus the acted flag of a new profiling record
// when kernels of this kind are being timed.
template <typename F>
void timed(int kind, const Batch& b, cudaStream_t st, F&& launch) {
  if (!t_prof || !t_prof->on || !(t_prof->mask & (1 << kind))) {
    launch(b);
    return;
  }
  Batch bb = b;
  int idx = -1;
  bb.acted = t_prof->flag_for(&idx);
  if (!bb.acted) idx = -1;
  cudaEvent_t e0 = t_prof->get(), e1 = t_prof->get();
  cudaEventRecord(e0, st);
  launch(bb);
  cudaEventRecord(e1, st);
  t_prof->pending.push_back({kind, e0, e1, idx});
}

// ----------------------------------------------------------------- shapes --

struct Shape {
  gps_grid grid;
  size_t n = 0;
  int Px = 0, Py = 0, Pz = 0, Hx = 0, Hp = 0;
  int periodic = 0;
  double inv_p = 0.0;
  PassGeom g;                 // heuristic geometry (reduction sizing)
  FftSched fx, fy, fz;
  struct Sched {
    bool tuned = false;
    PassGeom g;
    FftSched fx, fy, fz;
  } sp[3];                    // per spectrum precision (Spec), set by the autotuner
  double2 *twx64 = nullptr, *twy64 = nullptr, *twz64 = nullptr;
  float2 *twx32 = nullptr, *twy32 = nullptr, *twz32 = nullptr;
  dfc *twxdf = nullptr, *twydf = nullptr, *twzdf = nullptr;
  double* table = nullptr;
  float* table32 = nullptr;   // table rounded to float (FP32 spectrum)
  float2* tabledf = nullptr;  // table as double-float (df64 spectrum)
  double* lap = nullptr;
  DevMem mem;
};

int batch_lines(int L, int units) { return default_lines(L, units, sizeof(double2)); }

void upload_twiddles(Shape* S, int L, double2** t64, float2** t32, dfc** tdf) {
  std::vector<double2> h64(L);
  std::vector<float2> h32(L);
  std::vector<dfc> hdf(L);
  for (int m = 0; m < L; ++m) {
    const long double ang = 2.0L * 3.141592653589793238462643383279502884L * m / L;
    const long double c = cosl(ang), s = -sinl(ang);
    h64[m].x = (double)c;
    h64[m].y = (double)s;
    h32[m].x = (float)h64[m].x;
    h32[m].y = (float)h64[m].y;
    // double-float split taken from the long double value
    const float cx = (float)c, sy = (float)s;
    hdf[m].x = df(cx, (float)(c - (long double)cx));
    hdf[m].y = df(sy, (float)(s - (long double)sy));
  }
  // FP32 and df64 tables carry, after the plain table, the per-stage layouts
  // of the register-resident column passes (zeros where L is not served).
  std::vector<int> idx(2 * (size_t)L, 0);
  const bool col = col_stage_twiddle_index(L, idx.data());
  h32.resize(3 * (size_t)L);
  hdf.resize(3 * (size_t)L);
  for (size_t i = 0; i < 2 * (size_t)L; ++i) {
    h32[L + i] = col ? h32[idx[i]] : float2{0.f, 0.f};
    hdf[L + i] = col ? hdf[idx[i]] : dfc{df(0.f, 0.f), df(0.f, 0.f)};
  }
  *t64 = S->mem.alloc<double2>(L);
  *t32 = S->mem.alloc<float2>(3 * (size_t)L);
  *tdf = S->mem.alloc<dfc>(3 * (size_t)L);
  ck(cudaMemcpy(*t64, h64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(*t32, h32.data(), 3 * (size_t)L * sizeof(float2), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(*tdf, hdf.data(), 3 * (size_t)L * sizeof(dfc), cudaMemcpyHostToDevice));
}

// Free-BC table: h^3 g on the octant from the 4x oversampled truncated-Coulomb
// transform (three even transforms), then its 2n-periodic transform (three
// more), normalized by 1/(Px Py Pz).
void build_free_table(Shape* S, cudaStream_t st) {
  const int nx = S->grid.nx, ny = S->grid.ny, nz = S->grid.nz;
  const double hx = S->grid.hx, hy = S->grid.hy, hz = S->grid.hz;
  const int Mx = 4 * nx, My = 4 * ny, Mz = 4 * nz;
  const int mx = Mx / 2 + 1, my = My / 2 + 1, mz = Mz / 2 + 1;
  const double R = std::sqrt(std::pow(nx * hx, 2) + std::pow(ny * hy, 2) + std::pow(nz * hz, 2));
  const int hxo = nx + 1, hyo = ny + 1, hzo = nz + 1;
  DevMem tmp;
  auto up = [&](const std::vector<double>& h) {
    double* d = tmp.alloc<double>(h.size());
    ck(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    return d;
  };
  double* ghat = tmp.alloc<double>((size_t)mx * my * mz);
  launch_free_ghat(ghat, mx, my, mz, 2 * kPi / (Mx * hx), 2 * kPi / (My * hy), 2 * kPi / (Mz * hz), R, st);
  double* cx = up(cosine_matrix(Mx, hxo, 1.0 / Mx));
  double* cy = up(cosine_matrix(My, hyo, 1.0 / My));
  double* cz = up(cosine_matrix(Mz, hzo, 1.0 / Mz));
  double* t1 = tmp.alloc<double>((size_t)mz * my * hxo);
  launch_axis_matrix(ghat, t1, cx, mz * my, mx, 1, hxo, st);
  double* t2 = tmp.alloc<double>((size_t)mz * hyo * hxo);
  launch_axis_matrix(t1, t2, cy, mz, my, hxo, hyo, st);
  double* g = tmp.alloc<double>((size_t)hzo * hyo * hxo);
  launch_axis_matrix(t2, g, cz, 1, mz, hyo * hxo, hzo, st);
  // transform of the 2n-periodic even extension: M = 2n, entries m = 0..n
  double* dx = up(cosine_matrix(2 * nx, hxo, 1.0 / (2 * nx)));
  double* dy = up(cosine_matrix(2 * ny, hyo, 1.0 / (2 * ny)));
  double* dz = up(cosine_matrix(2 * nz, hzo, 1.0 / (2 * nz)));
  double* u1 = tmp.alloc<double>((size_t)hzo * hyo * hxo);
  double* u2 = tmp.alloc<double>((size_t)hzo * hyo * hxo);
  launch_axis_matrix(g, u1, dx, hzo * hyo, hxo, 1, hxo, st);
  launch_axis_matrix(u1, u2, dy, hzo, hyo, hxo, hyo, st);
  launch_axis_matrix(u2, S->table, dz, 1, hzo, hyo * hxo, hzo, st);
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
}

// Wire-BC table: per |kz| index, h_x h_y g on the (x, y) quadrant from the
// 4x oversampled transform of the transversely truncated Green's function
// (two even transforms), then the transform of its 2n-periodic extension
// (two more); z needs none (periodic, DFT wavevectors).  Normalized by
// 1/(Px Py Pz).  K0, K1 at kz R are evaluated here on the host (one pair per
// kz); J0, J1 on the device.
void build_wire_table(Shape* S, cudaStream_t st) {
  const int nx = S->grid.nx, ny = S->grid.ny, nz = S->grid.nz;
  const double hx = S->grid.hx, hy = S->grid.hy, hz = S->grid.hz;
  const int Mx = 4 * nx, My = 4 * ny;
  const int mx = Mx / 2 + 1, my = My / 2 + 1, mz = nz / 2 + 1;
  const double R = std::sqrt(std::pow(nx * hx, 2) + std::pow(ny * hy, 2));
  const double dkz = 2 * kPi / (nz * hz);
  const int hxo = nx + 1, hyo = ny + 1;
  std::vector<double> k0(mz, 0.0), k1(mz, 0.0);
  for (int k = 1; k < mz; ++k) {
    const double a = k * dkz * R;
    // K0, K1 below the smallest double for a > ~700; their terms vanish there
    if (a < 700.0) {
      k0[k] = std::cyl_bessel_k(0.0, a);
      k1[k] = std::cyl_bessel_k(1.0, a);
    }
  }
  DevMem tmp;
  auto up = [&](const std::vector<double>& h) {
    double* d = tmp.alloc<double>(h.size());
    ck(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    return d;
  };
  double* k0d = up(k0);
  double* k1d = up(k1);
  double* ghat = tmp.alloc<double>((size_t)mx * my * mz);
  launch_wire_ghat(ghat, mx, my, mz, 2 * kPi / (Mx * hx), 2 * kPi / (My * hy), dkz, R, k0d, k1d, st);
  double* cx = up(cosine_matrix(Mx, hxo, 1.0 / Mx));
  double* cy = up(cosine_matrix(My, hyo, 1.0 / My));
  double* t1 = tmp.alloc<double>((size_t)mz * my * hxo);
  launch_axis_matrix(ghat, t1, cx, mz * my, mx, 1, hxo, st);
  double* g = tmp.alloc<double>((size_t)mz * hyo * hxo);
  launch_axis_matrix(t1, g, cy, mz, my, hxo, hyo, st);
  double* dx = up(cosine_matrix(2 * nx, hxo, 1.0 / (2 * nx)));
  double* dy = up(cosine_matrix(2 * ny, hyo, 1.0 / (2.0 * ny * nz)));
  double* u1 = tmp.alloc<double>((size_t)mz * hyo * hxo);
  launch_axis_matrix(g, u1, dx, mz * hyo, hxo, 1, hxo, st);
  launch_axis_matrix(u1, S->table, dy, mz, hyo, hxo, hyo, st);
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
}

std::shared_ptr<Shape> build_shape(const gps_grid* gr, cudaStream_t st) {
  auto S = std::make_shared<Shape>();
  S->grid = *gr;
  const bool fx = gr->bc == GPS_BC_FREE || gr->bc == GPS_BC_WIRE;
  const bool fz = gr->bc == GPS_BC_FREE || gr->bc == GPS_BC_SURFACE;
  S->Px = fx ? 2 * gr->nx : gr->nx;
  S->Py = fx ? 2 * gr->ny : gr->ny;
  S->Pz = fz ? 2 * gr->nz : gr->nz;
  S->Hx = S->Px / 2 + 1;
  S->Hp = spectrum_pitch(S->Hx);
  S->n = (size_t)gr->nx * gr->ny * gr->nz;
  S->periodic = gr->bc == GPS_BC_PERIODIC;
  S->inv_p = 1.0 / ((double)S->Px * S->Py * S->Pz);
  PassGeom& g = S->g;
  g.nx = gr->nx; g.ny = gr->ny; g.nz = gr->nz;
  g.Px = S->Px; g.Py = S->Py; g.Pz = S->Pz; g.Hx = S->Hx; g.Hp = S->Hp;
  g.nrows = gr->ny * gr->nz;
  g.lines_x = batch_lines(S->Px, (g.nrows + 1) / 2);
  g.tile_y = batch_lines(S->Py, S->Hx * gr->nz);
  g.tile_z = batch_lines(S->Pz, S->Hx * S->Py);
  if (!make_sched(S->Px, &S->fx) || !make_sched(S->Py, &S->fy) || !make_sched(S->Pz, &S->fz))
    throw std::bad_alloc();
  for (auto& sp : S->sp) {
    sp.g = S->g;
    sp.fx = S->fx;
    sp.fy = S->fy;
    sp.fz = S->fz;
  }
  upload_twiddles(S.get(), S->Px, &S->twx64, &S->twx32, &S->twxdf);
  upload_twiddles(S.get(), S->Py, &S->twy64, &S->twy32, &S->twydf);
  upload_twiddles(S.get(), S->Pz, &S->twz64, &S->twz32, &S->twzdf);
  const int hy = S->Py / 2 + 1, hz = S->Pz / 2 + 1;
  const size_t tab = (size_t)S->Hx * hy * hz;
  S->table = S->mem.alloc<double>(tab);
  const double dkx = 2 * kPi / (S->Px * gr->hx), dky = 2 * kPi / (S->Py * gr->hy),
               dkz = 2 * kPi / (S->Pz * gr->hz);
  if (gr->bc == GPS_BC_PERIODIC) {
    S->lap = S->mem.alloc<double>(tab);
    launch_table_periodic(S->table, S->lap, S->Hx, hy, hz, dkx, dky, dkz, S->inv_p, st);
  } else if (gr->bc == GPS_BC_SURFACE) {
    launch_table_surface(S->table, S->Hx, hy, hz, dkx, dky, dkz, gr->nz * gr->hz, S->inv_p, st);
  } else if (gr->bc == GPS_BC_WIRE) {
    build_wire_table(S.get(), st);
  } else {
    build_free_table(S.get(), st);
  }
  S->table32 = S->mem.alloc<float>(tab);
  S->tabledf = S->mem.alloc<float2>(tab);
  launch_table_split(S->table, S->table32, S->tabledf, tab, st);
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
  return S;
}

// ------------------------------------------------------------------ pools --

}  // namespace

struct Request {
  gps_request req;
  unsigned long long ticket = 0;
  double t0 = 0.0;
  // set by the engine's thread after rep and status; read by the threads
  // that poll or wait on the ticket
  std::atomic<bool> done{false};
  int status = GPS_PENDING;
  gps_report rep{};
};

namespace {

// Work arrays of the comparison solvers (Algorithm 1, PSD, DIIS) on slot 0
// of a direct pool, allocated on first use.
struct ScWork {
  double *gx = nullptr, *gy = nullptr, *gz = nullptr, *isc = nullptr, *tmp = nullptr;
  double *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr;
  double *hist = nullptr;   // DIIS ring: phi, r, v blocks of hist_m * n
  int hist_m = 0;
  double *part = nullptr, *dpart = nullptr, *small = nullptr;
  unsigned int* cnt = nullptr;
  int pstride = 0;
};

struct Pool {
  std::shared_ptr<Shape> shape;
  int cap = 1;
  size_t n = 0, wn = 0;
  int pstride = 0;
  Fields f{};
  double *own_rho = nullptr, *own_eps = nullptr, *own_phi = nullptr, *own_gam = nullptr;
  double2* W64 = nullptr;
  float2* W32 = nullptr;
  double *partials = nullptr, *partials2 = nullptr, *partials3 = nullptr;
  SlotState* st = nullptr;
  SlotState* st_host = nullptr;
  int* active = nullptr;
  int* active_host = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool has_nlpb = false, has_mixed = false, has_cert = false, has_fp64 = false, has_df64 = false;
  std::vector<Request*> slot_req;
  std::map<int, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;
  unsigned long long last_use = 0;
  bool in_flight = false;     // engine: a round was launched and not yet collected
  // warm start: eps, phi and b - r of the last solve that asked for it (in
  // an engine pool: the last such request that completed in it), and the
  // flag of the same-eps test; ws_el (single solves) or ws_ion (engine
  // pools) identifies its electrolyte
  double *ws_eps = nullptr, *ws_phi = nullptr, *ws_d = nullptr;
  int* ws_flag = nullptr;
  bool ws_valid = false;
  int ws_kind = -1;
  gps_electrolyte ws_el{};
  IonParams ws_ion{};
  ScWork sc;
  double *dft_tmp = nullptr, *dft_part = nullptr;   // DFT-facing passes: scratch, partial sums
  DevMem mem;

  ~Pool() {
    for (auto& kv : graphs) {
      cudaGraphExecDestroy(kv.second.second);
      cudaGraphDestroy(kv.second.first);
    }
    if (st_host) cudaFreeHost(st_host);
    if (active_host) cudaFreeHost(active_host);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  int busy() const {
    int b = 0;
    for (auto* r : slot_req) b += r != nullptr;
    return b;
  }
};

size_t slot_bytes(const Shape& S) {
  const size_t wn = (size_t)S.Hp * S.Py * S.grid.nz;
  return 18 * S.n * sizeof(double) + S.n * sizeof(float) + wn * (sizeof(double2) + sizeof(float2)) +
         3 * 4096 * sizeof(double);
}

// Electrolyte parameters equal value by value (the warm-start test of
// served requests, whose electrolyte arrays may live at other addresses).
bool same_ion(const IonParams& a, const IonParams& b) {
  if (a.nspecies != b.nspecies || a.steric != b.steric || a.inv_kt != b.inv_kt ||
      a.inv_eps0m1 != b.inv_eps0m1 || a.exp_cap != b.exp_cap || a.lambda0 != b.lambda0)
    return false;
  for (int k = 0; k < a.nspecies && k < GPS_MAX_SPECIES; ++k)
    if (a.zq[k] != b.zq[k] || a.zn[k] != b.zn[k] || a.z2n_kt[k] != b.z2n_kt[k] || a.a[k] != b.a[k])
      return false;
  return true;
}

std::unique_ptr<Pool> make_pool(std::shared_ptr<Shape> shape, int cap, bool own_stream) {
  auto P = std::make_unique<Pool>();
  P->shape = shape;
  P->cap = cap;
  P->n = shape->n;
  P->wn = (size_t)shape->Hp * shape->Py * shape->grid.nz;
  P->pstride = std::max((shape->g.nrows + 1) / 2, vec_blocks(shape->n, cap)) + 32;
  const size_t N = P->n * cap;
  Fields& f = P->f;
  P->own_rho = f.rho = P->mem.alloc<double>(N);
  P->own_eps = f.eps = P->mem.alloc<double>(N);
  P->own_phi = f.phi = P->mem.alloc<double>(N);
  f.s = P->mem.alloc<double>(N);
  f.s32 = P->mem.alloc<float>(N);
  f.sq = P->mem.alloc<double>(N);
  f.q = P->mem.alloc<double>(N);
  f.qlam = P->mem.alloc<double>(N);
  f.r = P->mem.alloc<double>(N);
  f.p = P->mem.alloc<double>(N);
  f.Ap = P->mem.alloc<double>(N);
  f.v = P->mem.alloc<double>(N);
  f.rions = P->mem.alloc<double>(N);
  f.rp = P->mem.alloc<double>(N);
  f.fresh = P->mem.alloc<double>(N);
  f.lam = P->mem.alloc<double>(N);
  f.dphi = P->mem.alloc<double>(N);
  f.src = P->mem.alloc<double>(N);
  f.tmp = P->mem.alloc<double>(N);
  P->W64 = P->mem.alloc<double2>(P->wn * cap);
  P->W32 = P->mem.alloc<float2>(P->wn * cap);
  P->partials = P->mem.alloc<double>((size_t)P->pstride * cap);
  P->partials2 = P->mem.alloc<double>((size_t)P->pstride * cap);
  P->partials3 = P->mem.alloc<double>((size_t)P->pstride * cap);
  P->st = P->mem.alloc<SlotState>(cap);
  P->active = P->mem.alloc<int>(cap + 1);
  ck(cudaMemset(P->st, 0, sizeof(SlotState) * cap));
  ck(cudaMemset(P->active, 0, sizeof(int) * (cap + 1)));
  ck(cudaMallocHost((void**)&P->st_host, sizeof(SlotState) * cap));
  ck(cudaMallocHost((void**)&P->active_host, sizeof(int) * (cap + 1)));
  std::memset(P->st_host, 0, sizeof(SlotState) * cap);
  std::memset(P->active_host, 0, sizeof(int) * (cap + 1));
  P->slot_req.assign(cap, nullptr);
  if (own_stream) {
    ck(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    P->own_stream = true;
  }
  return P;
}

Batch batch_of(Pool& P, int phase, int prec) {
  Batch b;
  b.active = P.active;
  b.st = P.st;
  b.phase = phase;
  b.prec = prec;
  b.vstride = P.n;
  b.partials = P.partials;
  b.partials2 = P.partials2;
  b.partials3 = P.partials3;
  b.pstride = P.pstride;
  b.acted = nullptr;
  return b;
}

template <typename V> constexpr int spec_of() {
  return std::is_same<V, double2>::value ? SPEC_FP64 : std::is_same<V, float2>::value ? SPEC_FP32 : SPEC_DF64;
}

// One spectrum pipeline (five passes) for the slots of `b`.
template <typename V>
void pipeline(Pool& P, const Batch& b, PipeArgs a, cudaStream_t st) {
  const Shape& S = *P.shape;
  const V *twx, *twy, *twz;
  if constexpr (std::is_same<V, double2>::value) {
    twx = reinterpret_cast<const V*>(S.twx64);
    twy = reinterpret_cast<const V*>(S.twy64);
    twz = reinterpret_cast<const V*>(S.twz64);
    a.W = P.W64;
  } else if constexpr (std::is_same<V, dfc>::value) {
    twx = S.twxdf;
    twy = S.twydf;
    twz = S.twzdf;
    a.W = P.W64;   // same 16 bytes per complex; a slot uses one of the two at a time
  } else {
    twx = reinterpret_cast<const V*>(S.twx32);
    twy = reinterpret_cast<const V*>(S.twy32);
    twz = reinterpret_cast<const V*>(S.twz32);
    a.W = P.W32;
  }
  a.wstride = P.wn;
  const int ns = P.cap;
  const Shape::Sched& sc = S.sp[spec_of<V>()];
  // profile kinds of the passes: 0-4 FP64 spectrum, 10-14 df64, 15-19 FP32
  constexpr int k0 = spec_of<V>() == SPEC_FP64 ? 0 : spec_of<V>() == SPEC_DF64 ? 10 : 15;
  timed(k0 + 0, b, st, [&](const Batch& bb) { launch_x_fwd<V>(sc.g, sc.fx, twx, bb, a, ns, st); });
  timed(k0 + 1, b, st, [&](const Batch& bb) { launch_y<V>(sc.g, sc.fy, twy, bb, a, false, ns, st); });
  timed(k0 + 2, b, st, [&](const Batch& bb) { launch_z<V>(sc.g, sc.fz, twz, bb, a, ns, st); });
  timed(k0 + 3, b, st, [&](const Batch& bb) { launch_y<V>(sc.g, sc.fy, twy, bb, a, true, ns, st); });
  timed(k0 + 4, b, st, [&](const Batch& bb) { launch_x_inv<V>(sc.g, sc.fx, twx, bb, a, ns, st); });
}

// ------------------------------------------------------------- autotuner --
//
// For every grid and spectrum precision the lines per CTA of the x passes,
// the columns per CTA of the y and z passes and the radix order of each axis
// are chosen by timing the passes on the device (1 warm-up + 3 timed
// launches each, fastest kept).  Results are cached for the process, keyed by
// grid and precision, so every solve of a grid -- alone or batched -- uses
// the same schedule (and therefore the same rounding).

struct TuneKey {
  int nx, ny, nz, bc, spec;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, bc, spec) < std::tie(o.nx, o.ny, o.nz, o.bc, o.spec);
  }
};
struct TuneVal {
  PassGeom g;
  FftSched fx, fy, fz;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
int g_radix_order = -1;   // gps_set_radix_order: -1 tunes the radix order, else this one
int g_x_kernel = -1;      // gps_set_x_kernel: -1 tuned, 0 shared-memory, 1 register-resident (FP32)
int g_z_kernel = -1;      // gps_set_z_kernel: -1 tuned, 0 plain column kernel, 1 TMA-staged (FP32, df64)
int g_engine_async = 1;   // gps_set_engine_mode: 1 pools advance independently, 0 in lockstep

template <typename F>
float time_launch(F&& launch, cudaStream_t st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up launch, timed: long launches (> 1 ms, large grids) vary little
  // between repetitions, so one more is enough; short ones take the best of 3
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float warm = 0.f;
  cudaEventElapsedTime(&warm, e0, e1);
  const int reps = warm > 1.0f ? 1 : warm > 0.1f ? 3 : 7;
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ck(cudaGetLastError());
  return best;
}

// Lines (x passes) or columns (y, z passes) per CTA to try: every count from
// 1 to 16 that fits in shared memory.  Counts that are not powers of two
// matter: they set how full the last wave of CTAs is (at 128^3 the power-of-
// two choices leave 1.7-1.9 waves).  fixed: the pass runs a kernel with its
// own tiling (register-resident kernels), so only the heuristic is kept.
std::vector<int> batch_candidates(int b0, int L, size_t vbytes, bool fixed) {
  std::vector<int> c;
  if (fixed) {
    c.push_back(b0 < 1 ? 1 : b0);
    return c;
  }
  for (int b = 1; b <= kMaxLinesPerCta; ++b)
    if (x_lines_smem_bytes(L, b, vbytes) <= kMaxLinesSmem) c.push_back(b);
  if (c.empty()) c.push_back(1);
  return c;
}

// The radix orders the tuner may try for a transform of length L: all of
// them, or the one gps_set_radix_order chose (order 0 where that one does
// not apply to L).
bool order_allowed(int L, int order, int norders) {
  if (g_radix_order < 0) return true;
  FftSched tmp;
  const bool applies = g_radix_order < norders && make_sched(L, &tmp, g_radix_order);
  return order == (applies ? g_radix_order : 0);
}

template <typename V>
void tune_spec(Shape& S, cudaStream_t st) {
  constexpr int sp = spec_of<V>();
  Shape::Sched& out = S.sp[sp];
  if (out.tuned) return;
  const TuneKey key{S.grid.nx, S.grid.ny, S.grid.nz, S.grid.bc, sp};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto hit = g_tune.find(key);
  if (hit == g_tune.end()) {
    const V *twx, *twy, *twz;
    if constexpr (std::is_same<V, double2>::value) {
      twx = reinterpret_cast<const V*>(S.twx64);
      twy = reinterpret_cast<const V*>(S.twy64);
      twz = reinterpret_cast<const V*>(S.twz64);
    } else if constexpr (std::is_same<V, dfc>::value) {
      twx = S.twxdf;
      twy = S.twydf;
      twz = S.twzdf;
    } else {
      twx = reinterpret_cast<const V*>(S.twx32);
      twy = reinterpret_cast<const V*>(S.twy32);
      twz = reinterpret_cast<const V*>(S.twz32);
    }
    DevMem tmp;
    const size_t wn = (size_t)S.Hp * S.Py * S.grid.nz;
    V* W = tmp.alloc<V>(wn);
    double* in = tmp.alloc<double>(S.n);
    double* outv = tmp.alloc<double>(S.n);
    double* sc = tmp.alloc<double>(S.n);
    float* sc32 = tmp.alloc<float>(S.n);
    ck(cudaMemsetAsync(in, 0, S.n * sizeof(double), st));
    ck(cudaMemsetAsync(sc, 0, S.n * sizeof(double), st));
    ck(cudaMemsetAsync(sc32, 0, S.n * sizeof(float), st));
    ck(cudaMemsetAsync(W, 0, wn * sizeof(V), st));
    Batch b{};
    PipeArgs a{};
    // the arrays the PCG's passes read: scale factors (FP64 and the FP32
    // copy) on both sides and r for (v, r), so that candidates are timed on
    // the loads they will do
    a.in = in;
    a.out = outv;
    a.in_scale = sc;
    a.out_scale = sc;
    a.in_scale32 = sc32;
    a.out_scale32 = sc32;
    a.dot_with = in;
    a.table = S.table;
    a.table32 = S.table32;
    a.tabledf = S.tabledf;
    a.W = W;
    TuneVal best;
    best.g = S.g;
    best.fx = S.fx;
    best.fy = S.fy;
    best.fz = S.fz;
    // passes served by the register-resident kernels (fixed tiling, compile-time radix plan)
    const bool f64 = std::is_same<V, double2>::value;
    const bool fixx = std::is_same<V, dfc>::value && col_pass_supported(S.Px);
    const bool fixy = !f64 && col_pass_supported(S.Py);
    const bool fixz = !f64 && col_pass_supported(S.Pz);
    // radix orders: 8s first, 8s last, 4s, and for FP64 16s first
    const int norders = f64 ? 4 : 3;
    // x passes: lines per CTA and radix order of Px
    float tbest = 1e30f;
    best.g.x_reg = 0;
    for (int lines : batch_candidates(S.g.lines_x, S.Px, sizeof(V), fixx))
      for (int order = 0; order < (fixx ? 1 : norders); ++order) {
        if (!fixx && !order_allowed(S.Px, order, norders)) continue;
        PassGeom g = best.g;
        g.lines_x = lines;
        FftSched fx;
        if (!make_sched(S.Px, &fx, order)) continue;
        const float t = time_launch([&] { launch_x_fwd<V>(g, fx, twx, b, a, 1, st); }, st) +
                        time_launch([&] { launch_x_inv<V>(g, fx, twx, b, a, 1, st); }, st);
        if (t < tbest) { tbest = t; best.g.lines_x = lines; best.fx = fx; }
      }
    // FP32 spectrum: the register-resident x kernels (power-of-two Px) as
    // one more candidate against the shared-memory ones
    if (std::is_same<V, float2>::value && col_pass_supported(S.Px) && g_x_kernel != 0) {
      PassGeom g = best.g;
      g.x_reg = 1;
      const float t = time_launch([&] { launch_x_fwd<V>(g, best.fx, twx, b, a, 1, st); }, st) +
                      time_launch([&] { launch_x_inv<V>(g, best.fx, twx, b, a, 1, st); }, st);
      if (t < tbest || g_x_kernel == 1) { tbest = t; best.g.x_reg = 1; }
    }
    tbest = 1e30f;
    for (int tile : batch_candidates(S.g.tile_y, S.Py, sizeof(V), fixy))
      for (int order = 0; order < (fixy ? 1 : norders); ++order) {
        if (!fixy && !order_allowed(S.Py, order, norders)) continue;
        PassGeom g = best.g;
        g.tile_y = tile;
        FftSched fy;
        if (!make_sched(S.Py, &fy, order)) continue;
        const float t = time_launch([&] { launch_y<V>(g, fy, twy, b, a, false, 1, st); }, st) +
                        time_launch([&] { launch_y<V>(g, fy, twy, b, a, true, 1, st); }, st);
        if (t < tbest) { tbest = t; best.g.tile_y = tile; best.fy = fy; }
      }
    tbest = 1e30f;
    best.g.z_tma = 0;
    for (int tile : batch_candidates(S.g.tile_z, S.Pz, sizeof(V), fixz))
      for (int order = 0; order < (fixz ? 1 : norders); ++order) {
        if (!fixz && !order_allowed(S.Pz, order, norders)) continue;
        PassGeom g = best.g;
        g.tile_z = tile;
        FftSched fz;
        if (!make_sched(S.Pz, &fz, order)) continue;
        const float t = time_launch([&] { launch_z<V>(g, fz, twz, b, a, 1, st); }, st);
        if (t < tbest) { tbest = t; best.g.tile_z = tile; best.fz = fz; }
      }
    // column kernels: the TMA-staged z pass as one more candidate
    if (fixz && g_z_kernel != 0) {
      PassGeom g = best.g;
      g.z_tma = 1;
      const float t = time_launch([&] { launch_z<V>(g, best.fz, twz, b, a, 1, st); }, st);
      if (t < tbest || g_z_kernel == 1) { tbest = t; best.g.z_tma = 1; }
    }
    ck(cudaStreamSynchronize(st));
    hit = g_tune.emplace(key, best).first;
  }
  out.g = hit->second.g;
  out.fx = hit->second.fx;
  out.fy = hit->second.fy;
  out.fz = hit->second.fz;
  out.tuned = true;
}

// Tune the spectrum precisions a launch sequence may use (FP64 is always
// needed: setup of periodic q and the certificate run in FP64).  Must run
// outside stream capture.
void ensure_tuned(Shape& S, bool fp32, bool df64, cudaStream_t st) {
  tune_spec<double2>(S, st);
  if (fp32) tune_spec<float2>(S, st);
  if (df64) tune_spec<dfc>(S, st);
}

void launch_setup_group(Pool& P, cudaStream_t st) {
  const Shape& S = *P.shape;
  const Batch b = batch_of(P, PH_SETUP, -1);
  timed(7, b, st, [&](const Batch& bb) { launch_setup_s(bb, P.f, P.n, P.cap, st); });
  if (S.periodic) {
    PipeArgs a{};
    a.in = P.f.sq;
    a.out = P.f.q;
    a.out_scale = P.f.sq;
    a.table = S.lap;
    pipeline<double2>(P, b, a, st);
  } else {
    const int per_xy = S.grid.bc == GPS_BC_SURFACE ? 1 : 0;   // surface: x, y wrap; z free
    const int per_z = S.grid.bc == GPS_BC_WIRE ? 1 : 0;       // wire: z wraps; x, y free
    launch_fd16_q(b, P.f, S.grid.nx, S.grid.ny, S.grid.nz, S.grid.hx, S.grid.hy, S.grid.hz, per_xy,
                  per_xy, per_z, fd16_coeffs(), P.cap, st);
  }
}

// One round: every stage of the phase machine once and `m` PCG iterations.
void launch_round(Pool& P, int m, bool setup, bool init, cudaStream_t st) {
  const Shape& S = *P.shape;
  const size_t n = P.n;
  const int ns = P.cap;
  const Fields& f = P.f;
  const int periodic = S.periodic;
  if (setup) {
    launch_setup_group(P, st);
    launch_setup_final(batch_of(P, PH_SETUP, -1), f, n, S.inv_p, periodic, ns, st);
  }
  if (P.has_nlpb) launch_nl_eval(batch_of(P, PH_NLEVAL, -1), f, n, S.inv_p, periodic, ns, st);
  if (init || P.has_nlpb) launch_init(batch_of(P, PH_INIT, -1), f, n, ns, st);
  PipeArgs it{};
  it.in = f.r;
  it.in_scale = f.s;
  it.out = f.v;
  it.out_scale = f.s;
  it.dot_with = f.r;
  it.table = S.table;
  it.table32 = S.table32;
  it.tabledf = S.tabledf;
  it.slot_k0 = 1;
  it.red_mu = periodic;
  it.red_wsum = periodic;
  it.in_scale32 = f.s32;
  it.out_scale32 = f.s32;
  const Batch bi64 = batch_of(P, PH_ITER, SPEC_FP64), bi32 = batch_of(P, PH_ITER, SPEC_FP32);
  const Batch bidf = batch_of(P, PH_ITER, SPEC_DF64);
  const Batch bi = batch_of(P, PH_ITER, -1);
  for (int i = 0; i < m; ++i) {
    if (P.has_fp64) pipeline<double2>(P, bi64, it, st);
    if (P.has_df64) pipeline<dfc>(P, bidf, it, st);
    if (P.has_mixed) pipeline<float2>(P, bi32, it, st);
    timed(5, bi, st, [&](const Batch& bb) { launch_update_p(bb, f, n, periodic, ns, st); });
    timed(6, bi, st, [&](const Batch& bb) { launch_update_r(bb, f, n, ns, st); });
  }
  if (P.has_nlpb) {
    launch_nl_step(batch_of(P, PH_TRIAL, -1), f, n, 0, ns, st);
    launch_nl_step(batch_of(P, PH_COMMIT, -1), f, n, 1, ns, st);
  }
  if (P.has_cert) {
    const Batch bc = batch_of(P, PH_CERT, -1);
    launch_fp_source(bc, f, n, ns, st);
    PipeArgs c{};
    c.in = f.tmp;
    c.in_scale = f.s;
    c.out = f.Ap;
    c.out_scale = f.s;
    c.table = S.table;
    c.table32 = S.table32;
    c.tabledf = S.tabledf;
    c.slot_k0 = 1;
    pipeline<double2>(P, bc, c, st);
    launch_fp_residual(bc, f, n, periodic, ns, st);
  }
}

// The slot state of a new request.
// kind GPS_MPB runs as GPS_NLPB with the steric ionic charge.
SlotState initial_state(int kind, const gps_electrolyte* el, const gps_opts& o) {
  SlotState s;
  std::memset(&s, 0, sizeof(s));
  const bool steric = kind == GPS_MPB;
  if (steric) kind = GPS_NLPB;
  s.ion = ion_params(kind == GPS_GPE ? nullptr : el, steric);
  s.phase = PH_SETUP;
  s.kind = kind;
  s.status = GPS_OK;
  s.tol_abs = o.tol_abs;
  s.tol_rel = o.tol_rel;
  s.max_iter = o.max_iter > 0 ? o.max_iter : 1;
  const bool df = o.precision == GPS_DF64 || o.precision == GPS_MIXED_DF64;
  s.spec_hi = df ? SPEC_DF64 : SPEC_FP64;
  s.spec = s.spec_hi;
  s.mixed = (o.precision == GPS_MIXED || o.precision == GPS_MIXED_DF64) ? 1 : 0;
  s.mixed_req = s.mixed;
  s.mixed_switch = o.mixed_switch;
  s.certify = (o.certify || s.mixed) ? 1 : 0;
  s.newton = o.outer_mode == GPS_OUTER_NEWTON ? 1 : 0;
  s.eta = o.eta;
  s.forcing = o.forcing;
  s.forcing_ew = o.forcing_rule == GPS_FORCING_EW2 ? 1 : 0;
  s.F_prev = -1.0;
  s.eta_prev = 0.0;
  s.tol_outer = o.tol_outer;
  s.max_outer = o.max_outer;
  s.neutralize = kind == GPS_GPE ? 1 : 0;
  s.cert = -1.0;
  s.F0 = -1.0;
  return s;
}

void fill_report(gps_report* rep, const SlotState& s, double t0) {
  if (!rep) return;
  std::memset(rep, 0, sizeof(*rep));
  rep->status = s.status;
  rep->iters = s.iters_total;
  rep->outer_iters = s.outer;
  rep->fp64_iters = s.fp64_iters;
  rep->res0 = std::sqrt(s.rr0);
  rep->res = std::sqrt(s.rr);
  rep->outer_res = s.F;
  rep->background = s.background;
  rep->fixed_point_res = s.cert;
  rep->time_ms = now_ms() - t0;
  rep->warm = s.warm;
}

void put_state(Pool& P, int slot, const SlotState& s, cudaStream_t st) {
  P.st_host[slot] = s;
  ck(cudaMemcpyAsync(P.st + slot, P.st_host + slot, sizeof(SlotState), cudaMemcpyHostToDevice, st));
}

void put_active(Pool& P, cudaStream_t st) {
  int c = 0;
  for (int k = 0; k < P.cap; ++k)
    if (P.slot_req[k]) P.active_host[1 + c++] = k;
  P.active_host[0] = c;
  ck(cudaMemcpyAsync(P.active, P.active_host, sizeof(int) * (P.cap + 1), cudaMemcpyHostToDevice, st));
}

void get_states(Pool& P, cudaStream_t st) {
  ck(cudaMemcpyAsync(P.st_host, P.st, sizeof(SlotState) * P.cap, cudaMemcpyDeviceToHost, st));
}

// Engine: continuous batching over pools of one device.
struct Engine {
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  std::vector<std::shared_ptr<Shape>> shapes;
  std::vector<std::unique_ptr<Pool>> pools;
  std::deque<Request*> queue;
  unsigned long long clock = 0;
  int max_concurrent = 0;
  bool use_graphs = true;
  unsigned long long finished_total = 0;   // requests completed (solved or failed) so far

  size_t bytes() const {
    size_t b = 0;
    for (auto& s : shapes) b += s->mem.bytes;
    for (auto& p : pools) b += p->mem.bytes;
    return b;
  }

  int capacity_for(const Shape& S) const {
    int c = (int)std::lround(4.0e6 / (double)S.n);
    c = std::max(2, std::min(16, c));
    if (max_slots > 0) c = std::min(c, max_slots);
    return c;
  }

  // Pool for a request's grid: an existing one with a free slot, or a new one
  // if the budget allows (evicting idle pools first).  nullptr: not now.
  Pool* pool_for(const gps_grid& g) {
    for (auto& p : pools)
      if (same_grid(p->shape->grid, g) && p->busy() < p->cap && !p->in_flight) return p.get();
    for (auto& p : pools)
      if (same_grid(p->shape->grid, g)) return nullptr;   // full or mid-round: wait for it
    std::shared_ptr<Shape> shape;
    for (auto& s : shapes)
      if (same_grid(s->grid, g)) shape = s;
    if (!shape) {
      shape = build_shape(&g, nullptr);
      shapes.push_back(shape);
    }
    const int cap = capacity_for(*shape);
    const size_t need = slot_bytes(*shape) * cap;
    while (budget && bytes() + need > budget) {
      int victim = -1;
      bool any_busy = false;
      for (size_t i = 0; i < pools.size(); ++i) {
        any_busy |= pools[i]->busy() > 0;
        if (pools[i]->busy() == 0 && (victim < 0 || pools[i]->last_use < pools[victim]->last_use))
          victim = (int)i;
      }
      if (victim < 0) {
        if (any_busy) return nullptr;   // memory frees when a busy pool drains: wait
        throw std::bad_alloc();         // the request can never fit the budget
      }
      pools.erase(pools.begin() + victim);
    }
    pools.push_back(make_pool(shape, cap, true));
    // warm starts of this pool's requests: INIT reads phi_0 and
    // b_prev - r_prev from the slot's own phi and A p (see admit)
    Fields& f = pools.back()->f;
    f.wphi = f.phi;
    f.wd = f.Ap;
    return pools.back().get();
  }

  // Warm start of a batched or served request (opts.warm_start; GPe and
  // linear PB, as for single solves): from the pool's retained state -- eps,
  // phi and b - r of the last warm-start request of the same kind and
  // electrolyte that completed in this pool -- when the request's eps equals
  // the retained one value by value.  phi_0 and b_prev - r_prev go into the
  // slot's own phi and A p, where INIT reads them (engine pools have
  // Fields wphi = phi, wd = Ap); nothing between admission and INIT writes
  // either for these kinds.
  static bool warm_request(const gps_request& q) {
    return q.opts.warm_start && (q.kind == GPS_GPE || q.kind == GPS_LPB);
  }

  static bool warm_from_retained(Pool& P, int k, const SlotState& s) {
    if (!P.ws_valid || P.ws_kind != s.kind || !same_ion(P.ws_ion, s.ion)) return false;
    int differ = 1;
    ck(cudaMemsetAsync(P.ws_flag, 0, sizeof(int), P.stream));
    launch_eps_differ(P.f.eps + k * P.n, P.ws_eps, P.n, P.ws_flag, P.stream);
    ck(cudaMemcpyAsync(&differ, P.ws_flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    ck(cudaStreamSynchronize(P.stream));
    if (differ) return false;
    const size_t b = P.n * sizeof(double);
    ck(cudaMemcpyAsync(P.f.phi + k * P.n, P.ws_phi, b, cudaMemcpyDeviceToDevice, P.stream));
    ck(cudaMemcpyAsync(P.f.Ap + k * P.n, P.ws_d, b, cudaMemcpyDeviceToDevice, P.stream));
    return true;
  }

  // Keeps slot k's finished warm-start request as the pool's retained state
  // (three more fields of the pool's size; none if they cannot be had).
  static void retain(Pool& P, int k, const SlotState& s) {
    if (!P.ws_eps) {
      try {
        double* e = P.mem.alloc<double>(P.n);
        double* f = P.mem.alloc<double>(P.n);
        double* d = P.mem.alloc<double>(P.n);
        int* fl = P.mem.alloc<int>(1);
        P.ws_eps = e;
        P.ws_phi = f;
        P.ws_d = d;
        P.ws_flag = fl;
      } catch (std::bad_alloc&) {
        return;   // what was allocated stays with the pool until it is freed
      }
    }
    launch_warm_store(batch_of(P, PH_DONE, -1), P.f, k, P.ws_eps, P.ws_phi, P.ws_d, P.n, P.stream);
    P.ws_valid = true;
    P.ws_kind = s.kind;
    P.ws_ion = s.ion;
  }

  void admit(Pool& P, Request* r) {
    int k = 0;
    while (P.slot_req[k]) ++k;
    P.slot_req[k] = r;
    const gps_request& q = r->req;
    const size_t b = P.n * sizeof(double);
    ck(cudaMemcpyAsync(P.f.rho + k * P.n, q.rho_host, b, cudaMemcpyHostToDevice, P.stream));
    ck(cudaMemcpyAsync(P.f.eps + k * P.n, q.eps_host, b, cudaMemcpyHostToDevice, P.stream));
    SlotState s = initial_state(q.kind, &q.el, q.opts);
    if (warm_request(q) && warm_from_retained(P, k, s)) s.warm = 1;
    put_state(P, k, s, P.stream);
    P.has_nlpb |= q.kind == GPS_NLPB || q.kind == GPS_MPB;
    P.has_mixed |= s.mixed != 0;
    P.has_cert |= s.certify != 0;
    P.has_fp64 |= s.spec_hi == SPEC_FP64;
    P.has_df64 |= s.spec_hi == SPEC_DF64;
  }

  // PCG iterations per round: more for small pools, whose iterations are
  // short, so that a round amortizes its host-side state read (and
  // admission) over at least about a millisecond of device work; fewer with
  // nonlinear-PB slots, whose line-search trials take one round each.
  static int round_iters(const Pool& P) {
    if (!g_engine_async) return 4;
    const double pts = (double)P.n * std::max(1, P.busy());
    const int m = pts >= 2.0e6 ? 4 : pts >= 5.0e5 ? 8 : 16;
    return P.has_nlpb ? std::min(m, 8) : m;
  }

  void run_round(Pool& P) {
    ensure_tuned(*P.shape, P.has_mixed, P.has_df64, P.stream);
    put_active(P, P.stream);
    const int m = round_iters(P);
    // Pipelines of this round: the FP32 one if a slot iterates in (or, for
    // mixed nonlinear PB, may enter) FP32, a high-precision one if a slot is
    // in (or, for nonlinear PB, may return to) that precision.  A slot that switches in mid-round waits for the
    // next round (the update kernels act only after their pipeline ran).
    const bool acc_mixed = P.has_mixed, acc_fp64 = P.has_fp64, acc_df64 = P.has_df64;
    bool lo = false, h64 = false, hdf = false;
    for (int k = 0; k < P.cap; ++k) {
      if (!P.slot_req[k]) continue;
      const SlotState& s = P.st_host[k];
      if (s.phase == PH_DONE || s.phase == PH_IDLE) continue;
      const bool in_lo = s.spec == SPEC_FP32;
      // a mixed nonlinear-PB slot may enter FP32 at any inner solve
      lo |= in_lo || (s.kind == GPS_NLPB && s.mixed_req);
      if (!in_lo || s.kind == GPS_NLPB) (s.spec_hi == SPEC_FP64 ? h64 : hdf) = true;
    }
    P.has_mixed = acc_mixed && lo;
    P.has_fp64 = acc_fp64 && h64;
    P.has_df64 = acc_df64 && hdf;
    const int key = (P.has_nlpb ? 1 : 0) | (P.has_mixed ? 2 : 0) | (P.has_cert ? 4 : 0) |
                    (P.has_fp64 ? 8 : 0) | (P.has_df64 ? 16 : 0) | (m << 5);
    const bool graphs_ok = use_graphs && !(t_prof && t_prof->on);
    if (graphs_ok) {
      auto it = P.graphs.find(key);
      if (it == P.graphs.end()) {
        cudaGraph_t g;
        cudaGraphExec_t ge;
        ck(cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeRelaxed));
        launch_round(P, m, true, true, P.stream);
        ck(cudaStreamEndCapture(P.stream, &g));
        ck(cudaGraphInstantiate(&ge, g, 0));
        it = P.graphs.emplace(key, std::make_pair(g, ge)).first;
      }
      ck(cudaGraphLaunch(it->second.second, P.stream));
    } else {
      launch_round(P, m, true, true, P.stream);
    }
    P.has_mixed = acc_mixed;
    P.has_fp64 = acc_fp64;
    P.has_df64 = acc_df64;
    get_states(P, P.stream);
  }

  // Copy out and release the finished slots of P (after its stream synced).
  int collect(Pool& P) {
    int finished = 0;
    for (int k = 0; k < P.cap; ++k) {
      Request* r = P.slot_req[k];
      if (!r) continue;
      const SlotState s = P.st_host[k];
      if (s.phase != PH_DONE) continue;
      ck(cudaMemcpyAsync(r->req.phi_host, P.f.phi + k * P.n, P.n * sizeof(double),
                         cudaMemcpyDeviceToHost, P.stream));
      if (warm_request(r->req) && (s.status == GPS_OK || s.status == GPS_ERR_NOT_CONVERGED)) retain(P, k, s);
      ck(cudaStreamSynchronize(P.stream));
      fill_report(&r->rep, s, r->t0);
      r->status = s.status;
      r->done = true;
      ++finished_total;
      P.slot_req[k] = nullptr;
      SlotState idle;
      std::memset(&idle, 0, sizeof(idle));
      put_state(P, k, idle, P.stream);
      ++finished;
    }
    return finished;
  }

  // Admit what fits, advance every busy pool by one round, collect.
  // Returns the number of requests still queued or in slots.
  size_t step() {
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = *it;
      int v = validate_grid(&r->req.grid);
      if (v == GPS_OK && r->req.kind != GPS_GPE) v = validate_el(&r->req.el);
      if (v == GPS_OK && (r->req.kind < GPS_GPE || r->req.kind > GPS_MPB)) v = GPS_ERR_INVALID;
      if (v == GPS_OK && r->req.kind == GPS_MPB) v = validate_steric(&r->req.el);
      if (v == GPS_OK && r->req.opts.method != GPS_PCG) v = GPS_ERR_INVALID;   // single solves only
      if (v == GPS_OK && r->req.opts.forcing_rule != GPS_FORCING_EW2 && r->req.opts.forcing_rule != GPS_FORCING_RATIO)
        v = GPS_ERR_INVALID;
      if (v == GPS_OK && r->req.el.exclusion) v = GPS_ERR_INVALID;            // single solves only
      if (v == GPS_OK && (!r->req.rho_host || !r->req.eps_host || !r->req.phi_host)) v = GPS_ERR_INVALID;
      if (v != GPS_OK) {
        r->status = v;
        r->rep.status = v;
        r->done = true;
        ++finished_total;
        it = queue.erase(it);
        continue;
      }
      Pool* P = nullptr;
      try {
        P = pool_for(r->req.grid);
      } catch (std::bad_alloc&) {
        P = nullptr;
        bool any_busy = false;
        for (auto& p : pools) any_busy |= p->busy() > 0;
        if (!any_busy) {   // nothing will free memory: fail the request
          r->status = GPS_ERR_NOMEM;
          r->rep.status = GPS_ERR_NOMEM;
          r->done = true;
          ++finished_total;
          it = queue.erase(it);
          continue;
        }
      }
      if (P) {
        admit(*P, r);
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
    int busy_total = 0;
    for (auto& p : pools) busy_total += p->busy();
    max_concurrent = std::max(max_concurrent, busy_total);
    if (!g_engine_async) {
      // lockstep: one round on every busy pool, then every pool is synced
      for (auto& p : pools)
        if (p->busy()) {
          p->last_use = ++clock;
          run_round(*p);
        }
      for (auto& p : pools)
        if (p->busy()) {
          ck(cudaStreamSynchronize(p->stream));
          collect(*p);
        }
      size_t left = queue.size();
      for (auto& p : pools) left += p->busy();
      return left;
    }
    // Pools advance independently: a pool whose round has finished on its
    // stream is collected and, if it still has work, gets its next round at
    // once, while the rounds of the other pools keep running.
    bool progressed = false;
    for (auto& p : pools) {
      if (p->in_flight) {
        const cudaError_t q = cudaStreamQuery(p->stream);
        if (q == cudaErrorNotReady) continue;
        ck(q);
        p->in_flight = false;
        collect(*p);
        progressed = true;
        // queued requests of this grid (validated above) take the freed slots
        // before the pool's next round
        for (auto it = queue.begin(); it != queue.end() && p->busy() < p->cap;) {
          if (same_grid((*it)->req.grid, p->shape->grid)) {
            admit(*p, *it);
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      if (p->busy()) {
        p->last_use = ++clock;
        run_round(*p);
        p->in_flight = true;
        progressed = true;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    size_t left = queue.size();
    for (auto& p : pools) left += p->busy();
    return left;
  }
};

}  // namespace

// ----------------------------------------------------------- the context --

struct gps_ctx {
  Profiler prof;
  int device = 0;
  size_t budget = 0;
  std::vector<std::shared_ptr<Shape>> shapes;
  std::vector<std::unique_ptr<Pool>> direct;   // one-slot pools of the single-solve path
  unsigned long long clock = 0;
  size_t in_use() const {
    size_t b = 0;
    for (auto& s : shapes) b += s->mem.bytes;
    for (auto& p : direct) b += p->mem.bytes;
    return b;
  }
};

namespace {

std::shared_ptr<Shape> get_shape(std::vector<std::shared_ptr<Shape>>& shapes, const gps_grid* gr,
                                 cudaStream_t st) {
  for (auto& s : shapes)
    if (same_grid(s->grid, *gr)) return s;
  auto s = build_shape(gr, st);
  shapes.push_back(s);
  return s;
}

// Single solve in the context's one-slot pool of this grid, on `st`.
// rho/eps/phi are device pointers (the caller's, or the pool's own).
int solve_direct(Pool& P, const double* rho, const double* eps, double* phi, int kind,
                 const gps_electrolyte* el, const gps_opts& o, gps_report* rep, cudaStream_t st,
                 double t0) {
  P.f.rho = const_cast<double*>(rho);
  P.f.eps = const_cast<double*>(eps);
  P.f.phi = phi;
  P.slot_req[0] = reinterpret_cast<Request*>(&P);   // marks slot 0 busy
  SlotState s = initial_state(kind, el, o);
  // warm start: same kind, same electrolyte (LPB) and eps equal value by
  // value to the previous warm-start solve's
  const bool keep = o.warm_start && kind != GPS_NLPB && kind != GPS_MPB && !(el && el->exclusion);
  P.f.gam = (kind != GPS_GPE && el) ? el->exclusion : nullptr;
  P.f.wphi = nullptr;
  P.f.wd = nullptr;
  if (keep) {
    if (!P.ws_eps) {
      P.ws_eps = P.mem.alloc<double>(P.n);
      P.ws_phi = P.mem.alloc<double>(P.n);
      P.ws_d = P.mem.alloc<double>(P.n);
      P.ws_flag = P.mem.alloc<int>(1);
    }
    bool same = P.ws_valid && P.ws_kind == kind;
    if (same && kind == GPS_LPB) same = el && std::memcmp(el, &P.ws_el, sizeof(gps_electrolyte)) == 0;
    if (same) {
      int differ = 1;
      ck(cudaMemsetAsync(P.ws_flag, 0, sizeof(int), st));
      launch_eps_differ(eps, P.ws_eps, P.n, P.ws_flag, st);
      ck(cudaMemcpyAsync(&differ, P.ws_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      if (!differ) {
        s.warm = 1;
        P.f.wphi = P.ws_phi;
        P.f.wd = P.ws_d;
      }
    }
  }
  put_state(P, 0, s, st);
  P.has_nlpb = kind == GPS_NLPB || kind == GPS_MPB;
  P.has_mixed = s.mixed != 0;
  P.has_cert = s.certify != 0;
  P.has_fp64 = s.spec_hi == SPEC_FP64;
  P.has_df64 = s.spec_hi == SPEC_DF64;
  put_active(P, st);
  ensure_tuned(*P.shape, P.has_mixed, P.has_df64, st);
  // A single GPe / LPB solve runs the pipeline of its current spectrum
  // precision only (read from the slot state after each round); a switch in
  // mid-round leaves the rest of that round's iterations without work (the
  // update kernels wait for their pipeline's flag), the next round runs the
  // new precision.  Nonlinear PB re-enters the high precision at every outer
  // step and keeps every pipeline of its pool.
  const bool hi64 = s.spec_hi == SPEC_FP64, mixed = P.has_mixed;
  const bool pick = mixed && !P.has_nlpb;
  if (pick) {
    P.has_mixed = false;   // the first round starts in the high precision
  }
  int m = 2;
  bool first = true;
  for (;;) {
    launch_round(P, m, first, first || P.has_nlpb, st);
    first = false;
    get_states(P, st);
    ck(cudaStreamSynchronize(st));
    if (t_prof) t_prof->resolve();
    if (P.st_host[0].phase == PH_DONE || P.st_host[0].phase == PH_IDLE) break;
    if (pick) {
      const bool lo = P.st_host[0].spec == SPEC_FP32;
      P.has_mixed = lo;
      P.has_fp64 = !lo && hi64;
      P.has_df64 = !lo && !hi64;
    }
    if (m < 8) m *= 2;
  }
  if (keep) {
    const int stt = P.st_host[0].status;
    P.ws_valid = stt == GPS_OK || stt == GPS_ERR_NOT_CONVERGED;
    if (P.ws_valid) {
      launch_warm_store(batch_of(P, PH_DONE, -1), P.f, 0, P.ws_eps, P.ws_phi, P.ws_d, P.n, st);
      P.ws_kind = kind;
      if (el) P.ws_el = *el;
    }
  }
  P.f.wphi = nullptr;
  P.f.wd = nullptr;
  P.slot_req[0] = nullptr;
  P.f.rho = P.own_rho;
  P.f.eps = P.own_eps;
  P.f.phi = P.own_phi;
  P.f.gam = nullptr;
  fill_report(rep, P.st_host[0], t0);
  return P.st_host[0].status;
}

// Comparison solvers of the GPe (gps_opts.method GPS_SC / GPS_PSD) on slot 0
// of a direct pool: the FP64 spectrum pipeline is the vacuum solve of every
// iteration, the kernels of sc.cu the rest.  Iterations are launched in
// growing chunks; the slot's phase turns every later launch into a no-op
// once the solve has converged.
int solve_comparison(Pool& P, const double* rho, const double* eps, double* phi, const gps_opts& o,
                     gps_report* rep, cudaStream_t st, double t0) {
  const Shape& S = *P.shape;
  const gps_grid& g = S.grid;
  const size_t n = P.n;
  ScWork& w = P.sc;
  if (!w.gx) {
    w.pstride = sc_blocks(n) + 32;
    w.gx = P.mem.alloc<double>(n);
    w.gy = P.mem.alloc<double>(n);
    w.gz = P.mem.alloc<double>(n);
    w.isc = P.mem.alloc<double>(n);
    w.tmp = P.mem.alloc<double>(n);
    w.a = P.mem.alloc<double>(n);
    w.b = P.mem.alloc<double>(n);
    w.c = P.mem.alloc<double>(n);
    w.d = P.mem.alloc<double>(n);
    w.part = P.mem.alloc<double>(4 * (size_t)w.pstride);
    w.dpart = P.mem.alloc<double>((size_t)kMaxDiis * w.pstride);
    w.small = P.mem.alloc<double>(128);
    w.cnt = P.mem.alloc<unsigned int>(8);
    ck(cudaMemsetAsync(w.cnt, 0, 8 * sizeof(unsigned int), st));
  }
  const bool psd = o.method == GPS_PSD;
  const int m = psd && o.diis >= 2 ? o.diis : 0;
  if (m > w.hist_m) {
    w.hist = P.mem.alloc<double>(3 * (size_t)m * n);
    w.hist_m = m;
  }
  ScArgs a{};
  a.S = P.st;
  a.part = w.part;
  a.dpart = w.dpart;
  a.pstride = w.pstride;
  a.cnt = w.cnt;
  a.eps = eps;
  a.rho = rho;
  a.phi = phi;
  a.gx = w.gx;
  a.gy = w.gy;
  a.gz = w.gz;
  a.isc = w.isc;
  a.tmp = w.tmp;
  a.rho_eps = w.a;
  a.rho_iter = w.b;
  a.src = w.c;
  a.hist_m = m;
  a.hist_phi = w.hist;
  a.hist_r = m ? w.hist + (size_t)m * n : nullptr;
  a.hist_v = m ? w.hist + 2 * (size_t)m * n : nullptr;
  a.hist_mr = w.small;
  a.diis_B = w.small + 16;
  a.diis_c = w.small + 16 + kMaxDiis * kMaxDiis;
  a.s16 = stencil16_of(g);
  a.n = n;
  a.periodic = g.bc == GPS_BC_PERIODIC;
  a.inv_n = 1.0 / (double)n;
  a.alpha = o.alpha;

  SlotState s{};
  s.kind = GPS_GPE;
  s.phase = PH_ITER;
  s.spec = s.spec_hi = SPEC_FP64;
  s.max_iter = o.max_iter;
  s.tol_abs = o.tol_abs;
  s.tol_rel = o.tol_rel;
  s.eta = o.eta;
  s.cert = -1.0;
  P.slot_req[0] = reinterpret_cast<Request*>(&P);   // marks slot 0 busy
  put_state(P, 0, s, st);
  put_active(P, st);

  // PSD vectors: plain, phi (the output) and r, v, A v; DIIS, the ring plus
  // the combination phi_w, r_w, v_w and its A v.
  double *r = w.a, *v = w.b, *Av = w.c;
  double *phi_w = w.a, *r_w = w.b, *v_w = w.c, *Av_w = w.d;
  const Batch b = batch_of(P, PH_ITER, SPEC_FP64);
  const Batch bt{};   // profiling records only
  // runs launch(a') with a' = a plus the acted flag of the profiling record
  auto prof = [&](int kind, auto&& launch) {
    timed(kind, bt, st, [&](const Batch& bb) {
      ScArgs aa = a;
      aa.acted = bb.acted;
      launch(aa);
    });
  };
  prof(7, [&](const ScArgs& aa) {
    if (!psd) launch_sc_prep(aa, 0, nullptr, nullptr, st);
    else if (!m) launch_sc_prep(aa, 1, phi, r, st);
    else launch_sc_prep(aa, 1, aa.hist_phi, aa.hist_r, st);
  });
  PipeArgs pa{};
  pa.table = S.table;
  pa.slot_k0 = 0;
  auto iteration = [&](int k) {
    if (!psd) {
      pa.in = w.c;
      pa.in_scale = nullptr;
      pa.out = phi;
      pipeline<double2>(P, b, pa, st);
      prof(8, [&](const ScArgs& aa) { launch_sc_step(aa, st); });
    } else if (!m) {
      pa.in = r;
      pa.in_scale = w.isc;
      pa.out = v;
      pipeline<double2>(P, b, pa, st);
      prof(8, [&](const ScArgs& aa) { launch_psd_av(aa, v, r, Av, 0, st); });
      prof(9, [&](const ScArgs& aa) { launch_psd_update(aa, phi, r, v, Av, phi, r, -1, st); });
    } else {
      const int j = k % m, cnt = std::min(k + 1, m), jn = (k + 1) % m;
      pa.in = a.hist_r + (size_t)j * n;
      pa.in_scale = w.isc;
      pa.out = a.hist_v + (size_t)j * n;
      pipeline<double2>(P, b, pa, st);
      DiisSlots sl{};
      sl.cnt = cnt;
      for (int q = 0; q < cnt; ++q) sl.slot[q] = (k - cnt + 1 + q) % m;
      prof(9, [&](const ScArgs& aa) { launch_diis(aa, sl, phi_w, r_w, v_w, st); });
      prof(8, [&](const ScArgs& aa) { launch_psd_av(aa, v_w, r_w, Av_w, 1, st); });
      prof(9, [&](const ScArgs& aa) {
        launch_psd_update(aa, phi_w, r_w, v_w, Av_w, aa.hist_phi + (size_t)jn * n, aa.hist_r + (size_t)jn * n,
                          jn, st);
      });
    }
  };
  int k = 0, chunk = 4;
  for (;;) {
    for (int c = 0; c < chunk && k < o.max_iter; ++c) iteration(k++);
    get_states(P, st);
    ck(cudaStreamSynchronize(st));
    if (t_prof) t_prof->resolve();
    if (P.st_host[0].phase != PH_ITER || k >= o.max_iter) break;
    chunk = std::min(2 * chunk, 32);
  }
  const SlotState& f = P.st_host[0];
  if (m) {
    const int last = f.iter % m;
    ck(cudaMemcpyAsync(phi, a.hist_phi + (size_t)last * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  fill_report(rep, f, t0);
  P.slot_req[0] = nullptr;
  return f.status;
}

Pool* direct_pool(gps_ctx* ctx, const gps_grid* gr, cudaStream_t st) {
  ++ctx->clock;
  for (auto& p : ctx->direct)
    if (same_grid(p->shape->grid, *gr)) {
      p->last_use = ctx->clock;
      return p.get();
    }
  auto shape = get_shape(ctx->shapes, gr, st);
  const size_t need = slot_bytes(*shape);
  while (ctx->budget && ctx->in_use() + need > ctx->budget && !ctx->direct.empty()) {
    size_t lru = 0;
    for (size_t i = 1; i < ctx->direct.size(); ++i)
      if (ctx->direct[i]->last_use < ctx->direct[lru]->last_use) lru = i;
    auto victim_shape = ctx->direct[lru]->shape;
    ctx->direct.erase(ctx->direct.begin() + lru);
    for (size_t i = 0; i < ctx->shapes.size(); ++i)
      if (ctx->shapes[i] == victim_shape && victim_shape != shape) {
        ctx->shapes.erase(ctx->shapes.begin() + i);
        break;
      }
  }
  if (ctx->budget && ctx->in_use() + need > ctx->budget) throw std::bad_alloc();
  ctx->direct.push_back(make_pool(shape, 1, false));
  ctx->direct.back()->last_use = ctx->clock;
  return ctx->direct.back().get();
}

struct ProfScope {
  explicit ProfScope(gps_ctx* c) { t_prof = c ? &c->prof : nullptr; }
  ~ProfScope() {
    if (t_prof) t_prof->resolve();
    t_prof = nullptr;
  }
};

int finish(int status, cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return GPS_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return GPS_ERR_CUDA;
  if (take_wait_timeouts()) return GPS_ERR_TIMEOUT;   // a bounded device wait gave up
  return status;
}

}  // namespace

// ------------------------------------------------------------- the server --

struct gps_server {
  Engine eng;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Request*> incoming;
  std::map<unsigned long long, std::unique_ptr<Request>> reqs;
  unsigned long long next_ticket = 1;
  bool stop = false;
  int fatal = GPS_OK;
  std::thread worker;
  // engine figures for gps_server_stats, copied by the worker under mu
  size_t stat_bytes = 0;
  int stat_max_concurrent = 0;

  size_t busy() const {
    size_t b = eng.queue.size();
    for (auto& p : eng.pools) b += p->busy();
    return b;
  }

  void loop() {
    cudaSetDevice(eng.device);
    for (;;) {
      if (busy() == 0) {
        // nothing in the engine: sleep until a request arrives
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !incoming.empty(); });
        if (stop) return;
        while (!incoming.empty()) {
          eng.queue.push_back(incoming.front());
          incoming.pop_front();
        }
      } else {
        // work in flight: take new requests only if the lock is free now, so
        // that submitting and waiting threads are never held off by this loop
        std::unique_lock<std::mutex> lk(mu, std::try_to_lock);
        if (lk.owns_lock()) {
          if (stop) return;
          while (!incoming.empty()) {
            eng.queue.push_back(incoming.front());
            incoming.pop_front();
          }
        }
      }
      bool failed = false;
      size_t before = 0, after = 0;
      const unsigned long long done_before = eng.finished_total;
      try {
        before = busy();
        after = eng.step();
      } catch (...) {
        failed = true;
      }
      bool idle_pools = true;
      for (auto& p : eng.pools) idle_pools &= p->busy() == 0;
      if (!failed && after > 0 && after == before && idle_pools)
        std::this_thread::sleep_for(std::chrono::milliseconds(1));   // queued work waiting for memory
      if (!failed && eng.finished_total == done_before) {   // nothing to report
        std::unique_lock<std::mutex> lk(mu, std::try_to_lock);
        if (lk.owns_lock()) {
          stat_bytes = eng.bytes();
          stat_max_concurrent = eng.max_concurrent;
        }
        continue;
      }
      std::lock_guard<std::mutex> lk(mu);
      stat_bytes = eng.bytes();
      stat_max_concurrent = eng.max_concurrent;
      if (failed) {
        fatal = GPS_ERR_CUDA;
        for (auto& kv : reqs)
          if (!kv.second->done) {
            kv.second->status = GPS_ERR_CUDA;
            kv.second->rep.status = GPS_ERR_CUDA;
            kv.second->done = true;
          }
        eng.queue.clear();
        done_cv.notify_all();
        return;
      }
      done_cv.notify_all();
    }
  }
};

// ---------------------------------------------------------------- ABI ------

extern "C" {

void gps_default_opts(gps_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol_abs = 1e-10;
  o->tol_rel = 0.0;
  o->max_iter = 500;
  o->max_outer = 100;
  o->tol_outer = 1e-10;
  o->eta = 0.6;
  o->outer_mode = GPS_OUTER_NEWTON;
  // inexact Newton: with the line search any cap below 1 converges; 0.3 was
  // the fastest of 1e-2, 3e-2, 0.1, 0.3 on the free 256^3 nonlinear-PB workload
  o->forcing = 0.3;
  // Eisenstat-Walker choice 2: on a 128^3 analogue of that workload (oracle)
  // 19 % fewer inner iterations than min(forcing, F/F0), same fixed point
  o->forcing_rule = GPS_FORCING_EW2;
  o->precision = GPS_FP64;
  o->mixed_switch = 1e-2;
  o->certify = 0;
}

const char* gps_status_string(int s) {
  switch (s) {
    case GPS_OK: return "ok";
    case GPS_ERR_INVALID: return "invalid argument";
    case GPS_ERR_NOMEM: return "out of device memory or over the HBM budget";
    case GPS_ERR_NOT_CONVERGED: return "not converged";
    case GPS_ERR_BREAKDOWN: return "PCG breakdown";
    case GPS_ERR_TIMEOUT: return "device wait timed out";
    case GPS_ERR_CUDA: return "CUDA error";
    case GPS_PENDING: return "pending";
    default: return "unknown status";
  }
}

int gps_create(gps_ctx** out, int device, size_t budget) {
  if (!out) return GPS_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) return GPS_ERR_CUDA;
  if (device < 0 || device >= count) return GPS_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return GPS_ERR_CUDA;
  gps_ctx* c = new (std::nothrow) gps_ctx;
  if (!c) return GPS_ERR_NOMEM;
  c->device = device;
  c->budget = budget;
  *out = c;
  return GPS_OK;
}

void gps_destroy(gps_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  delete c;
}

size_t gps_bytes_in_use(const gps_ctx* c) { return c ? c->in_use() : 0; }

#define GPS_GUARD_BEGIN try {
#define GPS_GUARD_END                  \
  }                                    \
  catch (CudaError&) {                 \
    cudaGetLastError();                \
    return GPS_ERR_CUDA;               \
  }                                    \
  catch (std::bad_alloc&) {            \
    return GPS_ERR_NOMEM;              \
  }

int gps_pb_solve(gps_ctx* ctx, const gps_grid* grid, const double* rho, const double* eps,
                 const gps_electrolyte* el, int kind, double* phi, const gps_opts* opts,
                 gps_report* rep, void* stream) {
  const double t0 = now_ms();
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (!ctx || !rho || !eps || !phi) return GPS_ERR_INVALID;
  if (kind < GPS_GPE || kind > GPS_MPB) return GPS_ERR_INVALID;
  if (kind == GPS_MPB && validate_steric(el) != GPS_OK) return GPS_ERR_INVALID;
  int v = validate_grid(grid);
  if (v != GPS_OK) return v;
  if (kind != GPS_GPE && (v = validate_el(el)) != GPS_OK) return v;
  gps_opts o;
  if (opts) o = *opts; else gps_default_opts(&o);
  if ((v = validate_method(o, kind, grid)) != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  ProfScope prof_scope(ctx);
  Pool* P = direct_pool(ctx, grid, st);
  int s = o.method == GPS_PCG ? solve_direct(*P, rho, eps, phi, kind, el, o, rep, st, t0)
                              : solve_comparison(*P, rho, eps, phi, o, rep, st, t0);
  s = finish(s, st);
  if (rep) rep->time_ms = now_ms() - t0;
  return s;
  GPS_GUARD_END
}

int gps_gpe_solve(gps_ctx* ctx, const gps_grid* grid, const double* rho, const double* eps,
                  double* phi, const gps_opts* opts, gps_report* rep, void* stream) {
  return gps_pb_solve(ctx, grid, rho, eps, nullptr, GPS_GPE, phi, opts, rep, stream);
}

int gps_pb_solve_host(gps_ctx* ctx, const gps_grid* grid, const double* rho_h, const double* eps_h,
                      const gps_electrolyte* el, int kind, double* phi_h, const gps_opts* opts,
                      gps_report* rep, void* stream) {
  const double t0 = now_ms();
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (!ctx || !rho_h || !eps_h || !phi_h) return GPS_ERR_INVALID;
  if (kind < GPS_GPE || kind > GPS_MPB) return GPS_ERR_INVALID;
  if (kind == GPS_MPB && validate_steric(el) != GPS_OK) return GPS_ERR_INVALID;
  int v = validate_grid(grid);
  if (v != GPS_OK) return v;
  if (kind != GPS_GPE && (v = validate_el(el)) != GPS_OK) return v;
  gps_opts o;
  if (opts) o = *opts; else gps_default_opts(&o);
  if ((v = validate_method(o, kind, grid)) != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  ProfScope prof_scope(ctx);
  Pool* P = direct_pool(ctx, grid, st);
  const size_t b = P->n * sizeof(double);
  ck(cudaMemcpyAsync(P->own_rho, rho_h, b, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(P->own_eps, eps_h, b, cudaMemcpyHostToDevice, st));
  gps_electrolyte eld{};
  const gps_electrolyte* elp = el;
  if (el && el->exclusion && kind != GPS_GPE) {   // host array: copied next to rho and eps
    if (!P->own_gam) P->own_gam = P->mem.alloc<double>(P->n);
    ck(cudaMemcpyAsync(P->own_gam, el->exclusion, b, cudaMemcpyHostToDevice, st));
    eld = *el;
    eld.exclusion = P->own_gam;
    elp = &eld;
  }
  int s = o.method == GPS_PCG ? solve_direct(*P, P->own_rho, P->own_eps, P->own_phi, kind, elp, o, rep, st, t0)
                              : solve_comparison(*P, P->own_rho, P->own_eps, P->own_phi, o, rep, st, t0);
  ck(cudaMemcpyAsync(phi_h, P->own_phi, b, cudaMemcpyDeviceToHost, st));
  s = finish(s, st);
  if (rep) rep->time_ms = now_ms() - t0;
  return s;
  GPS_GUARD_END
}

int gps_gpe_solve_host(gps_ctx* ctx, const gps_grid* grid, const double* rho_h, const double* eps_h,
                       double* phi_h, const gps_opts* opts, gps_report* rep, void* stream) {
  return gps_pb_solve_host(ctx, grid, rho_h, eps_h, nullptr, GPS_GPE, phi_h, opts, rep, stream);
}

int gps_setup_fields(gps_ctx* ctx, const gps_grid* grid, const double* eps, double* s_out,
                     double* q_out, void* stream) {
  if (!ctx || !eps || !s_out || !q_out) return GPS_ERR_INVALID;
  int v = validate_grid(grid);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  ProfScope prof_scope(ctx);
  Pool* P = direct_pool(ctx, grid, st);
  gps_opts o;
  gps_default_opts(&o);
  P->f.eps = const_cast<double*>(eps);
  P->slot_req[0] = reinterpret_cast<Request*>(P);
  put_state(*P, 0, initial_state(GPS_GPE, nullptr, o), st);
  put_active(*P, st);
  ensure_tuned(*P->shape, false, false, st);
  launch_setup_group(*P, st);
  get_states(*P, st);
  ck(cudaStreamSynchronize(st));
  P->slot_req[0] = nullptr;
  P->f.eps = P->own_eps;
  if (P->st_host[0].bad_eps) return finish(GPS_ERR_INVALID, st);
  const size_t nb = P->n * sizeof(double);
  ck(cudaMemcpyAsync(s_out, P->f.s, nb, cudaMemcpyDeviceToDevice, st));
  ck(cudaMemcpyAsync(q_out, P->f.q, nb, cudaMemcpyDeviceToDevice, st));
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_vacuum_solve(gps_ctx* ctx, const gps_grid* grid, const double* sigma, double* w,
                     void* stream) {
  if (!ctx || !sigma || !w) return GPS_ERR_INVALID;
  int v = validate_grid(grid);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  ProfScope prof_scope(ctx);
  Pool* P = direct_pool(ctx, grid, st);
  ensure_tuned(*P->shape, false, false, st);
  Batch b{};
  PipeArgs a{};
  a.in = sigma;
  a.out = w;
  a.table = P->shape->table;
  a.table32 = P->shape->table32;
  a.tabledf = P->shape->tabledf;
  pipeline<double2>(*P, b, a, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_precondition(gps_ctx* ctx, const gps_grid* grid, const double* s, const double* r, double* v,
                     int precision, void* stream) {
  if (!ctx || !s || !r || !v) return GPS_ERR_INVALID;
  if (precision < GPS_FP64 || precision > GPS_DF64) return GPS_ERR_INVALID;
  int e = validate_grid(grid);
  if (e != GPS_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  ProfScope prof_scope(ctx);
  Pool* P = direct_pool(ctx, grid, st);
  ensure_tuned(*P->shape, precision == GPS_MIXED, precision == GPS_DF64, st);
  Batch b{};
  PipeArgs a{};
  a.in = r;
  a.in_scale = s;
  a.out = v;
  a.out_scale = s;
  a.table = P->shape->table;
  a.table32 = P->shape->table32;
  a.tabledf = P->shape->tabledf;
  if (precision == GPS_MIXED) {
    // the FP32 passes read s as float, as inside the PCG (a copy made at setup)
    launch_to_float(s, P->f.s32, P->n, st);
    a.in_scale32 = P->f.s32;
    a.out_scale32 = P->f.s32;
  }
  if (precision == GPS_MIXED) pipeline<float2>(*P, b, a, st);
  else if (precision == GPS_DF64) pipeline<dfc>(*P, b, a, st);
  else pipeline<double2>(*P, b, a, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_ionic_charge(gps_ctx* ctx, const gps_grid* grid, const double* phi, const double* eps,
                     const gps_electrolyte* el, double* out, void* stream) {
  if (!ctx || !phi || !eps || !out || !grid) return GPS_ERR_INVALID;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return GPS_ERR_INVALID;   // pointwise: any size
  int v = validate_el(el);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  const size_t n = (size_t)grid->nx * grid->ny * grid->nz;
  const bool steric = el->packing > 0;
  if (steric && validate_steric(el) != GPS_OK) return GPS_ERR_INVALID;
  launch_ionic_charge(phi, eps, el->exclusion, out, n, ion_params(el, steric), st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

// grids of the stencil passes: validate_grid, and periodic axes >= 8 points
int validate_stencil_grid(const gps_grid* g) {
  const int v = validate_grid(g);
  if (v != GPS_OK) return v;
  const Stencil16 s = stencil16_of(*g);
  if ((s.perx && g->nx < 8) || (s.pery && g->ny < 8) || (s.perz && g->nz < 8)) return GPS_ERR_INVALID;
  return GPS_OK;
}

int gps_sccs_eps(gps_ctx* ctx, size_t n, const double* rho_elec, double rho_max, double rho_min, double eps0,
                 double* eps, double* deps, void* stream) {
  if (!ctx || !rho_elec || !eps || n == 0) return GPS_ERR_INVALID;
  if (!(rho_min > 0.0 && rho_max > rho_min && eps0 > 1.0)) return GPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  launch_sccs(rho_elec, eps, deps, n, rho_max, rho_min, eps0, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_polarization_charge(gps_ctx* ctx, const gps_grid* grid, const double* rho, const double* eps,
                            const double* phi, double* out, void* stream) {
  if (!ctx || !grid || !rho || !eps || !phi || !out) return GPS_ERR_INVALID;
  int v = validate_stencil_grid(grid);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  Pool* P = direct_pool(ctx, grid, st);
  if (!P->dft_tmp) P->dft_tmp = P->mem.alloc<double>(P->n);
  launch_polarization(stencil16_of(*grid), rho, eps, phi, P->dft_tmp, out, P->n, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_v_eps(gps_ctx* ctx, const gps_grid* grid, const double* deps, const double* phi, double* out,
              void* stream) {
  if (!ctx || !grid || !deps || !phi || !out) return GPS_ERR_INVALID;
  int v = validate_stencil_grid(grid);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  const size_t n = (size_t)grid->nx * grid->ny * grid->nz;
  launch_veps(stencil16_of(*grid), deps, phi, out, n, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_electrostatic_energy(gps_ctx* ctx, const gps_grid* grid, const double* rho, const double* eps,
                             const double* phi, double* e_rho_phi, double* e_eps_grad, void* stream) {
  if (!ctx || !grid || !rho || !eps || !phi) return GPS_ERR_INVALID;
  int v = validate_stencil_grid(grid);
  if (v != GPS_OK) return v;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  Pool* P = direct_pool(ctx, grid, st);
  const int nb = dft_blocks(P->n);
  if (!P->dft_part) P->dft_part = P->mem.alloc<double>(2 * (size_t)nb);
  launch_energy(stencil16_of(*grid), rho, eps, phi, P->n, P->dft_part, st);
  std::vector<double> part(2 * (size_t)nb);
  ck(cudaMemcpyAsync(part.data(), P->dft_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  double a = 0.0, b = 0.0;   // fixed order: the same bits on every call
  for (int i = 0; i < nb; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  const double dv = grid->hx * grid->hy * grid->hz;
  if (e_rho_phi) *e_rho_phi = 0.5 * a * dv;
  if (e_eps_grad) *e_eps_grad = b * dv / (8.0 * kPi);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_batch_solve(gps_ctx* ctx, int count, const gps_request* reqs, gps_report* reps) {
  if (!ctx || count < 0 || (count > 0 && !reqs)) return GPS_ERR_INVALID;
  GPS_GUARD_BEGIN
  cudaSetDevice(ctx->device);
  const double t0 = now_ms();
  Engine eng;
  eng.device = ctx->device;
  eng.budget = ctx->budget;
  eng.shapes = ctx->shapes;   // tables and plans of the grids the context already has
  std::vector<std::unique_ptr<Request>> rs;
  for (int i = 0; i < count; ++i) {
    rs.emplace_back(new Request);
    rs.back()->req = reqs[i];
    rs.back()->t0 = t0;
    eng.queue.push_back(rs.back().get());
  }
  while (eng.step() > 0) {
  }
  ctx->shapes = eng.shapes;   // keep the new grids' tables for later calls
  int status = GPS_OK;
  for (int i = 0; i < count; ++i) {
    if (reps) reps[i] = rs[i]->rep;
    if (status == GPS_OK && rs[i]->status != GPS_OK) status = rs[i]->status;
  }
  return status;
  GPS_GUARD_END
}

int gps_server_create(gps_server** out, int device, size_t budget, int max_slots) {
  if (!out) return GPS_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) return GPS_ERR_CUDA;
  if (device < 0 || device >= count || max_slots < 0) return GPS_ERR_INVALID;
  gps_server* s = new (std::nothrow) gps_server;
  if (!s) return GPS_ERR_NOMEM;
  s->eng.device = device;
  s->eng.budget = budget;
  s->eng.max_slots = max_slots;
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return GPS_OK;
}

int gps_server_submit(gps_server* s, const gps_request* req, unsigned long long* ticket) {
  if (!s || !req || !ticket) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != GPS_OK) return s->fatal;
  auto r = std::make_unique<Request>();
  r->req = *req;
  r->t0 = now_ms();
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->incoming.push_back(r.get());
  s->reqs.emplace(r->ticket, std::move(r));
  s->cv.notify_all();
  return GPS_OK;
}

int gps_server_poll(gps_server* s, unsigned long long ticket, gps_report* rep) {
  if (!s) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GPS_ERR_INVALID;
  if (!it->second->done) return GPS_PENDING;
  if (rep) *rep = it->second->rep;
  const int st = it->second->status;
  s->reqs.erase(it);
  return st;
}

int gps_server_wait(gps_server* s, unsigned long long ticket, gps_report* rep) {
  if (!s) return GPS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return GPS_ERR_INVALID;
  Request* r = it->second.get();
  s->done_cv.wait(lk, [&] { return r->done.load(); });
  if (rep) *rep = r->rep;
  const int st = r->status;
  s->reqs.erase(ticket);
  return st;
}

int gps_server_stats(gps_server* s, size_t* bytes, int* max_concurrent) {
  if (!s) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes) *bytes = s->stat_bytes;
  if (max_concurrent) *max_concurrent = s->stat_max_concurrent;
  return GPS_OK;
}

void gps_server_destroy(gps_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->eng.device);
  cudaDeviceSynchronize();
  delete s;
}

int gps_set_radix_order(int order) {
  if (order < -1 || order > 3) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_radix_order = order;
  g_tune.clear();
  return GPS_OK;
}

int gps_set_x_kernel(int kind) {
  if (kind < -1 || kind > 1) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_x_kernel = kind;
  g_tune.clear();
  return GPS_OK;
}

int gps_set_z_kernel(int kind) {
  if (kind < -1 || kind > 1) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_z_kernel = kind;
  g_tune.clear();
  return GPS_OK;
}

int gps_set_engine_mode(int async) {
  if (async != 0 && async != 1) return GPS_ERR_INVALID;
  g_engine_async = async;
  return GPS_OK;
}

int gps_set_profiling(gps_ctx* ctx, int mask) {
  if (!ctx) return GPS_ERR_INVALID;
  ctx->prof.on = mask != 0;
  ctx->prof.mask = mask;
  return GPS_OK;
}

int gps_get_profile(gps_ctx* ctx, long long* launches, double* total_ms, int reset) {
  if (!ctx || !launches || !total_ms) return GPS_ERR_INVALID;
  ctx->prof.resolve();
  for (int k = 0; k < GPS_PROFILE_KINDS; ++k) {
    launches[k] = ctx->prof.launches[k];
    total_ms[k] = ctx->prof.ms[k];
    if (reset) {
      ctx->prof.launches[k] = 0;
      ctx->prof.ms[k] = 0.0;
    }
  }
  return GPS_OK;
}

unsigned long long gps_kernel_launches(void) { return launch_count(); }

}  // extern "C"
