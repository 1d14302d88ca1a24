// C ABI of the solver (include/gps.h): context, cached plans, and the
// drivers of Algorithm 2 (PCG) and Algorithm 4 (nonlinear PB outer loop).
//
// A plan is everything that depends on (grid, spacing, BC): FFT schedules
// and twiddles, the Green's-function table, the spectrum workspace and the
// PCG vectors.  Plans are cached per context and evicted least-recently-used
// under the context's HBM budget.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <vector>

#include "gps_internal.h"
#include "kernels.h"

using namespace gps;

namespace {

// ---------------------------------------------------------------- helpers --

bool factorable(int L) {
  int r = L;
  for (int p : {2, 3, 5})
    while (r % p == 0) r /= p;
  return r == 1;
}

bool make_sched(int L, FftSched* s) {
  if (L < 2 || L > kMaxLen || !factorable(L)) return false;
  std::memset(s, 0, sizeof(*s));
  s->L = L;
  int rem = L, ns = 1, k = 0;
  auto push = [&](int R) {
    s->radix[k] = R;
    s->ns[k] = ns;
    ns *= R;
    rem /= R;
    ++k;
  };
  while (rem % 8 == 0) push(8);
  if (rem % 4 == 0) push(4);
  if (rem % 2 == 0) push(2);
  while (rem % 5 == 0) push(5);
  while (rem % 3 == 0) push(3);
  s->nst = k;
  return rem == 1 && k <= kMaxStages;
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

struct CudaError {};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaError{};
}

struct Dev {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

// ------------------------------------------------------------------ plans --

struct FftLen {
  FftSched sched;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
};

struct Plan {
  int nx, ny, nz, bc;
  double hx, hy, hz;
  int Px, Py, Pz, Hx;
  size_t n;
  PassGeom g64, g32;
  FftLen fx, fy, fz;
  double* table = nullptr;
  double* lap_table = nullptr;
  double2* W64 = nullptr;
  float2* W32 = nullptr;
  double *s = nullptr, *sq = nullptr, *q = nullptr, *qlam = nullptr;
  double *r = nullptr, *p = nullptr, *Ap = nullptr, *v = nullptr;
  double *rions = nullptr, *rp = nullptr, *fresh = nullptr, *lam = nullptr, *dphi = nullptr,
         *src = nullptr;
  double *io_rho = nullptr, *io_eps = nullptr, *io_phi = nullptr;
  double* partials = nullptr;
  double* partials2 = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  unsigned long long last_use = 0;

  template <typename T>
  T* alloc(size_t count) {
    void* ptr = nullptr;
    const size_t b = count * sizeof(T);
    if (cudaMalloc(&ptr, b) != cudaSuccess) throw std::bad_alloc();
    allocs.push_back(ptr);
    bytes += b;
    return static_cast<T*>(ptr);
  }
  ~Plan() {
    for (void* a : allocs) cudaFree(a);
    if (sc_host) cudaFreeHost(sc_host);
  }
};

// Opt-in per-kernel timing with CUDA events on the launching stream.
struct Profiler {
  bool on = false;
  int mask = 0;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
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
  void resolve() {
    if (pending.empty()) return;
    cudaEventSynchronize(pending.back().b);
    for (auto& r : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        launches[r.kind] += 1;
        ms[r.kind] += t;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  // Drop the records of loop kernels (kinds 0..6) launched after the PCG had
  // converged (they return at once) -- keep the first `iters` of each kind.
  void trim_loop(size_t from, int iters) {
    int seen[GPS_PROFILE_KINDS] = {0};
    std::vector<Rec> keep(pending.begin(), pending.begin() + from);
    for (size_t i = from; i < pending.size(); ++i) {
      const Rec& r = pending[i];
      if (r.kind < 7 && seen[r.kind]++ >= iters) {
        pool.push_back(r.a);
        pool.push_back(r.b);
      } else {
        keep.push_back(r);
      }
    }
    pending.swap(keep);
  }
  ~Profiler() {
    for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

static thread_local Profiler* t_prof = nullptr;

template <typename F>
static void timed(int kind, cudaStream_t st, F&& f) {
  if (!t_prof || !t_prof->on || !(t_prof->mask & (1 << kind))) {
    f();
    return;
  }
  cudaEvent_t a = t_prof->get(), b = t_prof->get();
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  t_prof->pending.push_back({kind, a, b});
}

struct gps_ctx {
  Profiler prof;
  int device = 0;
  size_t budget = 0;
  std::vector<std::unique_ptr<Plan>> plans;
  unsigned long long clock = 0;
  size_t in_use() const {
    size_t b = 0;
    for (auto& p : plans) b += p->bytes;
    return b;
  }
};

namespace {

int validate_grid(const gps_grid* g) {
  if (!g) return GPS_ERR_INVALID;
  if (g->nx < 4 || g->ny < 4 || g->nz < 4) return GPS_ERR_INVALID;
  if (!(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) return GPS_ERR_INVALID;
  if (g->bc < GPS_BC_FREE || g->bc > GPS_BC_SURFACE) return GPS_ERR_INVALID;
  const bool fx = g->bc == GPS_BC_FREE, fy = fx, fz = g->bc != GPS_BC_PERIODIC;
  const int Px = fx ? 2 * g->nx : g->nx, Py = fy ? 2 * g->ny : g->ny, Pz = fz ? 2 * g->nz : g->nz;
  for (int P : {Px, Py, Pz})
    if (P % 2 || P > kMaxLen || !factorable(P)) return GPS_ERR_INVALID;
  if (g->bc == GPS_BC_FREE) {
    const double R = std::sqrt(std::pow(g->nx * g->hx, 2) + std::pow(g->ny * g->hy, 2) +
                               std::pow(g->nz * g->hz, 2));
    if (4 * g->nx * g->hx < g->nx * g->hx + R || 4 * g->ny * g->hy < g->ny * g->hy + R ||
        4 * g->nz * g->hz < g->nz * g->hz + R)
      return GPS_ERR_INVALID;   // aspect ratio too large for the 4x oversampled kernel
  }
  return GPS_OK;
}

int batch_lines(int L, int units) {
  int b = 2048 / L;
  if (b < 1) b = 1;
  const int want = units / 304;   // keep >= ~2 CTAs per SM
  if (want < b) b = want < 1 ? 1 : want;
  return b;
}

void fill_twiddles(Plan* P, FftLen* f, int L) {
  if (!make_sched(L, &f->sched)) throw std::bad_alloc();
  std::vector<double2> h64(L);
  std::vector<float2> h32(L);
  for (int m = 0; m < L; ++m) {
    const long double ang = 2.0L * 3.141592653589793238462643383279502884L * m / L;
    h64[m].x = (double)cosl(ang);
    h64[m].y = (double)-sinl(ang);
    h32[m].x = (float)h64[m].x;
    h32[m].y = (float)h64[m].y;
  }
  f->tw64 = P->alloc<double2>(L);
  f->tw32 = P->alloc<float2>(L);
  ck(cudaMemcpy(f->tw64, h64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(f->tw32, h32.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
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

// Free-BC table: h^3 g on the octant from the 4x oversampled truncated-Coulomb
// transform (three even transforms), then its 2n-periodic transform (three
// more), normalized by 1/(Px Py Pz).
void build_free_table(Plan* P, cudaStream_t st) {
  const int nx = P->nx, ny = P->ny, nz = P->nz;
  const int Mx = 4 * nx, My = 4 * ny, Mz = 4 * nz;
  const int mx = Mx / 2 + 1, my = My / 2 + 1, mz = Mz / 2 + 1;
  const double R = std::sqrt(std::pow(nx * P->hx, 2) + std::pow(ny * P->hy, 2) + std::pow(nz * P->hz, 2));
  double *ghat = nullptr, *t1 = nullptr, *t2 = nullptr, *g = nullptr, *u1 = nullptr, *u2 = nullptr;
  double *cx = nullptr, *cy = nullptr, *cz = nullptr, *dx = nullptr, *dy = nullptr, *dz = nullptr;
  auto tmp = [&](size_t cnt) {
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, cnt * sizeof(double)) != cudaSuccess) throw std::bad_alloc();
    return static_cast<double*>(ptr);
  };
  auto up = [&](const std::vector<double>& h) {
    double* d = tmp(h.size());
    ck(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    return d;
  };
  const int hxo = nx + 1, hyo = ny + 1, hzo = nz + 1;
  try {
    ghat = tmp((size_t)mx * my * mz);
    launch_free_ghat(ghat, mx, my, mz, 2 * kPi / (Mx * P->hx), 2 * kPi / (My * P->hy),
                     2 * kPi / (Mz * P->hz), R, st);
    cx = up(cosine_matrix(Mx, hxo, 1.0 / Mx));
    cy = up(cosine_matrix(My, hyo, 1.0 / My));
    cz = up(cosine_matrix(Mz, hzo, 1.0 / Mz));
    t1 = tmp((size_t)mz * my * hxo);
    launch_axis_matrix(ghat, t1, cx, mz * my, mx, 1, hxo, st);
    ck(cudaStreamSynchronize(st));
    cudaFree(ghat);
    ghat = nullptr;
    t2 = tmp((size_t)mz * hyo * hxo);
    launch_axis_matrix(t1, t2, cy, mz, my, hxo, hyo, st);
    g = tmp((size_t)hzo * hyo * hxo);
    launch_axis_matrix(t2, g, cz, 1, mz, hyo * hxo, hzo, st);
    // transform of the 2n-periodic even extension: M = 2n, entries m = 0..n
    dx = up(cosine_matrix(2 * nx, hxo, 1.0 / (2 * nx)));
    dy = up(cosine_matrix(2 * ny, hyo, 1.0 / (2 * ny)));
    dz = up(cosine_matrix(2 * nz, hzo, 1.0 / (2 * nz)));
    u1 = tmp((size_t)hzo * hyo * hxo);
    u2 = tmp((size_t)hzo * hyo * hxo);
    launch_axis_matrix(g, u1, dx, hzo * hyo, hxo, 1, hxo, st);
    launch_axis_matrix(u1, u2, dy, hzo, hyo, hxo, hyo, st);
    launch_axis_matrix(u2, P->table, dz, 1, hzo, hyo * hxo, hzo, st);
    ck(cudaStreamSynchronize(st));
    ck(cudaGetLastError());
  } catch (...) {
    for (double* d : {ghat, t1, t2, g, u1, u2, cx, cy, cz, dx, dy, dz})
      if (d) cudaFree(d);
    throw;
  }
  for (double* d : {t1, t2, g, u1, u2, cx, cy, cz, dx, dy, dz})
    if (d) cudaFree(d);
}

Plan* build_plan(const gps_grid* gr, cudaStream_t st) {
  auto P = std::make_unique<Plan>();
  P->nx = gr->nx; P->ny = gr->ny; P->nz = gr->nz; P->bc = gr->bc;
  P->hx = gr->hx; P->hy = gr->hy; P->hz = gr->hz;
  const bool fx = gr->bc == GPS_BC_FREE, fz = gr->bc != GPS_BC_PERIODIC;
  P->Px = fx ? 2 * gr->nx : gr->nx;
  P->Py = fx ? 2 * gr->ny : gr->ny;
  P->Pz = fz ? 2 * gr->nz : gr->nz;
  P->Hx = P->Px / 2 + 1;
  P->n = (size_t)gr->nx * gr->ny * gr->nz;
  PassGeom g;
  g.nx = gr->nx; g.ny = gr->ny; g.nz = gr->nz;
  g.Px = P->Px; g.Py = P->Py; g.Pz = P->Pz; g.Hx = P->Hx;
  g.nrows = gr->ny * gr->nz;
  g.lines_x = batch_lines(P->Px, (g.nrows + 1) / 2);
  g.tile_y = batch_lines(P->Py, P->Hx * gr->nz);
  g.tile_z = batch_lines(P->Pz, P->Hx * P->Py);
  P->g64 = g;
  P->g32 = g;
  fill_twiddles(P.get(), &P->fx, P->Px);
  fill_twiddles(P.get(), &P->fy, P->Py);
  fill_twiddles(P.get(), &P->fz, P->Pz);
  const int hy = P->Py / 2 + 1, hz = P->Pz / 2 + 1;
  const size_t tab = (size_t)P->Hx * hy * hz;
  const double inv_n = 1.0 / ((double)P->Px * P->Py * P->Pz);
  P->table = P->alloc<double>(tab);
  if (gr->bc == GPS_BC_PERIODIC) {
    P->lap_table = P->alloc<double>(tab);
    launch_table_periodic(P->table, P->lap_table, P->Hx, hy, hz, 2 * kPi / (P->Px * gr->hx),
                          2 * kPi / (P->Py * gr->hy), 2 * kPi / (P->Pz * gr->hz), inv_n, st);
  } else if (gr->bc == GPS_BC_SURFACE) {
    launch_table_surface(P->table, P->Hx, hy, hz, 2 * kPi / (P->Px * gr->hx),
                         2 * kPi / (P->Py * gr->hy), 2 * kPi / (P->Pz * gr->hz), gr->nz * gr->hz,
                         inv_n, st);
  } else {
    build_free_table(P.get(), st);
  }
  P->W64 = P->alloc<double2>((size_t)P->Hx * P->Py * gr->nz);
  const size_t n = P->n;
  P->s = P->alloc<double>(n);
  P->sq = P->alloc<double>(n);
  P->q = P->alloc<double>(n);
  P->qlam = P->alloc<double>(n);
  P->r = P->alloc<double>(n);
  P->p = P->alloc<double>(n);
  P->Ap = P->alloc<double>(n);
  P->v = P->alloc<double>(n);
  size_t maxblocks = 152 * 8;
  const size_t xb = ((g.nrows + 1) / 2 + g.lines_x - 1) / g.lines_x;
  if (xb > maxblocks) maxblocks = xb;
  P->partials = P->alloc<double>(maxblocks);
  P->partials2 = P->alloc<double>(maxblocks);
  P->sc = P->alloc<PcgScalars>(1);
  ck(cudaMemsetAsync(P->sc, 0, sizeof(PcgScalars), st));
  ck(cudaMallocHost((void**)&P->sc_host, sizeof(PcgScalars)));
  ck(cudaStreamSynchronize(st));
  ck(cudaGetLastError());
  return P.release();
}

void ensure_nl(Plan* P) {
  if (P->rions) return;
  P->rions = P->alloc<double>(P->n);
  P->rp = P->alloc<double>(P->n);
  P->fresh = P->alloc<double>(P->n);
  P->lam = P->alloc<double>(P->n);
  P->dphi = P->alloc<double>(P->n);
  P->src = P->alloc<double>(P->n);
}

void ensure_io(Plan* P) {
  if (P->io_rho) return;
  P->io_rho = P->alloc<double>(P->n);
  P->io_eps = P->alloc<double>(P->n);
  P->io_phi = P->alloc<double>(P->n);
}

void ensure_w32(Plan* P) {
  if (!P->W32) P->W32 = P->alloc<float2>((size_t)P->Hx * P->Py * P->nz);
}

int get_plan(gps_ctx* c, const gps_grid* gr, cudaStream_t st, Plan** out) {
  int v = validate_grid(gr);
  if (v != GPS_OK) return v;
  ++c->clock;
  for (auto& p : c->plans) {
    if (p->nx == gr->nx && p->ny == gr->ny && p->nz == gr->nz && p->bc == gr->bc &&
        p->hx == gr->hx && p->hy == gr->hy && p->hz == gr->hz) {
      p->last_use = c->clock;
      *out = p.get();
      return GPS_OK;
    }
  }
  Plan* P = nullptr;
  try {
    P = build_plan(gr, st);
  } catch (std::bad_alloc&) {
    return GPS_ERR_NOMEM;
  } catch (CudaError&) {
    return GPS_ERR_CUDA;
  }
  // evict least-recently-used plans while over budget
  while (c->budget && c->in_use() + P->bytes > c->budget && !c->plans.empty()) {
    size_t lru = 0;
    for (size_t i = 1; i < c->plans.size(); ++i)
      if (c->plans[i]->last_use < c->plans[lru]->last_use) lru = i;
    c->plans.erase(c->plans.begin() + lru);
  }
  if (c->budget && P->bytes > c->budget) {
    delete P;
    return GPS_ERR_NOMEM;
  }
  P->last_use = c->clock;
  c->plans.emplace_back(P);
  *out = P;
  return GPS_OK;
}

// ------------------------------------------------------------- pipelines --

// Vacuum solve on the spectrum pipeline: out = out_scale * S(in_scale * in),
// with `table` the normalized octant multiplier.  Optionally reduces
// (out, dot_with) into sc->vr and records the k = 0 sum in sc->mu_sum.
template <typename V>
void vacuum_pipeline(Plan* P, const double* in, const double* in_scale, const double* table,
                     double k0, int use_k0, double* out, const double* out_scale,
                     const double* dot_with, bool track, cudaStream_t st, bool gauge = false) {
  V* W;
  const V *twx, *twy, *twz;
  if constexpr (sizeof(V) == sizeof(double2)) {
    W = reinterpret_cast<V*>(P->W64);
    twx = reinterpret_cast<const V*>(P->fx.tw64);
    twy = reinterpret_cast<const V*>(P->fy.tw64);
    twz = reinterpret_cast<const V*>(P->fz.tw64);
  } else {
    W = reinterpret_cast<V*>(P->W32);
    twx = reinterpret_cast<const V*>(P->fx.tw32);
    twy = reinterpret_cast<const V*>(P->fy.tw32);
    twz = reinterpret_cast<const V*>(P->fz.tw32);
  }
  const PassGeom& g = P->g64;
  const int* done = track ? &P->sc->done : nullptr;
  const bool periodic_track = track && P->bc == GPS_BC_PERIODIC;
  timed(0, st, [&] {
    launch_x_fwd<V>(g, P->fx.sched, twx, in, in_scale, W, done, st, P->partials, P->sc,
                    periodic_track ? &P->sc->mu_sum : nullptr);
  });
  timed(1, st, [&] { launch_y<V>(g, P->fy.sched, twy, W, false, done, st); });
  timed(2, st, [&] { launch_z<V>(g, P->fz.sched, twz, W, table, k0, use_k0, nullptr, done, st); });
  timed(3, st, [&] { launch_y<V>(g, P->fy.sched, twy, W, true, done, st); });
  timed(4, st, [&] {
    launch_x_inv<V>(g, P->fx.sched, twx, W, out, out_scale, dot_with, dot_with ? P->partials : nullptr,
                    P->sc, CNT_VR, &P->sc->vr, done, st, P->partials2,
                    gauge ? &P->sc->wsum : nullptr);
  });
}

void read_scalars(Plan* P, cudaStream_t st) {
  ck(cudaMemcpyAsync(P->sc_host, P->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
}

// S1: s, sqrt(eps), q (spectral for periodic, FD-16 otherwise).
int setup_fields(Plan* P, const double* eps, cudaStream_t st) {
  timed(7, st, [&] { launch_setup_s(eps, P->s, P->sq, P->n, P->sc, st); });
  if (P->bc == GPS_BC_PERIODIC) {
    vacuum_pipeline<double2>(P, P->sq, nullptr, P->lap_table, 0.0, 0, P->q, P->sq, nullptr, false, st);
  } else {
    const int per_xy = P->bc == GPS_BC_SURFACE ? 1 : 0;   // surface: x, y wrap; z free
    launch_fd16_q(P->sq, P->q, P->nx, P->ny, P->nz, P->hx, P->hy, P->hz, per_xy, per_xy, 0,
                  fd16_coeffs(), st);
  }
  return GPS_OK;
}

struct PcgResult {
  int status, iters, fp64_iters;
  double res0, res, background;
};

// Algorithm 2 from phi = 0 on the current plan state: operator term `qlam`
// (q + lambda), source rho.  Iterations are enqueued in chunks; the device
// sets `done`, after which every queued kernel returns at once.
PcgResult run_pcg(Plan* P, const double* rho, double* phi, const double* qlam, double k0, int use_k0,
                  bool neutralize, const gps_opts* o, cudaStream_t st) {
  PcgScalars* sc = P->sc;
  const bool periodic = P->bc == GPS_BC_PERIODIC;
  const size_t prof_from = t_prof ? t_prof->pending.size() : 0;
  double* bg_sum = nullptr;
  if (neutralize) {
    launch_sum(rho, P->n, P->partials, &sc->counter[CNT_AUX], &sc->aux[3], st);
    bg_sum = &sc->aux[3];
  }
  launch_init(rho, P->r, phi, P->p, P->Ap, P->n, o->tol_abs, o->tol_rel, o->max_iter, P->partials, sc,
              1, bg_sum, st);
  read_scalars(P, st);
  PcgResult res{GPS_OK, 0, 0, std::sqrt(P->sc_host->rr0), std::sqrt(P->sc_host->rr0),
                P->sc_host->background};
  const bool mixed = o->precision == GPS_MIXED;
  if (mixed) ensure_w32(P);
  const bool gauge = periodic && !use_k0;   // singular periodic operator: keep v on the gauge
  bool use32 = false;
  int chunk = 2;
  while (!P->sc_host->done) {
    for (int c = 0; c < chunk; ++c) {
      if (use32)
        vacuum_pipeline<float2>(P, P->r, P->s, P->table, k0, use_k0, P->v, P->s, P->r, true, st, gauge);
      else
        vacuum_pipeline<double2>(P, P->r, P->s, P->table, k0, use_k0, P->v, P->s, P->r, true, st, gauge);
      timed(5, st, [&] {
        launch_update_p(P->v, P->r, qlam, P->sq, P->s, P->p, P->Ap, P->n, periodic ? 1 : 0,
                        gauge ? 1 : 0, P->partials, sc, st);
      });
      timed(6, st, [&] { launch_update_r(phi, P->r, P->p, P->Ap, P->n, P->partials, sc, st); });
    }
    const int before = P->sc_host->iter;
    read_scalars(P, st);
    if (!use32) res.fp64_iters += P->sc_host->iter - before;
    if (mixed && !use32 && std::sqrt(P->sc_host->rr) <= o->mixed_switch * res.res0) use32 = true;
    if (chunk < 8) chunk *= 2;
  }
  res.status = P->sc_host->status;
  res.iters = P->sc_host->iter;
  if (t_prof && t_prof->on) t_prof->trim_loop(prof_from, res.iters);
  res.res = std::sqrt(P->sc_host->rr);
  return res;
}

// Certificate of a result (FP64): ||g|| / ||phi|| with
// g = M(rho - bg [+ rions] - qlam phi / 4pi) [+ <sqrt(eps) phi> s] - phi.
// Uses P->p and P->Ap as scratch.
double certify(Plan* P, const double* rho, double bg, const double* rions, const double* qlam,
               const double* phi, double k0, int use_k0, cudaStream_t st) {
  const bool periodic = P->bc == GPS_BC_PERIODIC;
  launch_fp_source(rho, rions, qlam, phi, P->sq, P->p, P->n, bg, P->partials, P->sc, st);
  vacuum_pipeline<double2>(P, P->p, P->s, P->table, k0, use_k0, P->Ap, P->s, nullptr, false, st);
  read_scalars(P, st);
  const double c = periodic ? P->sc_host->aux[5] / (double)P->n : 0.0;
  launch_fp_residual(P->Ap, P->s, phi, P->n, c, P->partials, P->partials2, P->sc, st);
  read_scalars(P, st);
  const double nphi = std::sqrt(P->sc_host->aux[7]);
  return nphi > 0 ? std::sqrt(P->sc_host->aux[6]) / nphi : std::sqrt(P->sc_host->aux[6]);
}

IonParams ion_params(const gps_electrolyte* el) {
  const double NA = 6.02214076e23, a0 = 5.29177210903e-11, kB = 3.1668115634556e-6;
  IonParams ip;
  std::memset(&ip, 0, sizeof(ip));
  ip.nspecies = el->nspecies;
  const double kt = kB * el->temperature;
  ip.inv_kt = 1.0 / kt;
  ip.inv_eps0m1 = 1.0 / (el->eps0 - 1.0);
  ip.exp_cap = 40.0;
  for (int s = 0; s < el->nspecies; ++s) {
    const double nb = el->c_molar[s] * 1000.0 * NA * a0 * a0 * a0;
    ip.zq[s] = el->z[s];
    ip.zn[s] = el->z[s] * nb;
    ip.z2n_kt[s] = (double)el->z[s] * el->z[s] * nb / kt;
  }
  return ip;
}

double lambda0_of(const gps_electrolyte* el) {
  const IonParams ip = ion_params(el);
  double l = 0.0;
  for (int s = 0; s < ip.nspecies; ++s) l += ip.z2n_kt[s];
  return kFourPi * l;
}

int validate_el(const gps_electrolyte* el) {
  if (!el || el->nspecies < 0 || el->nspecies > GPS_MAX_SPECIES) return GPS_ERR_INVALID;
  if (!(el->temperature > 0) || !(el->eps0 > 1.0)) return GPS_ERR_INVALID;
  for (int s = 0; s < el->nspecies; ++s)
    if (!(el->c_molar[s] >= 0)) return GPS_ERR_INVALID;
  return GPS_OK;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

void fill_report(gps_report* rep, const PcgResult& r, double t0) {
  if (!rep) return;
  rep->status = r.status;
  rep->iters = r.iters;
  rep->fp64_iters = r.fp64_iters;
  rep->res0 = r.res0;
  rep->res = r.res;
  rep->background = r.background;
  rep->fixed_point_res = -1.0;
  rep->time_ms = now_ms() - t0;
}

// Core solve on device pointers (shared by the device and host entry points).
int solve_core(gps_ctx* ctx, const gps_grid* gr, const double* rho, const double* eps,
               const gps_electrolyte* el, int kind, double* phi, const gps_opts* oin,
               gps_report* rep, cudaStream_t st, double t0, Plan* P) {
  gps_opts o;
  if (oin) o = *oin; else gps_default_opts(&o);
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (kind != GPS_GPE) {
    int e = validate_el(el);
    if (e != GPS_OK) return e;
  }
  setup_fields(P, eps, st);
  read_scalars(P, st);
  if (P->sc_host->bad_eps) {
    P->sc_host->bad_eps = 0;
    ck(cudaMemsetAsync(&P->sc->bad_eps, 0, sizeof(int), st));
    return GPS_ERR_INVALID;
  }
  const bool periodic = P->bc == GPS_BC_PERIODIC;
  const double N = (double)P->n;
  const double invN = 1.0 / ((double)P->Px * P->Py * P->Pz);
  const bool want_cert = o.certify || o.precision == GPS_MIXED;
  if (kind == GPS_GPE) {
    PcgResult r = run_pcg(P, rho, phi, P->q, 0.0, 0, periodic, &o, st);
    fill_report(rep, r, t0);
    if (rep && want_cert && r.status == GPS_OK)
      rep->fixed_point_res = certify(P, rho, r.background, nullptr, P->q, phi, 0.0, 0, st);
    return r.status;
  }
  const double lam0 = lambda0_of(el);
  const IonParams ip = ion_params(el);
  double eps_mean = 0.0;
  if (periodic) {
    launch_sum(eps, P->n, P->partials, &P->sc->counter[CNT_AUX], &P->sc->aux[4], st);
    read_scalars(P, st);
    eps_mean = P->sc_host->aux[4] / N;
  }
  if (kind == GPS_LPB) {
    launch_qlam_linear(P->q, eps, P->qlam, P->n, lam0, ip.inv_eps0m1, P->partials, P->sc, st);
    read_scalars(P, st);
    const double lam_mean = P->sc_host->aux[1] / N;
    const bool k0 = periodic && lam_mean > 0;
    const double k0v = k0 ? kFourPi * eps_mean / lam_mean * invN : 0.0;
    PcgResult r = run_pcg(P, rho, phi, P->qlam, k0v, k0 ? 1 : 0, periodic && !k0, &o, st);
    fill_report(rep, r, t0);
    if (rep && want_cert && r.status == GPS_OK)
      rep->fixed_point_res = certify(P, rho, r.background, nullptr, P->qlam, phi, k0v, k0 ? 1 : 0, st);
    return r.status;
  }
  if (kind != GPS_NLPB) return GPS_ERR_INVALID;
  // Algorithm 4 (see gps.h): bookkeeping A phi = -4 pi (rho + rions - rp).
  try {
    ensure_nl(P);
  } catch (std::bad_alloc&) {
    return GPS_ERR_NOMEM;
  }
  const bool newton = o.outer_mode == GPS_OUTER_NEWTON;
  ck(cudaMemsetAsync(phi, 0, P->n * sizeof(double), st));
  launch_ionic_charge(phi, eps, P->rions, P->n, ip, st);
  ck(cudaMemcpyAsync(P->rp, rho, P->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double F0 = -1.0, F = 0.0;
  int outer = 0, total_iters = 0, status = GPS_ERR_NOT_CONVERGED, fp64_iters = 0;
  PcgResult last{GPS_OK, 0, 0, 0, 0, 0};
  for (; outer <= o.max_outer; ++outer) {
    launch_nl_eval(phi, eps, P->rions, P->rp, P->fresh, P->lam, P->n, ip, newton ? 1 : 0,
                   P->partials, P->sc, st);
    read_scalars(P, st);
    F = std::sqrt(P->sc_host->aux[0]);
    if (F0 < 0) F0 = F;
    if (!std::isfinite(F)) { status = GPS_ERR_BREAKDOWN; break; }
    if (F <= o.tol_outer) { status = GPS_OK; break; }
    if (outer == o.max_outer) break;
    const double e = newton ? 1.0 : o.eta;
    launch_nl_source(P->fresh, P->rions, P->rp, P->q, P->lam, P->src, P->qlam, P->n, e, P->partials,
                     P->sc, st);
    read_scalars(P, st);
    const double lam_mean = P->sc_host->aux[1] / N;
    const bool k0 = periodic && lam_mean > 0;
    gps_opts io = o;
    if (newton) {
      io.tol_abs = 0.1 * kFourPi * o.tol_outer;
      io.tol_rel = std::fmin(o.forcing, F / F0);
    } else if (outer < 2) {
      io.tol_abs = 0.0;
      io.tol_rel = 1e-4;
    } else {
      io.tol_abs = kFourPi * o.tol_outer;
      io.tol_rel = 0.0;
    }
    last = run_pcg(P, P->src, P->dphi, P->qlam, k0 ? kFourPi * eps_mean / lam_mean * invN : 0.0,
                   k0 ? 1 : 0, periodic && !k0, &io, st);
    total_iters += last.iters;
    fp64_iters += last.fp64_iters;
    if (last.status == GPS_ERR_BREAKDOWN) { status = last.status; break; }
    double t = 1.0;
    if (newton) {
      while (t > 1e-4) {
        launch_nl_step(phi, eps, P->rions, P->rp, P->fresh, P->lam, P->dphi, P->r, P->n, ip, e, t, 0,
                       P->partials, P->sc, st);
        read_scalars(P, st);
        if (std::sqrt(P->sc_host->aux[2]) < F) break;
        t *= 0.5;
      }
    }
    launch_nl_step(phi, eps, P->rions, P->rp, P->fresh, P->lam, P->dphi, P->r, P->n, ip, e, t, 1,
                   P->partials, P->sc, st);
  }
  double cert = -1.0;
  if (want_cert && status == GPS_OK) {
    launch_ionic_charge(phi, eps, P->fresh, P->n, ip, st);
    cert = certify(P, rho, 0.0, P->fresh, P->q, phi, 0.0, 0, st);
  }
  ck(cudaStreamSynchronize(st));
  if (rep) {
    rep->fixed_point_res = cert;
    rep->status = status;
    rep->iters = total_iters;
    rep->fp64_iters = fp64_iters;
    rep->outer_iters = outer;
    rep->res0 = last.res0;
    rep->res = last.res;
    rep->outer_res = F;
    rep->time_ms = now_ms() - t0;
  }
  return status;
}

}  // namespace

// ---------------------------------------------------------------- ABI ------

extern "C" {

void gps_default_opts(gps_opts* o) {
  if (!o) return;
  o->tol_abs = 1e-10;
  o->tol_rel = 0.0;
  o->max_iter = 500;
  o->max_outer = 100;
  o->tol_outer = 1e-10;
  o->eta = 0.6;
  o->outer_mode = GPS_OUTER_NEWTON;
  o->forcing = 1e-2;
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

struct ProfScope {
  explicit ProfScope(gps_ctx* c) { t_prof = c ? &c->prof : nullptr; }
  ~ProfScope() {
    if (t_prof) t_prof->resolve();
    t_prof = nullptr;
  }
};

#define GPS_GUARD_BEGIN try {
#define GPS_GUARD_END                  \
  }                                    \
  catch (CudaError&) {                 \
    return GPS_ERR_CUDA;               \
  }                                    \
  catch (std::bad_alloc&) {            \
    return GPS_ERR_NOMEM;              \
  }

static int finish(int status, cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return GPS_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return GPS_ERR_CUDA;
  return status;
}

int gps_pb_solve(gps_ctx* ctx, const gps_grid* grid, const double* rho, const double* eps,
                 const gps_electrolyte* el, int kind, double* phi, const gps_opts* opts,
                 gps_report* rep, void* stream) {
  const double t0 = now_ms();
  if (!ctx || !rho || !eps || !phi) return GPS_ERR_INVALID;
  if (kind < GPS_GPE || kind > GPS_NLPB) return GPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  ProfScope prof_scope(ctx);
  cudaSetDevice(ctx->device);
  Plan* P = nullptr;
  int e = get_plan(ctx, grid, st, &P);
  if (e != GPS_OK) return e;
  int s = solve_core(ctx, grid, rho, eps, el, kind, phi, opts, rep, st, t0, P);
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
  if (!ctx || !rho_h || !eps_h || !phi_h) return GPS_ERR_INVALID;
  if (kind < GPS_GPE || kind > GPS_NLPB) return GPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  ProfScope prof_scope(ctx);
  cudaSetDevice(ctx->device);
  Plan* P = nullptr;
  int e = get_plan(ctx, grid, st, &P);
  if (e != GPS_OK) return e;
  ensure_io(P);
  const size_t b = P->n * sizeof(double);
  ck(cudaMemcpyAsync(P->io_rho, rho_h, b, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(P->io_eps, eps_h, b, cudaMemcpyHostToDevice, st));
  int s = solve_core(ctx, grid, P->io_rho, P->io_eps, el, kind, P->io_phi, opts, rep, st, t0, P);
  ck(cudaMemcpyAsync(phi_h, P->io_phi, b, cudaMemcpyDeviceToHost, st));
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
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  ProfScope prof_scope(ctx);
  cudaSetDevice(ctx->device);
  Plan* P = nullptr;
  int e = get_plan(ctx, grid, st, &P);
  if (e != GPS_OK) return e;
  setup_fields(P, eps, st);
  read_scalars(P, st);
  if (P->sc_host->bad_eps) {
    ck(cudaMemsetAsync(&P->sc->bad_eps, 0, sizeof(int), st));
    return finish(GPS_ERR_INVALID, st);
  }
  const size_t b = P->n * sizeof(double);
  ck(cudaMemcpyAsync(s_out, P->s, b, cudaMemcpyDeviceToDevice, st));
  ck(cudaMemcpyAsync(q_out, P->q, b, cudaMemcpyDeviceToDevice, st));
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_vacuum_solve(gps_ctx* ctx, const gps_grid* grid, const double* sigma, double* w,
                     void* stream) {
  if (!ctx || !sigma || !w) return GPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  ProfScope prof_scope(ctx);
  cudaSetDevice(ctx->device);
  Plan* P = nullptr;
  int e = get_plan(ctx, grid, st, &P);
  if (e != GPS_OK) return e;
  vacuum_pipeline<double2>(P, sigma, nullptr, P->table, 0.0, 0, w, nullptr, nullptr, false, st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
}

int gps_precondition(gps_ctx* ctx, const gps_grid* grid, const double* s, const double* r, double* v,
                     int precision, void* stream) {
  if (!ctx || !s || !r || !v) return GPS_ERR_INVALID;
  if (precision != GPS_FP64 && precision != GPS_MIXED) return GPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  GPS_GUARD_BEGIN
  ProfScope prof_scope(ctx);
  cudaSetDevice(ctx->device);
  Plan* P = nullptr;
  int e = get_plan(ctx, grid, st, &P);
  if (e != GPS_OK) return e;
  if (precision == GPS_MIXED) {
    ensure_w32(P);
    vacuum_pipeline<float2>(P, r, s, P->table, 0.0, 0, v, s, nullptr, false, st);
  } else {
    vacuum_pipeline<double2>(P, r, s, P->table, 0.0, 0, v, s, nullptr, false, st);
  }
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
  launch_ionic_charge(phi, eps, out, n, ion_params(el), st);
  return finish(GPS_OK, st);
  GPS_GUARD_END
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
