// Vacuum Poisson solve that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: plugins hosted by an
// application that owns the whole device-memory budget, processes whose
// framework has already reserved (nearly) all of HBM in its own pool so
// that any further cudaMalloc would fail, and latency-critical loops in which
// the implicit device synchronization of cudaMalloc/cudaFree would stall
// work on other streams.  For them gps_vacuum_solve_noalloc runs the same
// five FFT passes as gps_vacuum_solve, but keeps every buffer the passes need
// (twiddle tables, Green's-function table, spectrum) in one file-scope
// __device__ array of fixed size.  The array belongs to the loaded module:
// every GPU that loads this library holds it until the process exits.
#include <mutex>

#include "gps_internal.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Host-side address of the array on the current device, found once per
// device with that device current.  The symbol itself is only a host-side
// stand-in and must never be passed to a kernel.  The cached address belongs
// to the device's primary context: it must not be used after
// cudaDeviceReset (which the caller of this library must not mix with it).
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return GPS_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return GPS_ERR_CUDA;
    g_scratch_addr[device] = ptr;
  }
  *out = g_scratch_addr[device];
  return GPS_OK;
}

bool radix_schedule(int L, gps::FftSched* s) {
  if (L < 2 || L > gps::kMaxLen) return false;
  *s = gps::FftSched{};
  s->L = L;
  int rem = L, ns = 1, k = 0;
  auto push = [&](int R) {
    s->radix[k] = R;
    s->ns[k] = ns;
    ns *= R;
    rem /= R;
    ++k;
  };
  while (rem % 8 == 0 && k < gps::kMaxStages) push(8);
  if (rem % 4 == 0 && k < gps::kMaxStages) push(4);
  if (rem % 2 == 0 && k < gps::kMaxStages) push(2);
  while (rem % 5 == 0 && k < gps::kMaxStages) push(5);
  while (rem % 3 == 0 && k < gps::kMaxStages) push(3);
  s->nst = k;
  return rem == 1;
}

// tw[m] = exp(-2 pi i m / L) in FP64.
__global__ void k_noalloc_twiddles(double2* tw, int L) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);
    tw[m] = make_double2(c, -s);
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int gps_vacuum_solve_noalloc(const gps_grid* grid, const double* sigma_dev,
                                        double* w_dev, void* cuda_stream) {
  using namespace gps;
  if (!grid || !sigma_dev || !w_dev) return GPS_ERR_INVALID;
  if (grid->bc != GPS_BC_PERIODIC && grid->bc != GPS_BC_SURFACE) return GPS_ERR_INVALID;
  if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4) return GPS_ERR_INVALID;
  if (!(grid->hx > 0) || !(grid->hy > 0) || !(grid->hz > 0)) return GPS_ERR_INVALID;
  const int Px = grid->nx, Py = grid->ny;
  const int Pz = grid->bc == GPS_BC_SURFACE ? 2 * grid->nz : grid->nz;
  if (Px % 2 || Py % 2 || Pz % 2) return GPS_ERR_INVALID;
  FftSched sx, sy, sz;
  if (!radix_schedule(Px, &sx) || !radix_schedule(Py, &sy) || !radix_schedule(Pz, &sz))
    return GPS_ERR_INVALID;
  const int Hx = Px / 2 + 1, hy = Py / 2 + 1, hz = Pz / 2 + 1;
  const size_t table_n = (size_t)Hx * hy * hz;
  // scratch layout: twiddles x, y, z | Green's-function table | spectrum
  const size_t off_twx = 0;
  const size_t off_twy = off_twx + align256((size_t)Px * sizeof(double2));
  const size_t off_twz = off_twy + align256((size_t)Py * sizeof(double2));
  const size_t off_tab = off_twz + align256((size_t)Pz * sizeof(double2));
  const size_t off_w = off_tab + align256(table_n * sizeof(double));
  const int Hp = spectrum_pitch(Hx);
  const size_t need = off_w + (size_t)Hp * Py * grid->nz * sizeof(double2);
  if (need > kScratchBytes) return GPS_ERR_INVALID;   // beyond the fixed scratch size

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return GPS_ERR_CUDA;
  unsigned char* base = nullptr;
  int e = scratch_address(device, reinterpret_cast<void**>(&base));
  if (e != GPS_OK) return e;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double2* twx = reinterpret_cast<double2*>(base + off_twx);
  double2* twy = reinterpret_cast<double2*>(base + off_twy);
  double2* twz = reinterpret_cast<double2*>(base + off_twz);
  double* table = reinterpret_cast<double*>(base + off_tab);
  double2* W = reinterpret_cast<double2*>(base + off_w);

  // Tables are rebuilt on every call: the array keeps whatever the previous
  // call (of any grid) left in it.  The spectrum needs no clearing: every
  // entry a pass reads was written by the pass before it.
  (void)cudaGetLastError();   // an earlier failed launch is not this call's error
  count_launch();
  k_noalloc_twiddles<<<(Px + 255) / 256, 256, 0, st>>>(twx, Px);
  count_launch();
  k_noalloc_twiddles<<<(Py + 255) / 256, 256, 0, st>>>(twy, Py);
  count_launch();
  k_noalloc_twiddles<<<(Pz + 255) / 256, 256, 0, st>>>(twz, Pz);
  const double inv_n = 1.0 / ((double)Px * Py * Pz);
  const double dkx = 2 * kPi / (Px * grid->hx), dky = 2 * kPi / (Py * grid->hy),
               dkz = 2 * kPi / (Pz * grid->hz);
  if (grid->bc == GPS_BC_PERIODIC)
    launch_table_periodic(table, nullptr, Hx, hy, hz, dkx, dky, dkz, inv_n, st);
  else
    launch_table_surface(table, Hx, hy, hz, dkx, dky, dkz, grid->nz * grid->hz, inv_n, st);

  PassGeom g;
  g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
  g.Px = Px; g.Py = Py; g.Pz = Pz; g.Hx = Hx; g.Hp = Hp;
  g.nrows = grid->ny * grid->nz;
  g.lines_x = default_lines(Px, (g.nrows + 1) / 2, sizeof(double2));
  g.tile_y = default_lines(Py, Hx * grid->nz, sizeof(double2));
  g.tile_z = default_lines(Pz, Hx * Py, sizeof(double2));
  Batch b{};                 // one slot, no phase machine
  PipeArgs a{};
  a.in = sigma_dev;
  a.out = w_dev;
  a.table = table;
  a.W = W;
  launch_x_fwd<double2>(g, sx, twx, b, a, 1, st);
  launch_y<double2>(g, sy, twy, b, a, false, 1, st);
  launch_z<double2>(g, sz, twz, b, a, 1, st);
  launch_y<double2>(g, sy, twy, b, a, true, 1, st);
  launch_x_inv<double2>(g, sx, twx, b, a, 1, st);
  if (cudaGetLastError() != cudaSuccess) return GPS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GPS_ERR_CUDA;
  return GPS_OK;
}
