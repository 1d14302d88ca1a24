// Mixed-radix (2, 3, 4, 5, 8) Stockham FFT passes of the vacuum Poisson
// solve used as the PCG preconditioner (Eq. PCGdef).  The 3D transform of the
// zero-padded, sqrt(eps)-scaled residual is done as five HBM passes:
//
//   x_fwd : real rows (scaled) -> half spectra, two rows per complex FFT
//   y     : columns along y (zero padding folded into the load)
//   z     : columns along z: forward FFT, multiply by the Green's-function
//           table, inverse FFT, crop (padding never touches HBM)
//   y inv : columns along y, crop
//   x_inv : half spectra -> real rows, crop, scale, and the (v, r) dot product
//
// Each CTA stages a batch of lines in shared memory; the radix stages run
// out of a shared-memory ping-pong pair with the twiddle table staged once.
// The spectrum buffer holds only z < nz planes: [nz][Py][Hx] complex.
#include <cstdio>

#include "device_util.cuh"
#include "gps_internal.h"

namespace gps {

// Radix-R butterflies, DIR = -1 forward (e^{-2 pi i/R}), +1 inverse.
template <typename V, int DIR>
__device__ __forceinline__ V rot_i(V a) {  // a * (DIR * i)
  return DIR < 0 ? mk<V>(a.y, -a.x) : mk<V>(-a.y, a.x);
}

template <typename V, int DIR, int R> struct Dft;

template <typename V, int DIR> struct Dft<V, DIR, 2> {
  __device__ __forceinline__ static void run(V* x) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <typename V, int DIR> struct Dft<V, DIR, 4> {
  __device__ __forceinline__ static void run(V* x) {
    V a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    V a2 = cadd(x[1], x[3]), a3 = rot_i<V, DIR>(csub(x[1], x[3]));
    x[0] = cadd(a0, a2);
    x[2] = csub(a0, a2);
    x[1] = cadd(a1, a3);
    x[3] = csub(a1, a3);
  }
};

template <typename V, int DIR> struct Dft<V, DIR, 8> {
  __device__ __forceinline__ static void run(V* x) {
    using T = typename Real<V>::T;
    const T c = (T)0.70710678118654752440;  // sqrt(1/2)
    V e[4] = {x[0], x[2], x[4], x[6]};
    V o[4] = {x[1], x[3], x[5], x[7]};
    Dft<V, DIR, 4>::run(e);
    Dft<V, DIR, 4>::run(o);
    // o_k *= e^{DIR 2 pi i k / 8}
    if (DIR < 0) {
      o[1] = mk<V>(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
      o[2] = mk<V>(o[2].y, -o[2].x);
      o[3] = mk<V>(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
    } else {
      o[1] = mk<V>(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y));
      o[2] = mk<V>(-o[2].y, o[2].x);
      o[3] = mk<V>(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x[k] = cadd(e[k], o[k]);
      x[k + 4] = csub(e[k], o[k]);
    }
  }
};

template <typename V, int DIR> struct Dft<V, DIR, 3> {
  __device__ __forceinline__ static void run(V* x) {
    using T = typename Real<V>::T;
    const T s3 = (T)0.86602540378443864676;  // sqrt(3)/2
    V t1 = cadd(x[1], x[2]);
    V t2 = mk<V>(x[0].x - (T)0.5 * t1.x, x[0].y - (T)0.5 * t1.y);
    V d = csub(x[1], x[2]);
    V u = mk<V>((T)DIR * s3 * d.x, (T)DIR * s3 * d.y);   // u = DIR s3 (x1 - x2)
    V iu = mk<V>(-u.y, u.x);
    x[0] = cadd(x[0], t1);
    x[1] = cadd(t2, iu);
    x[2] = csub(t2, iu);
  }
};

template <typename V, int DIR> struct Dft<V, DIR, 5> {
  __device__ __forceinline__ static void run(V* x) {
    using T = typename Real<V>::T;
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi/5) = (sqrt5 - 1)/4
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi/5) = -(sqrt5 + 1)/4
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi/5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi/5)
    V a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]);
    V a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
    V p1 = mk<V>(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
    V p2 = mk<V>(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
    V q1 = mk<V>((T)DIR * (s1 * b1.x + s2 * b2.x), (T)DIR * (s1 * b1.y + s2 * b2.y));
    V q2 = mk<V>((T)DIR * (s2 * b1.x - s1 * b2.x), (T)DIR * (s2 * b1.y - s1 * b2.y));
    V iq1 = mk<V>(-q1.y, q1.x), iq2 = mk<V>(-q2.y, q2.x);
    x[0] = cadd(x[0], cadd(a1, a2));
    x[1] = cadd(p1, iq1);
    x[4] = csub(p1, iq1);
    x[2] = cadd(p2, iq2);
    x[3] = csub(p2, iq2);
  }
};

// Shared-memory layout of a line: one pad element after every 128 bytes
// (8 complex doubles, 16 complex floats), so that the stride-R scatters of
// the early Stockham stages spread over all banks.
template <typename V> struct PadShift;
template <> struct PadShift<double2> { static constexpr int v = 3; };
template <> struct PadShift<float2> { static constexpr int v = 4; };
template <> struct PadShift<dfc> { static constexpr int v = 3; };

template <typename V> struct SpecOf;
template <> struct SpecOf<double2> { static constexpr int v = SPEC_FP64; };
template <> struct SpecOf<float2> { static constexpr int v = SPEC_FP32; };
template <> struct SpecOf<dfc> { static constexpr int v = SPEC_DF64; };

template <typename V>
__device__ __forceinline__ int pidx(int i) { return i + (i >> PadShift<V>::v); }

template <typename V>
__host__ __device__ __forceinline__ int line_stride(int L) { return L + (L >> PadShift<V>::v) + 1; }

// One Stockham stage over `nlines` lines of length L (line stride ls):
// butterfly j gathers in[j + r L/R], twiddles by W_(Ns R)^(r k), k = j mod Ns,
// and scatters to out[(j - k) R + k + r Ns].
template <typename V, int DIR, int R>
__device__ __forceinline__ void stage(const V* __restrict__ in, V* __restrict__ out, int L, int Ns,
                                      int ls, int nlines, const V* __restrict__ tw) {
  const int nb = L / R;
  const int total = nb * nlines;
  const int tstep = L / (Ns * R);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int line = idx / nb;
    const int j = idx - line * nb;
    const V* src = in + line * ls;
    V* dst = out + line * ls;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = src[pidx<V>(j + r * nb)];
    const int k = j % Ns;
    if (k != 0) {
      const int step = tstep * k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = tw[r * step];
        x[r] = DIR < 0 ? cmul(x[r], w) : cmulc(x[r], w);
      }
    }
    Dft<V, DIR, R>::run(x);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[pidx<V>(base + r * Ns)] = x[r];
  }
}

// Full 1D transform of a batch of lines held in a; b is the ping-pong partner.
// Returns the buffer holding the result.  Ends with a __syncthreads().
template <typename V, int DIR>
__device__ V* fft_lines(V* a, V* b, const FftSched& s, int ls, int nlines, const V* tw) {
  V* in = a;
  V* out = b;
  for (int st = 0; st < s.nst; ++st) {
    const int R = s.radix[st], Ns = s.ns[st];
    switch (R) {
      case 2: stage<V, DIR, 2>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 3: stage<V, DIR, 3>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 4: stage<V, DIR, 4>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 5: stage<V, DIR, 5>(in, out, s.L, Ns, ls, nlines, tw); break;
      default: stage<V, DIR, 8>(in, out, s.L, Ns, ls, nlines, tw); break;
    }
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
  }
  return in;
}

__device__ __forceinline__ size_t row_offset(const PassGeom& g, int row) {
  const int y = row % g.ny, z = row / g.ny;
  return ((size_t)z * g.Py + y) * g.Hx;
}

constexpr int kThreads = 256;

// Slot served by this block for a spectrum pass of precision V, or -1.
template <typename V>
__device__ __forceinline__ int pass_slot(const Batch& b) {
  int s = batch_slot(b);
  if (s >= 0 && b.st && b.prec >= 0 && b.st[s].spec != SpecOf<V>::v) s = -1;
  if (s >= 0) mark_acted(b);
  return s;
}

template <typename V>
__global__ void __launch_bounds__(kThreads) k_x_fwd(PassGeom g, FftSched s, const V* __restrict__ twg,
                                                   Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const double* __restrict__ in = a.in + slot * b.vstride;
  const double* __restrict__ scale = a.in_scale ? a.in_scale + slot * b.vstride : nullptr;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L);
  V* b0 = tw + L;
  V* b1 = b0 + g.lines_x * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int npairs = (g.nrows + 1) >> 1;
  const int p0 = blockIdx.x * g.lines_x;
  const int nl = min(g.lines_x, npairs - p0);
  double sum = 0.0;
  for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
    const int l = idx / L, j = idx - l * L;
    const int ra = 2 * (p0 + l);
    double va = 0.0, vb = 0.0;
    if (j < g.nx) {
      const size_t oa = (size_t)ra * g.nx + j;
      va = in[oa];
      if (scale) va *= scale[oa];
      if (ra + 1 < g.nrows) {
        vb = in[oa + g.nx];
        if (scale) vb *= scale[oa + g.nx];
      }
    }
    sum += va + vb;
    b0[l * ls + pidx<V>(j)] = mk<V>((T)va, (T)vb);
  }
  __syncthreads();
  const V* res = fft_lines<V, -1>(b0, b1, s, ls, nl, tw);
  for (int idx = threadIdx.x; idx < nl * g.Hx; idx += blockDim.x) {
    const int l = idx / g.Hx, k = idx - l * g.Hx;
    const V zk = res[l * ls + pidx<V>(k)];
    const V zm = res[l * ls + pidx<V>(k == 0 ? 0 : L - k)];
    const int ra = 2 * (p0 + l);
    // A_k = (Z_k + conj Z_(L-k))/2 ; B_k = -i (Z_k - conj Z_(L-k))/2
    W[row_offset(g, ra) + k] = mk<V>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
    if (ra + 1 < g.nrows) W[row_offset(g, ra + 1) + k] = mk<V>((T)0.5 * (zk.y + zm.y), (T)0.5 * (zm.x - zk.x));
  }
  if (a.red_mu && b.st)
    grid_reduce(sum, b.partials + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_MU], &b.st[slot].mu_sum);
}

template <typename V, int DIR>
__global__ void __launch_bounds__(kThreads) k_y(PassGeom g, FftSched s, const V* __restrict__ twg,
                                               Batch b, PipeArgs a) {
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L), tile = g.tile_y;
  V* b0 = tw + L;
  V* b1 = b0 + tile * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int kx0 = blockIdx.x * tile;
  const int nl = min(tile, g.Hx - kx0);   // valid columns of this tile
  const int z = blockIdx.y;
  const size_t plane = (size_t)z * g.Py * g.Hx;
  const int nload = DIR < 0 ? g.ny : L;   // forward: rows y >= ny are the zero padding
  for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
    const int y = idx / nl, c = idx - y * nl;
    V v = czero<V>();
    if (y < nload) v = W[plane + (size_t)y * g.Hx + kx0 + c];
    b0[c * ls + pidx<V>(y)] = v;
  }
  __syncthreads();
  const V* res = fft_lines<V, DIR>(b0, b1, s, ls, nl, tw);
  const int nstore = DIR < 0 ? L : g.ny;  // inverse: crop to y < ny
  for (int idx = threadIdx.x; idx < nl * nstore; idx += blockDim.x) {
    const int y = idx / nl, c = idx - y * nl;
    W[plane + (size_t)y * g.Hx + kx0 + c] = res[c * ls + pidx<V>(y)];
  }
}

template <typename V>
__global__ void __launch_bounds__(kThreads) k_z(PassGeom g, FftSched s, const V* __restrict__ twg,
                                               Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  const bool use_k0 = a.slot_k0 && b.st && b.st[slot].use_k0;
  const double k0 = use_k0 ? b.st[slot].k0 : 0.0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L), tile = g.tile_z;
  V* b0 = tw + L;
  V* b1 = b0 + tile * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int kx0 = blockIdx.x * tile;
  const int nl = min(tile, g.Hx - kx0);
  const int ky = blockIdx.y;
  const size_t colbase = (size_t)ky * g.Hx + kx0;
  const size_t zstride = (size_t)g.Py * g.Hx;
  for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
    const int z = idx / nl, c = idx - z * nl;
    V v = czero<V>();
    if (z < g.nz) v = W[(size_t)z * zstride + colbase + c];
    b0[c * ls + pidx<V>(z)] = v;
  }
  __syncthreads();
  V* res = fft_lines<V, -1>(b0, b1, s, ls, nl, tw);
  V* other = (res == b0) ? b1 : b0;
  const int kyp = min(ky, g.Py - ky);
  const int hy = g.Py / 2 + 1;
  for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
    const int kz = idx / nl, c = idx - kz * nl;
    const int kx = kx0 + c;
    const int kzp = min(kz, L - kz);
    double t = a.table[((size_t)kzp * hy + kyp) * g.Hx + kx];
    if (use_k0 && kx == 0 && ky == 0 && kz == 0) t = k0;
    const int pk = c * ls + pidx<V>(kz);
    res[pk] = cscale(res[pk], (T)t);
  }
  __syncthreads();
  const V* fin = fft_lines<V, +1>(res, other, s, ls, nl, tw);
  for (int idx = threadIdx.x; idx < nl * g.nz; idx += blockDim.x) {
    const int z = idx / nl, c = idx - z * nl;
    W[(size_t)z * zstride + colbase + c] = fin[c * ls + pidx<V>(z)];
  }
}

template <typename V>
__global__ void __launch_bounds__(kThreads) k_x_inv(PassGeom g, FftSched s, const V* __restrict__ twg,
                                                   Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const V* __restrict__ W = reinterpret_cast<const V*>(a.W) + slot * a.wstride;
  double* __restrict__ out = a.out + slot * b.vstride;
  const double* __restrict__ out_scale = a.out_scale ? a.out_scale + slot * b.vstride : nullptr;
  const double* __restrict__ dot_with = a.dot_with ? a.dot_with + slot * b.vstride : nullptr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L);
  V* b0 = tw + L;
  V* b1 = b0 + g.lines_x * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int npairs = (g.nrows + 1) >> 1;
  const int p0 = blockIdx.x * g.lines_x;
  const int nl = min(g.lines_x, npairs - p0);
  for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
    const int l = idx / L, k = idx - l * L;
    const int ra = 2 * (p0 + l);
    const bool hasb = ra + 1 < g.nrows;
    V A, B;
    if (k < g.Hx) {
      A = W[row_offset(g, ra) + k];
      B = hasb ? W[row_offset(g, ra + 1) + k] : czero<V>();
      if (k == 0 || 2 * k == L) { A.y = T(0); B.y = T(0); }   // DC and Nyquist are real
    } else {
      const int m = L - k;
      A = cconj(W[row_offset(g, ra) + m]);
      B = hasb ? cconj(W[row_offset(g, ra + 1) + m]) : czero<V>();
    }
    b0[l * ls + pidx<V>(k)] = mk<V>(A.x - B.y, A.y + B.x);   // Z = A + i B
  }
  __syncthreads();
  const V* res = fft_lines<V, +1>(b0, b1, s, ls, nl, tw);
  double dot = 0.0, wsum = 0.0;
  for (int idx = threadIdx.x; idx < nl * g.nx; idx += blockDim.x) {
    const int l = idx / g.nx, j = idx - l * g.nx;
    const int ra = 2 * (p0 + l);
    const V zz = res[l * ls + pidx<V>(j)];
    const size_t oa = (size_t)ra * g.nx + j;
    wsum += (double)zz.x;
    double va = (double)zz.x;
    if (out_scale) va *= out_scale[oa];
    out[oa] = va;
    if (dot_with) dot += va * dot_with[oa];
    if (ra + 1 < g.nrows) {
      const size_t ob = oa + g.nx;
      wsum += (double)zz.y;
      double vb = (double)zz.y;
      if (out_scale) vb *= out_scale[ob];
      out[ob] = vb;
      if (dot_with) dot += vb * dot_with[ob];
    }
  }
  if (dot_with && b.st)
    grid_reduce(dot, b.partials + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_VR], &b.st[slot].vr);
  if (a.red_wsum && b.st && b.st[slot].gauge)
    grid_reduce(wsum, b.partials2 + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_WSUM],
                &b.st[slot].wsum);
}

// ---------------------------------------------------------------------------
// Launchers.

size_t x_lines_smem_bytes(int L, int lines, size_t vbytes) {
  const int ls = vbytes == sizeof(double2) ? line_stride<double2>(L) : line_stride<float2>(L);
  return (size_t)(L + 2 * lines * ls) * vbytes;
}

int x_pass_blocks(const PassGeom& g) {
  const int npairs = (g.nrows + 1) / 2;
  return (npairs + g.lines_x - 1) / g.lines_x;
}

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename V>
void launch_x_fwd(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st) {
  const size_t sm = x_lines_smem_bytes(s.L, g.lines_x, sizeof(V));
  set_smem(k_x_fwd<V>, sm);
  count_launch();
  k_x_fwd<V><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
}

template <typename V>
void launch_y(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, bool inverse, int nslots, cudaStream_t st) {
  dim3 grid((g.Hx + g.tile_y - 1) / g.tile_y, g.nz, nslots);
  const size_t sm = x_lines_smem_bytes(s.L, g.tile_y, sizeof(V));
  count_launch();
  if (inverse) {
    set_smem(k_y<V, +1>, sm);
    k_y<V, +1><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  } else {
    set_smem(k_y<V, -1>, sm);
    k_y<V, -1><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  }
}

template <typename V>
void launch_z(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, int nslots, cudaStream_t st) {
  dim3 grid((g.Hx + g.tile_z - 1) / g.tile_z, g.Py, nslots);
  const size_t sm = x_lines_smem_bytes(s.L, g.tile_z, sizeof(V));
  set_smem(k_z<V>, sm);
  count_launch();
  k_z<V><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
}

template <typename V>
void launch_x_inv(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st) {
  const size_t sm = x_lines_smem_bytes(s.L, g.lines_x, sizeof(V));
  set_smem(k_x_inv<V>, sm);
  count_launch();
  k_x_inv<V><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
}

#define GPS_INSTANTIATE(V)                                                                       \
  template void launch_x_fwd<V>(const PassGeom&, const FftSched&, const V*, const Batch&,       \
                                const PipeArgs&, int, cudaStream_t);                             \
  template void launch_y<V>(const PassGeom&, const FftSched&, const V*, const Batch&,           \
                            const PipeArgs&, bool, int, cudaStream_t);                           \
  template void launch_z<V>(const PassGeom&, const FftSched&, const V*, const Batch&,           \
                            const PipeArgs&, int, cudaStream_t);                                 \
  template void launch_x_inv<V>(const PassGeom&, const FftSched&, const V*, const Batch&,       \
                                const PipeArgs&, int, cudaStream_t);

GPS_INSTANTIATE(double2)
GPS_INSTANTIATE(float2)
GPS_INSTANTIATE(dfc)

}  // namespace gps
