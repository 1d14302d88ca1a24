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
// The spectrum buffer holds only z < nz planes: [nz][Py][Hp] complex (Hx
// values per row, row pitch Hp).
#include <cstdio>
#include <type_traits>

#include "fft_common.cuh"

namespace gps {

// One Stockham stage over `nlines` lines of length L (line stride ls):
// butterfly j gathers in[j + r L/R], twiddles by W_(Ns R)^(r k), k = j mod Ns,
// and scatters to out[(j - k) R + k + r Ns].  Butterflies are dealt to the
// threads round-robin over (line, j); a thread's next (line, j, k) follows
// from the current one by constant steps (Ns divides L/R, so a wrap of j
// leaves k unchanged), without a division per butterfly.  When L/R (FL) or
// Ns (FS) is a multiple of the padding period, the padded index of element
// r is the padded index of element 0 plus a constant times r.
// HALF (first stage only, Ns = 1): elements L/2.. of every line are the zero
// padding, i.e. x[R/2..R-1] of every butterfly; they are neither read nor
// used (Dft::run_half).
template <typename V, int DIR, int R, bool FL, bool FS, bool HALF = false>
__device__ __forceinline__ void stage(const V* __restrict__ in, V* __restrict__ out, int L, int Ns,
                                      int ls, int nlines, const V* __restrict__ tw) {
  constexpr int P = 1 << PadShift<V>::v;
  const int nb = L / R;
  const int tstep = L / (Ns * R);
  const int snb = nb + nb / P, sns = Ns + Ns / P;
  const int bd = blockDim.x;
  const int dl = bd / nb, dj = bd - dl * nb, dk = dj % Ns;
  int line = threadIdx.x / nb;
  int j = threadIdx.x - line * nb;
  int k = j % Ns;
  while (line < nlines) {
    const V* src = in + line * ls;
    V* dst = out + line * ls;
    V x[R];
    const int s0 = pidx<V>(j);
#pragma unroll
    for (int r = 0; r < (HALF ? R / 2 : R); ++r) x[r] = src[FL ? s0 + r * snb : pidx<V>(j + r * nb)];
    if (!HALF && k != 0) {
      const int step = tstep * k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = tw[r * step];
        x[r] = DIR < 0 ? cmul(x[r], w) : cmulc(x[r], w);
      }
    }
    if constexpr (HALF) Dft<V, DIR, R>::run_half(x);
    else Dft<V, DIR, R>::run(x);
    const int base = (j - k) * R + k;
    const int d0 = pidx<V>(base);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[FS ? d0 + r * sns : pidx<V>(base + r * Ns)] = x[r];
    line += dl;
    j += dj;
    k += dk;
    if (j >= nb) {
      j -= nb;
      ++line;
    }
    if (k >= Ns) k -= Ns;
  }
}

template <typename V, int DIR, int R>
__device__ __forceinline__ void stage_any(const V* in, V* out, int L, int Ns, int ls, int nlines,
                                          const V* tw) {
  constexpr int P = 1 << PadShift<V>::v;
  const bool fl = (L / R) % P == 0, fs = Ns % P == 0;
  if (fl && fs) stage<V, DIR, R, true, true>(in, out, L, Ns, ls, nlines, tw);
  else if (fl) stage<V, DIR, R, true, false>(in, out, L, Ns, ls, nlines, tw);
  else if (fs) stage<V, DIR, R, false, true>(in, out, L, Ns, ls, nlines, tw);
  else stage<V, DIR, R, false, false>(in, out, L, Ns, ls, nlines, tw);
}

// First stage (Ns = 1, so FS holds) of a line whose upper half is zero.
template <typename V, int DIR, int R>
__device__ __forceinline__ void stage_half(const V* in, V* out, int L, int ls, int nlines, const V* tw) {
  constexpr int P = 1 << PadShift<V>::v;
  if ((L / R) % P == 0) stage<V, DIR, R, true, false, true>(in, out, L, 1, ls, nlines, tw);
  else stage<V, DIR, R, false, false, true>(in, out, L, 1, ls, nlines, tw);
}

// Full 1D transform of a batch of lines held in a; b is the ping-pong partner.
// Returns the buffer holding the result.  Ends with a __syncthreads().
// MR: the largest radix the kernel is built for (16 only in the FP64 kernels
// launched for schedules that contain a radix-16 stage, so that the other
// kernels keep their register budget).
// nin: elements of each line that may be nonzero (the rest is zero padding);
// when it is exactly half the length the first stage is pruned (every padded
// axis pads n to 2n, and the first radix of every schedule is even).
template <typename V, int DIR, int MR = 8, bool PRUNE = true>
__device__ __forceinline__ V* fft_lines(V* a, V* b, const FftSched& s, int ls, int nlines, const V* tw,
                                        int nin) {
  V* in = a;
  V* out = b;
  for (int st = 0; st < s.nst; ++st) {
    const int R = s.radix[st], Ns = s.ns[st];
    if (PRUNE && st == 0 && 2 * nin == s.L && R % 2 == 0) {
      switch (R) {
        case 2: stage_half<V, DIR, 2>(in, out, s.L, ls, nlines, tw); break;
        case 4: stage_half<V, DIR, 4>(in, out, s.L, ls, nlines, tw); break;
        case 16:
          if constexpr (MR == 16) stage_half<V, DIR, 16>(in, out, s.L, ls, nlines, tw);
          break;
        default: stage_half<V, DIR, 8>(in, out, s.L, ls, nlines, tw); break;
      }
      __syncthreads();
      V* t = in;
      in = out;
      out = t;
      continue;
    }
    switch (R) {
      case 2: stage_any<V, DIR, 2>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 3: stage_any<V, DIR, 3>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 4: stage_any<V, DIR, 4>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 5: stage_any<V, DIR, 5>(in, out, s.L, Ns, ls, nlines, tw); break;
      case 16:
        if constexpr (MR == 16) stage_any<V, DIR, 16>(in, out, s.L, Ns, ls, nlines, tw);
        break;
      default: stage_any<V, DIR, 8>(in, out, s.L, Ns, ls, nlines, tw); break;
    }
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
  }
  return in;
}

// Round-robin walk of the block's threads over (l, j) in [0, nl) x [0, J),
// with one division at the start.
struct LineIter {
  int l, j, dl, dj, J;
  __device__ explicit LineIter(int J_) : J(J_) {
    l = threadIdx.x / J;
    j = threadIdx.x - l * J;
    dl = blockDim.x / J;
    dj = blockDim.x - dl * J;
  }
  __device__ void next() {
    l += dl;
    j += dj;
    if (j >= J) {
      j -= J;
      ++l;
    }
  }
};

constexpr int kMaxLinesX = 64;
static_assert(kMaxLinesX >= kMaxLinesPerCta, "row-offset table of the x passes too small");
static_assert(kThreads >= kMaxLinesPerCta, "the y and z passes need one thread per column");

// Loads issued before their shared-memory stores, per thread and batch: the
// stores go through generic pointers that the compiler must assume may alias
// the loads, so without batching each thread would keep a single HBM load in
// flight.
template <typename V> struct LoadBatch { static constexpr int v = sizeof(V) == 8 ? 8 : 4; };

// line[pidx(y)] = y < nload ? col[y * stride] : 0 for y = y0, y0 + ystep, ... < L.
template <typename V>
__device__ __forceinline__ void load_column(V* line, const V* __restrict__ col, size_t stride, int y0,
                                            int ystep, int L, int nload) {
  constexpr int U = LoadBatch<V>::v;
  for (int yb = y0; yb < L; yb += U * ystep) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = yb + u * ystep;
      v[u] = y < nload ? col[(size_t)y * stride] : czero<V>();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = yb + u * ystep;
      if (y < L) line[pidx<V>(y)] = v[u];
    }
  }
}

// Spectrum offsets of the two rows of each pair handled by the block
// (row_offset needs a division per row).
template <typename V>
__device__ __forceinline__ void pair_offsets(const PassGeom& g, int p0, int nl, size_t* off) {
  for (int t = threadIdx.x; t < 2 * nl; t += blockDim.x) {
    const int row = 2 * p0 + t;
    off[t] = row < g.nrows ? row_offset(g, row) : 0;
  }
}

// XH: the rows are zero-padded to twice their length (free and wire BC); a
// separate build so that the unpadded one keeps its register budget.
template <typename V, int MR, bool XH>
__global__ void __launch_bounds__(kThreads) k_x_fwd(PassGeom g, FftSched s, const V* __restrict__ twg,
                                                   Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const double* __restrict__ in = a.in + slot * b.vstride;
  const double* __restrict__ scale = a.in_scale ? a.in_scale + slot * b.vstride : nullptr;
  const float* __restrict__ scale32 = a.in_scale32 ? a.in_scale32 + slot * b.vstride : nullptr;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ size_t woff[2 * kMaxLinesX];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L);
  V* b0 = tw + L;
  V* b1 = b0 + g.lines_x * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int npairs = (g.nrows + 1) >> 1;
  const int p0 = blockIdx.x * g.lines_x;
  const int nl = min(g.lines_x, npairs - p0);
  pair_offsets<V>(g, p0, nl, woff);
  const bool red = a.red_mu && b.st;
  double sum = 0.0;
  {
    constexpr int U = 4;
    // XH: the padded half (j >= nx = L/2) is never read -- the first stage
    // runs on the lower half only (fft_lines prunes it) -- so only the data
    // positions are staged
    LineIter it(XH ? g.nx : L);
    while (it.l < nl) {
      T va[U], vb[U];
      int dst[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        va[u] = T(0);
        vb[u] = T(0);
        dst[u] = -1;
        if (it.l < nl) {
          const int l = it.l, j = it.j;
          const int ra = 2 * (p0 + l);
          if (j < g.nx) {
            const size_t oa = (size_t)ra * g.nx + j;
            va[u] = load_scaled<V>(in, scale, oa, red, sum, scale32);
            if (ra + 1 < g.nrows) vb[u] = load_scaled<V>(in, scale, oa + g.nx, red, sum, scale32);
          }
          dst[u] = l * ls + pidx<V>(j);
          it.next();
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u] >= 0) b0[dst[u]] = mk<V>(va[u], vb[u]);
    }
  }
  __syncthreads();
  const V* res = fft_lines<V, -1, MR, XH>(b0, b1, s, ls, nl, tw, g.nx);
  const T half = T(0.5);
  for (LineIter it(g.Hx); it.l < nl; it.next()) {
    const int l = it.l, k = it.j;
    const V* line = res + l * ls;
    const V zk = line[pidx<V>(k)];
    const V zm = line[pidx<V>(k == 0 ? 0 : L - k)];
    // A_k = (Z_k + conj Z_(L-k))/2 ; B_k = -i (Z_k - conj Z_(L-k))/2
    W[woff[2 * l] + k] = mk<V>(half * (zk.x + zm.x), half * (zk.y - zm.y));
    if (2 * (p0 + l) + 1 < g.nrows) W[woff[2 * l + 1] + k] = mk<V>(half * (zk.y + zm.y), half * (zm.x - zk.x));
  }
  if (red)
    grid_reduce(sum, b.partials + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_MU], &b.st[slot].mu_sum);
}

template <typename V, int DIR, int MR>
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
  const size_t plane = (size_t)z * g.Py * g.Hp;
  const int nload = DIR < 0 ? g.ny : L;   // forward: rows y >= ny are the zero padding
  // thread -> (column c, first row y0); rows advance by ystep
  const int c = threadIdx.x % tile, y0 = threadIdx.x / tile, ystep = blockDim.x / tile;
  const bool act = c < nl && y0 < ystep;
  V* col = W + plane + kx0 + c;
  if (act) load_column<V>(b0 + c * ls, col, g.Hp, y0, ystep, L, nload);
  __syncthreads();
  const V* res = fft_lines<V, DIR, MR>(b0, b1, s, ls, nl, tw, nload);
  const int nstore = DIR < 0 ? L : g.ny;  // inverse: crop to y < ny
  if (act) {
    const V* line = res + c * ls;
    for (int y = y0; y < nstore; y += ystep) col[(size_t)y * g.Hp] = line[pidx<V>(y)];
  }
}

// ZH: the columns are zero-padded to twice their length (free and surface BC);
// a separate build, as for the x pass.
template <typename V, int MR, bool ZH>
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
  const size_t colbase = (size_t)ky * g.Hp + kx0;
  const size_t zstride = (size_t)g.Py * g.Hp;
  // thread -> (column c, first plane z0); planes advance by zstep
  const int c = threadIdx.x % tile, z0 = threadIdx.x / tile, zstep = blockDim.x / tile;
  const bool act = c < nl && z0 < zstep;
  V* col = W + colbase + c;
  if (act) load_column<V>(b0 + c * ls, col, zstride, z0, zstep, L, g.nz);
  __syncthreads();
  V* res = fft_lines<V, -1, MR, ZH>(b0, b1, s, ls, nl, tw, g.nz);
  V* other = (res == b0) ? b1 : b0;
  const int kyp = min(ky, g.Py - ky);
  const int hy = g.Py / 2 + 1;
  if (act) {
    const int kx = kx0 + c;
    const size_t t0 = (size_t)kyp * g.Hx + kx;   // + kzp * hy * Hx
    const size_t tz = (size_t)hy * g.Hx;
    V* line = res + c * ls;
    const bool at0 = use_k0 && kx == 0 && ky == 0;
    constexpr int U = 8;
    for (int kb = z0; kb < L; kb += U * zstep) {
      T t[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kz = min(kb + u * zstep, L - 1);
        const int kzp = min(kz, L - kz);
        const size_t ti = t0 + kzp * tz;
        if constexpr (std::is_same<V, float2>::value) {
          t[u] = a.table32 ? a.table32[ti] : d2f_rn(a.table[ti]);
        } else if constexpr (std::is_same<V, dfc>::value) {
          if (a.tabledf) {
            const float2 h = a.tabledf[ti];
            t[u] = df(h.x, h.y);
          } else {
            t[u] = df_of(a.table[ti]);
          }
        } else {
          t[u] = a.table[ti];
        }
      }
      if (at0 && kb == 0) {
        if constexpr (std::is_same<V, float2>::value) t[0] = d2f_rn(k0);
        else if constexpr (std::is_same<V, dfc>::value) t[0] = df_of(k0);
        else t[0] = k0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kz = kb + u * zstep;
        if (kz < L) {
          const int pk = pidx<V>(kz);
          line[pk] = cscale(line[pk], t[u]);
        }
      }
    }
  }
  __syncthreads();
  const V* fin = fft_lines<V, +1, MR, false>(res, other, s, ls, nl, tw, L);
  if (act) {
    const V* line = fin + c * ls;
    for (int z = z0; z < g.nz; z += zstep) col[(size_t)z * zstride] = line[pidx<V>(z)];
  }
}

template <typename V, int MR>
__global__ void __launch_bounds__(kThreads) k_x_inv(PassGeom g, FftSched s, const V* __restrict__ twg,
                                                   Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const V* __restrict__ W = reinterpret_cast<const V*>(a.W) + slot * a.wstride;
  double* __restrict__ out = a.out + slot * b.vstride;
  const double* __restrict__ out_scale = a.out_scale ? a.out_scale + slot * b.vstride : nullptr;
  const float* __restrict__ out_scale32 = a.out_scale32 ? a.out_scale32 + slot * b.vstride : nullptr;
  const double* __restrict__ dot_with = a.dot_with ? a.dot_with + slot * b.vstride : nullptr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ size_t woff[2 * kMaxLinesX];
  V* tw = reinterpret_cast<V*>(smem_raw);
  const int L = s.L, ls = line_stride<V>(L);
  V* b0 = tw + L;
  V* b1 = b0 + g.lines_x * ls;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
  const int npairs = (g.nrows + 1) >> 1;
  const int p0 = blockIdx.x * g.lines_x;
  const int nl = min(g.lines_x, npairs - p0);
  pair_offsets<V>(g, p0, nl, woff);
  __syncthreads();
  {
    // Each stored value k < Hx is loaded once and gives both Z_k and, by
    // Hermitian symmetry, Z_(L-k) = conj A_k + i conj B_k.
    constexpr int U = LoadBatch<V>::v / 2;
    LineIter it(g.Hx);
    while (it.l < nl) {
      V A[U], B[U];
      int dst[U], dstm[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        dst[u] = -1;
        dstm[u] = -1;
        A[u] = czero<V>();
        B[u] = czero<V>();
        if (it.l < nl) {
          const int l = it.l, k = it.j;
          const bool hasb = 2 * (p0 + l) + 1 < g.nrows;
          const V* wa = W + woff[2 * l];
          const V* wb = W + woff[2 * l + 1];
          A[u] = wa[k];
          if (hasb) B[u] = wb[k];
          if (k == 0 || 2 * k == L) { A[u].y = T(0); B[u].y = T(0); }   // DC and Nyquist are real
          dst[u] = l * ls + pidx<V>(k);
          if (k > 0 && 2 * k < L) dstm[u] = l * ls + pidx<V>(L - k);
          it.next();
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u] >= 0) {
          b0[dst[u]] = mk<V>(A[u].x - B[u].y, A[u].y + B[u].x);             // Z = A + i B
          if (dstm[u] >= 0) b0[dstm[u]] = mk<V>(A[u].x + B[u].y, B[u].x - A[u].y);   // conj A + i conj B
        }
    }
  }
  __syncthreads();
  const V* res = fft_lines<V, +1, MR, false>(b0, b1, s, ls, nl, tw, L);
  const bool want_wsum = a.red_wsum && b.st && b.st[slot].gauge;
  double dot = 0.0, wsum = 0.0;
  for (LineIter it(g.nx); it.l < nl; it.next()) {
    const int l = it.l, j = it.j;
    const int ra = 2 * (p0 + l);
    const V zz = res[l * ls + pidx<V>(j)];
    const size_t oa = (size_t)ra * g.nx + j;
    const double va = out_value<V>(zz.x, out_scale, oa, out_scale32);
    out[oa] = va;
    if (dot_with) dot += va * dot_with[oa];
    if (want_wsum) wsum += unscaled<V>(zz.x);
    if (ra + 1 < g.nrows) {
      const size_t ob = oa + g.nx;
      const double vb = out_value<V>(zz.y, out_scale, ob, out_scale32);
      out[ob] = vb;
      if (dot_with) dot += vb * dot_with[ob];
      if (want_wsum) wsum += unscaled<V>(zz.y);
    }
  }
  if (dot_with && b.st)
    if (grid_reduce(dot, b.partials + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_VR],
                    &b.st[slot].vr) && threadIdx.x == 0)
      b.st[slot].vdone = 1;
  if (want_wsum)
    grid_reduce(wsum, b.partials2 + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_WSUM],
                &b.st[slot].wsum);
}

// ---------------------------------------------------------------------------
// Launchers.

size_t x_lines_smem_bytes(int L, int lines, size_t vbytes) {
  const int ls = vbytes == sizeof(double2) ? line_stride<double2>(L) : line_stride<float2>(L);
  return (size_t)(L + 2 * lines * ls) * vbytes;
}

int default_lines(int L, int units, size_t vbytes) {
  int b = 2048 / (L > 0 ? L : 1);
  const int want = units / 304;   // keep >= ~2 CTAs per SM
  if (want < b) b = want;
  if (b > kMaxLinesPerCta) b = kMaxLinesPerCta;
  if (b < 1) b = 1;
  while (b > 1 && x_lines_smem_bytes(L, b, vbytes) > kMaxLinesSmem) --b;
  return b;
}

int x_pass_blocks(const PassGeom& g) {
  const int npairs = (g.nrows + 1) / 2;
  return (npairs + g.lines_x - 1) / g.lines_x;
}

// Opt a kernel in to `bytes` of dynamic shared memory.  The default limit
// (48 KB) covers static plus dynamic shared memory, and these kernels carry up
// to ~1.5 KB of static arrays (row offsets, reduction scratch), so the opt-in
// starts below 48 KB of dynamic memory.
template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes + kStaticSmemAllowance > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Whether the schedule takes the radix-16 build of a kernel (FP64 only).
template <typename V>
static bool radix16(const FftSched& s) {
  if constexpr (!std::is_same<V, double2>::value) {
    return false;
  } else {
    for (int k = 0; k < s.nst; ++k)
      if (s.radix[k] == 16) return true;
    return false;
  }
}

template <typename V, int MR>
static void x_fwd_mr(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b, const PipeArgs& a,
                     int nslots, size_t sm, cudaStream_t st) {
  count_launch();
  if (2 * g.nx == s.L) {
    set_smem(k_x_fwd<V, MR, true>, sm);
    k_x_fwd<V, MR, true><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
  } else {
    set_smem(k_x_fwd<V, MR, false>, sm);
    k_x_fwd<V, MR, false><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
  }
}

template <typename V>
void launch_x_fwd(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st) {
  if (launch_xr_pass<V>(false, s.L, g, tw, b, a, nslots, st)) return;
  const size_t sm = x_lines_smem_bytes(s.L, g.lines_x, sizeof(V));
  if constexpr (std::is_same<V, double2>::value)
    if (radix16<V>(s)) return x_fwd_mr<V, 16>(g, s, tw, b, a, nslots, sm, st);
  x_fwd_mr<V, 8>(g, s, tw, b, a, nslots, sm, st);
}

template <typename V>
void launch_y(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, bool inverse, int nslots, cudaStream_t st) {
  if (launch_col_pass<V>(inverse ? 1 : 0, s.L, g, tw, b, a, nslots, st)) return;
  dim3 grid((g.Hx + g.tile_y - 1) / g.tile_y, g.nz, nslots);
  const size_t sm = x_lines_smem_bytes(s.L, g.tile_y, sizeof(V));
  count_launch();
  if constexpr (std::is_same<V, double2>::value) {
    if (radix16<V>(s)) {
      if (inverse) {
        set_smem(k_y<V, +1, 16>, sm);
        k_y<V, +1, 16><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
      } else {
        set_smem(k_y<V, -1, 16>, sm);
        k_y<V, -1, 16><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
      }
      return;
    }
  }
  if (inverse) {
    set_smem(k_y<V, +1, 8>, sm);
    k_y<V, +1, 8><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  } else {
    set_smem(k_y<V, -1, 8>, sm);
    k_y<V, -1, 8><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  }
}

template <typename V>
void launch_z(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
              const PipeArgs& a, int nslots, cudaStream_t st) {
  if (launch_col_pass<V>(2, s.L, g, tw, b, a, nslots, st)) return;
  dim3 grid((g.Hx + g.tile_z - 1) / g.tile_z, g.Py, nslots);
  const size_t sm = x_lines_smem_bytes(s.L, g.tile_z, sizeof(V));
  count_launch();
  const bool zh = 2 * g.nz == s.L;
  if constexpr (std::is_same<V, double2>::value) {
    if (radix16<V>(s)) {
      if (zh) {
        set_smem(k_z<V, 16, true>, sm);
        k_z<V, 16, true><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
      } else {
        set_smem(k_z<V, 16, false>, sm);
        k_z<V, 16, false><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
      }
      return;
    }
  }
  if (zh) {
    set_smem(k_z<V, 8, true>, sm);
    k_z<V, 8, true><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  } else {
    set_smem(k_z<V, 8, false>, sm);
    k_z<V, 8, false><<<grid, kThreads, sm, st>>>(g, s, tw, b, a);
  }
}

template <typename V>
void launch_x_inv(const PassGeom& g, const FftSched& s, const V* tw, const Batch& b,
                  const PipeArgs& a, int nslots, cudaStream_t st) {
  if (launch_xr_pass<V>(true, s.L, g, tw, b, a, nslots, st)) return;
  const size_t sm = x_lines_smem_bytes(s.L, g.lines_x, sizeof(V));
  count_launch();
  if constexpr (std::is_same<V, double2>::value) {
    if (radix16<V>(s)) {
      set_smem(k_x_inv<V, 16>, sm);
      k_x_inv<V, 16><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
      return;
    }
  }
  set_smem(k_x_inv<V, 8>, sm);
  k_x_inv<V, 8><<<dim3(x_pass_blocks(g), 1, nslots), kThreads, sm, st>>>(g, s, tw, b, a);
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
