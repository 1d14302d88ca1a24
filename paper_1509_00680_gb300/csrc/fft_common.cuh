// Pieces shared by the spectrum-pass kernels: radix-R butterflies, the padded
// shared-memory line layout, and the slot test of a pass.
#pragma once

#include <type_traits>

#include "device_util.cuh"
#include "gps_internal.h"

namespace gps {

// Radix-R butterflies, DIR = -1 forward (e^{-2 pi i/R}), +1 inverse.
template <typename V, int DIR>
__device__ __forceinline__ V rot_i(V a) {  // a * (DIR * i)
  return DIR < 0 ? mk<V>(a.y, -a.x) : mk<V>(-a.y, a.x);
}

template <typename V, int DIR, int R> struct Dft;

// run_half(x): the same transform when x[R/2..R-1] are zero (the zero-padded
// half of a line in the first stage of a forward pass): X_(2m) is the R/2-point
// transform of x[0..R/2-1], X_(2m+1) that of x_r w^r, w = e^{DIR 2 pi i / R}.
template <typename V, int DIR> struct Dft<V, DIR, 2> {
  __device__ __forceinline__ static void run(V* x) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
  __device__ __forceinline__ static void run_half(V* x) { x[1] = x[0]; }
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
  __device__ __forceinline__ static void run_half(V* x) {
    const V o = rot_i<V, DIR>(x[1]);
    const V e0 = x[0], e1 = x[1];
    x[0] = cadd(e0, e1);
    x[2] = csub(e0, e1);
    x[1] = cadd(e0, o);
    x[3] = csub(e0, o);
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
  __device__ __forceinline__ static void run_half(V* x) {
    using T = typename Real<V>::T;
    const T c = (T)0.70710678118654752440;  // sqrt(1/2)
    V e[4] = {x[0], x[1], x[2], x[3]};
    V o[4] = {x[0], x[1], x[2], x[3]};
    // o_r *= e^{DIR 2 pi i r / 8}
    if (DIR < 0) {
      o[1] = mk<V>(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
      o[2] = mk<V>(o[2].y, -o[2].x);
      o[3] = mk<V>(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
    } else {
      o[1] = mk<V>(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y));
      o[2] = mk<V>(-o[2].y, o[2].x);
      o[3] = mk<V>(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y));
    }
    Dft<V, DIR, 4>::run(e);
    Dft<V, DIR, 4>::run(o);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      x[2 * m] = e[m];
      x[2 * m + 1] = o[m];
    }
  }
};

// 16 points as two 8-point transforms of the even and odd elements joined by
// the twiddles e^{DIR 2 pi i k / 16}, k = 0..7.
template <typename V, int DIR> struct Dft<V, DIR, 16> {
  __device__ __forceinline__ static V rot(V a, typename Real<V>::T cr, typename Real<V>::T sr) {
    // a (cr + i DIR sr)
    using T = typename Real<V>::T;
    const T si = DIR < 0 ? -sr : sr;
    return mk<V>(a.x * cr - a.y * si, a.x * si + a.y * cr);
  }
  __device__ __forceinline__ static void run(V* x) {
    using T = typename Real<V>::T;
    const T c1 = (T)0.92387953251128675613;   // cos(pi/8)
    const T s1 = (T)0.38268343236508977173;   // sin(pi/8)
    const T c = (T)0.70710678118654752440;    // sqrt(1/2)
    V e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      e[k] = x[2 * k];
      o[k] = x[2 * k + 1];
    }
    Dft<V, DIR, 8>::run(e);
    Dft<V, DIR, 8>::run(o);
    o[1] = rot(o[1], c1, s1);
    o[2] = rot(o[2], c, c);
    o[3] = rot(o[3], s1, c1);
    o[4] = DIR < 0 ? mk<V>(o[4].y, -o[4].x) : mk<V>(-o[4].y, o[4].x);
    o[5] = rot(o[5], -s1, c1);
    o[6] = rot(o[6], -c, c);
    o[7] = rot(o[7], -c1, s1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x[k] = cadd(e[k], o[k]);
      x[k + 8] = csub(e[k], o[k]);
    }
  }
  __device__ __forceinline__ static void run_half(V* x) {
    using T = typename Real<V>::T;
    const T c1 = (T)0.92387953251128675613;   // cos(pi/8)
    const T s1 = (T)0.38268343236508977173;   // sin(pi/8)
    const T c = (T)0.70710678118654752440;    // sqrt(1/2)
    V e[8], o[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) e[r] = x[r];
    o[0] = x[0];
    o[1] = rot(x[1], c1, s1);
    o[2] = rot(x[2], c, c);
    o[3] = rot(x[3], s1, c1);
    o[4] = DIR < 0 ? mk<V>(x[4].y, -x[4].x) : mk<V>(-x[4].y, x[4].x);
    o[5] = rot(x[5], -s1, c1);
    o[6] = rot(x[6], -c, c);
    o[7] = rot(x[7], -c1, s1);
    Dft<V, DIR, 8>::run(e);
    Dft<V, DIR, 8>::run(o);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      x[2 * m] = e[m];
      x[2 * m + 1] = o[m];
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
__host__ __device__ constexpr int line_stride(int L) { return L + (L >> PadShift<V>::v) + 1; }

__device__ __forceinline__ size_t row_offset(const PassGeom& g, int row) {
  const int y = row % g.ny, z = row / g.ny;
  return ((size_t)z * g.Py + y) * g.Hp;
}

constexpr int kThreads = 256;

// Upper bound on the static shared memory of a spectrum-pass kernel; a
// launcher opts a kernel in to more dynamic shared memory once dynamic plus
// this allowance may exceed the default 48 KB per block.
constexpr size_t kStaticSmemAllowance = 4096;


// Slot served by this block for a spectrum pass of precision V, or -1.
template <typename V>
__device__ __forceinline__ int pass_slot(const Batch& b) {
  int s = batch_slot(b);
  if (s >= 0 && b.st && b.prec >= 0 && b.st[s].spec != SpecOf<V>::v) s = -1;
  if (s >= 0) mark_acted(b);
  return s;
}

// Input value of the x pass: in * scale, rounded to the spectrum's real type.
// The FP32 spectrum multiplies in FP32 unless the FP64 sum of the products is
// wanted; conversions run on the integer pipe.
template <typename V>
__device__ __forceinline__ typename Real<V>::T load_scaled(const double* in, const double* scale,
                                                           size_t o, bool red, double& sum,
                                                           const float* scale32 = nullptr) {
  if constexpr (std::is_same<V, float2>::value) {
    if (red) {
      double v = in[o];
      if (scale) v *= scale[o];
      sum += v;
      return d2f_rn(v);
    }
    float v = d2f_rn(in[o]);
    if (scale32) v *= scale32[o];
    else if (scale) v *= d2f_rn(scale[o]);
    return v;
  } else {
    double v = in[o];
    if (scale) v *= scale[o];
    if (red) sum += v;
    if constexpr (std::is_same<V, dfc>::value) return df_of(v);
    else return v;
  }
}

// Real output value of the x inverse pass as a double (integer-pipe
// conversions; the FP32 spectrum scales in FP32).
template <typename V>
__device__ __forceinline__ double out_value(typename Real<V>::T z, const double* scale, size_t o,
                                            const float* scale32 = nullptr) {
  if constexpr (std::is_same<V, float2>::value) {
    float v = z;
    if (scale32) v *= scale32[o];
    else if (scale) v *= d2f_rn(scale[o]);
    return f2d(v);
  } else {
    double v;
    if constexpr (std::is_same<V, dfc>::value) v = dbl_of(z);
    else v = z;
    if (scale) v *= scale[o];
    return v;
  }
}

template <typename V>
__device__ __forceinline__ double unscaled(typename Real<V>::T z) {
  if constexpr (std::is_same<V, float2>::value) return f2d(z);
  else if constexpr (std::is_same<V, dfc>::value) return dbl_of(z);
  else return z;
}

}  // namespace gps
