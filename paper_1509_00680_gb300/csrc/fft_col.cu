// Register-resident column transforms of the y and z spectrum passes for
// power-of-two lengths L = 64 .. 1024 (the padded lengths of the common
// grids).  Other lengths use the shared-memory Stockham kernels of fft.cu.
//
// A CTA of 256 threads transforms TC = 256 / (L/E) adjacent columns of the
// spectrum; each thread holds E (8 or 16) elements of one column in
// registers.  The
// first Stockham stage reads its elements straight from HBM and the last one
// writes straight back; between stages the elements go through one padded
// shared-memory line per column.  All index arithmetic is compile-time.
//
// The z pass (Eq. PCGdef: forward FFT, multiply by the Green's-function
// table, inverse FFT, crop) runs the inverse with the forward's radices in
// reverse order: the forward's last stage leaves in each thread the elements
// b + r L/R that the inverse's first stage reads, so the table multiply and
// the hand-over between the two transforms happen in registers.
#include <cstdio>

#include "fft_common.cuh"
#include "tma.cuh"



namespace gps {
namespace {

// Radix plan: radix-8 stages, then one stage of radix L / 8^k when L is not a
// power of 8.  rev = true gives the stages in reverse order.
template <int L> struct ColPlan {
  static_assert(L == 64 || L == 128 || L == 256 || L == 512 || L == 1024, "unsupported length");
  static constexpr int nst = L == 64 ? 2 : L == 1024 ? 4 : 3;
  static constexpr int last = L == 128 ? 2 : L == 256 ? 4 : L == 1024 ? 2 : 8;
  __host__ __device__ static constexpr int radix(int s, bool rev) {
    return (rev ? nst - 1 - s : s) == nst - 1 ? last : 8;
  }
  __host__ __device__ static constexpr int ns(int s, bool rev) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix(i, rev);
    return p;
  }
};

// Twiddles of the stages, laid out per stage as W[s][r - 1][k] (k < Ns, the
// factor W_(Ns R)^(r k)), so that the threads of a warp, which hold
// consecutive k, read consecutive addresses (the index r k L/(Ns R) into the
// plain table scatters them).  The twiddle array of a length L served here
// holds three tables of L entries: the plain e^{-2 pi i m/L}, this layout for
// the forward radix order, and for the reversed order (built once per shape
// by the engine, col_stage_twiddle_index).  Offset of stage s in the layout:
template <int L, bool REV>
__host__ __device__ constexpr int stage_tw_offset(int s) {
  int o = 0;
  for (int i = 0; i < s; ++i) o += (ColPlan<L>::radix(i, REV) - 1) * ColPlan<L>::ns(i, REV);
  return o;
}
template <int L, bool REV>
__host__ __device__ constexpr int stage_tw_size() { return stage_tw_offset<L, REV>(ColPlan<L>::nst); }

// Butterflies of one stage (radix R, Ns = NS) on the thread's E elements:
// butterfly q is b = t + q L/E with inputs x[q R + r] = in[b + r L/R].
// tws: this stage's twiddles W[r - 1][k].  HALF (first stage only): the
// inputs r >= R/2 are the zero padding of the line (rows >= L/2), so each
// butterfly runs as two R/2-point ones (Dft::run_half).
template <typename V, int L, int E, int DIR, int R, int NS, bool HALF = false>
__device__ __forceinline__ void col_butterflies(V (&x)[E], int t, const V* tws) {
  constexpr int TPC = L / E, Q = E / R;
  static_assert(!HALF || NS == 1, "zero-half pruning applies to the first stage");
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if constexpr (NS > 1) {
      const int k = (t + q * TPC) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = tws[(r - 1) * NS + k];
        x[q * R + r] = DIR < 0 ? cmul(x[q * R + r], w) : cmulc(x[q * R + r], w);
      }
    }
    if constexpr (HALF) Dft<V, DIR, R>::run_half(x + q * R);
    else Dft<V, DIR, R>::run(x + q * R);
  }
}

// Scatter of a stage's outputs to out[(b - k) R + k + r Ns] in the column's
// shared line, then gather of the next stage's inputs in[b + r L/R2].
template <typename V, int L, int E, int R, int NS, int R2>
__device__ __forceinline__ void col_exchange(V (&x)[E], int t, V* line) {
  constexpr int TPC = L / E;
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int b = t + q * TPC;
    const int k = b & (NS - 1);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) line[pidx<V>(base + r * NS)] = x[q * R + r];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E / R2; ++q) {
    const int b = t + q * TPC;
#pragma unroll
    for (int r = 0; r < R2; ++r) x[q * R2 + r] = line[pidx<V>(b + r * (L / R2))];
  }
  __syncthreads();
}

// Stages S .. nst-1 of one transform.  On return x[q RL + r] = out[b + r L/RL]
// with RL the radix of the last stage.  HALF: the transform's input is zero
// beyond L/2 (pruned first stage).
template <typename V, int L, int E, int DIR, bool REV, int S, bool HALF = false>
__device__ __forceinline__ void col_stages(V (&x)[E], int t, const V* tw, V* line) {
  constexpr int R = ColPlan<L>::radix(S, REV), NS = ColPlan<L>::ns(S, REV);
  col_butterflies<V, L, E, DIR, R, NS, HALF && S == 0>(x, t, tw + stage_tw_offset<L, REV>(S));
  if constexpr (S + 1 < ColPlan<L>::nst) {
    col_exchange<V, L, E, R, NS, ColPlan<L>::radix(S + 1, REV)>(x, t, line);
    col_stages<V, L, E, DIR, REV, S + 1>(x, t, tw, line);
  }
}

enum ColMode { COL_Y_FWD = 0, COL_Y_INV = 1, COL_Z = 2 };

// Elements per thread: 16 for the FP32 spectrum at L >= 256 (wider column
// tiles, more loads in flight per thread), 8 otherwise.  MODE 3: x passes.
template <typename V, int L, int MODE> struct ColCfg {
  static constexpr bool f32 = std::is_same<V, float2>::value;
  static constexpr int E = (f32 && L >= 256) ? 16 : 8;
  // Resident CTAs per SM asked of the register allocator: 2 (128 registers a
  // thread) at 16 elements, 3 (85) otherwise.  Measured: the FP32 z pass at
  // 16 elements takes ~146 registers uncapped, fits one CTA per SM and runs
  // 1.6x slower; the df64 passes gain 2-3 % from the third CTA.
  static constexpr int B = (f32 && E == 16) ? 2 : 3;
};

template <typename V>
__device__ __forceinline__ typename Real<V>::T table_value(const PipeArgs& a, size_t i) {
  if constexpr (std::is_same<V, float2>::value) {
    return a.table32 ? a.table32[i] : d2f_rn(a.table[i]);
  } else if constexpr (std::is_same<V, dfc>::value) {
    if (a.tabledf) {
      const float2 h = a.tabledf[i];
      return df(h.x, h.y);
    }
    return df_of(a.table[i]);
  } else {
    return a.table[i];
  }
}

template <typename V>
__device__ __forceinline__ typename Real<V>::T real_of(double v) {
  if constexpr (std::is_same<V, float2>::value) return d2f_rn(v);
  else if constexpr (std::is_same<V, dfc>::value) return df_of(v);
  else return v;
}


// HALF (forward y and z passes of zero-padded axes): rows >= L/2 of every
// column are the padding; they are neither read nor transformed.
template <typename V, int L, int MODE, bool HALF>
__global__ void __launch_bounds__(kThreads, (ColCfg<V, L, MODE>::B)) k_col(PassGeom g, const V* __restrict__ twg, Batch b,
                                                 PipeArgs a) {
  constexpr int E = ColCfg<V, L, MODE>::E;
  constexpr int TPC = L / E, TC = kThreads / TPC, LS = line_stride<V>(L);
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const V* tw = twg + L;                           // forward-order stage twiddles (global, cached)
  const V* twr = twg + 2 * L;                      // reversed-order stage twiddles (z inverse)
  const int c = threadIdx.x % TC, t = threadIdx.x / TC;
  const int kx = blockIdx.x * TC + c;
  const bool act = kx < g.Hx;
  V* line = reinterpret_cast<V*>(smem_raw) + c * LS;
  size_t stride;
  V* col;
  int nload, nstore;
  if constexpr (MODE == COL_Z) {
    stride = (size_t)g.Py * g.Hp;
    col = W + (size_t)blockIdx.y * g.Hp + kx;
    nload = g.nz;
    nstore = g.nz;
  } else {
    stride = g.Hp;
    col = W + (size_t)blockIdx.y * g.Py * g.Hp + kx;
    nload = MODE == COL_Y_FWD ? g.ny : L;    // forward: rows y >= ny are the zero padding
    nstore = MODE == COL_Y_FWD ? L : g.ny;   // inverse: crop to y < ny
  }
  constexpr int R0 = ColPlan<L>::radix(0, false);
  V x[E];
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int row = t + q * TPC + r * (L / R0);
      if (HALF && r >= R0 / 2) x[q * R0 + r] = czero<V>();
      else x[q * R0 + r] = (act && row < nload) ? col[(size_t)row * stride] : czero<V>();
    }
  col_stages<V, L, E, MODE == COL_Y_INV ? +1 : -1, false, 0, HALF>(x, t, tw, line);
  constexpr int RL = ColPlan<L>::radix(ColPlan<L>::nst - 1, false);
  if constexpr (MODE == COL_Z) {
    const int ky = blockIdx.y;
    const int kyp = min(ky, g.Py - ky);
    const int hy = g.Py / 2 + 1;
    const size_t t0 = (size_t)kyp * g.Hx + (act ? kx : 0);
    const size_t tz = (size_t)hy * g.Hx;
    const bool use_k0 = a.slot_k0 && b.st && b.st[slot].use_k0;
    const bool at0 = use_k0 && kx == 0 && ky == 0;
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int kz = t + q * TPC + r * (L / RL);
        const int kzp = min(kz, L - kz);
        typename Real<V>::T tv = table_value<V>(a, t0 + (size_t)kzp * tz);
        if (at0 && kz == 0) tv = real_of<V>(b.st[slot].k0);
        x[q * RL + r] = cscale(x[q * RL + r], tv);
      }
    col_stages<V, L, E, +1, true, 0>(x, t, twr, line);
    // the reversed transform ends with radix R0
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int row = t + q * TPC + r * (L / R0);
        if (act && row < nstore) col[(size_t)row * stride] = x[q * R0 + r];
      }
  } else {
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int row = t + q * TPC + r * (L / RL);
        if (act && row < nstore) col[(size_t)row * stride] = x[q * RL + r];
      }
  }
}

template <typename V, int L, int MODE, bool HALF>
void launch_col_build(const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a, int nslots,
                      cudaStream_t st) {
  constexpr int TC = kThreads / (L / ColCfg<V, L, MODE>::E);
  const size_t sm = (size_t)(TC * line_stride<V>(L)) * sizeof(V);
  if (sm + kStaticSmemAllowance > 48 * 1024)
    cudaFuncSetAttribute(k_col<V, L, MODE, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const dim3 grid((g.Hx + TC - 1) / TC, MODE == COL_Z ? g.Py : g.nz, nslots);
  count_launch();
  k_col<V, L, MODE, HALF><<<grid, kThreads, sm, st>>>(g, tw, b, a);
}

template <typename V, int L, int MODE>
void launch_col_len(const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a, int nslots,
                    cudaStream_t st) {
  // zero-padded forward transforms: y of free and wire grids, z of free and surface grids
  const bool half = (MODE == COL_Y_FWD && 2 * g.ny == L) || (MODE == COL_Z && 2 * g.nz == L);
  if constexpr (MODE == COL_Y_INV) {
    launch_col_build<V, L, MODE, false>(g, tw, b, a, nslots, st);
  } else {
    if (half) launch_col_build<V, L, MODE, true>(g, tw, b, a, nslots, st);
    else launch_col_build<V, L, MODE, false>(g, tw, b, a, nslots, st);
  }
}

// ---- z pass with TMA-staged column tiles ----------------------------------
// The same transform, table multiply and inverse as k_col's z mode, but a
// persistent CTA walks over column tiles (TC adjacent kx of one ky, the nz
// planes that hold data), and each tile reaches shared memory by tensor
// loads (boxes of up to 256 planes) issued by one thread, double-buffered:
// the next tile is in flight while the current one is transformed.  Results
// go back into the tile and leave by tensor stores.  Per-thread global loads
// and their address arithmetic disappear from the loop, and the CTA's warps
// no longer wait on HBM latency between tiles.

constexpr uint32_t kTmaWaitLimit = 1u << 24;   // tests of a barrier before a wait gives up
__device__ unsigned int g_wait_timeouts;       // waits that gave up since the last check

template <typename V, int L>
struct ZTile {
  static constexpr int E = ColCfg<V, L, COL_Z>::E;
  static constexpr int TPC = L / E, TC = kThreads / TPC, LS = line_stride<V>(L);
  static constexpr int K8 = (int)(sizeof(V) / 8);   // 8-byte tensor elements per value
  // resident CTAs per SM asked of the register allocator: 2 (128 registers);
  // at 3 the df64 tiles spill (the loop keeps more state than k_col)
  static constexpr int B = 2;
};

template <typename V, int L, bool HALF>
__global__ void __launch_bounds__(kThreads, (ZTile<V, L>::B))
    k_colz_tma(PassGeom g, const V* __restrict__ twg, Batch b, PipeArgs a,
               const __grid_constant__ CUtensorMap tmap) {
  using Z = ZTile<V, L>;
  constexpr int E = Z::E, TPC = Z::TPC, TC = Z::TC, LS = Z::LS, K8 = Z::K8;
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int give_up;
  const int nz = g.nz;
  const size_t tile_elems = (size_t)nz * TC;
  V* tile0 = reinterpret_cast<V*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  V* tile1 = tile0 + tile_elems;
  V* lines = tile1 + tile_elems;
  const int c = threadIdx.x % TC, t = threadIdx.x / TC;
  V* line = lines + c * LS;
  const V* tw = twg + L;
  const V* twr = twg + 2 * L;
  const int nkb = (g.Hx + TC - 1) / TC;
  const int ntiles = nkb * g.Py;
  const uint32_t tile_bytes = (uint32_t)(tile_elems * sizeof(V));
  const int nbox = (nz + 255) / 256;
  auto issue = [&](int tile, V* dst, uint64_t* br) {
    const int kb = tile % nkb, ky = tile / nkb;
    mbar_arrive_expect_tx(br, tile_bytes);
    for (int bx = 0; bx < nbox; ++bx)
      tma_load_4d(dst + (size_t)bx * 256 * TC, &tmap, kb * TC * K8, ky, bx * 256, slot, br);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    give_up = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, tile0, &bar[0]);
  const int hy = g.Py / 2 + 1;
  const size_t tz = (size_t)hy * g.Hx;
  const bool use_k0 = a.slot_k0 && b.st && b.st[slot].use_k0;
  constexpr int R0 = ColPlan<L>::radix(0, false);
  constexpr int RL = ColPlan<L>::radix(ColPlan<L>::nst - 1, false);
  int i = 0;
  bool pending_next = false;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    V* cur = (i & 1) ? tile1 : tile0;
    V* nxt = (i & 1) ? tile0 : tile1;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0) {
      pending_next = false;
      if (next < ntiles) {
        bulk_wait_read_all();             // the store of the previous tile has read nxt
        issue(next, nxt, &bar[(i + 1) & 1]);
        pending_next = true;
      }
    }
    if (!mbar_wait_bounded(&bar[i & 1], (uint32_t)(i >> 1) & 1u, kTmaWaitLimit)) give_up = 1;
    __syncthreads();
    if (give_up) break;
    const int kb = tile % nkb, ky = tile / nkb;
    const int kx = kb * TC + c;
    const bool act = kx < g.Hx;
    V x[E];
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int row = t + q * TPC + r * (L / R0);
        if (HALF && r >= R0 / 2) x[q * R0 + r] = czero<V>();
        else x[q * R0 + r] = row < nz ? cur[(size_t)row * TC + c] : czero<V>();
      }
    col_stages<V, L, E, -1, false, 0, HALF>(x, t, tw, line);
    const int kyp = min(ky, g.Py - ky);
    const size_t t0 = (size_t)kyp * g.Hx + (act ? kx : 0);
    const bool at0 = use_k0 && kx == 0 && ky == 0;
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int kz = t + q * TPC + r * (L / RL);
        const int kzp = min(kz, L - kz);
        typename Real<V>::T tv = table_value<V>(a, t0 + (size_t)kzp * tz);
        if (at0 && kz == 0) tv = real_of<V>(b.st[slot].k0);
        x[q * RL + r] = cscale(x[q * RL + r], tv);
      }
    col_stages<V, L, E, +1, true, 0>(x, t, twr, line);
#pragma unroll
    for (int q = 0; q < E / R0; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const int row = t + q * TPC + r * (L / R0);
        if (row < nz) cur[(size_t)row * TC + c] = x[q * R0 + r];
      }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int bx = 0; bx < nbox; ++bx)
        tma_store_4d(&tmap, kb * TC * K8, ky, bx * 256, slot, cur + (size_t)bx * 256 * TC);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) {
    if (give_up) {
      // this tile's load and the prefetch of the next may still be in
      // flight: wait for them (bounded) before the CTA's shared memory goes
      mbar_wait_bounded(&bar[i & 1], (uint32_t)(i >> 1) & 1u, kTmaWaitLimit);
      if (pending_next) mbar_wait_bounded(&bar[(i + 1) & 1], (uint32_t)((i + 1) >> 1) & 1u, kTmaWaitLimit);
      atomicAdd(&g_wait_timeouts, 1u);
      if (b.st) {
        b.st[slot].status = GPS_ERR_TIMEOUT;
        b.st[slot].phase = PH_DONE;
      }
    }
    bulk_wait_all();                      // stores done before shared memory is released
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library); null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor map of the spectrum seen by the z pass: dims (8-byte elements of a
// row, ky, z, slot), strides from the row pitch Hp and the slot stride; box
// TC values x 1 x min(nz, 256) x 1.
template <typename V, int L>
bool encode_z_map(CUtensorMap* map, void* W, const PassGeom& g, size_t wstride, int nslots) {
  using Z = ZTile<V, L>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !W || (reinterpret_cast<uintptr_t>(W) & 15)) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.Hx * Z::K8, (cuuint64_t)g.Py, (cuuint64_t)g.nz,
                              (cuuint64_t)(nslots > 0 ? nslots : 1)};
  const cuuint64_t strides[3] = {(cuuint64_t)g.Hp * sizeof(V), (cuuint64_t)g.Py * g.Hp * sizeof(V),
                                 (cuuint64_t)(wstride ? wstride : (size_t)g.Py * g.Hp * g.nz) * sizeof(V)};
  for (cuuint64_t s : strides)
    if (s % 16) return false;
  const cuuint32_t box[4] = {(cuuint32_t)(Z::TC * Z::K8), 1u, (cuuint32_t)(g.nz < 256 ? g.nz : 256), 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, W, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename V, int L, bool HALF>
bool launch_colz_tma_build(const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a, int nslots,
                           cudaStream_t st) {
  using Z = ZTile<V, L>;
  // boxes of 256 planes must tile nz exactly (the tile in shared memory holds nz planes)
  if (g.nz % 2 || g.nz > 1024 || (g.nz > 256 && g.nz % 256)) return false;
  CUtensorMap map;
  if (!encode_z_map<V, L>(&map, a.W, g, a.wstride, nslots)) return false;
  const size_t sm = 128 + 2 * (size_t)g.nz * Z::TC * sizeof(V) + (size_t)Z::TC * Z::LS * sizeof(V);
  if (sm + kStaticSmemAllowance > 227 * 1024) return false;
  if (cudaFuncSetAttribute(k_colz_tma<V, L, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
      cudaSuccess)
    return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colz_tma<V, L, HALF>, kThreads, sm) !=
          cudaSuccess ||
      per_sm < 1)
    return false;
  const int ntiles = ((g.Hx + Z::TC - 1) / Z::TC) * g.Py;
  const int ns = nslots > 0 ? nslots : 1;
  int nb = (152 * per_sm + ns - 1) / ns;
  if (nb > ntiles) nb = ntiles;
  if (nb < 1) nb = 1;
  count_launch();
  k_colz_tma<V, L, HALF><<<dim3(nb, 1, ns), kThreads, sm, st>>>(g, tw, b, a, map);
  return true;
}

template <typename V, int L>
bool launch_colz_tma_len(const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a, int nslots,
                         cudaStream_t st) {
  if (2 * g.nz == L) return launch_colz_tma_build<V, L, true>(g, tw, b, a, nslots, st);
  return launch_colz_tma_build<V, L, false>(g, tw, b, a, nslots, st);
}

template <typename V, int MODE>
bool launch_col_mode(int L, const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a,
                     int nslots, cudaStream_t st) {
  switch (L) {
    case 64: launch_col_len<V, 64, MODE>(g, tw, b, a, nslots, st); return true;
    case 128: launch_col_len<V, 128, MODE>(g, tw, b, a, nslots, st); return true;
    case 256: launch_col_len<V, 256, MODE>(g, tw, b, a, nslots, st); return true;
    case 512: launch_col_len<V, 512, MODE>(g, tw, b, a, nslots, st); return true;
    case 1024: launch_col_len<V, 1024, MODE>(g, tw, b, a, nslots, st); return true;
    default: return false;
  }
}

// ---- register-resident x passes -----------------------------------------
// Lines are row pairs: two real rows of length nx, zero-padded to L = Px, as
// one complex transform (two-for-one real FFT).  A CTA transforms NL =
// 256 / (L/E) pairs; thread t of a pair holds elements t + q L/E + r L/R, so
// consecutive threads read and write consecutive elements of a row.

template <typename V, int L>
__global__ void __launch_bounds__(kThreads, (ColCfg<V, L, 3>::B)) k_xr_fwd(PassGeom g, const V* __restrict__ twg,
                                                                         Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  constexpr int E = ColCfg<V, L, 3>::E;
  constexpr int TPC = L / E, NL = kThreads / TPC, LS = line_stride<V>(L);
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const double* __restrict__ in = a.in + slot * b.vstride;
  const double* __restrict__ scale = a.in_scale ? a.in_scale + slot * b.vstride : nullptr;
  const float* __restrict__ scale32 = a.in_scale32 ? a.in_scale32 + slot * b.vstride : nullptr;
  V* __restrict__ W = reinterpret_cast<V*>(a.W) + slot * a.wstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = threadIdx.x / TPC, t = threadIdx.x % TPC;
  V* line = reinterpret_cast<V*>(smem_raw) + l * LS;
  const int npairs = (g.nrows + 1) >> 1;
  const int pr = blockIdx.x * NL + l;
  const bool act = pr < npairs;
  const int ra = 2 * pr;
  const bool hasb = act && ra + 1 < g.nrows;
  const bool red = a.red_mu && b.st;
  double sum = 0.0;
  constexpr int R0 = ColPlan<L>::radix(0, false);
  V x[E];
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int j = t + q * TPC + r * (L / R0);
      T va = T(0), vb = T(0);
      if (act && j < g.nx) {
        const size_t o = (size_t)ra * g.nx + j;
        va = load_scaled<V>(in, scale, o, red, sum, scale32);
        if (hasb) vb = load_scaled<V>(in, scale, o + g.nx, red, sum, scale32);
      }
      x[q * R0 + r] = mk<V>(va, vb);
    }
  col_stages<V, L, E, -1, false, 0>(x, t, twg + L, line);
  // Z in natural order; Z_k and Z_(L-k) meet through the line
  constexpr int RL = ColPlan<L>::radix(ColPlan<L>::nst - 1, false);
#pragma unroll
  for (int q = 0; q < E / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) line[pidx<V>(t + q * TPC + r * (L / RL))] = x[q * RL + r];
  __syncthreads();
  if (act) {
    V* wa = W + row_offset(g, ra);
    V* wb = hasb ? W + row_offset(g, ra + 1) : nullptr;
    const T half = T(0.5);
    for (int k = t; k < g.Hx; k += TPC) {
      const V zk = line[pidx<V>(k)];
      const V zm = line[pidx<V>(k == 0 ? 0 : L - k)];
      // A_k = (Z_k + conj Z_(L-k))/2 ; B_k = -i (Z_k - conj Z_(L-k))/2
      wa[k] = mk<V>(half * (zk.x + zm.x), half * (zk.y - zm.y));
      if (hasb) wb[k] = mk<V>(half * (zk.y + zm.y), half * (zm.x - zk.x));
    }
  }
  if (red)
    grid_reduce(sum, b.partials + (size_t)slot * b.pstride, &b.st[slot].counter[CNT_MU], &b.st[slot].mu_sum);
}

template <typename V, int L>
__global__ void __launch_bounds__(kThreads, (ColCfg<V, L, 3>::B)) k_xr_inv(PassGeom g, const V* __restrict__ twg,
                                                                         Batch b, PipeArgs a) {
  using T = typename Real<V>::T;
  constexpr int E = ColCfg<V, L, 3>::E;
  constexpr int TPC = L / E, NL = kThreads / TPC, LS = line_stride<V>(L);
  const int slot = pass_slot<V>(b);
  if (slot < 0) return;
  const V* __restrict__ W = reinterpret_cast<const V*>(a.W) + slot * a.wstride;
  double* __restrict__ out = a.out + slot * b.vstride;
  const double* __restrict__ out_scale = a.out_scale ? a.out_scale + slot * b.vstride : nullptr;
  const float* __restrict__ out_scale32 = a.out_scale32 ? a.out_scale32 + slot * b.vstride : nullptr;
  const double* __restrict__ dot_with = a.dot_with ? a.dot_with + slot * b.vstride : nullptr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = threadIdx.x / TPC, t = threadIdx.x % TPC;
  V* line = reinterpret_cast<V*>(smem_raw) + l * LS;
  const int npairs = (g.nrows + 1) >> 1;
  const int pr = blockIdx.x * NL + l;
  const bool act = pr < npairs;
  const int ra = 2 * pr;
  const bool hasb = act && ra + 1 < g.nrows;
  const V* wa = act ? W + row_offset(g, ra) : W;
  const V* wb = hasb ? W + row_offset(g, ra + 1) : W;
  constexpr int R0 = ColPlan<L>::radix(0, false);
  V x[E];
#pragma unroll
  for (int q = 0; q < E / R0; ++q)
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int k = t + q * TPC + r * (L / R0);
      V A = czero<V>(), B = czero<V>();
      if (act) {
        if (k < g.Hx) {
          A = wa[k];
          if (hasb) B = wb[k];
          if (k == 0 || 2 * k == L) { A.y = T(0); B.y = T(0); }   // DC and Nyquist are real
        } else {
          A = cconj(wa[L - k]);
          if (hasb) B = cconj(wb[L - k]);
        }
      }
      x[q * R0 + r] = mk<V>(A.x - B.y, A.y + B.x);   // Z = A + i B
    }
  col_stages<V, L, E, +1, false, 0>(x, t, twg + L, line);
  constexpr int RL = ColPlan<L>::radix(ColPlan<L>::nst - 1, false);
  const bool want_wsum = a.red_wsum && b.st && b.st[slot].gauge;
  double dot = 0.0, wsum = 0.0;
#pragma unroll
  for (int q = 0; q < E / RL; ++q)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int j = t + q * TPC + r * (L / RL);
      if (act && j < g.nx) {
        const V zz = x[q * RL + r];
        const size_t oa = (size_t)ra * g.nx + j;
        const double va = out_value<V>(zz.x, out_scale, oa, out_scale32);
        out[oa] = va;
        if (dot_with) dot += va * dot_with[oa];
        if (want_wsum) wsum += unscaled<V>(zz.x);
        if (hasb) {
          const size_t ob = oa + g.nx;
          const double vb = out_value<V>(zz.y, out_scale, ob, out_scale32);
          out[ob] = vb;
          if (dot_with) dot += vb * dot_with[ob];
          if (want_wsum) wsum += unscaled<V>(zz.y);
        }
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

template <typename V, int L>
void launch_xr_len(bool inverse, const PassGeom& g, const V* tw, const Batch& b, const PipeArgs& a,
                   int nslots, cudaStream_t st) {
  constexpr int NL = kThreads / (L / ColCfg<V, L, 3>::E);
  const size_t sm = (size_t)(NL * line_stride<V>(L)) * sizeof(V);
  const int npairs = (g.nrows + 1) / 2;
  const dim3 grid((npairs + NL - 1) / NL, 1, nslots);
  count_launch();
  if (inverse) {
    if (sm + kStaticSmemAllowance > 48 * 1024) cudaFuncSetAttribute(k_xr_inv<V, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_xr_inv<V, L><<<grid, kThreads, sm, st>>>(g, tw, b, a);
  } else {
    if (sm + kStaticSmemAllowance > 48 * 1024) cudaFuncSetAttribute(k_xr_fwd<V, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_xr_fwd<V, L><<<grid, kThreads, sm, st>>>(g, tw, b, a);
  }
}

}  // namespace

template <typename V>
bool launch_xr_pass(bool inverse, int L, const PassGeom& g, const V* tw, const Batch& b,
                    const PipeArgs& a, int nslots, cudaStream_t st) {
  // The df64 spectrum always takes these kernels (measured faster); the FP32
  // spectrum where the tuner found them faster than the shared-memory ones
  // (g.x_reg); the FP64 x passes are bound by the FP64 pipe and keep the
  // shared-memory kernels.
  if (std::is_same<V, double2>::value) return false;
  if (std::is_same<V, float2>::value && !g.x_reg) return false;
  switch (L) {
    case 64: launch_xr_len<V, 64>(inverse, g, tw, b, a, nslots, st); return true;
    case 128: launch_xr_len<V, 128>(inverse, g, tw, b, a, nslots, st); return true;
    case 256: launch_xr_len<V, 256>(inverse, g, tw, b, a, nslots, st); return true;
    case 512: launch_xr_len<V, 512>(inverse, g, tw, b, a, nslots, st); return true;
    case 1024: launch_xr_len<V, 1024>(inverse, g, tw, b, a, nslots, st); return true;
    default: return false;
  }
}

template bool launch_xr_pass<double2>(bool, int, const PassGeom&, const double2*, const Batch&,
                                      const PipeArgs&, int, cudaStream_t);
template bool launch_xr_pass<float2>(bool, int, const PassGeom&, const float2*, const Batch&,
                                     const PipeArgs&, int, cudaStream_t);
template bool launch_xr_pass<dfc>(bool, int, const PassGeom&, const dfc*, const Batch&,
                                  const PipeArgs&, int, cudaStream_t);

unsigned int take_wait_timeouts() {
  unsigned int n = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof(n)) != cudaSuccess) return 0;
  if (n) cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero));
  return n;
}

bool col_pass_supported(int L) {
  return L == 64 || L == 128 || L == 256 || L == 512 || L == 1024;
}

namespace {
template <int L>
void stage_index(int* idx) {
  for (int rev = 0; rev < 2; ++rev) {
    int* out = idx + rev * L;
    for (int i = 0; i < L; ++i) out[i] = 0;
    for (int s = 0; s < ColPlan<L>::nst; ++s) {
      const int R = ColPlan<L>::radix(s, rev != 0), NS = ColPlan<L>::ns(s, rev != 0);
      const int o = rev ? stage_tw_offset<L, true>(s) : stage_tw_offset<L, false>(s);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < NS; ++k) out[o + (r - 1) * NS + k] = r * k * (L / (NS * R));
    }
  }
}
}  // namespace

bool col_stage_twiddle_index(int L, int* idx) {
  switch (L) {
    case 64: stage_index<64>(idx); return true;
    case 128: stage_index<128>(idx); return true;
    case 256: stage_index<256>(idx); return true;
    case 512: stage_index<512>(idx); return true;
    case 1024: stage_index<1024>(idx); return true;
    default: return false;
  }
}

template <typename V>
bool launch_col_pass(int mode, int L, const PassGeom& g, const V* tw, const Batch& b,
                     const PipeArgs& a, int nslots, cudaStream_t st) {
  // The FP64 passes are bound by the FP64 pipe; they keep the shared-memory
  // kernels, which measured faster for them.
  if (std::is_same<V, double2>::value) return false;
  switch (mode) {
    case COL_Y_FWD: return launch_col_mode<V, COL_Y_FWD>(L, g, tw, b, a, nslots, st);
    case COL_Y_INV: return launch_col_mode<V, COL_Y_INV>(L, g, tw, b, a, nslots, st);
    default:
      // z pass: the TMA-staged kernel where the tuner chose it (and a tensor
      // map could be made), else the plain register-resident one
      if (g.z_tma) {
        bool done = false;
        switch (L) {
          case 64: done = launch_colz_tma_len<V, 64>(g, tw, b, a, nslots, st); break;
          case 128: done = launch_colz_tma_len<V, 128>(g, tw, b, a, nslots, st); break;
          case 256: done = launch_colz_tma_len<V, 256>(g, tw, b, a, nslots, st); break;
          case 512: done = launch_colz_tma_len<V, 512>(g, tw, b, a, nslots, st); break;
          case 1024: done = launch_colz_tma_len<V, 1024>(g, tw, b, a, nslots, st); break;
          default: break;
        }
        if (done) return true;
      }
      return launch_col_mode<V, COL_Z>(L, g, tw, b, a, nslots, st);
  }
}

template bool launch_col_pass<double2>(int, int, const PassGeom&, const double2*, const Batch&,
                                       const PipeArgs&, int, cudaStream_t);
template bool launch_col_pass<float2>(int, int, const PassGeom&, const float2*, const Batch&,
                                      const PipeArgs&, int, cudaStream_t);
template bool launch_col_pass<dfc>(int, int, const PassGeom&, const dfc*, const Batch&,
                                   const PipeArgs&, int, cudaStream_t);

}  // namespace gps
