// Per-precision engine: the pointwise kernels (x/r update with fused inner
// products, coefficient scaling, casts) and the host functions that launch
// every kernel of one storage type.  Included once per storage type by
// s7_engine_<type>.cu, which instantiates EngineImpl for its types.
#pragma once

#include <algorithm>
#include <type_traits>

#include <string.h>

#include "s7_handle.h"
#include "s7_resid.cuh"
#include "s7_step.cuh"
#include "s7_sweep.cuh"
#include "s7_sweep9.cuh"

namespace s7 {

// ---------------------------------------------------------------------------
// x_{i+1} = x_i + alpha p_i + omega q_i;  r_{i+1} = q_i - omega y_i;
// (r0, r_{i+1}) and (r_{i+1}, r_{i+1}) reduced;  beta_i, rho, history and
// the stopping test in the last block (Algorithm 1, lines after omega).
// ---------------------------------------------------------------------------
__device__ inline void finish_step(Scalars* sc, double rho_new, double rr, double* hist) {
  const int it = sc->iter + 1;
  const double h = sqrt(rr) / sc->bnorm;
  if (hist) hist[it] = h;
  sc->iter = it;
  sc->res[2] = h;
  if (sc->special) {
    sc->status = (h <= sc->tol) ? 0 : 3;
    sc->done = 1;
  } else if (h <= sc->tol) {
    sc->status = 0;
    sc->done = 1;
  } else if (rho_new == 0.0 || !isfinite(rho_new)) {
    sc->status = 3;
    sc->done = 1;
  } else {
    sc->beta = (sc->alpha / sc->omega) * (rho_new / sc->rho);
    sc->rho = rho_new;
    if (it >= sc->maxit) {
      sc->status = 4;
      sc->done = 1;
    }
  }
}

// Block `bid` of `nblk` blocks of the update over one system of n cells.
template <class T, class X, class A, int VEC>
__device__ __forceinline__ void update_body(long long n, const T* p0, const T* p1, const T* s0,
                                            const T* s1, const T* __restrict__ y,
                                            const T* __restrict__ rh, T* __restrict__ r,
                                            X* __restrict__ x, Scalars* sc, double* parts,
                                            double* hist, int bid, int nblk, double* red) {
  const int it = sc->iter;
  const T* __restrict__ p = (it & 1) ? p1 : p0;
  const T* __restrict__ s = (it & 1) ? s1 : s0;
  const A alpha = (A)sc->alpha, omega = (A)sc->omega;
  DotAcc<A, 2> acc;
  acc.init();
  const long long nvec = n / VEC;
  const long long stride = (long long)nblk * blockDim.x;
  int cnt = 0;
  for (long long v = (long long)bid * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    const long long i = v * VEC;
    A pv[VEC], sv[VEC], yv[VEC], rv[VEC], hv[VEC], xv[VEC];
    ldv<T, VEC, LD_STREAM>(r + i, rv);
    ldv<T, VEC, LD_STREAM>(s + i, sv);
    ldv<T, VEC, LD_STREAM>(p + i, pv);
    ldv<T, VEC, LD_STREAM>(y + i, yv);
    ldv<T, VEC, LD_STREAM>(rh + i, hv);
    ldv<X, VEC, LD_STREAM>(x + i, xv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const A q = q_of<T>(rv[k], sv[k], alpha);
      xv[k] = fma(omega, q, fma(alpha, pv[k], xv[k]));
      const A rn = as_stored<T>(fma(-omega, yv[k], q));
      rv[k] = rn;
      acc.part[0] = fma(hv[k], rn, acc.part[0]);
      acc.part[1] = fma(rn, rn, acc.part[1]);
    }
    stv<X, VEC, true>(x + i, xv);
    stv<T, VEC, true>(r + i, rv);
    if (++cnt == 8) {
      acc.fold();
      cnt = 0;
    }
  }
  if (bid == 0) {
    for (long long i = nvec * VEC + threadIdx.x; i < n; i += blockDim.x) {
      const A rv = to_acc<A>(r[i]), sv = to_acc<A>(s[i]);
      const A q = q_of<T>(rv, sv, alpha);
      x[i] = from_acc<X>(fma(omega, q, fma(alpha, to_acc<A>(p[i]), to_acc<A>(x[i]))));
      const A rn = as_stored<T>(fma(-omega, to_acc<A>(y[i]), q));
      r[i] = from_acc<T>(rn);
      acc.part[0] = fma(to_acc<A>(rh[i]), rn, acc.part[0]);
      acc.part[1] = fma(rn, rn, acc.part[1]);
    }
  }
  acc.fold();
  double vv[2] = {acc.tot[0], acc.tot[1]}, tot[2];
  block_sum<2>(vv, red);
  if (grid_combine<2>(parts, &sc->counter[CNT_C], nblk, bid, vv, tot, red) && threadIdx.x == 0)
    finish_step(sc, tot[0], tot[1], hist);
}

template <class T, class X, class A, int VEC>
__global__ void __launch_bounds__(256) k_update(long long n, const T* p0, const T* p1,
                                                const T* s0, const T* s1,
                                                const T* __restrict__ y, const T* __restrict__ rh,
                                                T* __restrict__ r, X* __restrict__ x, Scalars* sc,
                                                double* parts, double* hist) {
  __shared__ double red[32 * 4];
  if (*((volatile int*)&sc->done)) return;
  update_body<T, X, A, VEC>(n, p0, p1, s0, s1, y, rh, r, x, sc, parts, hist, blockIdx.x,
                            gridDim.x, red);
}

// Coefficient scaling to a unit diagonal (Sec. IV): out = c / diag computed
// in float64 and rounded once to the storage type; or a plain rounding when
// the raw operator is kept.
template <class RT, class T>
__global__ void k_scale(long long n, const RT* __restrict__ c, const RT* __restrict__ diag,
                        T* __restrict__ out, int jacobi) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double cv = (double)c[i];
    out[i] = from_acc<T>(jacobi ? cv / (double)diag[i] : cv);
  }
}

// Kept diagonal (for b~ = D^-1 b) and a count of unusable entries.
template <class RT, class DT>
__global__ void k_keep_diag(long long n, const RT* __restrict__ diag, DT* __restrict__ out,
                            unsigned int* bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned int nbad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double dv = (double)diag[i];
    if (dv == 0.0 || !isfinite(dv)) ++nbad;
    if (out) out[i] = from_acc<DT>(dv);
  }
  if (nbad) atomicAdd(bad, nbad);
}

template <class S, class D>
__global__ void k_cast(long long n, const S* __restrict__ src, D* __restrict__ dst) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = from_acc<D>(to_acc<double>(src[i]));
}

template <class V> __global__ void k_fill(long long n, V* dst, V v) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = v;
}

}  // namespace s7

// the batched kernels reuse update_body above
#include "s7_batch.cuh"

namespace s7 {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline int pointwise_grid(long long n, int per_thread) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long want = (n + 256LL * per_thread - 1) / (256LL * per_thread);
  long long cap = (long long)nsm * 8;
  return (int)std::max(1LL, std::min(want, cap));
}

// A 2D 9-point mesh is a Geom with ny = 1, nz = rows, plane = nx, tiles
// of bx runs by one row (see s7_sweep9.cuh).
inline Geom make_geom9(const Handle* h, int vec) {
  Geom g;
  g.nx = h->nx;
  g.ny = 1;
  g.nz = h->ny;
  const int runs = (h->nx + vec - 1) / vec;
  g.bx = std::min(h->tile.bx, runs);
  g.by = 1;
  g.tiles_x = (runs + g.bx - 1) / g.bx;
  g.tiles_y = 1;
  g.zchunk = std::min(h->tile.zchunk, h->ny);
  g.nchunks = (h->ny + g.zchunk - 1) / g.zchunk;
  g.plane = h->nx;
  return g;
}

inline Geom make_geom(const Handle* h, int vec) {
  if (h->stencil == 9) return make_geom9(h, vec);
  Geom g;
  g.nx = h->nx;
  g.ny = h->ny;
  g.nz = h->nz;
  g.bx = h->tile.bx;
  g.by = h->tile.by;
  const int runs = (h->nx + vec - 1) / vec;
  if (g.bx > runs) g.bx = runs;
  g.tiles_x = (runs + g.bx - 1) / g.bx;
  g.tiles_y = (h->ny + g.by - 1) / g.by;
  g.zchunk = h->tile.zchunk;
  g.nchunks = (h->nz + g.zchunk - 1) / g.zchunk;
  g.plane = (long long)h->nx * h->ny;
  return g;
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Allow `smem` bytes of dynamic shared memory for `kern`.  While `st` is
// being captured into a graph the attribute cannot be set; the solve driver
// sets it for the step kernels (prepare_capture) before it captures.
// Static shared memory of the sweep kernels is about 1 KB (reduction
// scratch); the opt-in is needed once static + dynamic exceeds 48 KB.
constexpr size_t kSmemNoOptIn = 48 * 1024 - 4096;

inline int allow_smem(const void* kern, size_t smem, cudaStream_t st) {
  if (smem <= kSmemNoOptIn) return S7_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return S7_ECUDA;
  if (cs != cudaStreamCaptureStatusNone) return S7_OK;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess
             ? S7_OK
             : S7_ECUDA;
}

template <class CT, class A, int VEC, class Src, class Epi>
int launch_sweep(const Geom& g, const CoefView<CT, A>& cf, const Src& src, const Epi& epi,
                 Scalars* sc, bool vl, cudaStream_t st) {
  const int threads = ((g.bx * g.by + 31) / 32) * 32;
  const size_t smem = (size_t)3 * (g.by + 2) * (g.bx * VEC + 2 * VEC) * sizeof(A);
  void (*kern)(Geom, CoefView<CT, A>, Src, Epi, Scalars*) =
      vl ? k_sweep<CT, A, VEC, true, Src, Epi> : k_sweep<CT, A, VEC, false, Src, Epi>;
  if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
  kern<<<s7_nblocks(g), threads, smem, st>>>(g, cf, src, epi, sc);
  return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
}

template <class CT, class A, int VEC, class P>
int launch_sweep1(const Geom& g, const CoefView<CT, A>& cf, const P& pol, Scalars* sc, bool vl,
                  cudaStream_t st) {
  const int threads = ((g.bx * g.by + 31) / 32) * 32;
  const size_t smem = (size_t)3 * (g.by + 2) * (g.bx * VEC + 2 * VEC) * sizeof(A);
  void (*kern)(Geom, CoefView<CT, A>, P, Scalars*) =
      vl ? k_sweep1<CT, A, VEC, true, P> : k_sweep1<CT, A, VEC, false, P>;
  if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
  kern<<<s7_nblocks(g), threads, smem, st>>>(g, cf, pol, sc);
  return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
}

template <class CT, class A, int VEC, class Src, class Epi>
int launch_sweep9(const Geom& g, const CoefView9<CT, A>& cf, const Src& src, const Epi& epi,
                  Scalars* sc, bool vl, cudaStream_t st) {
  const int threads = ((g.bx + 31) / 32) * 32;
  const size_t smem = sweep9_smem<A, VEC>(g);
  void (*kern)(Geom, CoefView9<CT, A>, Src, Epi, Scalars*) =
      vl ? k_sweep9<CT, A, VEC, true, Src, Epi> : k_sweep9<CT, A, VEC, false, Src, Epi>;
  if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
  kern<<<s7_nblocks(g), threads, smem, st>>>(g, cf, src, epi, sc);
  return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
}

template <class CT, class A, int VEC, class P>
int launch_sweep9_1(const Geom& g, const CoefView9<CT, A>& cf, const P& pol, Scalars* sc,
                    bool vl, cudaStream_t st) {
  const int threads = ((g.bx + 31) / 32) * 32;
  const size_t smem = sweep9_smem<A, VEC>(g);
  void (*kern)(Geom, CoefView9<CT, A>, P, Scalars*) =
      vl ? k_sweep9_1<CT, A, VEC, true, P> : k_sweep9_1<CT, A, VEC, false, P>;
  if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
  kern<<<s7_nblocks(g), threads, smem, st>>>(g, cf, pol, sc);
  return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
}

// ---- TMA tensor maps (host side) ----
static_assert(sizeof(StepMaps) <= kMapsBytes, "tensor maps do not fit their slot");
static_assert(sizeof(SysQueue) == kQueueBytes && sizeof(QueueState) <= kQueueStateBytes,
              "work queue layout");

typedef CUresult (*TensorMapEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                           const cuuint64_t*, const cuuint64_t*,
                                           const cuuint32_t*, const cuuint32_t*,
                                           CUtensorMapInterleave, CUtensorMapSwizzle,
                                           CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once (NULL if unavailable).
inline TensorMapEncodeTiledFn tensor_map_encoder() {
  static TensorMapEncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return (TensorMapEncodeTiledFn)f;
  }();
  return fn;
}

template <class E> struct TmaType;
template <> struct TmaType<double> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; };
template <> struct TmaType<float> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <> struct TmaType<__nv_bfloat16> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; };
template <> struct TmaType<__half> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; };

// Map of an nx*ny*nz array of E (x fastest) read in boxes of bw x bh x 1;
// cells outside the array read as zero.
template <class E>
inline bool encode_box(CUtensorMap* m, const void* base, int nx, int ny, int nz, int bw, int bh) {
  TensorMapEncodeTiledFn fn = tensor_map_encoder();
  if (!fn || !base || ((uintptr_t)base & 15u) || bw > 256 || bh > 256 ||
      ((size_t)bw * sizeof(E)) % 16)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(E), (cuuint64_t)nx * ny * sizeof(E)};
  if (strides[0] % 16) return false;
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, TmaType<E>::v, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class T_, class X_, class DT_, class A_>
struct EngineImpl {
  typedef T_ T;
  typedef X_ X;
  typedef DT_ DT;
  typedef A_ A;
  // cells per thread: 16-byte vectors for 32/64-bit storage; 16-bit storage
  // keeps 4 cells (8-byte vectors) so per-thread state, and with it
  // occupancy, matches the float32 kernels
  static constexpr int VEC = sizeof(T) >= 4 ? 16 / (int)sizeof(T) : 4;
  // arithmetic of the float64-accuracy residual sweeps: binary64 for float64
  // storage; double words (binary32 pairs, about 48 bits) otherwise, since
  // GB300's float64 rate would bound those sweeps far below HBM bandwidth
  typedef typename std::conditional<sizeof(T) == 8, double, dfl>::type RA;
  // the other width the pipelined sweeps can take: 8 cells (16 bytes) of
  // 16-bit storage per thread, which halves their per-cell overhead
  static constexpr int VW = sizeof(T) == 2 ? 8 : VEC;

  template <class AA>
  static CoefView<T, AA> stored(const Handle* h) {
    typedef typename CoefOf<AA>::t CA;
    CoefView<T, AA> cf;
    for (int d = 0; d < 6; ++d) {
      cf.c[d] = (const T*)h->c[d];
      cf.cc[d] = (CA)h->cconst[d];
    }
    cf.constant = h->constant;
    cf.diag = h->jacobi ? nullptr : (const T*)h->diag;
    cf.cdiag = h->jacobi ? CA(1) : (CA)h->cconst[6];
    return cf;
  }

  template <class AA>
  static CoefView9<T, AA> stored9(const Handle* h) {
    CoefView9<T, AA> cf;
    for (int d = 0; d < 8; ++d) cf.c[d] = (const T*)h->c[d];
    cf.diag = h->jacobi ? nullptr : (const T*)h->diag;
    cf.cdiag = 1;
    return cf;
  }

  // One sweep of the stored operator (7- or 9-point) with policies src/epi.
  template <class AA, int V, class Src, class Epi>
  static int run_sweep(const Handle* h, const Src& src, const Epi& epi, Scalars* sc, bool vl,
                       cudaStream_t st) {
    const Geom g = make_geom(h, V);
    if (h->stencil == 9) return launch_sweep9<T, AA, V>(g, stored9<AA>(h), src, epi, sc, vl, st);
    return launch_sweep<T, AA, V>(g, stored<AA>(h), src, epi, sc, vl, st);
  }

  // One float64-accuracy sweep (arithmetic R) of the raw float32 operator kept
  // by keep_true.
  template <int V, class R, class Src, class Epi>
  static int run_true_sweep(const Handle* h, const Src& src, const Epi& epi, Scalars* sc,
                            bool vl, cudaStream_t st) {
    const Geom g = make_geom(h, V);
    if (h->stencil == 9) {
      CoefView9<float, R> cf;
      for (int d = 0; d < 8; ++d) cf.c[d] = h->tc[d];
      cf.diag = h->tc[8];
      cf.cdiag = 1;
      return launch_sweep9<float, R, V>(g, cf, src, epi, sc, vl, st);
    }
    CoefView<float, R> cf;
    for (int d = 0; d < 6; ++d) {
      cf.c[d] = h->tc[d];
      cf.cc[d] = 0;
    }
    cf.diag = h->tc[6];
    cf.cdiag = 1;
    cf.constant = 0;
    return launch_sweep<float, R, V>(g, cf, src, epi, sc, vl, st);
  }

  static int scale(Handle* h, const void* const raw[7], s7_dtype raw_dt, cudaStream_t st, int* bad) {
    const long long n = h->n;
    const int grid = pointwise_grid(n, 4);
    unsigned int* d_bad = (unsigned int*)h->small;
    cudaMemsetAsync(d_bad, 0, sizeof(unsigned int), st);
#define S7_SCALE(RT)                                                                              \
  {                                                                                               \
    const RT* dg = (const RT*)raw[6];                                                             \
    k_keep_diag<RT, DT><<<grid, 256, 0, st>>>(n, dg, (DT*)h->d, d_bad);                           \
    for (int d = 0; d < 6; ++d)                                                                   \
      k_scale<RT, T><<<grid, 256, 0, st>>>(n, (const RT*)raw[d], dg, (T*)h->c[d], h->jacobi);      \
    if (!h->jacobi) k_scale<RT, T><<<grid, 256, 0, st>>>(n, dg, dg, (T*)h->diag, 0);              \
    for (int d = 0; d < 7 && h->keep_true; ++d)                                                   \
      k_cast<RT, float><<<grid, 256, 0, st>>>(n, (const RT*)raw[d], h->tc[d]);                     \
  }
    if (raw_dt == S7_F64) S7_SCALE(double) else S7_SCALE(float)
#undef S7_SCALE
    unsigned int hb = 0;
    cudaMemcpyAsync(&hb, d_bad, sizeof hb, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return S7_ECUDA;
    *bad = (int)hb;
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  static int scale9(Handle* h, const void* const raw[9], s7_dtype raw_dt, int columns,
                    cudaStream_t st, int* bad) {
    // neighbour offsets of xm xp ym yp xmym xpym xmyp xpyp, and the index of
    // the opposite direction (the column array a row entry comes from)
    static const int DX[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
    static const int DY[8] = {0, 0, -1, 1, -1, -1, 1, 1};
    static const int OPP[8] = {1, 0, 3, 2, 7, 6, 5, 4};
    const long long n = h->n;
    const int grid = pointwise_grid(n, 4);
    unsigned int* d_bad = (unsigned int*)h->small;
    cudaMemsetAsync(d_bad, 0, sizeof(unsigned int), st);
#define S7_SCALE9(RT)                                                                             \
  {                                                                                               \
    const RT* dg = (const RT*)raw[8];                                                             \
    k_keep_diag<RT, DT><<<grid, 256, 0, st>>>(n, dg, (DT*)h->d, d_bad);                           \
    for (int d = 0; d < 8; ++d) {                                                                 \
      const RT* src = (const RT*)raw[columns ? OPP[d] : d];                                       \
      k_scale9<RT, T><<<grid, 256, 0, st>>>(n, h->nx, h->ny, src, DX[d], DY[d], columns, dg,      \
                                            (T*)h->c[d], h->jacobi);                              \
      if (h->keep_true)                                                                           \
        k_scale9<RT, float><<<grid, 256, 0, st>>>(n, h->nx, h->ny, src, DX[d], DY[d], columns,    \
                                                  dg, h->tc[d], 0);                               \
    }                                                                                             \
    if (!h->jacobi) k_scale<RT, T><<<grid, 256, 0, st>>>(n, dg, dg, (T*)h->diag, 0);              \
    if (h->keep_true) k_cast<RT, float><<<grid, 256, 0, st>>>(n, dg, h->tc[8]);                    \
  }
    if (raw_dt == S7_F64) S7_SCALE9(double) else S7_SCALE9(float)
#undef S7_SCALE9
    unsigned int hb = 0;
    cudaMemcpyAsync(&hb, d_bad, sizeof hb, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return S7_ECUDA;
    *bad = (int)hb;
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  static int apply(Handle* h, const void* x, void* y, cudaStream_t st) {
    SrcPlain<T, A> src{(const T*)x};
    EpiStore<T, A> epi{(T*)y};
    const bool vl = (h->nx % VEC == 0) && aligned16(x) && aligned16(y);
    return run_sweep<A, VEC>(h, src, epi, nullptr, vl, st);
  }

  static int init(Handle* h, const void* b, cudaStream_t st) {
    Workspace& w = h->ws;
    SrcPlain<X, A> src{(const X*)w.x};
    EpiResid<X, T, DT, A> epi;
    epi.b = (const X*)b;
    epi.dinv = (h->jacobi && !h->constant) ? (const DT*)h->d : nullptr;
    epi.dc = (h->jacobi && h->constant) ? (A)h->cconst[6] : A(1);
    epi.dmul = nullptr;
    epi.dmc = A(1);
    epi.r_out = (T*)w.r;
    epi.rh_out = (T*)w.rh;
    epi.parts = w.parts;
    epi.counter = CNT_INIT;
    epi.mode = 0;
    const bool vl = (h->nx % VEC == 0) && aligned16(b);
    return run_sweep<A, VEC>(h, src, epi, w.sc, vl, st);
  }

  // The pipelined sweeps serve the common case: Jacobi-scaled per-cell
  // coefficients, rows of whole 16-byte vectors, at most 256 threads.
  // Kinds 0, 3 (p/s sweeps) follow bit 0 of pipe_kinds, kinds 1, 2 (q/y
  // sweeps) bit 1.
  template <int V = VEC>
  static bool pipelined(const Handle* h, const Geom& g, int kind) {
    const int bit = (kind == 0 || kind == 3) ? 0 : 1;
    return h->stencil == 7 && h->stages >= 2 && ((h->pipe_kinds >> bit) & 1) && h->jacobi &&
           !h->constant &&
           h->nx % V == 0 &&
           g.bx * g.by <= 256 &&
           step_smem_bytes<T, A, V>(g.bx, g.by, h->stages, kind) <= 200 * 1024;
  }

  // Geometry of the pipelined sweeps at V cells per thread: the tile keeps
  // its width in cells and its thread count, so with V > VEC it has fewer
  // threads across and more rows (a 16-bit tile of 128 x 4 cells at 4 cells
  // per thread becomes 128 x 8 at 8: less halo per row, and the same
  // number of warps per block).
  static Geom step_geom(const Handle* h, int v) {
    if (v == VEC) return make_geom(h, VEC);
    Handle t = *h;
    t.tile.bx = std::max(1, h->tile.bx * VEC / v);
    t.tile.by = std::max(1, std::min(h->ny, h->tile.by * v / VEC));
    return make_geom(&t, v);
  }

  // Tensor maps of the handle's arrays for the pipelined sweeps of geometry
  // g at V cells per thread (see StepMaps).  TMA needs the halo'd tile's x
  // origin, one vector left of the tile, on a 16-byte boundary: V cells of T
  // must be 16 bytes.
  template <int V>
  static bool encode_step_maps(const Handle* h, const Geom& g, StepMaps* m) {
    if (V * sizeof(T) != 16 || h->stencil != 7) return false;
    const Workspace& w = h->ws;
    const int TW = g.bx * V, W = TW + 2 * V, nx = h->nx, ny = h->ny, nz = h->nz;
    bool ok = true;
    for (int d = 0; d < 6; ++d) ok = ok && encode_box<T>(&m->c[d], h->c[d], nx, ny, nz, TW, g.by);
    ok = ok && encode_box<T>(&m->rh, w.rh, nx, ny, nz, TW, g.by);
    const void* ins[MAP_NIN] = {w.r, w.r2 ? w.r2 : w.r, w.p[0], w.p[1], w.s[0], w.s[1], w.y};
    for (int k = 0; k < MAP_NIN; ++k)
      ok = ok && encode_box<T>(&m->in[k], ins[k], nx, ny, nz, W, g.by + 2);
    ok = ok && encode_box<X>(&m->x, w.x, nx, ny, nz, TW, g.by);
    return ok;
  }

  // The handle's maps for geometry g at V cells per thread (host memory,
  // built when the handle holds none for that tile); NULL when TMA does not
  // apply.
  template <int V>
  static const StepMaps* maps_for(const Handle* hc, const Geom& g) {
    Handle* h = const_cast<Handle*>(hc);
    Workspace& w = h->ws;
    if (!h->tma || !w.ready) return nullptr;
    StepMaps* m = reinterpret_cast<StepMaps*>(w.maps);
    int* key = w.maps_key;
    if (key[0] == g.bx && key[1] == g.by && key[2] == V) return m;
    key[0] = 0;
    memset(m, 0, sizeof *m);
    if (!encode_step_maps<V>(h, g, m)) return nullptr;
    key[0] = g.bx;
    key[1] = g.by;
    key[2] = V;
    return m;
  }

  template <int KIND, int STAGES, int V = VEC>
  static int launch_step(const Handle* h, const Geom& g, cudaStream_t st) {
    const Workspace& w = h->ws;
    StepArgs<T> a;
    for (int d = 0; d < 6; ++d) a.c[d] = (const T*)h->c[d];
    a.r = (const T*)w.r;
    a.rh = (const T*)w.rh;
    a.pbuf[0] = (T*)w.p[0];
    a.pbuf[1] = (T*)w.p[1];
    a.sbuf[0] = (T*)w.s[0];
    a.sbuf[1] = (T*)w.s[1];
    a.y = (T*)w.y;
    a.parts = w.parts;
    a.rbuf[0] = (T*)w.r;
    a.rbuf[1] = (T*)w.r2;
    a.x = w.x;
    a.hist = w.hist;
    a.maps = nullptr;
    static const StepMaps none = {};
    const StepMaps* maps = maps_for<V>(h, g);
    const size_t smem = step_smem_bytes<T, A, V>(g.bx, g.by, STAGES, KIND);
    void (*kern)(Geom, StepArgs<T>, Scalars*, const StepMaps, int) =
        k_step<T, A, V, KIND, STAGES>;
    if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
    const int threads = ((g.bx * g.by + 31) / 32) * 32;
    kern<<<s7_nblocks(g), threads, smem, st>>>(g, a, w.sc, maps ? *maps : none, maps ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  // Shared-memory attributes of the step kernels, set outside any capture.
  static int prepare_capture(Handle* h) {
    const Geom g = make_geom(h, VEC);
    int rc = S7_OK;
    auto set = [&](const void* k, size_t bytes) {
      if (bytes > kSmemNoOptIn &&
          cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
              cudaSuccess)
        rc = S7_ECUDA;
    };
    if (h->stencil == 9) {
      const size_t b9 = sweep9_smem<A, VEC>(g);
      set((const void*)k_sweep9<T, A, VEC, true, SrcPUpdate<T, A>, EpiS<T, A>>, b9);
      set((const void*)k_sweep9<T, A, VEC, false, SrcPUpdate<T, A>, EpiS<T, A>>, b9);
      set((const void*)k_sweep9<T, A, VEC, true, SrcQ<T, A>, EpiY<T, A>>, b9);
      set((const void*)k_sweep9<T, A, VEC, false, SrcQ<T, A>, EpiY<T, A>>, b9);
      set((const void*)k_sweep9<T, A, VEC, true, SrcQ2<T, A>, EpiYMerged<T, A>>, b9);
      set((const void*)k_sweep9<T, A, VEC, false, SrcQ2<T, A>, EpiYMerged<T, A>>, b9);
      set((const void*)k_sweep9_1<T, A, VEC, true, MergedPass<T, X, A>>, b9);
      set((const void*)k_sweep9_1<T, A, VEC, false, MergedPass<T, X, A>>, b9);
      return rc;
    }
    const Geom gw = step_geom(h, VW);
    for (int kind = 0; kind < 4; ++kind) {
      if (h->step_vec == VW && VW != VEC) {
        if (!pipelined<VW>(h, gw, kind)) continue;
        set(step_fn<VW>(kind, h->stages), step_smem_bytes<T, A, VW>(gw.bx, gw.by, h->stages, kind));
      } else {
        if (!pipelined(h, g, kind)) continue;
        set(step_fn<VEC>(kind, h->stages), step_smem_bytes<T, A, VEC>(g.bx, g.by, h->stages, kind));
      }
    }
    const size_t gb = (size_t)3 * (g.by + 2) * (g.bx * VEC + 2 * VEC) * sizeof(A);
    set((const void*)k_sweep<T, A, VEC, true, SrcPUpdate<T, A>, EpiS<T, A>>, gb);
    set((const void*)k_sweep<T, A, VEC, false, SrcPUpdate<T, A>, EpiS<T, A>>, gb);
    set((const void*)k_sweep<T, A, VEC, true, SrcQ<T, A>, EpiY<T, A>>, gb);
    set((const void*)k_sweep<T, A, VEC, false, SrcQ<T, A>, EpiY<T, A>>, gb);
    set((const void*)k_sweep<T, A, VEC, true, SrcQ2<T, A>, EpiYMerged<T, A>>, gb);
    set((const void*)k_sweep<T, A, VEC, false, SrcQ2<T, A>, EpiYMerged<T, A>>, gb);
    set((const void*)k_sweep1<T, A, VEC, true, MergedPass<T, X, A>>, gb);
    set((const void*)k_sweep1<T, A, VEC, false, MergedPass<T, X, A>>, gb);
    return rc;
  }

  template <int V>
  static const void* step_fn(int kind, int stages) {
    static const void* const fns[4][3] = {
        {(const void*)k_step<T, A, V, 0, 2>, (const void*)k_step<T, A, V, 0, 3>,
         (const void*)k_step<T, A, V, 0, 4>},
        {(const void*)k_step<T, A, V, 1, 2>, (const void*)k_step<T, A, V, 1, 3>,
         (const void*)k_step<T, A, V, 1, 4>},
        {(const void*)k_step<T, A, V, 2, 2>, (const void*)k_step<T, A, V, 2, 3>,
         (const void*)k_step<T, A, V, 2, 4>},
        {(const void*)k_step<T, A, V, 3, 2>, (const void*)k_step<T, A, V, 3, 3>,
         (const void*)k_step<T, A, V, 3, 4>}};
    return fns[kind][std::min(std::max(stages, 2), 4) - 2];
  }

  template <int KIND, int V = VEC>
  static int launch_step_any(const Handle* h, const Geom& g, cudaStream_t st) {
    return h->stages == 4 ? launch_step<KIND, 4, V>(h, g, st)
         : h->stages == 3 ? launch_step<KIND, 3, V>(h, g, st) : launch_step<KIND, 2, V>(h, g, st);
  }

  // The pipelined form of step kind `kind` if it applies (rc in *rc), at the
  // handle's width.
  template <int KIND>
  static bool try_pipelined(const Handle* h, cudaStream_t st, int* rc) {
    if (h->step_vec == VW && VW != VEC) {
      const Geom gw = step_geom(h, VW);
      if (!pipelined<VW>(h, gw, KIND)) return false;
      *rc = launch_step_any<KIND, VW>(h, gw, st);
      return true;
    }
    const Geom g = make_geom(h, VEC);
    if (!pipelined(h, g, KIND)) return false;
    *rc = launch_step_any<KIND>(h, g, st);
    return true;
  }

  static int step_kernel(Handle* h, int which, cudaStream_t st) {
    const Geom g = make_geom(h, VEC);
    Workspace& w = h->ws;
    const bool vl = (h->nx % VEC == 0);
    int rc = S7_OK;
    if (which == 0 && try_pipelined<0>(h, st, &rc)) return rc;
    if (which == 1 && try_pipelined<1>(h, st, &rc)) return rc;
    if (which == 0) {
      SrcPUpdate<T, A> sa;
      sa.r = (const T*)w.r;
      sa.pbuf[0] = (T*)w.p[0];
      sa.pbuf[1] = (T*)w.p[1];
      sa.sbuf[0] = (T*)w.s[0];
      sa.sbuf[1] = (T*)w.s[1];
      EpiS<T, A> ea;
      ea.sbuf[0] = (T*)w.s[0];
      ea.sbuf[1] = (T*)w.s[1];
      ea.rh = (const T*)w.rh;
      ea.parts = w.parts;
      return run_sweep<A, VEC>(h, sa, ea, w.sc, vl, st);
    }
    if (which == 1) {
      SrcQ<T, A> sb;
      sb.r = (const T*)w.r;
      sb.sbuf[0] = (T*)w.s[0];
      sb.sbuf[1] = (T*)w.s[1];
      EpiY<T, A> eb;
      eb.y_out = (T*)w.y;
      eb.parts = w.parts;
      return run_sweep<A, VEC>(h, sb, eb, w.sc, vl, st);
    }
    k_update<T, X, A, VEC><<<pointwise_grid(h->n / VEC + 1, 1), 256, 0, st>>>(
        h->n, (const T*)w.p[0], (const T*)w.p[1], (const T*)w.s[0], (const T*)w.s[1],
        (const T*)w.y, (const T*)w.rh, (T*)w.r, (X*)w.x, w.sc, w.parts, w.hist);
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  static int merged_kernel(Handle* h, int which, cudaStream_t st) {
    if (which == 0) return step_kernel(h, 0, st);   // s_0 = A p_0 at step 0
    const Geom g = make_geom(h, VEC);
    Workspace& w = h->ws;
    const bool vl = (h->nx % VEC == 0);
    int rc = S7_OK;
    if (which == 1 && try_pipelined<2>(h, st, &rc)) return rc;
    if (which == 2 && try_pipelined<3>(h, st, &rc)) return rc;
    if (which == 1) {
      SrcQ2<T, A> sb;
      sb.rbuf[0] = (T*)w.r;
      sb.rbuf[1] = (T*)w.r2;
      sb.sbuf[0] = (T*)w.s[0];
      sb.sbuf[1] = (T*)w.s[1];
      EpiYMerged<T, A> eb;
      eb.y_out = (T*)w.y;
      eb.rh = (const T*)w.rh;
      eb.parts = w.parts;
      return run_sweep<A, VEC>(h, sb, eb, w.sc, vl, st);
    }
    MergedPass<T, X, A> m;
    m.rbuf[0] = (T*)w.r;
    m.rbuf[1] = (T*)w.r2;
    m.pbuf[0] = (T*)w.p[0];
    m.pbuf[1] = (T*)w.p[1];
    m.sbuf[0] = (T*)w.s[0];
    m.sbuf[1] = (T*)w.s[1];
    m.y = (const T*)w.y;
    m.rh = (const T*)w.rh;
    m.x = (X*)w.x;
    m.parts = w.parts;
    m.hist = w.hist;
    if (h->stencil == 9) return launch_sweep9_1<T, A, VEC>(g, stored9<A>(h), m, w.sc, vl, st);
    return launch_sweep1<T, A, VEC>(g, stored<A>(h), m, w.sc, vl, st);
  }

  // The float64-accuracy residual sweeps run in binary64 when the handle asks
  // for it (and always for float64 storage), else in double words.
  static bool resid_f64(const Handle* h) { return h->resid_f64 != 0; }

  // ||b~ - A~ x|| and ||b~|| with float64 accuracy -> sc->res[0], res[1].
  // ---- the specialised double-word residual sweep (s7_resid.cuh) ----
  // It applies to 7-point operators with per-cell coefficients, rows of
  // whole 4-cell vectors and 16-byte aligned buffers, when the residual runs
  // in double words (not for float64 storage or residual_f64).
  static bool resid_dw_ok(const Handle* h, const void* b, const void* x, const void* r) {
    return std::is_same<RA, dfl>::value && !resid_f64(h) && h->stencil == 7 && !h->constant &&
           h->nx % 4 == 0 && aligned16(b) && aligned16(x) && (!r || aligned16(r));
  }
  template <class CT, class XT, bool UNIT>
  static int launch_resid_dw(const Handle* h, const void* const* c, const void* diag,
                             const void* dinv, const XT* x, const XT* b, XT* r, double* parts,
                             Scalars* sc, cudaStream_t st) {
    const Geom g = make_geom(h, 4);
    ResidArgs<CT, XT, DT> a;
    for (int d = 0; d < 6; ++d) a.c[d] = (const CT*)c[d];
    a.diag = (const CT*)diag;
    a.dinv = (const DT*)dinv;
    a.x = x;
    a.b = b;
    a.r = r;
    a.parts = parts;
    a.counter = CNT_RES;
    const size_t smem = resid_dw_smem<XT>(g);
    void (*kern)(Geom, ResidArgs<CT, XT, DT>, Scalars*) = k_resid_dw<CT, XT, DT, UNIT>;
    if (allow_smem((const void*)kern, smem, st)) return S7_ECUDA;
    const int threads = ((g.bx * g.by + 31) / 32) * 32;
    kern<<<s7_nblocks(g), threads, smem, st>>>(g, a, sc);
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  static int true_resid(Handle* h, const void* b, cudaStream_t st) {
    if (h->jacobi && resid_dw_ok(h, b, h->ws.x, nullptr)) {
      const Workspace& w = h->ws;
      return launch_resid_dw<T, X, true>(h, h->c, nullptr, h->d, (const X*)w.x, (const X*)b,
                                         nullptr, w.parts, w.sc, st);
    }
    return resid_f64(h) ? true_resid_r<double>(h, b, st) : true_resid_r<RA>(h, b, st);
  }

  template <class R>
  static int true_resid_r(Handle* h, const void* b, cudaStream_t st) {
    Workspace& w = h->ws;
    SrcPlain<X, R> src{(const X*)w.x};
    EpiResid<X, T, DT, R> epi;
    epi.b = (const X*)b;
    epi.dinv = (h->jacobi && !h->constant) ? (const DT*)h->d : nullptr;
    epi.dc = (h->jacobi && h->constant) ? h->cconst[6] : 1.0;
    epi.dmul = nullptr;
    epi.dmc = 1.0;
    epi.r_out = nullptr;
    epi.rh_out = nullptr;
    epi.parts = w.parts;
    epi.counter = CNT_RES;
    epi.mode = 1;
    const bool vl = (h->nx % VEC == 0) && aligned16(b);
    return run_sweep<R, VEC>(h, src, epi, w.sc, vl, st);
  }

  template <class R, class XT>
  static int raw_resid_t(Handle* h, const XT* b, const XT* x, XT* r, cudaStream_t st) {
    Workspace& w = h->ws;
    if (h->keep_true && resid_dw_ok(h, b, x, r))
      return launch_resid_dw<float, XT, false>(h, (const void* const*)h->tc, h->tc[6], nullptr,
                                               x, b, r, w.parts, w.sc, st);
    if (h->keep_true) {
      constexpr int V = 16 / (int)sizeof(XT) < 4 ? 16 / (int)sizeof(XT) : 4;
      SrcPlain<XT, R> src{x};
      EpiResid<XT, XT, float, R> epi;
      epi.b = b;
      epi.dinv = nullptr;
      epi.dc = 1.0;
      epi.dmul = nullptr;
      epi.dmc = 1.0;
      epi.r_out = r;
      epi.rh_out = nullptr;
      epi.parts = w.parts;
      epi.counter = CNT_RES;
      epi.mode = 1;
      const bool vl = (h->nx % V == 0) && aligned16(b) && aligned16(x) && (!r || aligned16(r));
      return run_true_sweep<V, R>(h, src, epi, w.sc, vl, st);
    }
    SrcPlain<XT, R> src{x};
    EpiResid<XT, XT, DT, R> epi;
    epi.b = b;
    epi.dinv = nullptr;
    epi.dc = 1.0;
    epi.dmul = (h->jacobi && !h->constant) ? (const DT*)h->d : nullptr;
    epi.dmc = (h->jacobi && h->constant) ? h->cconst[6] : 1.0;
    epi.r_out = r;
    epi.rh_out = nullptr;
    epi.parts = w.parts;
    epi.counter = CNT_RES;
    epi.mode = 1;
    const bool vl = (h->nx % VEC == 0) && aligned16(b) && aligned16(x) && (!r || aligned16(r));
    return run_sweep<R, VEC>(h, src, epi, w.sc, vl, st);
  }

  template <class R>
  static int raw_resid_r(Handle* h, const void* b, const void* x, void* r, s7_dtype dt,
                         cudaStream_t st) {
    if (dt == S7_F64)
      return raw_resid_t<R, double>(h, (const double*)b, (const double*)x, (double*)r, st);
    return raw_resid_t<R, float>(h, (const float*)b, (const float*)x, (float*)r, st);
  }

  static int raw_resid(Handle* h, const void* b, const void* x, void* r, s7_dtype dt, cudaStream_t st) {
    return resid_f64(h) ? raw_resid_r<double>(h, b, x, r, dt, st)
                        : raw_resid_r<RA>(h, b, x, r, dt, st);
  }

  // The raw-system residual sweep with caller-supplied combine scratch.
  template <class R, class XT>
  static int raw_resid_into_t(Handle* h, const XT* b, const XT* x, XT* r, double* parts,
                              Scalars* sc, cudaStream_t st) {
    const bool al = aligned16(b) && aligned16(x) && (!r || aligned16(r));
    EpiResid<XT, XT, DT, R> epi;
    epi.b = b;
    epi.dinv = nullptr;
    epi.dc = 1.0;
    epi.r_out = r;
    epi.rh_out = nullptr;
    epi.parts = parts;
    epi.counter = CNT_RES;
    epi.mode = 1;
    SrcPlain<XT, R> src{x};
    if (h->keep_true && resid_dw_ok(h, b, x, r))
      return launch_resid_dw<float, XT, false>(h, (const void* const*)h->tc, h->tc[6], nullptr,
                                               x, b, r, parts, sc, st);
    if (h->keep_true) {
      constexpr int V = 16 / (int)sizeof(XT) < 4 ? 16 / (int)sizeof(XT) : 4;
      EpiResid<XT, XT, float, R> e2;
      e2.b = b;
      e2.dinv = nullptr;
      e2.dc = 1.0;
      e2.dmul = nullptr;
      e2.dmc = 1.0;
      e2.r_out = r;
      e2.rh_out = nullptr;
      e2.parts = parts;
      e2.counter = CNT_RES;
      e2.mode = 1;
      return run_true_sweep<V, R>(h, src, e2, sc, (h->nx % V == 0) && al, st);
    }
    epi.dmul = (h->jacobi && !h->constant) ? (const DT*)h->d : nullptr;
    epi.dmc = (h->jacobi && h->constant) ? h->cconst[6] : 1.0;
    return run_sweep<R, VEC>(h, src, epi, sc, (h->nx % VEC == 0) && al, st);
  }

  template <class R>
  static int raw_resid_into_r(Handle* h, const void* b, const void* x, void* r, s7_dtype dt,
                              double* parts, Scalars* sc, cudaStream_t st) {
    if (dt == S7_F64)
      return raw_resid_into_t<R, double>(h, (const double*)b, (const double*)x, (double*)r,
                                         parts, sc, st);
    return raw_resid_into_t<R, float>(h, (const float*)b, (const float*)x, (float*)r, parts, sc,
                                      st);
  }

  static int raw_resid_into(Handle* h, const void* b, const void* x, void* r, s7_dtype dt,
                            double* parts, Scalars* sc, cudaStream_t st) {
    return resid_f64(h) ? raw_resid_into_r<double>(h, b, x, r, dt, parts, sc, st)
                        : raw_resid_into_r<RA>(h, b, x, r, dt, parts, sc, st);
  }

  // Blocks of the raw residual sweep (the noalloc entry point checks its
  // scratch against this; either sweep may run, so the larger count).
  static long long raw_resid_blocks(const Handle* h, s7_dtype dt) {
    const int v = h->keep_true ? (dt == S7_F64 ? 2 : 4) : VEC;
    return std::max(s7_nblocks(make_geom(h, v)), s7_nblocks(make_geom(h, 4)));
  }

  static int cast(const void* src, s7_dtype sdt, void* dst, s7_dtype ddt, long long n, cudaStream_t st) {
    const int grid = pointwise_grid(n, 4);
    if (sdt == S7_F64 && ddt == S7_F32)
      k_cast<double, float><<<grid, 256, 0, st>>>(n, (const double*)src, (float*)dst);
    else if (sdt == S7_F32 && ddt == S7_F64)
      k_cast<float, double><<<grid, 256, 0, st>>>(n, (const float*)src, (double*)dst);
    else
      return S7_EINVAL;
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  static size_t parts_needed(const Handle* h) {
    size_t m = 0;
    const int vecs[3] = {VEC, 2, 4};
    for (int v : vecs) m = std::max(m, (size_t)s7_nblocks(make_geom(h, v)));
    m = std::max(m, (size_t)s7_nblocks(step_geom(h, VW)));
    m = std::max(m, (size_t)pointwise_grid(h->n / VEC + 1, 1));
    return 4 * m;
  }

  static int smem_ok(const Handle* h) {
    const Geom g = make_geom(h, VEC);
    if (h->stencil == 9) return g.bx <= 512 && sweep9_smem<double, VEC>(g) <= 200 * 1024;
    const size_t smem = (size_t)3 * (g.by + 2) * (g.bx * VEC + 2 * VEC) * sizeof(double);
    return smem <= 200 * 1024 && g.bx * g.by <= 512;
  }

  // ---- batched solves ----
  typedef SysDesc<T, X> Desc;

  static Geom geom_tile(const Handle* h, const Tile& t, int v) {
    Geom g;
    g.nx = h->nx;
    g.ny = h->ny;
    g.nz = h->nz;
    const int runs = (h->nx + v - 1) / v;
    g.bx = std::min(t.bx, runs);
    g.by = std::min(t.by, h->ny);
    g.tiles_x = (runs + g.bx - 1) / g.bx;
    g.tiles_y = (h->ny + g.by - 1) / g.by;
    g.zchunk = std::min(t.zchunk, h->nz);
    g.nchunks = (h->nz + g.zchunk - 1) / g.zchunk;
    g.plane = (long long)h->nx * h->ny;
    return g;
  }

  // Batched pipelined sweeps: VW cells per thread, 2 stages; the q/y sweep
  // too for 16-bit storage (as for single solves).
  static constexpr int SB = 2;
  static constexpr bool kPipeQ = sizeof(T) == 2;

  static int batch_pipe_ok(const Handle* h) {
    return h->stencil == 7 && h->jacobi && !h->constant && h->nx % VW == 0;
  }

  static void fill_desc(Handle* h, void* out, const Tile& t, const void* b, double* parts,
                        double* hist, Scalars* sc, int block0, int ublock0, int* nb, int* unb,
                        int pipe) {
    const int v = pipe ? VW : VEC;
    Desc d;
    memset(&d, 0, sizeof d);
    d.g = geom_tile(h, t, v);
    d.vl = (h->nx % v == 0) && aligned16(b);
    d.block0 = block0;
    d.nblocks = s7_nblocks(d.g);
    d.ublock0 = ublock0;
    const long long nvec = h->n / VEC;
    d.unblocks = (int)std::max(1LL, std::min(4096LL, (nvec + 1023) / 1024));
    // the persistent launch claims update tiles one by one: 8192 vectors a
    // tile keeps the claim a small part of the tile's time
    d.punblocks = (int)std::max(1LL, std::min(4096LL, (nvec + 8191) / 8192));
    d.constant = h->constant;
    d.n = h->n;
    for (int k = 0; k < 6; ++k) {
      d.c[k] = (const T*)h->c[k];
      d.cc[k] = h->cconst[k];
    }
    d.diag = h->jacobi ? nullptr : (const T*)h->diag;
    d.cdiag = h->jacobi ? 1.0 : h->cconst[6];
    d.d = (h->jacobi && !h->constant) ? h->d : nullptr;
    d.cdiv = (h->jacobi && h->constant) ? h->cconst[6] : 1.0;
    const Workspace& w = h->ws;
    d.r = (T*)w.r;
    d.r2 = (T*)w.r2;
    d.rh = (T*)w.rh;
    d.p[0] = (T*)w.p[0];
    d.p[1] = (T*)w.p[1];
    d.s[0] = (T*)w.s[0];
    d.s[1] = (T*)w.s[1];
    d.y = (T*)w.y;
    d.x = (X*)w.x;
    d.b = (const X*)b;
    d.parts = parts;
    d.hist = hist;
    d.sc = sc;
    memcpy(out, &d, sizeof d);
    *nb = d.nblocks;
    *unb = d.unblocks;
  }

  static size_t batched_smem(const Handle* h, const Tile& t, int pipe, int kind) {
    const int v = pipe ? VW : VEC;
    const Geom g = geom_tile(h, t, v);
    const size_t reg = (size_t)3 * (g.by + 2) * (g.bx * v + 2 * v) * sizeof(A);
    if (!pipe) return reg;
    switch (kind) {
      case 0: return step_smem_bytes<T, A, VW>(g.bx, g.by, SB, 0);
      case 1: return kPipeQ ? step_smem_bytes<T, A, VW>(g.bx, g.by, SB, 1) : reg;
      case 6: return step_smem_bytes<T, A, VW>(g.bx, g.by, SB, 2);
      case 7: return step_smem_bytes<T, A, VW>(g.bx, g.by, SB, 3);
      default: return reg;
    }
  }

  static int batched_prepare(size_t smem, int pipe) {
    if (smem <= kSmemNoOptIn) return S7_OK;
    const void* reg[6] = {(const void*)k_sweep_batched<T, X, DT, A, VEC, 0>,
                          (const void*)k_sweep_batched<T, X, DT, A, VEC, 1>,
                          (const void*)k_sweep_batched<T, X, DT, A, VEC, 2>,
                          (const void*)k_sweep_batched<T, X, DT, A, VEC, 3>,
                          (const void*)k_sweep_batched<T, X, DT, A, VEC, 4>,
                          (const void*)k_sweep_batched<T, X, DT, A, VEC, 5>};
    const void* wide[7] = {(const void*)k_step_batched<T, X, A, VW, 0, SB>,
                           (const void*)k_step_batched<T, X, A, VW, 1, SB>,
                           (const void*)k_step_batched<T, X, A, VW, 2, SB>,
                           (const void*)k_step_batched<T, X, A, VW, 3, SB>,
                           (const void*)k_sweep_batched<T, X, DT, A, VW, 1>,
                           (const void*)k_sweep_batched<T, X, DT, A, VW, 2>,
                           (const void*)k_sweep_batched<T, X, DT, A, VW, 3>};
    const void* const* ks = pipe ? wide : reg;
    const int nk = pipe ? 7 : 6;
    for (int k = 0; k < nk; ++k)
      if (cudaFuncSetAttribute(ks[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return S7_ECUDA;
    return S7_OK;
  }

  static int launch_batched(int kind, const void* descs, int nsys, int blocks, int threads,
                            size_t smem, cudaStream_t st, int pipe) {
    const Desc* d = (const Desc*)descs;
    if (pipe && (kind <= 3 || kind >= 6)) {
      switch (kind) {
        case 0: k_step_batched<T, X, A, VW, 0, SB><<<blocks, threads, smem, st>>>(d, nsys); break;
        case 6: k_step_batched<T, X, A, VW, 2, SB><<<blocks, threads, smem, st>>>(d, nsys); break;
        case 7: k_step_batched<T, X, A, VW, 3, SB><<<blocks, threads, smem, st>>>(d, nsys); break;
        case 1:
          if (kPipeQ) k_step_batched<T, X, A, VW, 1, SB><<<blocks, threads, smem, st>>>(d, nsys);
          else k_sweep_batched<T, X, DT, A, VW, 1><<<blocks, threads, smem, st>>>(d, nsys);
          break;
        case 2: k_sweep_batched<T, X, DT, A, VW, 2><<<blocks, threads, smem, st>>>(d, nsys); break;
        default: k_sweep_batched<T, X, DT, A, VW, 3><<<blocks, threads, smem, st>>>(d, nsys); break;
      }
      return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
    }
    switch (kind) {
      case 0: k_sweep_batched<T, X, DT, A, VEC, 0><<<blocks, threads, smem, st>>>(d, nsys); break;
      case 1: k_sweep_batched<T, X, DT, A, VEC, 1><<<blocks, threads, smem, st>>>(d, nsys); break;
      case 2: k_sweep_batched<T, X, DT, A, VEC, 2><<<blocks, threads, smem, st>>>(d, nsys); break;
      case 3: k_sweep_batched<T, X, DT, A, VEC, 3><<<blocks, threads, smem, st>>>(d, nsys); break;
      case 4: k_update_batched<T, X, A, VEC><<<blocks, 256, 0, st>>>(d, nsys); break;
      case 5: k_hist0_batched<T, X><<<(nsys + 127) / 128, 128, 0, st>>>(d, nsys); break;
      case 6: k_sweep_batched<T, X, DT, A, VEC, 4><<<blocks, threads, smem, st>>>(d, nsys); break;
      case 7: k_sweep_batched<T, X, DT, A, VEC, 5><<<blocks, threads, smem, st>>>(d, nsys); break;
      default: return S7_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? S7_OK : S7_ECUDA;
  }

  // ---- the persistent batched solve ----
  template <bool PIPE, bool MERGED>
  static const void* persistent_fn() {
    return (const void*)k_batched_persistent<T, X, DT, A, PIPE ? VW : VEC, VEC, SB, PIPE, MERGED,
                                             kPipeQ>;
  }
  static const void* persistent_of(int pipe, int merged) {
    return pipe ? (merged ? persistent_fn<true, true>() : persistent_fn<true, false>())
                : (merged ? persistent_fn<false, true>() : persistent_fn<false, false>());
  }

  static int persistent_occupancy(int threads, size_t smem, int pipe, int merged, int* per_sm) {
    const void* k = persistent_of(pipe, merged);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      return S7_ECUDA;
    }
    return S7_OK;
  }

  static int launch_persistent(const void* descs, const int* order, void* queues, void* qstate,
                               int nsys, int grid, int threads, size_t smem, long long budget,
                               cudaStream_t st, int pipe, int merged) {
    k_queue_init<T, X><<<(nsys + 255) / 256, 256, 0, st>>>((const Desc*)descs, nsys,
                                                           (SysQueue*)queues, (QueueState*)qstate);
    if (cudaGetLastError() != cudaSuccess) return S7_ECUDA;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all blocks resident at once
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[6] = {(void*)&descs, (void*)&order, (void*)&nsys, (void*)&queues, (void*)&qstate,
                     (void*)&budget};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, persistent_of(pipe, merged), args);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return S7_ECUDA;
    }
    return S7_OK;
  }

  static const Engine* get() {
    static const Engine e = {sizeof(T), sizeof(X), sizeof(DT), VEC, VW, &scale, &scale9, &apply,
                             &init, &step_kernel,
                             &true_resid, &raw_resid, &cast, &parts_needed, &smem_ok,
                             &raw_resid_into, &raw_resid_blocks, &prepare_capture,
                             &merged_kernel,
                             sizeof(Desc), &batch_pipe_ok, &fill_desc, &batched_smem,
                             &launch_batched, &batched_prepare, &persistent_occupancy,
                             &launch_persistent};
    return &e;
  }
};

}  // namespace s7
