// C ABI of the library (declared in include/stencil7.h): handle lifetime,
// workspace management, host/device staging, the solve driver that replays
// captured CUDA graphs of BiCGStab steps, and float64 iterative refinement.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cuda.h>

#include "s7_handle.h"
#include "s7_sweep.cuh"

using namespace s7;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? S7_ENOMEM : S7_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call)                                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

extern "C" const char* s7_last_error(void) { return g_err; }

namespace s7 {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace s7
extern "C" const char* s7_version(void) { return "stencil7-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static size_t dsize(s7_dtype t) {
  switch (t) {
    case S7_F64: return 8;
    case S7_F32: return 4;
    case S7_BF16:
    case S7_F16: return 2;
  }
  return 0;
}

namespace s7 {
const Engine* engine_for(s7_dtype t);
}
const Engine* s7::engine_for(s7_dtype t) {
  switch (t) {
    case S7_F64: return engine_f64();
    case S7_F32: return engine_f32();
    case S7_BF16: return engine_bf16();
    case S7_F16: return engine_f16();
  }
  return nullptr;
}

static s7_dtype xtype(const Handle* h) { return h->storage == S7_F64 ? S7_F64 : S7_F32; }

// True if p is device (or managed) memory; host memory otherwise.
static bool on_device(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of pinned (page-locked or registered) host memory that
// kernels can read in place; NULL for pageable host memory.
static const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The library carries its own CUDA runtime.  A caller (for instance PyTorch)
// selects a device by making that device's primary context current on the
// thread; bind this runtime to the same device before any work.
typedef CUresult (*CtxGetDeviceFn)(CUdevice*);

static void bind_caller_device() {
  static CtxGetDeviceFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetDevice", (void**)&fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
  }
  CUdevice d;
  if (fn && fn(&d) == CUDA_SUCCESS) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != (int)d) cudaSetDevice((int)d);
  }
  cudaGetLastError();
}


// ---------------------------------------------------------------------------
// device memory: one stream-ordered pool per device, owned by the library.
// A freed block stays in the pool (up to the cache limit) and the next
// operator of a similar size takes it without mapping memory again: mapping
// and unmapping tens of GB costs tens of milliseconds per create/destroy,
// as much as a few solver steps.  An allocation is synchronised on the stream
// it was made on, so any stream may use it on return; a block goes back to
// the pool ordered after the work already queued on the handle's stream.
// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static size_t g_cache_limit = (size_t)64 << 30;

static cudaError_t pool_of(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &pp);
    if (e != cudaSuccess) return e;
    unsigned long long thr = g_cache_limit;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// Pool allocation on device `dev` for use from any stream.  If the pool cannot
// grow, the blocks it caches are returned to the device and the call retried.
static cudaError_t pool_alloc(int dev, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool;
  cudaError_t e = pool_of(dev, &pool);
  if (e != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  }
  if (e == cudaErrorMemoryAllocation) {
    // a failed attempt can leave the pool holding memory it reserved while
    // growing: give back everything no live block uses
    cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}

cudaError_t s7::dev_alloc(int dev, void** p, size_t bytes, cudaStream_t st) {
  return pool_alloc(dev, p, bytes, st);
}

void s7::dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

static int dmalloc(Handle* h, void** p, size_t bytes, cudaStream_t st) {
  cudaError_t e = pool_alloc(h->device, p, bytes, st);
  if (e != cudaSuccess)
    return fail(S7_ENOMEM, "device allocation of %zu bytes failed: %s", bytes,
                cudaGetErrorString(e));
  h->bytes += bytes;
  return S7_OK;
}

static int dmalloc(Handle* h, void** p, size_t bytes) { return dmalloc(h, p, bytes, h->stream); }

// Return a block to the pool after the work queued on the handle's stream.
// Work on other streams that reads it must be complete (the API calls that
// issue such work finish it before they return; destroy synchronises the
// device first).
static void dfree(Handle* h, void** p, size_t bytes) {
  if (*p) {
    cudaFreeAsync(*p, h->stream);
    h->bytes -= bytes;
  }
  *p = nullptr;
}

// Pinned host buffers (scalar mirrors of handles and batches), kept on a free
// list for reuse: freeing pinned memory synchronises the whole device.
static std::mutex g_pin_mu;
static std::vector<std::pair<void*, size_t>> g_pin_free;
static std::map<void*, size_t> g_pin_size;   // capacity of every buffer made here

static cudaError_t pinned_get(void** out, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    size_t best = g_pin_free.size();
    for (size_t i = 0; i < g_pin_free.size(); ++i)
      if (g_pin_free[i].second >= bytes &&
          (best == g_pin_free.size() || g_pin_free[i].second < g_pin_free[best].second))
        best = i;
    if (best < g_pin_free.size()) {
      *out = g_pin_free[best].first;
      g_pin_free.erase(g_pin_free.begin() + best);
      return cudaSuccess;
    }
  }
  const size_t cap = std::max(bytes, (size_t)4096);
  cudaError_t e = cudaMallocHost(out, cap);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_size[*out] = cap;
  }
  return e;
}

static void pinned_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace_back(p, g_pin_size[p]);
}

static cudaError_t pinned_scalars(Scalars** out) {
  return pinned_get((void**)out, 2 * sizeof(Scalars));
}

static void pinned_scalars_put(Scalars* p) { pinned_put(p); }

extern "C" int s7_mem_stats(int device, size_t* reserved, size_t* used) {
  cudaMemPool_t pool;
  cudaError_t e = pool_of(device, &pool);
  if (e != cudaSuccess) return cuda_fail(e, "s7_mem_stats");
  unsigned long long r = 0, u = 0;
  if ((e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r)) != cudaSuccess ||
      (e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u)) != cudaSuccess)
    return cuda_fail(e, "s7_mem_stats");
  if (reserved) *reserved = (size_t)r;
  if (used) *used = (size_t)u;
  return S7_OK;
}

extern "C" int s7_mem_trim(int device, size_t keep) {
  cudaMemPool_t pool;
  cudaError_t e = pool_of(device, &pool);
  if (e != cudaSuccess) return cuda_fail(e, "s7_mem_trim");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "s7_mem_trim");
  e = cudaDeviceSynchronize();   // frees still queued on the device's streams
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, keep);
  if (cur >= 0 && cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(e, "s7_mem_trim");
  return S7_OK;
}

extern "C" int s7_mem_set_cache(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_cache_limit = bytes;
  unsigned long long thr = bytes;
  for (int d = 0; d < 64; ++d)
    if (g_pool[d]) cudaMemPoolSetAttribute(g_pool[d], cudaMemPoolAttrReleaseThreshold, &thr);
  return S7_OK;
}

// small kernels of the driver
__global__ void k_fill_f32(long long n, float* p, float v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// out = (X) (r / s): the refinement's inner right-hand side
template <class X>
__global__ void k_scaled_copy(long long n, const double* r, double inv_s, X* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (X)(r[i] * inv_s);
}

// x += s * d, in float64
template <class X>
__global__ void k_axpy_f64(long long n, double s, const X* d, double* x) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)d[i], x[i]);
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 16));
}

static int num_sms() {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

namespace s7 {
void default_tile(int nx, int ny, int nz, int vec, int nsm, Tile* t) {
  const int runs = (nx + vec - 1) / vec;
  const int ntx = (runs + 31) / 32;
  int bx = (runs + ntx - 1) / ntx;          // <= 32 runs per row, balanced tiles
  int by = std::max(1, std::min(ny, 128 / std::max(1, bx)));
  if (by > 16) by = 16;
  while (bx * by > 512) --by;
  const long long tiles = (long long)ntx * ((ny + by - 1) / by);
  // z chunk: long enough to amortise the two extra planes of each chunk,
  // short enough to give every SM several blocks
  const long long target = (long long)nsm * 8;
  long long zc = (tiles * nz + target - 1) / target;
  zc = std::max(4LL, std::min(64LL, zc));
  if (zc > nz) zc = nz;
  t->bx = bx;
  t->by = by;
  t->zchunk = (int)zc;
}

void default_tile9(int nx, int ny, int vec, int nsm, Tile* t) {
  const int runs = (nx + vec - 1) / vec;
  const int ntx = (runs + 127) / 128;
  const int bx = (runs + ntx - 1) / ntx;    // <= 128 runs per strip, balanced strips
  // rows per block: about 32 blocks per SM, so the last wave is a small
  // fraction of the sweep (measured on 22800^2: 97.7% of the copy peak per
  // step at ~200 rows against 92% at ~850), and at least 32 rows, so the two
  // extra rows each chunk reads stay a small fraction
  const long long target = (long long)nsm * 32;
  long long rc = ((long long)ntx * ny + target - 1) / target;
  rc = std::max(32LL, std::min(4096LL, rc));
  if (rc > ny) rc = ny;
  t->bx = bx;
  t->by = 1;
  t->zchunk = (int)rc;
}
}  // namespace s7

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
static void prof_free(Handle* h);

static void release(Handle* h) {
  Workspace& w = h->ws;
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w.graph = nullptr;
  const size_t ts = dsize(h->storage), xs = dsize(xtype(h));
  const size_t n = (size_t)h->n;
  dfree(h, &w.r, n * ts);
  dfree(h, &w.rh, n * ts);
  for (int k = 0; k < 2; ++k) {
    dfree(h, &w.p[k], n * ts);
    dfree(h, &w.s[k], n * ts);
  }
  dfree(h, &w.y, n * ts);
  dfree(h, &w.x, n * xs);
  dfree(h, &w.b, n * xs);
  dfree(h, &w.stage, n * 8);
  dfree(h, (void**)&w.parts, w.parts_n * 8);
  dfree(h, (void**)&w.hist, (size_t)w.hist_cap * 8);
  dfree(h, (void**)&w.sc, sizeof(Scalars));
  dfree(h, &w.r2, n * ts);
  dfree(h, &w.ref_x, n * 8);
  dfree(h, &w.ref_b, n * 8);
  dfree(h, &w.ref_r, n * 8);
  w.maps_key[0] = 0;
  pinned_scalars_put(w.h_sc);
  w.h_sc = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (w.snap[k]) cudaEventDestroy(w.snap[k]);
    w.snap[k] = nullptr;
  }
  w.ready = false;
  for (int d = 0; d < 8; ++d) dfree(h, &h->c[d], n * ts);
  dfree(h, &h->diag, n * ts);
  dfree(h, &h->d, n * dsize(xtype(h)));
  for (int d = 0; d < 9; ++d) dfree(h, (void**)&h->tc[d], n * 4);
  dfree(h, &h->small, 256);
  prof_free(h);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->aux_ev) cudaEventDestroy(h->aux_ev);
  if (h->aux) cudaStreamDestroy(h->aux);
  h->ev = nullptr;
  h->stream = nullptr;
  h->aux_ev = nullptr;
  h->aux = nullptr;
}

static double round_storage(double v, s7_dtype t) {
  switch (t) {
    case S7_F64: return v;
    case S7_F32: return (double)(float)v;
    case S7_BF16: return (double)__bfloat162float(__double2bfloat16(v));
    case S7_F16: return (double)__half2float(__double2half(v));
  }
  return v;
}

extern "C" int stencil7_create(stencil7_t* out, int nx, int ny, int nz, const s7_coeffs* c,
                               const s7_opts* o) {
  if (!out) return fail(S7_EINVAL, "stencil7_create: out is NULL");
  *out = nullptr;
  if (!c) return fail(S7_EINVAL, "stencil7_create: coeffs is NULL");
  if (nx < 1 || ny < 1 || nz < 1) return fail(S7_EINVAL, "stencil7_create: sizes must be >= 1");
  const long long n = (long long)nx * ny * nz;
  if (n >= (1LL << 40)) return fail(S7_EINVAL, "stencil7_create: mesh too large");
  if (c->dtype != S7_F64 && c->dtype != S7_F32)
    return fail(S7_EINVAL, "stencil7_create: raw coefficients must be S7_F64 or S7_F32");
  const void* raw_in[7] = {c->xm, c->xp, c->ym, c->yp, c->zm, c->zp, c->diag};
  for (int d = 0; d < 7; ++d)
    if (!raw_in[d]) return fail(S7_EINVAL, "stencil7_create: coefficient pointer %d is NULL", d);
  s7_opts opts;
  memset(&opts, 0, sizeof opts);
  if (o) opts = *o;
  bind_caller_device();
  const Engine* eng = engine_for(opts.storage);
  if (!eng) return fail(S7_EINVAL, "stencil7_create: unknown storage type %d", (int)opts.storage);

  stencil7_op* h = new (std::nothrow) stencil7_op();
  if (!h) return fail(S7_ENOMEM, "stencil7_create: host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->n = n;
  h->storage = opts.storage;
  h->jacobi = opts.no_jacobi ? 0 : 1;
  h->keep_true = opts.keep_true ? 1 : 0;
  h->constant = c->constant ? 1 : 0;
  cudaGetDevice(&h->device);
  default_tile(nx, ny, nz, eng->vec, num_sms(), &h->tile);
  if (opts.bx > 0) h->tile.bx = opts.bx;
  if (opts.by > 0) h->tile.by = opts.by;
  if (opts.zchunk > 0) h->tile.zchunk = std::min(opts.zchunk, nz);
  if (h->tile.bx * h->tile.by > 512) {
    delete h;
    return fail(S7_EINVAL, "stencil7_create: bx*by must be <= 512");
  }
  // iterations per graph launch: about a millisecond of work per launch
  {
    const double est_us = std::max(15.0, 120.0 * (double)n / 6.0e6);
    int ce = (int)std::min(64.0, std::max(2.0, 1000.0 / est_us));
    h->check_every = opts.check_every > 0 ? opts.check_every : ce;
  }
  // Defaults measured on GB300.  float32 (600x595 planes): a 2-stage
  // pipeline for both sweeps (the q/y sweep 2.91 ms pipelined against 3.18 ms
  // in registers at 600x595x1536, once the on-the-fly vector's ring held two
  // planes); float64: the p/s sweep only, whose register version is limited
  // by occupancy.  16-bit storage (512^2 planes):
  // both sweeps are bound by instruction issue at half the bytes per cell;
  // 8 cells (one 16-byte copy per array) per thread halve the per-cell
  // overhead, and both sweeps take a 2-stage pipeline (1.57 vs 1.84 ms per
  // step at 4 cells and 3 stages).  The two-reduction variant's passes
  // carry more streams per cell (r0 in the q/y pass; r, s, y, p and x in the
  // fused pass), and both run fastest with 2 stages for every storage type
  // (deeper stages cost occupancy).
  if (opts.variant < 0 || opts.variant > 1) {
    delete h;
    return fail(S7_EINVAL, "stencil7_create: variant must be 0 or 1");
  }
  const bool half = opts.storage == S7_BF16 || opts.storage == S7_F16;
  const int def_stages = 2;
  const int def_kinds = (opts.variant == 1 || half || opts.storage == S7_F32) ? 3 : 1;
  h->stages = opts.stages > 0 ? std::min(opts.stages, 4) : def_stages;
  h->pipe_kinds = opts.pipe_kinds > 0 ? (opts.pipe_kinds & 3) : def_kinds;
  if (opts.step_cells != 0 && opts.step_cells != eng->vec && !(half && opts.step_cells == 8)) {
    delete h;
    return fail(S7_EINVAL, "stencil7_create: step_cells must be 0, %d%s", eng->vec,
                half ? " or 8" : "");
  }
  h->step_vec = opts.step_cells > 0 ? opts.step_cells : (half ? 8 : eng->vec);
  h->variant = opts.variant;
  h->resid_f64 = opts.residual_f64 ? 1 : 0;
  h->tma = opts.tma ? 1 : 0;
  if (!eng->smem_ok(h)) {
    delete h;
    return fail(S7_EINVAL, "stencil7_create: tile too large for shared memory");
  }

  int rc = S7_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "stream/event creation");
    release(h);
    delete h;
    return rc;
  }
  const size_t ts = eng->t_size;
  if ((rc = dmalloc(h, &h->small, 256))) goto fail_out;

  if (h->constant) {
    // read the seven scalars (host or device) and scale on the host in float64
    double v[7];
    for (int d = 0; d < 7; ++d) {
      if (c->dtype == S7_F64) {
        double t;
        if ((e = cudaMemcpy(&t, raw_in[d], 8, cudaMemcpyDefault)) != cudaSuccess) break;
        v[d] = t;
      } else {
        float t;
        if ((e = cudaMemcpy(&t, raw_in[d], 4, cudaMemcpyDefault)) != cudaSuccess) break;
        v[d] = t;
      }
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "reading constant coefficients");
      goto fail_out;
    }
    if (v[6] == 0.0 || !isfinite(v[6])) {
      rc = fail(S7_EINVAL, "stencil7_create: zero or non-finite diagonal");
      goto fail_out;
    }
    for (int d = 0; d < 6; ++d)
      h->cconst[d] = round_storage(h->jacobi ? v[d] / v[6] : v[d], h->storage);
    h->cconst[6] = h->jacobi ? v[6] : round_storage(v[6], h->storage);
    if (h->keep_true) {
      // true operator as float32 arrays (the raw-residual sweep reads arrays)
      for (int d = 0; d < 7; ++d) {
        if ((rc = dmalloc(h, (void**)&h->tc[d], (size_t)n * 4))) goto fail_out;
      }
    }
  } else {
    for (int d = 0; d < 6; ++d)
      if ((rc = dmalloc(h, &h->c[d], (size_t)n * ts))) goto fail_out;
    if (!h->jacobi && (rc = dmalloc(h, &h->diag, (size_t)n * ts))) goto fail_out;
    if (h->jacobi && (rc = dmalloc(h, &h->d, (size_t)n * dsize(xtype(h))))) goto fail_out;
    if (h->keep_true)
      for (int d = 0; d < 7; ++d)
        if ((rc = dmalloc(h, (void**)&h->tc[d], (size_t)n * 4))) goto fail_out;
  }
  if (!h->constant) {
    // Raw arrays are read where they are when the kernels can reach them:
    // device memory, and for the six off-diagonals (each read once, unless
    // keep_true casts them again) pinned host memory, which the scaling
    // kernels stream over the host link as fast as a copy engine moves it.
    // Other host arrays are first copied to pool blocks.
    const size_t rs = dsize(c->dtype);
    const void* raw_dev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void* stage[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int d = 0; d < 7 && rc == S7_OK; ++d) {
      if (on_device(raw_in[d])) {
        raw_dev[d] = raw_in[d];
        continue;
      }
      const void* m = (d < 6 && !h->keep_true) ? mapped_host(raw_in[d]) : nullptr;
      if (m) {
        raw_dev[d] = m;
        continue;
      }
      if ((e = pool_alloc(h->device, &stage[d], (size_t)n * rs, h->stream)) != cudaSuccess)
        rc = fail(S7_ENOMEM, "staging coefficients: %s", cudaGetErrorString(e));
      raw_dev[d] = stage[d];
    }
    for (int d = 0; d < 7 && rc == S7_OK; ++d)
      if (stage[d] &&
          (e = cudaMemcpyAsync(stage[d], raw_in[d], (size_t)n * rs, cudaMemcpyDefault,
                               h->stream)) != cudaSuccess)
        rc = cuda_fail(e, "copying coefficients");
    if (rc == S7_OK) {
      int bad = 0;
      rc = eng->scale(h, raw_dev, c->dtype, h->stream, &bad);
      if (rc) rc = fail(rc, "coefficient scaling failed: %s", cudaGetErrorString(cudaGetLastError()));
      else if (bad) rc = fail(S7_EINVAL, "stencil7_create: %d zero or non-finite diagonal entries", bad);
    }
    cudaStreamSynchronize(h->stream);
    for (int d = 0; d < 7; ++d)
      if (stage[d]) cudaFreeAsync(stage[d], h->stream);
    if (rc) goto fail_out;
  } else if (h->keep_true) {
    // expand the constants into arrays
    for (int d = 0; d < 7 && rc == S7_OK; ++d) {
      float v;
      if (c->dtype == S7_F64) {
        double t;
        cudaMemcpy(&t, raw_in[d], 8, cudaMemcpyDefault);
        v = (float)t;
      } else {
        cudaMemcpy(&v, raw_in[d], 4, cudaMemcpyDefault);
      }
      k_fill_f32<<<grid_for(n), 256, 0, h->stream>>>(n, h->tc[d], v);
      if ((e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(e, "k_fill_f32");
    }
    cudaStreamSynchronize(h->stream);
    if (rc) goto fail_out;
  }
  *out = h;
  return S7_OK;

fail_out:
  release(h);
  delete h;
  return rc;
}

extern "C" int stencil9_create(stencil7_t* out, int nx, int ny, const s9_coeffs* c,
                               const s7_opts* o) {
  if (!out) return fail(S7_EINVAL, "stencil9_create: out is NULL");
  *out = nullptr;
  if (!c) return fail(S7_EINVAL, "stencil9_create: coeffs is NULL");
  if (nx < 1 || ny < 1) return fail(S7_EINVAL, "stencil9_create: sizes must be >= 1");
  const long long n = (long long)nx * ny;
  if (n >= (1LL << 40)) return fail(S7_EINVAL, "stencil9_create: mesh too large");
  if (c->dtype != S7_F64 && c->dtype != S7_F32)
    return fail(S7_EINVAL, "stencil9_create: raw coefficients must be S7_F64 or S7_F32");
  if (c->layout != S9_ROWS && c->layout != S9_COLUMNS)
    return fail(S7_EINVAL, "stencil9_create: layout must be S9_ROWS or S9_COLUMNS");
  const void* raw_in[9] = {c->xm, c->xp, c->ym, c->yp, c->xmym, c->xpym, c->xmyp, c->xpyp,
                           c->diag};
  for (int d = 0; d < 9; ++d)
    if (!raw_in[d]) return fail(S7_EINVAL, "stencil9_create: coefficient pointer %d is NULL", d);
  s7_opts opts;
  memset(&opts, 0, sizeof opts);
  if (o) opts = *o;
  if (opts.by > 1) return fail(S7_EINVAL, "stencil9_create: by must be 0 or 1");
  if (opts.variant < 0 || opts.variant > 1)
    return fail(S7_EINVAL, "stencil9_create: variant must be 0 or 1");
  bind_caller_device();
  const Engine* eng = engine_for(opts.storage);
  if (!eng) return fail(S7_EINVAL, "stencil9_create: unknown storage type %d", (int)opts.storage);

  stencil7_op* h = new (std::nothrow) stencil7_op();
  if (!h) return fail(S7_ENOMEM, "stencil9_create: host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->nz = 1;
  h->n = n;
  h->stencil = 9;
  h->storage = opts.storage;
  h->jacobi = opts.no_jacobi ? 0 : 1;
  h->keep_true = opts.keep_true ? 1 : 0;
  h->constant = 0;
  cudaGetDevice(&h->device);
  default_tile9(nx, ny, eng->vec, num_sms(), &h->tile);
  if (opts.bx > 0) h->tile.bx = opts.bx;
  if (opts.zchunk > 0) h->tile.zchunk = std::min(opts.zchunk, ny);
  if (h->tile.bx > 512) {
    delete h;
    return fail(S7_EINVAL, "stencil9_create: bx must be <= 512");
  }
  {
    const double est_us = std::max(15.0, 130.0 * (double)n / 6.0e6);
    int ce = (int)std::min(64.0, std::max(2.0, 1000.0 / est_us));
    h->check_every = opts.check_every > 0 ? opts.check_every : ce;
  }
  h->stages = 1;        // the 9-point sweeps load directly
  h->pipe_kinds = 0;
  h->step_vec = eng->vec;
  h->variant = opts.variant;
  h->resid_f64 = opts.residual_f64 ? 1 : 0;
  h->tma = opts.tma ? 1 : 0;
  if (!eng->smem_ok(h)) {
    delete h;
    return fail(S7_EINVAL, "stencil9_create: tile too large for shared memory");
  }

  int rc = S7_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "stream/event creation");
    release(h);
    delete h;
    return rc;
  }
  const size_t ts = eng->t_size;
  const void* raw_dev[9];
  void* stage[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if ((rc = dmalloc(h, &h->small, 256))) goto fail9;
  for (int d = 0; d < 8; ++d)
    if ((rc = dmalloc(h, &h->c[d], (size_t)n * ts))) goto fail9;
  if (!h->jacobi && (rc = dmalloc(h, &h->diag, (size_t)n * ts))) goto fail9;
  if (h->jacobi && (rc = dmalloc(h, &h->d, (size_t)n * dsize(xtype(h))))) goto fail9;
  if (h->keep_true)
    for (int d = 0; d < 9; ++d)
      if ((rc = dmalloc(h, (void**)&h->tc[d], (size_t)n * 4))) goto fail9;
  {
    // stage host arrays on the device, one at a time as needed
    const size_t rs = dsize(c->dtype);
    for (int d = 0; d < 9 && rc == S7_OK; ++d) {
      if (on_device(raw_in[d])) {
        raw_dev[d] = raw_in[d];
        continue;
      }
      void* p = nullptr;
      if ((e = pool_alloc(h->device, &p, (size_t)n * rs, h->stream)) != cudaSuccess) {
        rc = fail(S7_ENOMEM, "staging coefficients: %s", cudaGetErrorString(e));
        break;
      }
      stage[d] = p;
      if ((e = cudaMemcpyAsync(p, raw_in[d], (size_t)n * rs, cudaMemcpyDefault, h->stream)) !=
          cudaSuccess) {
        rc = cuda_fail(e, "copying coefficients");
        break;
      }
      raw_dev[d] = p;
    }
    if (rc == S7_OK) {
      int bad = 0;
      rc = eng->scale9(h, raw_dev, c->dtype, c->layout == S9_COLUMNS, h->stream, &bad);
      if (rc) rc = fail(rc, "coefficient scaling failed: %s", cudaGetErrorString(cudaGetLastError()));
      else if (bad) rc = fail(S7_EINVAL, "stencil9_create: %d zero or non-finite diagonal entries", bad);
    }
    cudaStreamSynchronize(h->stream);
    for (int d = 0; d < 9; ++d)
      if (stage[d]) cudaFreeAsync(stage[d], h->stream);
    if (rc) goto fail9;
  }
  *out = h;
  return S7_OK;

fail9:
  release(h);
  delete h;
  return rc;
}

void s7::destroy_idle(Handle* h) {
  if (!h) return;
  DeviceScope dev_scope(h->device);
  cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
}

extern "C" int stencil7_destroy(stencil7_t h) {
  if (!h) return S7_OK;
  DeviceScope dev_scope(h->device);
  // work queued on the caller's streams may still read the handle's memory
  // (stencil7_apply on device buffers returns before it runs): finish it
  // before the blocks go back to the pool
  cudaDeviceSynchronize();
  release(h);
  delete h;
  return S7_OK;
}

extern "C" int stencil7_info(stencil7_t h, int* nx, int* ny, int* nz, s7_dtype* storage,
                             size_t* bytes) {
  if (!h) return fail(S7_EINVAL, "stencil7_info: NULL handle");
  if (nx) *nx = h->nx;
  if (ny) *ny = h->ny;
  if (nz) *nz = h->nz;
  if (storage) *storage = h->storage;
  if (bytes) *bytes = h->bytes;
  return S7_OK;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
namespace s7 {
int ensure_ws(Handle* h, int maxit);
}
int s7::ensure_ws(Handle* h, int maxit) {
  Workspace& w = h->ws;
  const Engine* eng = engine_for(h->storage);
  const size_t n = (size_t)h->n, ts = eng->t_size, xs = eng->x_size;
  int rc;
  if (!w.ready) {
    void** vs[7] = {&w.r, &w.rh, &w.p[0], &w.p[1], &w.s[0], &w.s[1], &w.y};
    for (int k = 0; k < 7; ++k)
      if ((rc = dmalloc(h, vs[k], n * ts))) return rc;
    if ((rc = dmalloc(h, &w.x, n * xs))) return rc;
    if ((rc = dmalloc(h, &w.b, n * xs))) return rc;
    if (h->variant == 1 && (rc = dmalloc(h, &w.r2, n * ts))) return rc;
    w.parts_n = eng->parts_needed(h);
    if ((rc = dmalloc(h, (void**)&w.parts, w.parts_n * 8))) return rc;
    if ((rc = dmalloc(h, (void**)&w.sc, sizeof(Scalars)))) return rc;
    CK(cudaMemset(w.sc, 0, sizeof(Scalars)));

    if (!w.h_sc) CK(pinned_scalars(&w.h_sc));
    for (int k = 0; k < 2; ++k)
      if (!w.snap[k]) CK(cudaEventCreateWithFlags(&w.snap[k], cudaEventDisableTiming));
    w.ready = true;
  }
  if (maxit + 1 > w.hist_cap) {
    if (w.graph) {  // the graph holds the history pointer
      cudaGraphExecDestroy(w.graph);
      w.graph = nullptr;
    }
    dfree(h, (void**)&w.hist, (size_t)w.hist_cap * 8);
    w.hist_cap = 0;
    const int cap = std::max(maxit + 1, 1024);
    if ((rc = dmalloc(h, (void**)&w.hist, (size_t)cap * 8))) return rc;
    w.hist_cap = cap;
  }
  return S7_OK;
}

static int ensure_stage(Handle* h) {
  if (h->ws.stage) return S7_OK;
  return dmalloc(h, &h->ws.stage, (size_t)h->n * 8);
}

// Bring caller data (host or device, type `dt`) into a device buffer of type
// `want`.  If the caller's buffer is already suitable it is returned as is.
static int stage_in(Handle* h, const void* src, s7_dtype dt, s7_dtype want, void* dst,
                    const void** out, cudaStream_t st) {
  const Engine* eng = engine_for(h->storage);
  const size_t n = (size_t)h->n;
  const bool dev = on_device(src);
  if (dev && dt == want && ((uintptr_t)src & 15u) == 0) {
    *out = src;
    return S7_OK;
  }
  if (dt == want) {
    CK(cudaMemcpyAsync(dst, src, n * dsize(dt), cudaMemcpyDefault, st));
  } else {
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    CK(cudaMemcpyAsync(h->ws.stage, src, n * dsize(dt), cudaMemcpyDefault, st));
    if ((rc = eng->cast(h->ws.stage, dt, dst, want, (long long)n, st)))
      return fail(rc, "type conversion failed");
  }
  *out = dst;
  return S7_OK;
}

// Copy device buffer `src` (type `have`) to caller memory `dst` (type `dt`).
static int stage_out(Handle* h, const void* src, s7_dtype have, void* dst, s7_dtype dt,
                     cudaStream_t st) {
  const Engine* eng = engine_for(h->storage);
  const size_t n = (size_t)h->n;
  if (dt == have) {
    CK(cudaMemcpyAsync(dst, src, n * dsize(dt), cudaMemcpyDefault, st));
    return S7_OK;
  }
  int rc;
  if ((rc = ensure_stage(h))) return rc;
  if ((rc = eng->cast(src, have, h->ws.stage, dt, (long long)n, st)))
    return fail(rc, "type conversion failed");
  CK(cudaMemcpyAsync(dst, h->ws.stage, n * dsize(dt), cudaMemcpyDefault, st));
  return S7_OK;
}

// The handle's second stream and its event, created on first use.
static int ensure_aux(Handle* h) {
  if (h->aux) return S7_OK;
  CK(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->aux_ev, cudaEventDisableTiming));
  return S7_OK;
}

// The caller's stream waits for the handle's stream, or the reverse.
static int join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  if (from == to) return S7_OK;
  CK(cudaEventRecord(ev, from));
  CK(cudaStreamWaitEvent(to, ev, 0));
  return S7_OK;
}

// ---------------------------------------------------------------------------
// apply / residual
// ---------------------------------------------------------------------------
extern "C" int stencil7_apply(stencil7_t h, const void* x, void* y, s7_dtype dt, void* stream) {
  if (!h || !x || !y) return fail(S7_EINVAL, "stencil7_apply: NULL argument");
  if (dt != h->storage)
    return fail(S7_EINVAL, "stencil7_apply: dt (%d) must equal the storage type (%d)", (int)dt,
                (int)h->storage);
  if (x == y) return fail(S7_EINVAL, "stencil7_apply: x and y must not overlap");
  DeviceScope dev_scope(h->device);
  const Engine* eng = engine_for(h->storage);
  cudaStream_t st = (cudaStream_t)stream;
  const bool dx = on_device(x), dy = on_device(y);
  if (dx && dy) {
    int rc = eng->apply(h, x, y, st);
    return rc ? fail(rc, "stencil7_apply: launch failed: %s", cudaGetErrorString(cudaGetLastError()))
              : S7_OK;
  }
  // host buffers: stage through temporary device memory
  const size_t bytes = (size_t)h->n * eng->t_size;
  void *tx = nullptr, *ty = nullptr;
  int rc = S7_OK;
  if ((rc = dmalloc(h, &tx, bytes)) || (rc = dmalloc(h, &ty, bytes))) {
    dfree(h, &tx, bytes);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(tx, x, bytes, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    rc = eng->apply(h, tx, ty, st);
    if (rc == S7_OK) e = cudaMemcpyAsync(y, ty, bytes, cudaMemcpyDefault, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(h, &tx, bytes);
  dfree(h, &ty, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "stencil7_apply");
  return rc ? fail(rc, "stencil7_apply: launch failed") : S7_OK;
}

// Run the float64 raw-system residual on device buffers; returns norms.
static int raw_resid_dev(Handle* h, const void* b, const void* x, void* r, s7_dtype dt,
                         double* rn, double* bn, cudaStream_t st) {
  const Engine* eng = engine_for(h->storage);
  int rc = eng->raw_resid(h, b, x, r, dt, st);
  if (rc) return fail(rc, "residual launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  CK(cudaMemcpyAsync(h->ws.h_sc, h->ws.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (rn) *rn = sqrt(h->ws.h_sc->res[0]);
  if (bn) *bn = sqrt(h->ws.h_sc->res[1]);
  return S7_OK;
}

extern "C" int stencil7_residual(stencil7_t h, const void* b, const void* x, void* r, s7_dtype dt,
                                 double* rnorm, double* bnorm, void* stream) {
  if (!h || !b || !x) return fail(S7_EINVAL, "stencil7_residual: NULL argument");
  if (dt != S7_F64 && dt != S7_F32) return fail(S7_EINVAL, "stencil7_residual: dt must be F64 or F32");
  DeviceScope dev_scope(h->device);
  int rc;
  if ((rc = ensure_ws(h, 0))) return rc;
  cudaStream_t us = (cudaStream_t)stream, st = h->stream;
  if ((rc = join(us, st, h->ev))) return rc;
  const size_t bytes = (size_t)h->n * dsize(dt);
  const bool db = on_device(b), dx = on_device(x), dr = !r || on_device(r);
  void *tb = nullptr, *tx = nullptr, *tr = nullptr;
  const void *pb = b, *px = x;
  void* pr = r;
  if (!db) { if ((rc = dmalloc(h, &tb, bytes))) goto out; CK(cudaMemcpyAsync(tb, b, bytes, cudaMemcpyDefault, st)); pb = tb; }
  if (!dx) { if ((rc = dmalloc(h, &tx, bytes))) goto out; CK(cudaMemcpyAsync(tx, x, bytes, cudaMemcpyDefault, st)); px = tx; }
  if (!dr) { if ((rc = dmalloc(h, &tr, bytes))) goto out; pr = tr; }
  rc = raw_resid_dev(h, pb, px, pr, dt, rnorm, bnorm, st);
  if (rc == S7_OK && !dr) {
    cudaError_t e = cudaMemcpyAsync(r, tr, bytes, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "stencil7_residual: copy out");
  }
out:
  cudaStreamSynchronize(st);
  dfree(h, &tb, bytes);
  dfree(h, &tx, bytes);
  dfree(h, &tr, bytes);
  if (rc == S7_OK) rc = join(st, us, h->ev);
  return rc;
}

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
enum { PK_A = 0, PK_B = 1, PK_C = 2, PK_INIT = 3, PK_RES = 4, PK_OTHER = 5 };

// Fold finished event pairs into the totals (the stream must be idle).
static void prof_collect(Handle* h) {
  for (int i = 0; i < h->prof_ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) == cudaSuccess) {
      h->prof_ms[h->prof_kind[i]] += ms;
      h->prof_n[h->prof_kind[i]] += 1;
    }
  }
  cudaGetLastError();
  h->prof_ev_used = 0;
}

// Account the first m pending records (complete) and keep the rest pending.
static void prof_take(Handle* h, int m) {
  for (int i = 0; i < m; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) == cudaSuccess) {
      h->prof_ms[h->prof_kind[i]] += ms;
      h->prof_n[h->prof_kind[i]] += 1;
    }
  }
  cudaGetLastError();
  for (int i = m; i < h->prof_ev_used; ++i) {
    std::swap(h->prof_ev[2 * (i - m)], h->prof_ev[2 * i]);
    std::swap(h->prof_ev[2 * (i - m) + 1], h->prof_ev[2 * i + 1]);
    h->prof_kind[i - m] = h->prof_kind[i];
  }
  h->prof_ev_used -= m;
}

static int prof_begin(Handle* h, int kind, cudaStream_t st) {
  if (!h->prof) return -1;
  if (h->prof_ev_used == h->prof_ev_cap) {
    const int cap = std::max(64, 2 * h->prof_ev_cap);
    cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[2 * cap];
    int* kd = new (std::nothrow) int[cap];
    if (!ev || !kd) { delete[] ev; delete[] kd; return -1; }
    for (int i = 0; i < 2 * h->prof_ev_cap; ++i) ev[i] = h->prof_ev[i];
    for (int i = 0; i < h->prof_ev_cap; ++i) kd[i] = h->prof_kind[i];
    for (int i = 2 * h->prof_ev_cap; i < 2 * cap; ++i)
      if (cudaEventCreate(&ev[i]) != cudaSuccess) { delete[] ev; delete[] kd; return -1; }
    delete[] h->prof_ev;
    delete[] h->prof_kind;
    h->prof_ev = ev;
    h->prof_kind = kd;
    h->prof_ev_cap = cap;
  }
  const int i = h->prof_ev_used++;
  h->prof_kind[i] = kind;
  cudaEventRecord(h->prof_ev[2 * i], st);
  return i;
}

static void prof_end(Handle* h, int i, cudaStream_t st) {
  if (i >= 0) cudaEventRecord(h->prof_ev[2 * i + 1], st);
}

static void prof_free(Handle* h) {
  for (int i = 0; i < 2 * h->prof_ev_cap; ++i) cudaEventDestroy(h->prof_ev[i]);
  delete[] h->prof_ev;
  delete[] h->prof_kind;
  h->prof_ev = nullptr;
  h->prof_kind = nullptr;
  h->prof_ev_cap = h->prof_ev_used = 0;
}

extern "C" int stencil7_profile(stencil7_t h, int enable, double* ms, long long* launches) {
  if (!h) return fail(S7_EINVAL, "stencil7_profile: NULL handle");
  DeviceScope dev_scope(h->device);
  cudaStreamSynchronize(h->stream);
  prof_collect(h);
  for (int k = 0; k < S7_PROF_NKINDS; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_n[k];
    h->prof_ms[k] = 0.0;
    h->prof_n[k] = 0;
  }
  h->prof = enable ? 1 : 0;
  return S7_OK;
}

// One BiCGStab step: its three kernels, each timed when profiling.
static int run_step(Handle* h, cudaStream_t st) {
  const Engine* eng = engine_for(h->storage);
  if (h->variant == 1) {
    // the q/y pass, then the fused x, r update + p/s pass of the next step
    const int kinds[2] = {PK_B, PK_A};
    for (int k = 0; k < 2; ++k) {
      const int pi = prof_begin(h, kinds[k], st);
      int rc = eng->merged_kernel(h, k + 1, st);
      prof_end(h, pi, st);
      if (rc) return rc;
    }
    return S7_OK;
  }
  for (int k = 0; k < 3; ++k) {
    const int pi = prof_begin(h, k, st);
    int rc = eng->step_kernel(h, k, st);
    prof_end(h, pi, st);
    if (rc) return rc;
  }
  return S7_OK;
}

// ---------------------------------------------------------------------------
// the solve driver
// ---------------------------------------------------------------------------
static int capture_graph(Handle* h) {
  Workspace& w = h->ws;
  const Engine* eng = engine_for(h->storage);
  if (w.graph) return S7_OK;
  if (eng->prepare_capture(h)) return cuda_fail(cudaGetLastError(), "kernel attributes");
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = S7_OK;
  for (int k = 0; k < h->check_every && rc == S7_OK; ++k) {
    if (h->variant == 1)
      for (int j = 1; j <= 2 && rc == S7_OK; ++j) rc = eng->merged_kernel(h, j, h->stream);
    else
      for (int j = 0; j < 3 && rc == S7_OK; ++j) rc = eng->step_kernel(h, j, h->stream);
  }
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? fail(rc, "graph capture: step launch failed") : cuda_fail(e, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(&w.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    w.graph = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  w.graph_steps = h->check_every;
  return S7_OK;
}

struct SolveOut {
  int iters;
  int status;
  double bnorm;
};

// Solve A~ x = D^-1 b with the iterate in ws.x (already set to x0) and b a
// device buffer of the iterate's type.  Leaves the history in ws.hist.
static int solve_core(Handle* h, const void* bdev, double tol, int maxit, SolveOut* so) {
  Workspace& w = h->ws;
  const Engine* eng = engine_for(h->storage);
  cudaStream_t st = h->stream;
  Scalars* hs = w.h_sc;
  memset(hs, 0, sizeof(Scalars));
  hs->tol = tol;
  hs->maxit = maxit;
  hs->status = 4;
  CK(cudaMemcpyAsync(w.sc, hs, sizeof(Scalars), cudaMemcpyHostToDevice, st));
  const int pi = prof_begin(h, PK_INIT, st);
  int rc = eng->init(h, bdev, st);
  prof_end(h, pi, st);
  if (rc) return fail(rc, "init launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  // hist[0] = ||r_0|| / ||b~|| is left in res[2] by the start kernel
  CK(cudaMemcpyAsync(w.hist, &w.sc->res[2], sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (h->variant == 1) {
    // the two-reduction variant starts with s_0 = A p_0 and (r0, s_0)
    const int pf = prof_begin(h, PK_OTHER, st);
    rc = eng->merged_kernel(h, 0, st);
    prof_end(h, pf, st);
    if (rc) return fail(rc, "first pass launch failed");
  }
  if (!h->prof && (rc = capture_graph(h))) return rc;
  // Launches of `per` steps run one ahead of the host's check of the device
  // stop flag: while the host waits for the copy of the scalars after launch
  // k, launch k+1 is already queued, so the device never idles on the host.
  // Each launch is followed by a copy of the scalars into its own pinned
  // mirror.  The launch queued after the stop is seen runs kernels that
  // return at entry; its profiling records, if any, are dropped.
  const int per = std::max(1, h->check_every);
  const int max_launch = maxit / per + 3;
  int mark[2] = {0, 0};  // profiling records issued up to each snapshot
  auto snapshot = [&](int slot) -> int {
    CK(cudaMemcpyAsync(hs + slot, w.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(w.snap[slot], st));
    mark[slot] = h->prof_ev_used;
    return S7_OK;
  };
  if ((rc = snapshot(0))) return rc;
  int cur = 0, issued = 0;
  for (;;) {
    if (issued <= max_launch) {
      if (h->prof) {
        for (int k = 0; k < per; ++k)
          if ((rc = run_step(h, st))) return fail(rc, "step launch failed");
      } else {
        CK(cudaGraphLaunch(w.graph, st));
      }
      ++issued;
      if ((rc = snapshot(1 - cur))) return rc;
    }
    CK(cudaEventSynchronize(w.snap[cur]));
    if (h->prof) {
      prof_take(h, mark[cur]);
      mark[1 - cur] -= mark[cur];
      mark[cur] = 0;
    }
    if (hs[cur].done) break;
    if (issued > max_launch)
      return fail(S7_ECUDA, "solve did not terminate after %d launches", issued);
    cur = 1 - cur;
  }
  CK(cudaStreamSynchronize(st));
  if (h->prof) h->prof_ev_used = 0;
  so->iters = hs[cur].iter;
  so->status = hs[cur].status;
  so->bnorm = hs[cur].bnorm;
  return S7_OK;
}

extern "C" int bicgstab_solve(stencil7_t h, const void* b, void* x, s7_dtype dt, double tol,
                              int maxit, int* iters, double* resid_hist, double* true_resid,
                              void* stream) {
  if (!h || !b || !x) return fail(S7_EINVAL, "bicgstab_solve: NULL argument");
  if (dt != S7_F64 && dt != S7_F32) return fail(S7_EINVAL, "bicgstab_solve: dt must be F64 or F32");
  if (maxit < 0 || !(tol >= 0.0)) return fail(S7_EINVAL, "bicgstab_solve: bad tol or maxit");
  DeviceScope dev_scope(h->device);
  int rc;
  if ((rc = ensure_ws(h, maxit))) return rc;
  Workspace& w = h->ws;
  const Engine* eng = engine_for(h->storage);
  const s7_dtype xt = xtype(h);
  cudaStream_t us = (cudaStream_t)stream, st = h->stream;
  if ((rc = join(us, st, h->ev))) return rc;
  const void* bdev = nullptr;
  if ((rc = stage_in(h, b, dt, xt, w.b, &bdev, st))) return rc;
  const void* xin = nullptr;
  if ((rc = stage_in(h, x, dt, xt, w.x, &xin, st))) return rc;
  if (xin != w.x) CK(cudaMemcpyAsync(w.x, xin, (size_t)h->n * eng->x_size, cudaMemcpyDeviceToDevice, st));
  SolveOut so;
  if ((rc = solve_core(h, bdev, tol, maxit, &so))) return rc;
  if (so.bnorm == 0.0) CK(cudaMemsetAsync(w.x, 0, (size_t)h->n * eng->x_size, st));
  // The copy of x to host memory and the true residual both only read w.x,
  // and one is bound by the host link, the other by HBM and float64
  // arithmetic: run the copy on the second stream beside the residual.
  cudaStream_t xs = st;
  if (true_resid && !on_device(x)) {
    if ((rc = ensure_aux(h))) return rc;
    CK(cudaEventRecord(h->ev, st));
    CK(cudaStreamWaitEvent(h->aux, h->ev, 0));
    xs = h->aux;
    if ((rc = stage_out(h, w.x, xt, x, dt, xs))) return rc;
  }
  if (true_resid) {
    const int pr = prof_begin(h, PK_RES, st);
    rc = eng->true_resid(h, bdev, st);
    prof_end(h, pr, st);
    if (rc) return fail(rc, "true residual launch failed");
    CK(cudaMemcpyAsync(w.h_sc, w.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double bb = w.h_sc->res[1];
    *true_resid = bb > 0 ? sqrt(w.h_sc->res[0] / bb) : sqrt(w.h_sc->res[0]);
  }
  if (resid_hist)
    CK(cudaMemcpyAsync(resid_hist, w.hist, (size_t)(so.iters + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (xs == st) {
    if ((rc = stage_out(h, w.x, xt, x, dt, st))) return rc;
  } else {
    CK(cudaEventRecord(h->aux_ev, xs));
    CK(cudaStreamWaitEvent(st, h->aux_ev, 0));
  }
  CK(cudaStreamSynchronize(st));
  if (resid_hist && so.bnorm == 0.0) resid_hist[0] = 0.0;
  if (iters) *iters = so.iters;
  if ((rc = join(st, us, h->ev))) return rc;
  if (so.status == S7_EBREAKDOWN) return fail(S7_EBREAKDOWN, "BiCGStab breakdown after %d steps", so.iters);
  if (so.status == S7_ENOTCONV) return fail(S7_ENOTCONV, "not converged in %d steps", so.iters);
  return S7_OK;
}

// ---------------------------------------------------------------------------
// float64 iterative refinement around low-precision inner solves
// ---------------------------------------------------------------------------
extern "C" int bicgstab_solve_refined(stencil7_t h, const double* b, double* x, double tol,
                                      int max_outer, int inner_maxit, double inner_tol,
                                      int* outer, int* inner_total, double* hist, void* stream) {
  if (!h || !b || !x) return fail(S7_EINVAL, "bicgstab_solve_refined: NULL argument");
  if (max_outer < 0 || inner_maxit < 1 || !(tol >= 0) || !(inner_tol > 0))
    return fail(S7_EINVAL, "bicgstab_solve_refined: bad tolerances or limits");
  if ((h->storage == S7_BF16 || h->storage == S7_F16) && !h->keep_true)
    return fail(S7_EINVAL, "bicgstab_solve_refined: 16-bit storage needs keep_true");
  DeviceScope dev_scope(h->device);
  int rc;
  if ((rc = ensure_ws(h, inner_maxit))) return rc;
  Workspace& w = h->ws;
  const Engine* eng = engine_for(h->storage);
  const size_t n = (size_t)h->n;
  cudaStream_t us = (cudaStream_t)stream, st = h->stream;
  if ((rc = join(us, st, h->ev))) return rc;
  if (!w.ref_x && (rc = dmalloc(h, &w.ref_x, n * 8))) return rc;
  if (!w.ref_b && (rc = dmalloc(h, &w.ref_b, n * 8))) return rc;
  if (!w.ref_r && (rc = dmalloc(h, &w.ref_r, n * 8))) return rc;
  CK(cudaMemcpyAsync(w.ref_b, b, n * 8, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(w.ref_x, x, n * 8, cudaMemcpyDefault, st));
  const int grid = grid_for((long long)n);
  int total = 0, k = 0, status = S7_ENOTCONV;
  for (k = 0;; ++k) {
    double rn = 0, bn = 0;
    if ((rc = raw_resid_dev(h, w.ref_b, w.ref_x, w.ref_r, S7_F64, &rn, &bn, st))) return rc;
    const double rel = bn > 0 ? rn / bn : rn;
    if (hist) hist[k] = rel;
    if (rel <= tol) { status = S7_OK; break; }
    if (k >= max_outer) { status = S7_ENOTCONV; break; }
    // inner right-hand side with unit RMS
    const double s = rn / sqrt((double)n);
    if (h->storage == S7_F64)
      k_scaled_copy<double><<<grid, 256, 0, st>>>((long long)n, (const double*)w.ref_r, 1.0 / s, (double*)w.b);
    else
      k_scaled_copy<float><<<grid, 256, 0, st>>>((long long)n, (const double*)w.ref_r, 1.0 / s, (float*)w.b);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(w.x, 0, n * eng->x_size, st));
    SolveOut so;
    if ((rc = solve_core(h, w.b, inner_tol, inner_maxit, &so))) return rc;
    total += so.iters;
    if (so.status == S7_EBREAKDOWN && so.iters == 0) { status = S7_EBREAKDOWN; break; }
    if (h->storage == S7_F64)
      k_axpy_f64<double><<<grid, 256, 0, st>>>((long long)n, s, (const double*)w.x, (double*)w.ref_x);
    else
      k_axpy_f64<float><<<grid, 256, 0, st>>>((long long)n, s, (const float*)w.x, (double*)w.ref_x);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(x, w.ref_x, n * 8, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  if (outer) *outer = k;
  if (inner_total) *inner_total = total;
  if ((rc = join(st, us, h->ev))) return rc;
  if (status == S7_EBREAKDOWN) return fail(status, "inner solve broke down at outer step %d", k);
  if (status == S7_ENOTCONV) return fail(status, "refinement not converged in %d outer steps", k);
  return S7_OK;
}

// ---------------------------------------------------------------------------
// batched solves
// ---------------------------------------------------------------------------
namespace {

struct BatchPolicy {
  int threads;
  int zchunk;
  int sched;   // 1: one persistent launch; -1: one launch per step kernel
  int pipe;    // the pipelined step sweeps (wide vectors), else the register sweeps
  int merged;  // the two-reduction variant
};

// Autotuned policies by batch signature (storage, systems, log2 cells,
// pipelined sweeps possible, the handles' variant, variant chosen, schedule
// asked for).
std::map<std::tuple<int, int, int, int, int, int, int>, BatchPolicy> g_policy;
std::mutex g_policy_mu;
// the policy of the calling thread's last batched solve
thread_local BatchPolicy t_last_policy{0, 0, 0, 0, 0};
// steps a system in each timing trial of a fusion schedule
constexpr int kScheduleTrialSteps = 8;

Tile batch_tile(const Handle* h, int vec, const BatchPolicy& p) {
  const int runs = (h->nx + vec - 1) / vec;
  const int cap = std::min(32, p.threads);
  const int ntx = (runs + cap - 1) / cap;
  Tile t;
  t.bx = (runs + ntx - 1) / ntx;
  t.by = std::max(1, std::min(h->ny, p.threads / t.bx));
  t.zchunk = std::max(1, std::min(p.zchunk, h->nz));
  return t;
}

// Buffers of one batched solve, from the library's pools; released when the
// solve returns, after its stream has synchronised.
struct BatchBuffers {
  Scalars* sc = nullptr;
  Scalars* h_sc = nullptr;
  double* hist = nullptr;
  double* parts = nullptr;
  void* desc = nullptr;
  std::vector<unsigned char> h_desc;
  int upd_blocks = 0;  // blocks of the update launch (launch per kernel)
  ~BatchBuffers() {
    dev_free(sc, nullptr);
    pinned_put(h_sc);
    dev_free(hist, nullptr);
    dev_free(parts, nullptr);
    dev_free(desc, nullptr);
  }
};

}  // namespace

// Lay out the batch for policy p: descriptors (host + device), block offsets.
// `pipe`: the batch runs the pipelined step sweeps (tiles in units of the
// engine's wide vector).
static int batch_layout(int nsys, Handle* const* hs, const void* const* bdev, const Engine* eng,
                        const BatchPolicy& p, BatchBuffers& bb, const std::vector<size_t>& hist_off,
                        const std::vector<size_t>& parts_off, int* sweep_blocks, size_t smem[8],
                        int pipe, cudaStream_t st) {
  int b0 = 0, u0 = 0;
  for (int k = 0; k < 8; ++k) smem[k] = 0;
  for (int j = 0; j < nsys; ++j) {
    const Tile t = batch_tile(hs[j], pipe ? eng->vec_wide : eng->vec, p);
    int nb = 0, ub = 0;
    eng->fill_desc(hs[j], bb.h_desc.data() + (size_t)j * eng->desc_size, t, bdev[j],
                   bb.parts + parts_off[j], bb.hist + hist_off[j], bb.sc + j, b0, u0, &nb, &ub,
                   pipe);
    b0 += nb;
    u0 += ub;
    for (int k = 0; k < 8; ++k)
      if (k != 4 && k != 5) smem[k] = std::max(smem[k], eng->batched_smem(hs[j], t, pipe, k));
  }
  *sweep_blocks = b0;
  bb.upd_blocks = u0;
  CK(cudaMemcpyAsync(bb.desc, bb.h_desc.data(), (size_t)nsys * eng->desc_size,
                     cudaMemcpyHostToDevice, st));
  return S7_OK;
}

// x0 of every system into its workspace (again after the autotuner's trial
// runs, which advance x).
static int stage_x0(int nsys, Handle* const* hs, void* const* x, s7_dtype dt, s7_dtype xt,
                    const Engine* eng, cudaStream_t st) {
  for (int j = 0; j < nsys; ++j) {
    Handle* h = hs[j];
    const void* xin = nullptr;
    int rc = stage_in(h, x[j], dt, xt, h->ws.x, &xin, st);
    if (rc) return rc;
    if (xin != h->ws.x) {
      const cudaError_t e =
          cudaMemcpyAsync(h->ws.x, xin, (size_t)h->n * eng->x_size, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "x0 copy");
    }
  }
  return S7_OK;
}

// What one run of a laid-out batch needs.
struct BatchRun {
  int nsys;
  Handle* const* hs;
  const Engine* eng;
  BatchBuffers* bb;
  const double* tol;
  const int* maxit;
  int sweep_blocks, threads;
  const size_t* smem;  // dynamic shared memory by launch kind (8 kinds)
  int pipe, merged;    // pipelined step sweeps; the two-reduction variant
  int ce;              // steps per graph launch (launch per kernel)
  long long budget;    // wait budget of the persistent launch, SM cycles
  cudaStream_t st;
};

// One run of a laid-out batch from the staged x0: per-system scalars, the
// start sweeps, then the steps in one persistent launch (persistent = 1) or
// as one launch per step kernel replayed from a captured graph.  On return
// the host copy of the scalars holds every system's final state.  trial > 0:
// a timing run of at most `trial` steps a system with tolerance 0, *ms the
// device time of its steps.
static int batch_run(const BatchRun& R, int persistent, int trial, float* ms) {
  const int nsys = R.nsys;
  const Engine* eng = R.eng;
  BatchBuffers& bb = *R.bb;
  const cudaStream_t st = R.st;
  const int pipe = R.pipe, merged = R.merged, threads = R.threads;
  const size_t* smem = R.smem;
  const size_t psm = merged ? std::max(smem[6], smem[7]) : std::max(smem[0], smem[1]);
  int rc = S7_OK;
  cudaError_t e = cudaSuccess;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  void* d_queue = nullptr;
  void* d_qstate = nullptr;
  int* d_order = nullptr;
  int pgrid = 0, mx = 0;
  for (int j = 0; j < nsys; ++j) {
    Scalars& s = bb.h_sc[j];
    memset(&s, 0, sizeof s);
    s.tol = trial ? 0.0 : R.tol[j];
    s.maxit = trial ? std::min(trial, R.maxit[j]) : R.maxit[j];
    s.status = S7_ENOTCONV;
    mx = std::max(mx, s.maxit);
  }
  if (persistent) {
    // as many blocks as are resident on the device at once
    int per_sm = 0;
    if (eng->persistent_occupancy(threads, psm, pipe, merged, &per_sm) == S7_OK && per_sm > 0)
      pgrid = per_sm * num_sms();
    if (!pgrid) return fail(S7_EINVAL, "bicgstab_solve_batched: no block of the persistent launch fits");
  }
  if (ms && ((e = cudaEventCreate(&ev[0])) != cudaSuccess ||
             (e = cudaEventCreate(&ev[1])) != cudaSuccess)) { rc = cuda_fail(e, "events"); goto out; }
  if ((e = cudaMemcpyAsync(bb.sc, bb.h_sc, (size_t)nsys * sizeof(Scalars), cudaMemcpyHostToDevice, st)) != cudaSuccess) { rc = cuda_fail(e, "scalars"); goto out; }
  if ((rc = eng->launch_batched(2, bb.desc, nsys, R.sweep_blocks, threads, smem[2], st, pipe)) ||
      (rc = eng->launch_batched(5, bb.desc, nsys, 0, 0, 0, st, pipe)) ||
      // the two-reduction variant starts with s_0 = A p_0 and (r0, s_0)
      (merged && (rc = eng->launch_batched(0, bb.desc, nsys, R.sweep_blocks, threads, smem[0], st,
                                           pipe)))) {
    rc = fail(rc, "batched start launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    goto out;
  }
  if (persistent) {
    const int dev = R.hs[0]->device;
    // blocks look for work in the largest systems first: they set the end
    std::vector<int> order(nsys);
    for (int j = 0; j < nsys; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return R.hs[a]->n > R.hs[b]->n; });
    if ((e = dev_alloc(dev, &d_queue, (size_t)nsys * kQueueBytes, st)) != cudaSuccess ||
        (e = dev_alloc(dev, &d_qstate, kQueueStateBytes, st)) != cudaSuccess ||
        (e = dev_alloc(dev, (void**)&d_order, (size_t)nsys * sizeof(int), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_qstate, 0, kQueueStateBytes, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_order, order.data(), (size_t)nsys * sizeof(int),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      rc = cuda_fail(e, "persistent batch queues");
      goto out;
    }
    // captured as a graph of one launch; launched directly where the capture
    // of a cooperative launch is refused
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int lrc = eng->launch_persistent(bb.desc, d_order, d_queue, d_qstate, nsys, pgrid,
                                             threads, psm, R.budget, st, pipe, merged);
      e = cudaStreamEndCapture(st, &g);
      if (lrc != S7_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess)
        gexec = nullptr;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    if (ms) cudaEventRecord(ev[0], st);
    if (gexec) {
      if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) { rc = cuda_fail(e, "persistent graph launch"); goto out; }
    } else if ((rc = eng->launch_persistent(bb.desc, d_order, d_queue, d_qstate, nsys, pgrid,
                                            threads, psm, R.budget, st, pipe, merged))) {
      rc = fail(rc, "persistent batched launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      goto out;
    }
    if (ms) cudaEventRecord(ev[1], st);
    if ((e = cudaMemcpyAsync(bb.h_sc, bb.sc, (size_t)nsys * sizeof(Scalars), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "persistent batched solve"); goto out; }
  } else {
    // a trial runs all its steps in one graph launch
    const int ce = trial ? std::max(1, mx) : R.ce;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) { rc = cuda_fail(e, "capture"); goto out; }
    for (int k = 0; k < ce && rc == S7_OK; ++k) {
      if (merged) {
        // q/y pass, then the x, r updates fused with the next step's p/s pass
        rc = eng->launch_batched(6, bb.desc, nsys, R.sweep_blocks, threads, smem[6], st, pipe);
        if (!rc) rc = eng->launch_batched(7, bb.desc, nsys, R.sweep_blocks, threads, smem[7], st, pipe);
        continue;
      }
      rc = eng->launch_batched(0, bb.desc, nsys, R.sweep_blocks, threads, smem[0], st, pipe);
      if (!rc) rc = eng->launch_batched(1, bb.desc, nsys, R.sweep_blocks, threads, smem[1], st, pipe);
      if (!rc) rc = eng->launch_batched(4, bb.desc, nsys, bb.upd_blocks, 256, 0, st, pipe);
    }
    e = cudaStreamEndCapture(st, &g);
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      rc = rc ? fail(rc, "batched capture: launch failed") : cuda_fail(e, "cudaStreamEndCapture");
      goto out;
    }
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { gexec = nullptr; rc = cuda_fail(e, "cudaGraphInstantiate"); goto out; }
    if (ms) {
      cudaEventRecord(ev[0], st);
      if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) { rc = cuda_fail(e, "graph launch"); goto out; }
      cudaEventRecord(ev[1], st);
      if ((e = cudaMemcpyAsync(bb.h_sc, bb.sc, (size_t)nsys * sizeof(Scalars), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "batched trial"); goto out; }
    } else {
      const int max_launch = mx / ce + 3;
      for (int launches = 0;; ++launches) {
        if ((e = cudaMemcpyAsync(bb.h_sc, bb.sc, (size_t)nsys * sizeof(Scalars), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "batched poll"); goto out; }
        bool all = true;
        for (int j = 0; j < nsys && all; ++j) all = bb.h_sc[j].done != 0;
        if (all) break;
        if (launches >= max_launch) { rc = fail(S7_ECUDA, "batched solve did not terminate"); goto out; }
        if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) { rc = cuda_fail(e, "graph launch"); goto out; }
      }
    }
  }
  if (ms) cudaEventElapsedTime(ms, ev[0], ev[1]);
out:
  if (gexec) cudaGraphExecDestroy(gexec);
  cudaStreamSynchronize(st);
  dev_free(d_queue, st);
  dev_free(d_qstate, st);
  dev_free(d_order, st);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  return rc;
}

extern "C" int bicgstab_solve_batched(int nsys, const stencil7_t* hs_in, const void* const* b,
                                      void* const* x, s7_dtype dt, const double* tol,
                                      const int* maxit, int* iters, int* status, double* resid,
                                      const s7_batch_opts* o, void* stream) {
  if (nsys < 1 || !hs_in || !b || !x || !tol || !maxit)
    return fail(S7_EINVAL, "bicgstab_solve_batched: bad arguments");
  if (dt != S7_F64 && dt != S7_F32)
    return fail(S7_EINVAL, "bicgstab_solve_batched: dt must be F64 or F32");
  s7_batch_opts opts;
  memset(&opts, 0, sizeof opts);
  if (o) opts = *o;
  if (opts.schedule < -1 || opts.schedule > 1)
    return fail(S7_EINVAL, "bicgstab_solve_batched: schedule must be -1, 0 or 1");
  std::vector<Handle*> hs(nsys);
  for (int j = 0; j < nsys; ++j) {
    hs[j] = hs_in[j];
    if (!hs[j] || !b[j] || !x[j]) return fail(S7_EINVAL, "bicgstab_solve_batched: NULL system %d", j);
    if (hs[j]->stencil != 7)
      return fail(S7_EINVAL, "bicgstab_solve_batched: system %d is not a 7-point operator", j);
    if (hs[j]->storage != hs[0]->storage || hs[j]->device != hs[0]->device)
      return fail(S7_EINVAL, "bicgstab_solve_batched: mixed storage types or devices");
    if (maxit[j] < 0 || !(tol[j] >= 0.0))
      return fail(S7_EINVAL, "bicgstab_solve_batched: bad tol/maxit for system %d", j);
  }
  {
    std::vector<Handle*> sorted(hs);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(S7_EINVAL, "bicgstab_solve_batched: a handle appears twice");
  }
  // the handles' variant (they must agree); the autotuner may pick the other
  // one when asked to
  const int hvar = hs[0]->variant;
  for (int j = 1; j < nsys; ++j)
    if (hs[j]->variant != hvar)
      return fail(S7_EINVAL, "bicgstab_solve_batched: systems created with different variants");
  DeviceScope dev_scope(hs[0]->device);
  const Engine* eng = engine_for(hs[0]->storage);
  const s7_dtype xt = xtype(hs[0]);
  // the pipelined step sweeps are possible when every system qualifies
  int pipe_ok = 1;
  for (int j = 0; j < nsys; ++j) pipe_ok &= eng->batch_pipe_ok(hs[j]);
  const bool explicit_policy = opts.threads > 0 || opts.zchunk > 0 || opts.no_autotune;
  const bool try_variant = opts.choose_variant && !explicit_policy;
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int rc = S7_OK;
  BatchBuffers bb;
  std::vector<const void*> bdev(nsys);
  std::vector<size_t> hist_off(nsys), parts_off(nsys);
  size_t hist_total = 0, parts_total = 0;
  long long cells = 0;
  size_t smem[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // by launch kind
  BatchPolicy pol{128, 16, opts.schedule >= 0 ? 1 : -1, pipe_ok, hvar};
  BatchRun run;
  memset(&run, 0, sizeof run);
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) { rc = cuda_fail(e, "event"); goto out; }
  if ((rc = join(us, st, ev))) goto out;
  // workspaces and inputs
  for (int j = 0; j < nsys; ++j) {
    Handle* h = hs[j];
    if ((rc = ensure_ws(h, 0))) goto out;
    // the second r buffer of the two-reduction variant, for the trials too
    if ((hvar || try_variant) && !h->ws.r2 &&
        (rc = dmalloc(h, &h->ws.r2, (size_t)h->n * eng->t_size)))
      goto out;
    if ((rc = stage_in(h, b[j], dt, xt, h->ws.b, &bdev[j], st))) goto out;
    hist_off[j] = hist_total;
    hist_total += (size_t)maxit[j] + 1;
    cells += h->n;
  }
  if ((rc = stage_x0(nsys, hs.data(), x, dt, xt, eng, st))) goto out;
  // batch-owned scalars, histories, partial sums, descriptors
  {
    // partials: up to 3 per block, for the largest block count of any policy tried
    std::vector<BatchPolicy> pols;
    for (int t : {64, 128, 256})
      for (int z : {16, 32, 64}) pols.push_back(BatchPolicy{t, z, 0, 0, 0});
    pols.push_back(BatchPolicy{opts.threads > 0 ? std::max(64, std::min(256, opts.threads)) : 128,
                               opts.zchunk > 0 ? opts.zchunk : 16, 0, 0, 0});
    for (int j = 0; j < nsys; ++j) {
      Handle* h = hs[j];
      long long cap = 4096;  // update blocks
      for (int bvec : {eng->vec, eng->vec_wide}) {
        const long long runs = (h->nx + bvec - 1) / bvec;
        for (const BatchPolicy& q : pols) {
          const Tile t = batch_tile(h, bvec, q);
          const long long nb = ((runs + t.bx - 1) / t.bx) * ((h->ny + t.by - 1) / t.by) *
                               ((h->nz + t.zchunk - 1) / t.zchunk);
          cap = std::max(cap, nb);
        }
      }
      parts_off[j] = parts_total;
      // up to three sums per block (the two-reduction variant's passes)
      parts_total += 3 * (size_t)cap;
    }
    bb.h_desc.resize((size_t)nsys * eng->desc_size);
    void* p = nullptr;
    const int dev = hs[0]->device;
    if ((e = dev_alloc(dev, &p, (size_t)nsys * sizeof(Scalars), st)) != cudaSuccess) { rc = cuda_fail(e, "batch scalars"); goto out; }
    bb.sc = (Scalars*)p;
    if ((e = pinned_get(&p, (size_t)nsys * sizeof(Scalars))) != cudaSuccess) { rc = cuda_fail(e, "batch scalars (host)"); goto out; }
    bb.h_sc = (Scalars*)p;
    if ((e = dev_alloc(dev, &p, hist_total * 8, st)) != cudaSuccess) { rc = cuda_fail(e, "batch history"); goto out; }
    bb.hist = (double*)p;
    if ((e = dev_alloc(dev, &p, parts_total * 8, st)) != cudaSuccess) { rc = cuda_fail(e, "batch partials"); goto out; }
    bb.parts = (double*)p;
    if ((e = dev_alloc(dev, &p, (size_t)nsys * eng->desc_size, st)) != cudaSuccess) { rc = cuda_fail(e, "batch descriptors"); goto out; }
    bb.desc = p;
  }
  run.nsys = nsys;
  run.hs = hs.data();
  run.eng = eng;
  run.bb = &bb;
  run.tol = tol;
  run.maxit = maxit;
  run.smem = smem;
  run.ce = opts.check_every > 0 ? opts.check_every : 16;
  run.budget = opts.wait_cycles > 0 ? opts.wait_cycles : (1LL << 31);
  run.st = st;
  // policy: explicit, cached, or autotuned.  The autotuner first times the
  // block shapes with a batched SpMV probe over the batch's own operators,
  // then the fusion schedules with a few steps of the solve itself: the
  // persistent launch or one launch per step kernel, the pipelined step
  // sweeps (wide vectors) or the register sweeps, and on request the
  // two-reduction variant.
  {
    int l2 = 0;
    while ((1LL << l2) < cells) ++l2;
    const auto key = std::make_tuple((int)hs[0]->storage, nsys, l2, pipe_ok, hvar,
                                     (int)try_variant, opts.schedule);
    bool have = false;
    if (explicit_policy) {
      pol.threads = opts.threads > 0 ? std::max(64, std::min(256, opts.threads)) : 128;
      pol.zchunk = opts.zchunk > 0 ? opts.zchunk : 16;
      have = true;
    } else {
      std::lock_guard<std::mutex> lk(g_policy_mu);
      auto it = g_policy.find(key);
      if (it != g_policy.end()) {
        pol = it->second;
        have = true;
      }
    }
    if (!have) {
      const int cand_t[3] = {64, 128, 256};
      const int cand_z[3] = {16, 32, 64};
      float best = 1e30f;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int ti = 0; ti < 3; ++ti)
        for (int zi = 0; zi < 3; ++zi) {
          BatchPolicy c = pol;
          c.threads = cand_t[ti];
          c.zchunk = cand_z[zi];
          if ((rc = batch_layout(nsys, hs.data(), bdev.data(), eng, c, bb, hist_off, parts_off,
                                 &run.sweep_blocks, smem, c.pipe, st)))
            goto tune_out;
          if (eng->batched_prepare(*std::max_element(smem, smem + 8), c.pipe)) { rc = fail(S7_ECUDA, "batched kernel attributes"); goto tune_out; }
          // warm, then time two probes
          if ((rc = eng->launch_batched(3, bb.desc, nsys, run.sweep_blocks, c.threads, smem[3], st, c.pipe))) goto tune_out;
          cudaEventRecord(e0, st);
          for (int r = 0; r < 2 && rc == S7_OK; ++r)
            rc = eng->launch_batched(3, bb.desc, nsys, run.sweep_blocks, c.threads, smem[3], st, c.pipe);
          cudaEventRecord(e1, st);
          if (rc) goto tune_out;
          if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "autotune"); goto tune_out; }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) {
            best = ms;
            pol = c;
          }
        }
      // the fusion schedules, each timed over a few steps of every system
      {
        std::vector<BatchPolicy> scheds;
        for (int pp : {1, 0}) {
          if (pp && !pipe_ok) continue;
          for (int mg : {hvar, 1 - hvar}) {
            if (mg != hvar && !try_variant) continue;
            for (int sc : {1, -1}) {
              if (opts.schedule && sc != opts.schedule) continue;
              BatchPolicy c = pol;
              c.pipe = pp;
              c.merged = mg;
              c.sched = sc;
              scheds.push_back(c);
            }
          }
        }
        float sbest = 1e30f;
        const BatchPolicy tile = pol;
        for (const BatchPolicy& c : scheds) {
          if ((rc = batch_layout(nsys, hs.data(), bdev.data(), eng, c, bb, hist_off, parts_off,
                                 &run.sweep_blocks, smem, c.pipe, st)))
            goto tune_out;
          if (eng->batched_prepare(*std::max_element(smem, smem + 8), c.pipe)) { rc = fail(S7_ECUDA, "batched kernel attributes"); goto tune_out; }
          run.threads = c.threads;
          run.pipe = c.pipe;
          run.merged = c.merged;
          float ms = 0.f;
          const int trc = batch_run(run, c.sched > 0, kScheduleTrialSteps, &ms);
          if (trc == S7_EINVAL && c.sched > 0) continue;  // the persistent launch does not fit
          if (trc) { rc = trc; goto tune_out; }
          if (ms < sbest) {
            sbest = ms;
            pol = c;
          }
          if ((rc = stage_x0(nsys, hs.data(), x, dt, xt, eng, st))) goto tune_out;
        }
        if (sbest == 1e30f) pol = tile;
      }
    tune_out:
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (rc) goto out;
      std::lock_guard<std::mutex> lk(g_policy_mu);
      g_policy[key] = pol;
    }
  }
  t_last_policy = pol;
  if ((rc = batch_layout(nsys, hs.data(), bdev.data(), eng, pol, bb, hist_off, parts_off,
                         &run.sweep_blocks, smem, pol.pipe, st)))
    goto out;
  if (eng->batched_prepare(*std::max_element(smem, smem + 8), pol.pipe)) { rc = fail(S7_ECUDA, "batched kernel attributes"); goto out; }
  run.threads = pol.threads;
  run.pipe = pol.pipe;
  run.merged = pol.merged;
  {
    int prc = S7_EINVAL;
    if (pol.sched > 0) {
      prc = batch_run(run, 1, 0, nullptr);
      // schedule 0: one launch per kernel where the persistent launch does not fit
      if (prc == S7_EINVAL && opts.schedule == 0) {
        pol.sched = -1;
        t_last_policy = pol;
      } else if (prc) {
        rc = prc;
        goto out;
      }
    }
    if (pol.sched < 0 && (rc = batch_run(run, 0, 0, nullptr))) goto out;
  }
  // results
  {
    bool any_break = false, any_nc = false, any_timeout = false;
    for (int j = 0; j < nsys; ++j) {
      const Scalars& s = bb.h_sc[j];
      Handle* h = hs[j];
      if (s.bnorm == 0.0) {
        if ((e = cudaMemsetAsync(h->ws.x, 0, (size_t)h->n * eng->x_size, st)) != cudaSuccess) { rc = cuda_fail(e, "zero x"); goto out; }
      }
      if ((rc = stage_out(h, h->ws.x, xt, x[j], dt, st))) goto out;
      if (iters) iters[j] = s.iter;
      if (status) status[j] = s.status;
      if (resid) resid[j] = s.bnorm == 0.0 ? 0.0 : s.res[2];
      any_break |= s.status == S7_EBREAKDOWN;
      any_nc |= s.status == S7_ENOTCONV;
      any_timeout |= s.status == S7_ETIMEOUT;
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "batched results"); goto out; }
    if (any_timeout) rc = fail(S7_ETIMEOUT, "a group-barrier wait of the persistent launch ran out");
    else if (any_break) rc = fail(S7_EBREAKDOWN, "breakdown in at least one system");
    else if (any_nc) rc = fail(S7_ENOTCONV, "at least one system did not converge");
  }
out:
  if (st) {
    cudaStreamSynchronize(st);
    if (ev && us != st) {
      cudaEventRecord(ev, st);
      cudaStreamWaitEvent(us, ev, 0);
    }
  }
  if (ev) cudaEventDestroy(ev);
  if (st) cudaStreamDestroy(st);
  return rc;
}

extern "C" int bicgstab_batched_policy(int* threads, int* zchunk, int* schedule, int* pipelined,
                                       int* variant) {
  const BatchPolicy& p = t_last_policy;
  if (!p.threads) return fail(S7_EINVAL, "bicgstab_batched_policy: no batched solve on this thread");
  if (threads) *threads = p.threads;
  if (zchunk) *zchunk = p.zchunk;
  if (schedule) *schedule = p.sched;
  if (pipelined) *pipelined = p.pipe;
  if (variant) *variant = p.merged;
  return S7_OK;
}
