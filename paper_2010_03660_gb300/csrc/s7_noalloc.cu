// stencil7_residual_noalloc: the float64-accuracy residual sweep of stencil7_residual
// for callers that cannot allocate device memory at call time.  Its scratch
// (the per-block partial sums of the grid combine and the solver-scalar
// block with the arrival counter and the totals) lives in a file-scope
// __device__ array of fixed size instead of a cudaMalloc'd workspace.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "s7_handle.h"
#include "s7_sweep.cuh"

using namespace s7;

namespace {

// Largest sweep grid the static scratch can serve (blocks of the residual
// sweep; each block leaves two float64 partial sums).
constexpr long long kMaxBlocks = S7_NOALLOC_MAX_BLOCKS;
constexpr size_t kScalarsBytes = (sizeof(Scalars) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kScalarsBytes + 2 * kMaxBlocks * sizeof(double);
constexpr int kMaxDevices = 64;

}  // namespace

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char s7_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device with that
// device current.  (In host code the array's name is only a host-side
// stand-in; it must never be handed to a kernel.)
static void* g_scratch[kMaxDevices];
static std::mutex g_scratch_mu;

static int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(S7_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, s7_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      char msg[256];
      snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
      cudaGetLastError();
      return set_error(S7_ECUDA, msg);
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return S7_OK;
}

static bool device_memory(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static const Engine* engine_of(s7_dtype t) {
  switch (t) {
    case S7_F64: return engine_f64();
    case S7_F32: return engine_f32();
    case S7_BF16: return engine_bf16();
    case S7_F16: return engine_f16();
  }
  return nullptr;
}

extern "C" int stencil7_residual_noalloc(stencil7_t h, const void* b, const void* x, void* r,
                                         s7_dtype dt, double* rnorm, double* bnorm,
                                         void* stream) {
  if (!h || !b || !x) return set_error(S7_EINVAL, "stencil7_residual_noalloc: NULL argument");
  if (dt != S7_F64 && dt != S7_F32)
    return set_error(S7_EINVAL, "stencil7_residual_noalloc: dt must be S7_F64 or S7_F32");
  cudaStream_t st = (cudaStream_t)stream;
  // the call waits for its norms on the host: a capturing stream cannot
  // run it (the capture would be invalidated), so refuse before touching it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return set_error(S7_EINVAL, "stencil7_residual_noalloc: bad stream");
  }
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(S7_EINVAL,
                     "stencil7_residual_noalloc: synchronous call on a capturing stream");
  DeviceScope dev_scope(h->device);
  if (!device_memory(b) || !device_memory(x) || (r && !device_memory(r)))
    return set_error(S7_EINVAL,
                     "stencil7_residual_noalloc: b, x and r must be device memory (host buffers "
                     "would need staging)");
  const Engine* eng = engine_of(h->storage);
  const long long nb = eng->raw_resid_blocks(h, dt);
  if (nb > kMaxBlocks) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "stencil7_residual_noalloc: the sweep needs %lld blocks, the static scratch holds "
             "%lld; use stencil7_residual or a larger zchunk",
             nb, kMaxBlocks);
    return set_error(S7_EINVAL, msg);
  }
  void* base = nullptr;
  int rc = scratch_address(h->device, &base);
  if (rc) return rc;
  Scalars* sc = (Scalars*)base;
  double* parts = (double*)((char*)base + kScalarsBytes);
  // the arrival counters (and totals) must start at zero; the partials are
  // written before they are read, so they need no clearing
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(Scalars), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(S7_ECUDA, cudaGetErrorString(e));
  }
  rc = eng->raw_resid_into(h, b, x, r, dt, parts, sc, st);
  if (rc) {
    char msg[256];
    snprintf(msg, sizeof msg, "residual launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return set_error(rc, msg);
  }
  double tot[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(tot, &sc->res[0], sizeof tot, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(S7_ECUDA, cudaGetErrorString(e));
  }
  if (rnorm) *rnorm = sqrt(tot[0]);
  if (bnorm) *bnorm = sqrt(tot[1]);
  return S7_OK;
}
