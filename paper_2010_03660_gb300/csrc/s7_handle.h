// Host-side handle and workspace layout shared by the C ABI and the
// per-precision engines.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/stencil7.h"

namespace s7 {

struct Scalars;

constexpr size_t kMapsBytes = 2048;   // room for the tensor maps of one tile shape
constexpr size_t kQueueBytes = 16;     // work queue of one system (persistent batched solve)
constexpr size_t kQueueStateBytes = 16;

// Makes `dev` the calling thread's current device for the scope of an entry
// point and gives the caller's current device back when the scope ends, so
// a caller that works on several devices keeps the device it selected.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) changed_ = cudaSetDevice(dev) == cudaSuccess;
    cudaGetLastError();
  }
  ~DeviceScope() {
    if (changed_ && prev_ >= 0) cudaSetDevice(prev_);
    cudaGetLastError();
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;

 private:
  int prev_ = -1;
  bool changed_ = false;
};

// Krylov workspace of one handle (allocated on first solve, reused).
struct Workspace {
  void* r = nullptr;
  void* rh = nullptr;      // shadow residual r0_hat
  void* p[2] = {nullptr, nullptr};
  void* s[2] = {nullptr, nullptr};
  void* y = nullptr;
  void* x = nullptr;       // iterate (float64 or float32)
  void* b = nullptr;       // right-hand side in the iterate's type
  void* stage = nullptr;   // staging for host / other-typed inputs
  double* parts = nullptr; // grid-combine partials
  size_t parts_n = 0;
  double* hist = nullptr;  // device residual history
  int hist_cap = 0;
  Scalars* sc = nullptr;   // device scalars
  Scalars* h_sc = nullptr; // pinned host mirrors (two: the solve loop checks one
                           // while the next launch's copy is in flight)
  cudaEvent_t snap[2] = {nullptr, nullptr};  // completion of each mirror's copy
  void* r2 = nullptr;      // second r buffer (two-reduction variant)
  void* ref_x = nullptr;   // float64 iterate of the refined solver
  void* ref_b = nullptr;   // float64 right-hand side of the refined solver
  void* ref_r = nullptr;   // float64 true residual of the refined solver
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool ready = false;
  // TMA tensor maps of the pipelined sweeps for the handle's own solves
  // (host memory, passed to the kernels by value); key = (bx, by, cells per
  // thread) they were built for, bx = 0 when not built
  alignas(128) unsigned char maps[kMapsBytes];
  int maps_key[3] = {0, 0, 0};
};



// Launch shape of the sweeps.
struct Tile {
  int bx, by, zchunk;
};

struct Handle {
  int nx, ny, nz;             // a 2D 9-point mesh has nz = 1
  long long n;
  int stencil = 7;            // 7: 3D 7-point operator; 9: 2D 9-point operator
  s7_dtype storage;
  int jacobi;       // 1: stored operator is D^-1 A (unit diagonal)
  int keep_true;
  int constant;
  int device;
  // stored operator (element type = storage): xm xp ym yp zm zp, or for the
  // 9-point operator xm xp ym yp xmym xpym xmyp xpyp
  void* c[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* diag = nullptr;       // raw diagonal (no_jacobi) in storage type
  double cconst[7] = {0, 0, 0, 0, 0, 0, 0};  // constant scaled coefficients; [6] = diag
  void* d = nullptr;          // kept diagonal for b scaling (float64 / float32)
  // raw operator in float32 (keep_true): the directions, then the diagonal
  // (tc[6] for the 7-point operator, tc[8] for the 9-point one)
  float* tc[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  Tile tile;
  int check_every;
  int stages;                 // step-sweep pipeline depth (1 = direct loads)
  int pipe_kinds;             // bit k: sweep k of a step uses the pipeline
  int variant;                // 0: three reductions per step; 1: two (merged passes)
  int step_vec = 0;           // cells per thread in the pipelined sweeps
  int resid_f64 = 0;          // 1: float64-accuracy residual sweeps in binary64
  int tma = 0;                // 1: pipelined sweeps of single solves stage with TMA
  size_t bytes = 0;           // device bytes held
  void* small = nullptr;      // 256 bytes of device scratch (flags)
  cudaStream_t stream = nullptr;   // private stream (captures, solves)
  cudaEvent_t ev = nullptr;
  cudaStream_t aux = nullptr;      // second stream: copies that overlap the private one
  cudaEvent_t aux_ev = nullptr;
  Workspace ws;
  // per-kernel timing (stencil7_profile)
  int prof = 0;
  double prof_ms[S7_PROF_NKINDS] = {0, 0, 0, 0, 0, 0};
  long long prof_n[S7_PROF_NKINDS] = {0, 0, 0, 0, 0, 0};
  cudaEvent_t* prof_ev = nullptr;   // event pool, pairs
  int prof_ev_cap = 0, prof_ev_used = 0;
  int* prof_kind = nullptr;         // kind of each pending pair
};

// Per-precision engine: launches kernels for one storage type.
struct Engine {
  size_t t_size;   // storage element size
  size_t x_size;   // iterate element size (8 or 4)
  size_t d_size;   // kept-diagonal element size
  int vec;         // cells per thread in the sweeps
  int vec_wide;    // cells per thread of the pipelined sweeps at their widest
  // scale raw coefficients (device, dtype raw_dt) into the handle
  int (*scale)(Handle* h, const void* const raw[7], s7_dtype raw_dt, cudaStream_t st, int* bad);
  // the same for the 9-point operator: raw = xm xp ym yp xmym xpym xmyp xpyp
  // diag, in row layout or (columns = 1) the paper's column layout
  int (*scale9)(Handle* h, const void* const raw[9], s7_dtype raw_dt, int columns,
                cudaStream_t st, int* bad);
  int (*apply)(Handle* h, const void* x, void* y, cudaStream_t st);
  int (*init)(Handle* h, const void* b, cudaStream_t st);
  // one kernel of a BiCGStab step: 0 = p update + s = A p + (r0,s);
  // 1 = q + y = A q + (q,y),(y,y); 2 = x, r updates + (r0,r),(r,r)
  int (*step_kernel)(Handle* h, int which, cudaStream_t st);
  int (*true_resid)(Handle* h, const void* b, cudaStream_t st);
  int (*raw_resid)(Handle* h, const void* b, const void* x, void* r, s7_dtype dt, cudaStream_t st);
  int (*cast)(const void* src, s7_dtype sdt, void* dst, s7_dtype ddt, long long n, cudaStream_t st);
  size_t (*parts_needed)(const Handle* h);
  int (*smem_ok)(const Handle* h);
  // raw_resid with the grid-combine partials and scalars in memory the
  // caller supplies, and the number of blocks (partials per value) it uses
  int (*raw_resid_into)(Handle* h, const void* b, const void* x, void* r, s7_dtype dt,
                        double* parts, Scalars* sc, cudaStream_t st);
  long long (*raw_resid_blocks)(const Handle* h, s7_dtype dt);
  // set kernel attributes the step kernels need, before graph capture
  int (*prepare_capture)(Handle* h);
  // the two-reduction variant: 0 = first p/s pass, 1 = q/y pass, 2 = fused
  // x, r update + p/s pass of the next step
  int (*merged_kernel)(Handle* h, int which, cudaStream_t st);
  // ---- batched solves (s7_batch.cuh) ----
  // A batch is "pipelined" when every system qualifies (batch_pipe_ok):
  // its step sweeps then run the cp.async-pipelined bodies at vec_wide
  // cells per thread, and every sweep of the batch uses that geometry (the
  // tile t is then in units of vec_wide cells).
  size_t desc_size;
  int (*batch_pipe_ok)(const Handle* h);
  // Fill the batch descriptor of system h (host memory) for tile t with
  // sweep blocks starting at block0 and update blocks at ublock0; returns
  // the block counts.
  void (*fill_desc)(Handle* h, void* desc, const Tile& t, const void* b, double* parts,
                    double* hist, Scalars* sc, int block0, int ublock0, int* nblocks,
                    int* unblocks, int pipe);
  // dynamic shared memory of launch kind `kind` for system h
  size_t (*batched_smem)(const Handle* h, const Tile& t, int pipe, int kind);
  // kind 0..3: batched sweeps (see s7_batch.cuh), 4: update, 5: history
  // start; pipelined batches only: 6 = q/y pass and 7 = fused pass of the
  // two-reduction variant (systems created with variant 1)
  int (*launch_batched)(int kind, const void* descs, int nsys, int blocks, int threads,
                        size_t smem, cudaStream_t st, int pipe);
  int (*batched_prepare)(size_t smem, int pipe);
  // The persistent batched solve (s7_batch.cuh, k_batched_persistent):
  // resident blocks per SM for `threads` threads and `smem` bytes (setting
  // the kernel's shared-memory limit), and its cooperative launch over
  // `grid` blocks with work queues (kQueueBytes per system, set up by the
  // launch) and a zeroed queue state (kQueueStateBytes); `order` (device,
  // nsys entries) lists the systems in the order blocks look for work.
  int (*persistent_occupancy)(int threads, size_t smem, int pipe, int merged, int* per_sm);
  int (*launch_persistent)(const void* descs, const int* order, void* queues, void* qstate,
                           int nsys, int grid, int threads, size_t smem, long long budget,
                           cudaStream_t st, int pipe, int merged);
};

const Engine* engine_f64();
const Engine* engine_f32();
const Engine* engine_bf16();
const Engine* engine_f16();

// Record `msg` as the calling thread's error text; returns `code`.
int set_error(int code, const char* msg);
// The engine of a storage type.
const Engine* engine_for(s7_dtype t);
// Allocate (once) the solver workspace of a handle, with a history of
// maxit+1 entries.
int ensure_ws(Handle* h, int maxit);

// A block of `bytes` from the library's memory pool of device `dev`, usable
// from any stream on return, and its release ordered after the work queued
// on stream `st` (work on other streams that reads it must be complete).
cudaError_t dev_alloc(int dev, void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
// Release a handle whose memory no queued work reads any more (the caller
// synchronised the streams that used it), without synchronising the device.
void destroy_idle(Handle* h);

// Shape of the sweep grid for a handle (same for every sweep of the handle).
void default_tile(int nx, int ny, int nz, int vec, int nsm, Tile* t);
// The same for a 2D 9-point mesh: bx threads per row strip, zchunk rows.
void default_tile9(int nx, int ny, int vec, int nsm, Tile* t);

}  // namespace s7

// The opaque handle type of the C ABI.
struct stencil7_op : public s7::Handle {};
