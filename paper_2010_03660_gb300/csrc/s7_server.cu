// The solve server: continuous batching of independent solve requests.
//
// Requests (mesh, raw coefficients, right-hand side, tolerance) are queued
// by s7_server_submit and admitted by a scheduler thread while the device
// memory they will need fits the server's budget.  Each admitted request
// runs mixed-precision BiCGStab with float64 iterative refinement as a small
// state machine:
//
//   RESIDUAL  r = b - A x with float64 accuracy on the true float32 operator; stop if
//             ||r||/||b|| <= tol; else start an inner solve of
//             A~ d = D^-1 r / s (s = ||r||/sqrt(N)) in the storage precision
//   INNER     BiCGStab steps; every request in this state shares the same
//             batched kernel launches (one launch per step kernel covers
//             them all, each with its own grid combine and stop flag)
//   back to RESIDUAL after x += s d (float64)
//
// so requests that arrive while others are on the GPU join the running
// batch at the next tick, retire as soon as they meet their own tolerance,
// and give their memory back for the next admissions.  Every request's
// arithmetic is independent of the others in the batch (own blocks, own
// reductions, a fixed tile policy), so its result does not depend on what
// else was running.
//
// Every request is held with per-cell coefficient arrays (constants are
// expanded) and its x extent padded to a multiple of the engine's wide
// vector: padding cells have a unit diagonal, no couplings and a zero
// right-hand side, so every vector stays exactly zero there and the solution
// on the real cells is unchanged.  With all rows made of whole vectors, the
// batch's step sweeps run the cp.async-pipelined bodies; by default the
// inner solves take two reductions per step (a q/y pass and a fused pass,
// s7_opts.variant 1) after a first p/s pass at their start.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "s7_handle.h"
#include "s7_sweep.cuh"

using namespace s7;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

__global__ void k_rhs_scaled(long long n, const double* r, double inv_s, float* f, double* dd) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (f) f[i] = (float)(r[i] * inv_s);
    if (dd) dd[i] = r[i] * inv_s;
  }
}

template <class X>
__global__ void k_axpy_x(long long n, double s, const X* d, double* x) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)d[i], x[i]);
}

// dst (rows of nxp) from src (rows of nx): padding cells get `fill`.
template <class V>
__global__ void k_pad(long long rows, int nx, int nxp, const V* __restrict__ src,
                      V* __restrict__ dst, V fill) {
  const long long n = rows * nxp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / nxp;
    const int x = (int)(i - row * nxp);
    dst[i] = x < nx ? src[row * nx + x] : fill;
  }
}

// dst (rows of nxp) holding `v` on the real cells and `fill` in the padding.
template <class V>
__global__ void k_const_pad(long long rows, int nx, int nxp, V v, V* __restrict__ dst, V fill) {
  const long long n = rows * nxp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / nxp;
    dst[i] = (i - row * nxp) < nx ? v : fill;
  }
}

// dst (rows of nx) from src (rows of nxp).
template <class V>
__global__ void k_unpad(long long rows, int nx, int nxp, const V* __restrict__ src,
                        V* __restrict__ dst) {
  const long long n = rows * nx;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / nx;
    dst[i] = src[row * nxp + (i - row * nx)];
  }
}

template <class S, class D>
__global__ void k_conv(long long n, const S* a, D* b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (D)a[i];
}

int grid_of(long long n) {
  return (int)std::max(1LL, std::min((n + 255) / 256, 152LL * 16));
}

enum RState { QUEUED = 0, RESIDUAL = 1, INNER_START = 2, INNER = 3, FINISHED = 4 };

struct Req {
  uint64_t id = 0;
  s7_request in;
  double t_arrive = 0, t_admit = 0, t_done = 0;
  int state = QUEUED;
  int status = S7_EAGAIN;
  int outer = 0, inner_total = 0;
  double resid = 0, s = 0, rel0 = 0;
  long long n = 0;       // cells held (x extent padded to nxp)
  long long n_in = 0;    // cells of the request
  int nxp = 0;
  size_t bytes = 0;
  int slot = -1;
  stencil7_t h = nullptr;
  double *xr = nullptr, *br = nullptr, *rr = nullptr, *parts = nullptr;
  size_t parts_n = 0;
};

}  // namespace

struct s7_server {
  s7_server_opts o;
  int device = 0;
  std::thread th;        // scheduler: ticks of batched work
  std::thread th_admit;  // admission: operator set-up and uploads
  std::deque<Req*> ready;  // admitted, set up, not yet picked up by the scheduler
  cudaStream_t st_admit = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_ready;
  int admitting = 0;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> reqs;
  uint64_t next_id = 1;
  size_t mem_used = 0, mem_peak = 0;
  bool stop = false;
  // device state shared by all requests
  cudaStream_t st = nullptr;
  Scalars* d_sc = nullptr;
  Scalars* h_sc = nullptr;
  double* d_hist = nullptr;
  void* d_desc = nullptr;
  void* d_desc_start = nullptr;
  std::vector<int> free_slots;
  // statistics
  long long completed = 0, failed = 0;
  double cell_iters = 0;
  double busy_s = 0;
  const Engine* eng = nullptr;
};

namespace {

size_t request_bytes(const s7_server* S, long long n, int raw_size) {
  // stored operator, kept diagonal, true float32 operator, seven Krylov
  // vectors (eight with the two-reduction variant's second r), x and b in
  // float32, three float64 refinement vectors, and the staging of the raw
  // coefficients (seven arrays and one more while a padded operator is
  // formed) while the operator is created
  const size_t ts = S->eng->t_size;
  const size_t vecs = S->o.three_pass ? 7 : 8;
  return (size_t)n * (6 * ts + 4 + 28 + vecs * ts + 8 + 24 + 8 * (size_t)raw_size) + (1 << 20);
}

Tile serve_tile(const s7_server* S, int nx, int ny, int nz, int pipe) {
  const int vec = pipe ? S->eng->vec_wide : S->eng->vec;
  const int T = S->o.threads;
  const int runs = (nx + vec - 1) / vec;
  const int cap = std::min(32, T);
  const int ntx = (runs + cap - 1) / cap;
  Tile t;
  t.bx = (runs + ntx - 1) / ntx;
  t.by = std::max(1, std::min(ny, T / t.bx));
  t.zchunk = std::max(1, std::min(S->o.zchunk, nz));
  return t;
}

// Retire a request.  Its work on the scheduler's stream is finished first
// (a no-op after a normal completion, which synchronised it; needed when a
// failure or cancellation retires a request with launches still queued);
// admission synchronises its own stream before a request becomes active.  The
// blocks then go back to the library's pool without a device-wide
// synchronisation, which would stall the other thread's work.
void release_req(s7_server* S, Req* r) {
  if (S->st) cudaStreamSynchronize(S->st);
  dev_free(r->xr, S->st);
  dev_free(r->br, S->st);
  dev_free(r->rr, S->st);
  dev_free(r->parts, S->st);
  r->xr = r->br = r->rr = r->parts = nullptr;
  if (r->h) destroy_idle(r->h);
  r->h = nullptr;
  if (r->slot >= 0) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->free_slots.push_back(r->slot);
  }
  r->slot = -1;
}

// Bring an nx*ny*nz array (host or device, `es`-byte elements) into the
// padded layout `dst` (rows of nxp), staging it contiguously in `tmp`.
cudaError_t pad_in(void* dst, const void* src, void* tmp, int nx, int nxp, long long rows, int es,
                   double fill, cudaStream_t st) {
  const long long n = rows * nx;
  if (nx == nxp) return cudaMemcpyAsync(dst, src, (size_t)n * es, cudaMemcpyDefault, st);
  cudaError_t e = cudaMemcpyAsync(tmp, src, (size_t)n * es, cudaMemcpyDefault, st);
  if (e != cudaSuccess) return e;
  if (es == 8)
    k_pad<double><<<grid_of(rows * nxp), 256, 0, st>>>(rows, nx, nxp, (const double*)tmp,
                                                      (double*)dst, fill);
  else
    k_pad<float><<<grid_of(rows * nxp), 256, 0, st>>>(rows, nx, nxp, (const float*)tmp,
                                                     (float*)dst, (float)fill);
  return cudaGetLastError();
}

// The padded array `src` back to the caller's layout `dst` (rows of nx),
// through the contiguous device buffer `tmp`.
cudaError_t pad_out(void* dst, const void* src, void* tmp, int nx, int nxp, long long rows,
                    int es, cudaStream_t st) {
  const long long n = rows * nx;
  if (nx == nxp) return cudaMemcpyAsync(dst, src, (size_t)n * es, cudaMemcpyDefault, st);
  if (es == 8)
    k_unpad<double><<<grid_of(n), 256, 0, st>>>(rows, nx, nxp, (const double*)src, (double*)tmp);
  else
    k_unpad<float><<<grid_of(n), 256, 0, st>>>(rows, nx, nxp, (const float*)src, (float*)tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(dst, tmp, (size_t)n * es, cudaMemcpyDefault, st);
}

// The request's operator with its x extent padded to r->nxp (unit diagonal,
// zero couplings in the padding).
int create_padded(s7_server* S, Req* r, const s7_opts* oo) {
  const s7_coeffs& c = r->in.coeffs;
  const int es = c.dtype == S7_F64 ? 8 : 4;
  const size_t n = (size_t)r->n;
  const long long rows = (long long)r->in.ny * r->in.nz;
  cudaStream_t as = S->st_admit;
  unsigned char* buf = nullptr;
  if (dev_alloc(S->device, (void**)&buf, 8 * n * es, as) != cudaSuccess)
    return set_error(S7_ENOMEM, "s7_server: staging the padded operator");
  const void* src[7] = {c.xm, c.xp, c.ym, c.yp, c.zm, c.zp, c.diag};
  void* dst[7];
  void* tmp = buf + 7 * n * es;
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < 7 && e == cudaSuccess; ++d) {
    dst[d] = buf + d * n * es;
    const double fill = d == 6 ? 1.0 : 0.0;
    if (!c.constant) {
      e = pad_in(dst[d], src[d], tmp, r->in.nx, r->nxp, rows, es, fill, as);
      continue;
    }
    // a constant operator: one value per array, expanded to the cells
    double v = 0.0;
    if (es == 8) {
      e = cudaMemcpy(&v, src[d], 8, cudaMemcpyDefault);
    } else {
      float f = 0.f;
      e = cudaMemcpy(&f, src[d], 4, cudaMemcpyDefault);
      v = f;
    }
    if (e != cudaSuccess) break;
    if (es == 8)
      k_const_pad<double><<<grid_of(n), 256, 0, as>>>(rows, r->in.nx, r->nxp, v, (double*)dst[d],
                                                      fill);
    else
      k_const_pad<float><<<grid_of(n), 256, 0, as>>>(rows, r->in.nx, r->nxp, (float)v,
                                                     (float*)dst[d], (float)fill);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(as);
  int rc = S7_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = S7_ECUDA;
  } else {
    s7_coeffs pc = c;
    pc.constant = 0;
    pc.xm = dst[0];
    pc.xp = dst[1];
    pc.ym = dst[2];
    pc.yp = dst[3];
    pc.zm = dst[4];
    pc.zp = dst[5];
    pc.diag = dst[6];
    rc = stencil7_create(&r->h, r->nxp, r->in.ny, r->in.nz, &pc, oo);
  }
  cudaStreamSynchronize(as);   // nothing on the admission stream reads buf now
  dev_free(buf, as);
  return rc;
}

// Admit one request: operator, workspace, float64 vectors, slot.
int admit(s7_server* S, Req* r) {
  s7_opts oo;
  memset(&oo, 0, sizeof oo);
  oo.storage = S->o.storage;
  oo.keep_true = 1;
  oo.variant = S->o.three_pass ? 0 : 1;
  oo.residual_f64 = S->o.residual_f64;
  int rc = (r->nxp != r->in.nx || r->in.coeffs.constant)
               ? create_padded(S, r, &oo)
               : stencil7_create(&r->h, r->in.nx, r->in.ny, r->in.nz, &r->in.coeffs, &oo);
  if (rc) return rc;
  if ((rc = ensure_ws(r->h, S->o.inner_maxit))) return rc;
  const size_t n = (size_t)r->n;
  cudaError_t e = cudaSuccess;
  cudaStream_t as = S->st_admit;
  if ((e = dev_alloc(S->device, (void**)&r->xr, n * 8, as)) != cudaSuccess ||
      (e = dev_alloc(S->device, (void**)&r->br, n * 8, as)) != cudaSuccess ||
      (e = dev_alloc(S->device, (void**)&r->rr, n * 8, as)) != cudaSuccess)
    return S7_ENOMEM;
  long long nb = 0;
  for (int pipe = 0; pipe < 2; ++pipe) {
    const int v = pipe ? S->eng->vec_wide : S->eng->vec;
    const Tile t = serve_tile(S, r->nxp, r->in.ny, r->in.nz, pipe);
    const long long runs = (r->nxp + v - 1) / v;
    nb = std::max(nb, ((runs + t.bx - 1) / t.bx) * ((r->in.ny + t.by - 1) / t.by) *
                          ((r->in.nz + t.zchunk - 1) / t.zchunk));
  }
  const long long rb = S->eng->raw_resid_blocks(r->h, S7_F64);
  // up to three sums per block (the q/y and fused passes reduce three)
  r->parts_n = 3 * (size_t)std::max(std::max(nb, rb), 4096LL);
  if ((e = dev_alloc(S->device, (void**)&r->parts, r->parts_n * 8, as)) != cudaSuccess) return S7_ENOMEM;
  // b (host or device, f32/f64) -> float64 (zero in the padding); x0 = 0
  const long long rows = (long long)r->in.ny * r->in.nz;
  if (r->in.dt == S7_F64) {
    // r->rr (unused until the first residual) stages b
    e = pad_in(r->br, r->in.b, r->rr, r->in.nx, r->nxp, rows, 8, 0.0, as);
  } else {
    e = pad_in(r->h->ws.b, r->in.b, r->h->ws.x, r->in.nx, r->nxp, rows, 4, 0.0, as);
    if (e == cudaSuccess) {
      k_conv<float, double><<<grid_of(n), 256, 0, as>>>((long long)n, (const float*)r->h->ws.b, r->br);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(r->xr, 0, n * 8, as);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return S7_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->slot = S->free_slots.back();
    S->free_slots.pop_back();
  }
  Scalars z;
  memset(&z, 0, sizeof z);
  e = cudaMemcpyAsync(S->d_sc + r->slot, &z, sizeof z, cudaMemcpyHostToDevice, as);
  if (e == cudaSuccess) e = cudaStreamSynchronize(as);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return S7_ECUDA;
  }
  r->state = RESIDUAL;
  return S7_OK;
}

// Copy the float64 iterate to the caller's buffer and retire the request.
void finish(s7_server* S, Req* r, int status) {
  const size_t n = (size_t)r->n;
  if (status == S7_OK || status == S7_ENOTCONV) {
    cudaError_t e;
    const long long rows = (long long)r->in.ny * r->in.nz;
    if (r->in.dt == S7_F64) {
      e = pad_out(r->in.x, r->xr, r->rr, r->in.nx, r->nxp, rows, 8, S->st);
    } else {
      k_conv<double, float><<<grid_of(n), 256, 0, S->st>>>((long long)n, r->xr, (float*)r->h->ws.x);
      e = pad_out(r->in.x, r->h->ws.x, r->h->ws.b, r->in.nx, r->nxp, rows, 4, S->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      status = S7_ECUDA;
    }
  }
  release_req(S, r);
  std::lock_guard<std::mutex> lk(S->mu);
  r->t_done = now_s();
  r->status = status;
  r->state = FINISHED;
  S->mem_used -= r->bytes;
  if (status == S7_OK) S->completed++;
  else S->failed++;
  S->cv_done.notify_all();
  S->cv_work.notify_all();   // memory came back: the admission thread re-checks
}

void fail_all(s7_server* S, int status) {
  std::vector<Req*> all;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    all.swap(S->active);
  }
  for (Req* r : all) finish(S, r, status);
}

// Admission: first come, first served, while a slot is free and the request
// at the head of the queue fits the memory budget.  Set-up (operator
// creation, uploads) runs on the admission stream, overlapping the
// scheduler's batched work.
void admitter(s7_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        return S->stop || (!S->queue.empty() && !S->free_slots.empty() &&
                           S->mem_used + S->queue.front()->bytes <= S->o.hbm_budget_bytes);
      });
      if (S->stop) return;
      r = S->queue.front();
      S->queue.pop_front();
      S->mem_used += r->bytes;
      S->mem_peak = std::max(S->mem_peak, S->mem_used);
      S->admitting++;
    }
    r->t_admit = now_s();
    const int rc = admit(S, r);
    if (rc) {
      cudaStreamSynchronize(S->st_admit);   // uploads of a failed admission
      finish(S, r, rc);
      std::lock_guard<std::mutex> lk(S->mu);
      S->admitting--;
      continue;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->admitting--;
    S->ready.push_back(r);
    S->cv_ready.notify_all();
  }
}

void scheduler(s7_server* S) {
  cudaSetDevice(S->device);
  const Engine* eng = S->eng;
  const int K = S->o.steps_per_tick;
  std::vector<unsigned char> hd, hds;
  int sweep_blocks = 0, upd_blocks = 0;
  size_t smem_max[2] = {0, 0};   // by pipelined or not
  for (;;) {
    // ---- pick up requests the admission thread has set up
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->active.empty() && S->ready.empty())
        S->cv_ready.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->stop) break;
      while (!S->ready.empty()) {
        S->active.push_back(S->ready.front());
        S->ready.pop_front();
      }
    }
    if (S->active.empty()) continue;
    const double t0 = now_s();

    // ---- outer residuals
    bool any_res = false;
    for (Req* r : S->active)
      if (r->state == RESIDUAL) {
        if (eng->raw_resid_into(r->h, r->br, r->xr, r->rr, S7_F64, r->parts, S->d_sc + r->slot,
                                S->st)) {
          fail_all(S, S7_ECUDA);
          break;
        }
        any_res = true;
      }
    if (S->active.empty()) continue;
    if (any_res) {
      if (cudaMemcpyAsync(S->h_sc, S->d_sc, (size_t)S->o.max_active * sizeof(Scalars),
                          cudaMemcpyDeviceToHost, S->st) != cudaSuccess ||
          cudaStreamSynchronize(S->st) != cudaSuccess) {
        cudaGetLastError();
        fail_all(S, S7_ECUDA);
        continue;
      }
      std::vector<Req*> keep;
      for (Req* r : S->active) {
        if (r->state != RESIDUAL) {
          keep.push_back(r);
          continue;
        }
        const Scalars& sc = S->h_sc[r->slot];
        const double rn = sqrt(sc.res[0]), bn = sqrt(sc.res[1]);
        const double rel = bn > 0 ? rn / bn : rn;
        r->resid = rel;
        if (r->outer == 0) r->rel0 = rel;
        if (rel <= r->in.tol || rn == 0.0) {
          finish(S, r, S7_OK);
          continue;
        }
        if (r->outer >= S->o.max_outer) {
          finish(S, r, S7_ENOTCONV);
          continue;
        }
        // inner right-hand side r / s with unit RMS over the request's cells,
        // x_inner = 0
        r->s = rn / sqrt((double)r->n_in);
        const bool f64 = S->o.storage == S7_F64;
        k_rhs_scaled<<<grid_of(r->n), 256, 0, S->st>>>(
            r->n, r->rr, 1.0 / r->s, f64 ? nullptr : (float*)r->h->ws.b,
            f64 ? (double*)r->h->ws.b : nullptr);
        cudaMemsetAsync(r->h->ws.x, 0, (size_t)r->n * eng->x_size, S->st);
        Scalars z;
        memset(&z, 0, sizeof z);
        z.tol = S->o.inner_tol;
        z.maxit = S->o.inner_maxit;
        z.status = S7_ENOTCONV;
        cudaMemcpyAsync(S->d_sc + r->slot, &z, sizeof z, cudaMemcpyHostToDevice, S->st);
        r->outer++;
        r->state = INNER_START;
        keep.push_back(r);
      }
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->active.swap(keep);
      }
    }
    if (S->active.empty()) continue;

    // ---- batched inner solves: start the new ones, then K shared steps
    std::vector<Req*> inner, starting;
    for (Req* r : S->active)
      if (r->state == INNER_START || r->state == INNER) inner.push_back(r);
    for (Req* r : inner)
      if (r->state == INNER_START) starting.push_back(r);
    // the pipelined step sweeps when every request of the set qualifies
    auto pipe_of = [&](const std::vector<Req*>& set) {
      int p = 1;
      for (Req* r : set) p &= eng->batch_pipe_ok(r->h);
      return p;
    };
    auto layout = [&](const std::vector<Req*>& set, std::vector<unsigned char>& host, void* dev,
                      int* nb_total, int* ub_total, size_t smem[8], int pipe) {
      host.resize(set.size() * eng->desc_size);
      int b0 = 0, u0 = 0;
      for (int k = 0; k < 8; ++k) smem[k] = 0;
      for (size_t j = 0; j < set.size(); ++j) {
        Req* r = set[j];
        const Tile t = serve_tile(S, r->nxp, r->in.ny, r->in.nz, pipe);
        int nb = 0, ub = 0;
        eng->fill_desc(r->h, host.data() + j * eng->desc_size, t, r->h->ws.b, r->parts,
                       S->d_hist + (size_t)r->slot * (S->o.inner_maxit + 1), S->d_sc + r->slot,
                       b0, u0, &nb, &ub, pipe);
        b0 += nb;
        u0 += ub;
        for (int k = 0; k < 8; ++k)
          if (k != 4 && k != 5) smem[k] = std::max(smem[k], eng->batched_smem(r->h, t, pipe, k));
      }
      *nb_total = b0;
      *ub_total = u0;
      return cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, S->st);
    };
    // kernel attributes: dynamic shared memory up to the largest seen
    auto prepare = [&](const size_t sm[8], int pipe) {
      const size_t m = *std::max_element(sm, sm + 8);
      if (m <= smem_max[pipe]) return S7_OK;
      smem_max[pipe] = m;
      return eng->batched_prepare(m, pipe);
    };
    const bool merged = !S->o.three_pass;
    int rc = S7_OK;
    if (!starting.empty()) {
      int nbs = 0, ubs = 0;
      size_t sms[8];
      const int ps = pipe_of(starting);
      if (merged && !ps) rc = S7_EINVAL;   // held operators always qualify
      if (!rc && layout(starting, hds, S->d_desc_start, &nbs, &ubs, sms, ps) != cudaSuccess)
        rc = S7_ECUDA;
      if (!rc) rc = prepare(sms, ps);
      if (!rc) rc = eng->launch_batched(2, S->d_desc_start, (int)starting.size(), nbs,
                                        S->o.threads, sms[2], S->st, ps);
      if (!rc) rc = eng->launch_batched(5, S->d_desc_start, (int)starting.size(), 0, 0, 0, S->st, ps);
      // the two-reduction variant starts with s_0 = A p_0 and (r0, s_0)
      if (!rc && merged)
        rc = eng->launch_batched(0, S->d_desc_start, (int)starting.size(), nbs, S->o.threads,
                                 sms[0], S->st, ps);
      for (Req* r : starting) r->state = INNER;
    }
    const int pipe = pipe_of(inner);
    if (!rc && merged && !pipe) rc = S7_EINVAL;
    size_t smi[8];
    if (!rc) {
      // the membership changes as requests start and finish inner solves:
      // lay the batch out again every tick (a few hundred bytes per request)
      if (layout(inner, hd, S->d_desc, &sweep_blocks, &upd_blocks, smi, pipe) != cudaSuccess)
        rc = S7_ECUDA;
      if (!rc) rc = prepare(smi, pipe);
    }
    for (int k = 0; k < K && !rc; ++k) {
      const int n_in = (int)inner.size();
      if (merged) {
        rc = eng->launch_batched(6, S->d_desc, n_in, sweep_blocks, S->o.threads, smi[6], S->st,
                                 pipe);
        if (!rc) rc = eng->launch_batched(7, S->d_desc, n_in, sweep_blocks, S->o.threads, smi[7],
                                          S->st, pipe);
        continue;
      }
      rc = eng->launch_batched(0, S->d_desc, n_in, sweep_blocks, S->o.threads, smi[0], S->st, pipe);
      if (!rc) rc = eng->launch_batched(1, S->d_desc, n_in, sweep_blocks, S->o.threads, smi[1],
                                        S->st, pipe);
      if (!rc) rc = eng->launch_batched(4, S->d_desc, n_in, upd_blocks, 256, 0, S->st, pipe);
    }
    if (!rc && (cudaMemcpyAsync(S->h_sc, S->d_sc, (size_t)S->o.max_active * sizeof(Scalars),
                                cudaMemcpyDeviceToHost, S->st) != cudaSuccess ||
                cudaStreamSynchronize(S->st) != cudaSuccess))
      rc = S7_ECUDA;
    if (rc) {
      cudaGetLastError();
      fail_all(S, rc);
      continue;
    }
    std::vector<Req*> keep;
    for (Req* r : S->active) {
      if (r->state == INNER && S->h_sc[r->slot].done) {
        const Scalars& sc = S->h_sc[r->slot];
        r->inner_total += sc.iter;
        S->cell_iters += (double)r->n_in * sc.iter;
        if (sc.status == S7_EBREAKDOWN && sc.iter == 0) {
          finish(S, r, S7_EBREAKDOWN);
          continue;
        }
        if (S->o.storage == S7_F64)
          k_axpy_x<double><<<grid_of(r->n), 256, 0, S->st>>>(r->n, r->s, (const double*)r->h->ws.x, r->xr);
        else
          k_axpy_x<float><<<grid_of(r->n), 256, 0, S->st>>>(r->n, r->s, (const float*)r->h->ws.x, r->xr);
        r->state = RESIDUAL;
      }
      keep.push_back(r);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.swap(keep);
      S->busy_s += now_s() - t0;
    }
  }
  // shut down: fail what is left (the admission thread has stopped)
  fail_all(S, S7_ECANCELED);
  std::vector<Req*> left;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    left.assign(S->ready.begin(), S->ready.end());
    S->ready.clear();
  }
  for (Req* r : left) finish(S, r, S7_ECANCELED);
  std::lock_guard<std::mutex> lk(S->mu);
  for (Req* r : S->queue) {
    r->status = S7_ECANCELED;
    r->state = FINISHED;
  }
  S->queue.clear();
  S->cv_done.notify_all();
}

void fill_result(const Req* r, s7_result* out) {
  out->status = r->status;
  out->outer = r->outer;
  out->inner_iters = r->inner_total;
  out->resid = r->resid;
  out->t_arrive = r->t_arrive;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
}

}  // namespace

extern "C" int s7_server_create(s7_server_t* out, const s7_server_opts* o) {
  if (!out) return set_error(S7_EINVAL, "s7_server_create: out is NULL");
  *out = nullptr;
  s7_server_opts opts;
  memset(&opts, 0, sizeof opts);
  if (o) opts = *o;
  if (opts.storage == S7_F64 && !o) opts.storage = S7_BF16;
  if (opts.hbm_budget_bytes == 0) opts.hbm_budget_bytes = (size_t)150 << 30;
  if (opts.max_active <= 0) opts.max_active = 256;
  if (opts.steps_per_tick <= 0) opts.steps_per_tick = 4;
  if (opts.threads <= 0) opts.threads = 128;
  opts.threads = std::max(64, std::min(256, opts.threads));
  if (opts.zchunk <= 0) opts.zchunk = 16;
  // BF16's 8 significant bits cap what one refinement step can gain (the
  // stored operator is off by about 2^-9), so its inner solves stop at 1e-1:
  // fewer inner steps in total than at 1e-2 (measured on the served
  // request mix); the other types at 1e-2
  if (!(opts.inner_tol > 0)) opts.inner_tol = opts.storage == S7_BF16 ? 1e-1 : 1e-2;
  if (opts.inner_maxit <= 0) opts.inner_maxit = 100;
  if (opts.max_outer <= 0) opts.max_outer = 60;
  s7_server* S = new (std::nothrow) s7_server();
  if (!S) return set_error(S7_ENOMEM, "s7_server_create: host allocation failed");
  S->o = opts;
  S->eng = engine_for(opts.storage);
  if (!S->eng) {
    delete S;
    return set_error(S7_EINVAL, "s7_server_create: bad storage type");
  }
  cudaGetDevice(&S->device);
  cudaError_t e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st_admit, cudaStreamNonBlocking);
  const size_t ns = (size_t)opts.max_active;
  if (e == cudaSuccess) e = cudaMalloc(&S->d_sc, ns * sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMemset(S->d_sc, 0, ns * sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_sc, ns * sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_hist, ns * (opts.inner_maxit + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_desc, ns * S->eng->desc_size);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_desc_start, ns * S->eng->desc_size);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s7_server_destroy(S);
    return set_error(S7_ENOMEM, "s7_server_create: device allocation failed");
  }
  for (int i = (int)ns - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->th = std::thread(scheduler, S);
  S->th_admit = std::thread(admitter, S);
  *out = S;
  return S7_OK;
}

extern "C" int s7_server_submit(s7_server_t S, const s7_request* r, uint64_t* id) {
  if (!S || !r || !r->b || !r->x) return set_error(S7_EINVAL, "s7_server_submit: bad arguments");
  if (r->nx < 1 || r->ny < 1 || r->nz < 1 || (r->dt != S7_F64 && r->dt != S7_F32) || !(r->tol > 0))
    return set_error(S7_EINVAL, "s7_server_submit: bad sizes, dtype or tol");
  Req* q = new (std::nothrow) Req();
  if (!q) return set_error(S7_ENOMEM, "s7_server_submit: host allocation failed");
  q->in = *r;
  // operators are held per cell, with whole wide vectors per row
  const int vw = S->eng->vec_wide;
  q->nxp = (r->nx + vw - 1) / vw * vw;
  q->n_in = (long long)r->nx * r->ny * r->nz;
  q->n = (long long)q->nxp * r->ny * r->nz;
  q->bytes = request_bytes(S, q->n, r->coeffs.dtype == S7_F64 ? 8 : 4);
  if (q->bytes > S->o.hbm_budget_bytes) {
    delete q;
    return set_error(S7_ENOMEM, "s7_server_submit: request larger than the memory budget");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    delete q;
    return set_error(S7_ECANCELED, "s7_server_submit: server is stopping");
  }
  q->id = S->next_id++;
  q->t_arrive = now_s();
  S->reqs[q->id] = q;
  S->queue.push_back(q);
  if (id) *id = q->id;
  S->cv_work.notify_one();
  return S7_OK;
}

extern "C" int s7_server_poll(s7_server_t S, uint64_t id, s7_result* out) {
  if (!S || !out) return set_error(S7_EINVAL, "s7_server_poll: bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return set_error(S7_EINVAL, "s7_server_poll: unknown request");
  if (it->second->state != FINISHED) return S7_EAGAIN;
  fill_result(it->second, out);
  return S7_OK;
}

extern "C" int s7_server_wait(s7_server_t S, uint64_t id, s7_result* out, double timeout_s) {
  if (!S || !out) return set_error(S7_EINVAL, "s7_server_wait: bad arguments");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return set_error(S7_EINVAL, "s7_server_wait: unknown request");
  Req* r = it->second;
  const auto pred = [&] { return r->state == FINISHED; };
  if (timeout_s < 0) S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return set_error(S7_ETIMEOUT, "s7_server_wait: timed out");
  fill_result(r, out);
  return S7_OK;
}

extern "C" int s7_server_release(s7_server_t S, uint64_t id) {
  if (!S) return set_error(S7_EINVAL, "s7_server_release: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return set_error(S7_EINVAL, "s7_server_release: unknown request");
  if (it->second->state != FINISHED) return set_error(S7_EAGAIN, "s7_server_release: not finished");
  delete it->second;
  S->reqs.erase(it);
  return S7_OK;
}

extern "C" int s7_server_get_stats(s7_server_t S, s7_server_stats* out) {
  if (!S || !out) return set_error(S7_EINVAL, "s7_server_get_stats: bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (long long)(S->queue.size() + S->ready.size() + S->admitting);
  out->active = (long long)S->active.size();
  out->mem_used = S->mem_used;
  out->mem_peak = S->mem_peak;
  out->cell_iters = S->cell_iters;
  out->busy_s = S->busy_s;
  return S7_OK;
}

extern "C" int s7_server_destroy(s7_server_t S) {
  if (!S) return S7_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
    S->cv_ready.notify_all();
  }
  if (S->th_admit.joinable()) S->th_admit.join();
  if (S->th.joinable()) S->th.join();
  for (auto& kv : S->reqs) delete kv.second;
  S->reqs.clear();
  if (S->st) cudaStreamSynchronize(S->st);
  if (S->d_sc) cudaFree(S->d_sc);
  if (S->h_sc) cudaFreeHost(S->h_sc);
  if (S->d_hist) cudaFree(S->d_hist);
  if (S->d_desc) cudaFree(S->d_desc);
  if (S->d_desc_start) cudaFree(S->d_desc_start);
  if (S->st) cudaStreamDestroy(S->st);
  if (S->st_admit) cudaStreamDestroy(S->st_admit);
  delete S;
  return S7_OK;
}
