// Batched kernels: one launch advances many independent systems.
//
// Every system has a descriptor (its mesh, tile, operator, Krylov vectors,
// scalars, partial-sum area and history) and owns a contiguous range of the
// launch's blocks.  A block finds its system by binary search over the
// ranges' first blocks, then runs the same sweep or update body as the
// single-system kernels, with that system's grid combine (its own counter,
// partials and block count).  Systems that have stopped leave their blocks
// idle (they return at entry), so a captured graph of steps serves a batch
// whose members converge at different steps.
#pragma once

#include <type_traits>

#include "s7_step.cuh"
#include "s7_sweep.cuh"

namespace s7 {

template <class T, class X>
struct SysDesc {
  Geom g;
  int vl;            // rows of whole 16-byte vectors (vector loads)
  int block0;        // first sweep block of this system
  int nblocks;       // sweep blocks
  int ublock0;       // first update block
  int unblocks;      // update blocks
  int punblocks;     // update tiles of the persistent launch (larger: fewer claims)
  int constant;      // constant coefficients (cc / cdiag)
  long long n;
  const T* c[6];
  const T* diag;     // raw diagonal (operator kept without Jacobi scaling) or NULL
  double cc[6];
  double cdiag;
  const void* d;     // kept diagonal for b~ = D^-1 b (NULL: constant cdiv)
  double cdiv;       // constant divisor when d is NULL
  T* r;
  T* r2;             // second r buffer (two-reduction variant) or NULL
  T* rh;
  T* p[2];
  T* s[2];
  T* y;
  X* x;
  const X* b;
  double* parts;
  double* hist;
  Scalars* sc;
};

// Index of the system whose block range holds block `blk` (ranges ascend).
template <class D>
__device__ __forceinline__ int find_system(const D* sys, int nsys, int blk, bool update) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int first = update ? sys[mid].ublock0 : sys[mid].block0;
    if (first <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// KIND 0: p update + s = A p + (r0,s) -> alpha.  KIND 1: q + y = A q +
// (q,y),(y,y) -> omega.  KIND 2: start residual r0 = D^-1 b - A x0.
// KIND 3: y = A r (timing probe of the autotuner; no reductions).  The two
// passes of the two-reduction variant (systems created with variant 1):
// KIND 4: q + y = A q + (q,y),(y,y),(r0,y) -> omega, beta from the rho
// recurrence; KIND 5: x, r updates fused with p + s = A p of the next step
// + (r0,s),(r,r),(r0,r) -> alpha, history, stop test.
// Sweep block `bid` of system `d` (register form; kinds as above).
template <class T, class X, class DT, class A, int VEC, int KIND>
__device__ __forceinline__ void batched_sweep(const SysDesc<T, X>& d, int bid, unsigned char* s7_smem,
                                              double* red) {
  Scalars* sc = d.sc;
  const Geom g = d.g;
  CoefView<T, A> cf;
  for (int k = 0; k < 6; ++k) {
    cf.c[k] = d.c[k];
    cf.cc[k] = (A)d.cc[k];
  }
  cf.diag = d.diag;
  cf.cdiag = (A)d.cdiag;
  cf.constant = d.constant;
  A* sm = reinterpret_cast<A*>(s7_smem);
  if (KIND == 0) {
    SrcPUpdate<T, A> src;
    src.r = d.r;
    src.pbuf[0] = d.p[0];
    src.pbuf[1] = d.p[1];
    src.sbuf[0] = d.s[0];
    src.sbuf[1] = d.s[1];
    EpiS<T, A> epi;
    epi.sbuf[0] = d.s[0];
    epi.sbuf[1] = d.s[1];
    epi.rh = d.rh;
    epi.parts = d.parts;
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else if (KIND == 1) {
    SrcQ<T, A> src;
    src.r = d.r;
    src.sbuf[0] = d.s[0];
    src.sbuf[1] = d.s[1];
    EpiY<T, A> epi;
    epi.y_out = d.y;
    epi.parts = d.parts;
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else if (KIND == 2) {
    SrcPlain<X, A> src{d.x};
    EpiResid<X, T, DT, A> epi;
    epi.b = d.b;
    epi.dinv = (const DT*)d.d;
    epi.dc = (A)d.cdiv;
    epi.dmul = nullptr;
    epi.dmc = A(1);
    epi.r_out = d.r;
    epi.rh_out = d.rh;
    epi.parts = d.parts;
    epi.counter = CNT_INIT;
    epi.mode = 0;
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else if (KIND == 3) {
    SrcPlain<T, A> src{d.r};
    EpiStore<T, A> epi{d.y};
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, src, epi, nullptr, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, src, epi, nullptr, bid, d.nblocks, sm, red);
  } else if (KIND == 4) {
    SrcQ2<T, A> src;
    src.rbuf[0] = d.r;
    src.rbuf[1] = d.r2;
    src.sbuf[0] = d.s[0];
    src.sbuf[1] = d.s[1];
    EpiYMerged<T, A> epi;
    epi.y_out = d.y;
    epi.rh = d.rh;
    epi.parts = d.parts;
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else {
    MergedPass<T, X, A> m;
    m.rbuf[0] = d.r;
    m.rbuf[1] = d.r2;
    m.pbuf[0] = d.p[0];
    m.pbuf[1] = d.p[1];
    m.sbuf[0] = d.s[0];
    m.sbuf[1] = d.s[1];
    m.y = d.y;
    m.rh = d.rh;
    m.x = d.x;
    m.parts = d.parts;
    m.hist = d.hist;
    if (d.vl) sweep_body<T, A, VEC, true, true>(g, cf, m, m, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false, true>(g, cf, m, m, sc, bid, d.nblocks, sm, red);
  }
}

template <class T, class X, class DT, class A, int VEC, int KIND>
__global__ void __launch_bounds__(256) k_sweep_batched(const SysDesc<T, X>* __restrict__ sys,
                                                       int nsys) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(sys, nsys, (int)blockIdx.x, false);
  __syncthreads();
  const SysDesc<T, X>& d = sys[s_sys];
  if ((KIND == 0 || KIND == 1 || KIND == 4 || KIND == 5) && *((volatile int*)&d.sc->done)) return;
  batched_sweep<T, X, DT, A, VEC, KIND>(d, (int)blockIdx.x - d.block0, s7_smem, red);
}

// The pipelined sweeps (kinds 0-3 of s7_step.cuh) over a batch whose
// systems all qualify (Jacobi-scaled per-cell operators, rows of whole
// VEC-cell vectors); each system's geometry in its descriptor is for VEC
// cells per thread.  Kinds 2 and 3 (the two-reduction variant) need r2.
// Two 256-thread blocks per SM bound the registers (at most 128 a thread):
// the descriptor lookup otherwise takes the fused pass to 142 registers and
// three 128-thread blocks per SM (served BF16 to 1e-8: 0.405 -> 0.374 s).
// Pipelined sweep block `bid` of system `d`.
template <class T, class X, class A, int VEC, int KIND, int STAGES>
__device__ __forceinline__ void batched_step(const SysDesc<T, X>& d, int bid, unsigned char* s7_smem,
                                             double* red, unsigned long long* bars) {
  StepArgs<T> a;
  for (int k = 0; k < 6; ++k) a.c[k] = d.c[k];
  a.r = d.r;
  a.rh = d.rh;
  a.pbuf[0] = d.p[0];
  a.pbuf[1] = d.p[1];
  a.sbuf[0] = d.s[0];
  a.sbuf[1] = d.s[1];
  a.y = d.y;
  a.parts = d.parts;
  a.rbuf[0] = d.r;
  a.rbuf[1] = d.r2;
  a.x = d.x;
  a.hist = d.hist;
  a.maps = nullptr;   // batches stage with cp.async
  step_body<T, A, VEC, KIND, STAGES>(d.g, a, d.sc, bid, d.nblocks, s7_smem, red, bars);
}

template <class T, class X, class A, int VEC, int KIND, int STAGES>
__global__ void __launch_bounds__(256, 2) k_step_batched(const SysDesc<T, X>* __restrict__ sys,
                                                      int nsys) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(sys, nsys, (int)blockIdx.x, false);
  __syncthreads();
  const SysDesc<T, X>& d = sys[s_sys];
  if (*((volatile int*)&d.sc->done)) return;
  batched_step<T, X, A, VEC, KIND, STAGES>(d, (int)blockIdx.x - d.block0, s7_smem, red, bars);
}

template <class T, class X, class A, int VEC>
__global__ void __launch_bounds__(256) k_update_batched(const SysDesc<T, X>* __restrict__ sys,
                                                        int nsys) {
  __shared__ double red[32 * 4];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(sys, nsys, (int)blockIdx.x, true);
  __syncthreads();
  const SysDesc<T, X>& d = sys[s_sys];
  if (*((volatile int*)&d.sc->done)) return;
  update_body<T, X, A, VEC>(d.n, d.p[0], d.p[1], d.s[0], d.s[1], d.y, d.rh, d.r, d.x, d.sc,
                            d.parts, d.hist, (int)blockIdx.x - d.ublock0, d.unblocks, red);
}

// ---------------------------------------------------------------------------
// The persistent batched solve: one launch runs every step of every system.
//
// The grid (no larger than the blocks that fit on the device at once, a
// cooperative launch) works from a queue per system.  A system's step is a
// sequence of phases (p/s sweep, q/y sweep, update; or the two passes of the
// two-reduction variant), each a set of tiles: the sweep blocks (or update
// blocks) of the launch-per-kernel form.  A phase's tiles open once its
// previous phase has completed, and any block may claim any open tile of
// any system, so the device stays full while systems run their steps at
// their own pace, and the last large systems get every block in the end.
// Tiles are the same as in the launch-per-kernel form and each carries its
// own partial sums, so a system's arithmetic does not depend on which block
// ran which tile (the same bits alone and in any mix).
//
// Queue word per system: (phase << 32) | next tile to claim.  The block
// that completes a phase's last tile (it finds every other tile counted, and
// with them the phase's grid combine) opens the next phase by exchanging the
// word, or marks the system finished (a word whose tile count no claim can
// reach).  The first warp of a block looks for an open tile 32 systems at
// a time, starting from the system of its last claim (so a block stays with
// a system while it has open tiles instead of rescanning the batch from the
// top; the first scan starts at the largest systems, which set the end of
// the batch), and claims one tile at a time.  A block that finds no open tile waits at most
// `budget` SM clock cycles for one; when a wait runs out it aborts the
// launch: every unfinished system stops with status 5 (S7_ETIMEOUT) and
// every block leaves after its current tile, so nothing can hang the device.
// ---------------------------------------------------------------------------
struct SysQueue {
  unsigned long long word;   // (phase << 32) | next tile
  unsigned int tiles_done;   // tiles of the current phase completed
  unsigned int finished;     // 1 once the system has stopped
};
struct QueueState {
  unsigned int n_finished;
  int abort;
};
constexpr unsigned long long kQueueClosed = (0xffffffffull << 32) | 0x80000000ull;

// Queues of the systems that stopped before the launch (done at the start),
// closed; the others open at phase 0.
template <class T, class X>
__global__ void k_queue_init(const SysDesc<T, X>* __restrict__ sys, int nsys, SysQueue* q,
                             QueueState* qs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nsys) return;
  const bool done = *((volatile int*)&sys[j].sc->done) != 0;
  q[j].word = done ? kQueueClosed : 0ull;
  q[j].tiles_done = 0u;
  q[j].finished = done ? 1u : 0u;
  if (done) atomicAdd(&qs->n_finished, 1u);
}

// PIPE: the batch runs the pipelined sweeps (VEC = the wide vector; the q/y
// sweep of float32/float64 storage in its register form, as in the
// launch-per-kernel batches).  MERGED: the two-reduction variant.  VU: the
// update's cells per thread.  order: the systems, largest first.
// Registers: the blocks hide load latency by their number (the register
// sweeps keep their loads in registers), so Algorithm 1's form is bounded to
// 85 registers (three 256-thread blocks per SM: 5-6 blocks of 128 threads,
// a few spilled words), measured 4.66e10 against 4.01e10 cell-iters/s at 128
// registers on 512 mixed systems; the two-reduction form spills too much
// below 128 registers (3.36e10 at 85 against 3.95-4.11e10).
template <class T, class X, class DT, class A, int VEC, int VU, int STAGES, bool PIPE,
          bool MERGED, bool PIPE_Q>
__global__ void __launch_bounds__(256, MERGED ? 2 : 3)
    k_batched_persistent(const SysDesc<T, X>* __restrict__ sys, const int* __restrict__ order,
                         int nsys, SysQueue* q, QueueState* qs, long long budget) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  __shared__ int s_sys, s_phase, s_tile;
  constexpr int NPH = MERGED ? 2 : 3;   // phases per step
  auto tiles_of = [&](int j, unsigned int ph) -> unsigned int {
    return (unsigned int)((!MERGED && ph == 2) ? sys[j].punblocks : sys[j].nblocks);
  };
  int pos = 0;   // (first warp) where in `order` the next scan starts: the last claim's system
  for (;;) {
    // ---- the first warp claims a tile, or finds that none is left
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int got = 0;           // 1: claimed, -1: stop
      long long t0 = -1;
      while (got == 0) {
        if (*((volatile int*)&qs->abort) ||
            *((volatile unsigned int*)&qs->n_finished) >= (unsigned int)nsys) {
          got = -1;
          break;
        }
        for (int base = 0; base < nsys && got == 0; base += 32) {
          const int k = base + lane;
          const int idx = pos + k < nsys ? pos + k : pos + k - nsys;
          int j = -1;
          bool open = false;
          if (k < nsys) {
            j = order[idx];
            const unsigned long long w = *((volatile unsigned long long*)&q[j].word);
            open = (unsigned int)(w & 0xffffffffull) < tiles_of(j, (unsigned int)((w >> 32) % NPH));
          }
          unsigned int mask = __ballot_sync(0xffffffffu, open);
          while (mask) {
            const int src = __ffs(mask) - 1;
            int ok = 0;
            if (lane == src) {
              const unsigned long long old = atomicAdd(&q[j].word, 1ull);
              const unsigned int ph = (unsigned int)((old >> 32) % NPH);
              const unsigned int tile = (unsigned int)(old & 0xffffffffull);
              if (tile < tiles_of(j, ph) && !*((volatile unsigned int*)&q[j].finished)) {
                ok = 1;
                s_sys = j;
                s_phase = (int)ph;
                s_tile = (int)tile;
              }
            }
            if (__shfl_sync(0xffffffffu, ok, src)) {
              got = 1;
              pos = __shfl_sync(0xffffffffu, idx, src);
              break;
            }
            mask &= mask - 1u;
          }
        }
        if (got == 0) {   // every open tile is taken: wait for a phase to complete
          int stop = 0;
          if (lane == 0) {
            if (t0 < 0) t0 = clock64();
            else if (clock64() - t0 > budget) {
              qs->abort = 1;
              __threadfence();
              stop = 1;
            }
          }
          if (__shfl_sync(0xffffffffu, stop, 0)) got = -1;
          else __nanosleep(64);
        }
      }
      if (lane == 0) {
        if (got < 0) s_sys = -1;
        __threadfence();
      }
    }
    __syncthreads();
    const int j = s_sys;
    if (j < 0) break;
    const SysDesc<T, X>& d = sys[j];
    const int ph = s_phase, tile = s_tile;
    // ---- run the tile
    if constexpr (MERGED) {
      if (ph == 0) {
        if constexpr (PIPE) batched_step<T, X, A, VEC, 2, STAGES>(d, tile, s7_smem, red, bars);
        else batched_sweep<T, X, DT, A, VEC, 4>(d, tile, s7_smem, red);
      } else {
        if constexpr (PIPE) batched_step<T, X, A, VEC, 3, STAGES>(d, tile, s7_smem, red, bars);
        else batched_sweep<T, X, DT, A, VEC, 5>(d, tile, s7_smem, red);
      }
    } else {
      if (ph == 0) {
        if constexpr (PIPE) batched_step<T, X, A, VEC, 0, STAGES>(d, tile, s7_smem, red, bars);
        else batched_sweep<T, X, DT, A, VEC, 0>(d, tile, s7_smem, red);
      } else if (ph == 1) {
        if constexpr (PIPE && PIPE_Q) batched_step<T, X, A, VEC, 1, STAGES>(d, tile, s7_smem, red, bars);
        else batched_sweep<T, X, DT, A, VEC, 1>(d, tile, s7_smem, red);
      } else {
        update_body<T, X, A, VU>(d.n, d.p[0], d.p[1], d.s[0], d.s[1], d.y, d.rh, d.r, d.x, d.sc,
                                 d.parts, d.hist, tile, d.punblocks, red);
      }
    }
    __syncthreads();
    // ---- count the tile; the last one of the phase opens the next phase
    if (threadIdx.x == 0) {
      SysQueue* qj = q + j;
      __threadfence();
      if (atomicAdd(&qj->tiles_done, 1u) == tiles_of(j, (unsigned int)ph) - 1u) {
        qj->tiles_done = 0u;
        __threadfence();
        if (*((volatile int*)&d.sc->done)) {
          atomicExch(&qj->word, kQueueClosed);
          if (atomicCAS(&qj->finished, 0u, 1u) == 0u) atomicAdd(&qs->n_finished, 1u);
        } else {
          const unsigned long long next = (qj->word >> 32) + 1ull;
          atomicExch(&qj->word, next << 32);
        }
      }
    }
  }
  // an aborted launch: the systems still running stop timed out
  if (blockIdx.x == 0 && threadIdx.x == 0 && *((volatile int*)&qs->abort)) {
    for (int j = 0; j < nsys; ++j) {
      Scalars* sc = sys[j].sc;
      if (!*((volatile int*)&sc->done)) {
        sc->status = 5;
        sc->done = 1;
      }
    }
  }
}

// hist[0] = ||r0|| / ||b~|| for every system (after the start sweep).
template <class T, class X>
__global__ void k_hist0_batched(const SysDesc<T, X>* __restrict__ sys, int nsys) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nsys && sys[j].hist) sys[j].hist[0] = sys[j].sc->res[2];
}

}  // namespace s7
