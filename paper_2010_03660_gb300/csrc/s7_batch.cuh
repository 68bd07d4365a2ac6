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
template <class T, class X, class DT, class A, int VEC, int KIND>
__global__ void __launch_bounds__(256) k_sweep_batched(const SysDesc<T, X>* __restrict__ sys,
                                                       int nsys) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  __shared__ int s_sys;
  if (threadIdx.x == 0) s_sys = find_system(sys, nsys, (int)blockIdx.x, false);
  __syncthreads();
  const SysDesc<T, X>& d = sys[s_sys];
  Scalars* sc = d.sc;
  if ((KIND == 0 || KIND == 1 || KIND == 4 || KIND == 5) && *((volatile int*)&sc->done)) return;
  const int bid = (int)blockIdx.x - d.block0;
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
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else if (KIND == 1) {
    SrcQ<T, A> src;
    src.r = d.r;
    src.sbuf[0] = d.s[0];
    src.sbuf[1] = d.s[1];
    EpiY<T, A> epi;
    epi.y_out = d.y;
    epi.parts = d.parts;
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
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
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
  } else if (KIND == 3) {
    SrcPlain<T, A> src{d.r};
    EpiStore<T, A> epi{d.y};
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, src, epi, nullptr, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, src, epi, nullptr, bid, d.nblocks, sm, red);
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
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, src, epi, sc, bid, d.nblocks, sm, red);
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
    if (d.vl) sweep_body<T, A, VEC, true>(g, cf, m, m, sc, bid, d.nblocks, sm, red);
    else sweep_body<T, A, VEC, false>(g, cf, m, m, sc, bid, d.nblocks, sm, red);
  }
}

// The pipelined sweeps (kinds 0-3 of s7_step.cuh) over a batch whose
// systems all qualify (Jacobi-scaled per-cell operators, rows of whole
// VEC-cell vectors); each system's geometry in its descriptor is for VEC
// cells per thread.  Kinds 2 and 3 (the two-reduction variant) need r2.
// Two 256-thread blocks per SM bound the registers (at most 128 a thread):
// the descriptor lookup otherwise takes the fused pass to 142 registers and
// three 128-thread blocks per SM (served BF16 to 1e-8: 0.405 -> 0.374 s).
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
  step_body<T, A, VEC, KIND, STAGES>(d.g, a, d.sc, (int)blockIdx.x - d.block0, d.nblocks, s7_smem,
                                     red, bars);
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

// hist[0] = ||r0|| / ||b~|| for every system (after the start sweep).
template <class T, class X>
__global__ void k_hist0_batched(const SysDesc<T, X>* __restrict__ sys, int nsys) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nsys && sys[j].hist) sys[j].hist[0] = sys[j].sc->res[2];
}

}  // namespace s7
