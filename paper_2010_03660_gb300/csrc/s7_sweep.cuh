// The z-marching 7-point stencil sweep.
//
// The paper maps X and Y of the mesh across the processor fabric and keeps
// the whole Z column in each core, where the two z-neighbour terms of the
// SpMV come from shifted copies of the local column (Sec. IV, Sec. IV-A).
// The GB300 analogue: a thread block owns an xy tile of (bx*VEC) x by cells
// and a chunk of z planes, and marches along z.  Each thread owns VEC
// consecutive x cells of one row; it keeps the input vector at z-1, z, z+1
// for its own cells in registers, so the z terms cost no extra memory
// traffic.  The x and y neighbours come from the current plane staged in
// shared memory with a one-cell halo ring.
//
// The input of every SpMV in the solver is not stored: it is formed on the
// fly from other vectors (p_{i} = r + beta (p - omega s) before s = A p;
// q = r - alpha s before y = A q), by a `Src` policy that is evaluated for the
// block's own cells and for its halo ring.  An `Epi` policy consumes each
// output run (stores, fused inner products) and finishes the block with the
// deterministic grid combine.
//
// Shared memory: three plane buffers used as a ring, so one __syncthreads()
// per plane suffices: step k fills buffer (k+1)%3 with plane z+1 and then
// reads buffer k%3; buffer (k+2)%3, written at step k+1, was last read at
// step k-1, before step k's barrier.
#pragma once

#include "s7_common.cuh"

namespace s7 {

// Device-resident solver scalars (one per solve in flight).
struct Scalars {
  double rho;     // (r0, r_i)
  double alpha;
  double omega;
  double beta;
  double bnorm;   // ||b~||_2
  double tol;
  double res[4];  // totals of auxiliary reductions (residual norms)
  int iter;       // completed steps
  int maxit;
  int done;       // 1: no further step runs
  int status;     // S7_* code once done
  int special;    // 1: (y,y) = 0 in this step (q = 0): take the half step
  int pad_;
  double rho_next;  // merged variant: (r0, r_{i+1}) from its recurrence
  unsigned int counter[8];  // grid-combine arrival counters, one per kernel kind
};

enum { CNT_A = 0, CNT_B = 1, CNT_C = 2, CNT_INIT = 3, CNT_RES = 4, CNT_AUX = 5 };

struct Geom {
  int nx, ny, nz;
  int bx, by;          // tile: bx threads of VEC cells in x, by rows
  int tiles_x, tiles_y;
  int zchunk, nchunks;
  long long plane;     // nx * ny
};

__host__ __device__ inline int s7_nblocks(const Geom& g) { return g.tiles_x * g.tiles_y * g.nchunks; }

// Coefficients of the stored operator as seen by a sweep.
template <class CT, class A>
struct CoefView {
  typedef typename CoefOf<A>::t CA;   // coefficient values inside the sweep
  const CT* c[6];    // xm xp ym yp zm zp; unused when constant
  const CT* diag;    // NULL: unit (or constant) diagonal
  CA cc[6];          // constant coefficients
  CA cdiag;          // constant / unit diagonal value
  int constant;
};

template <class T, int VEC, bool VL, int POL = LD_DEFAULT, class A>
__device__ __forceinline__ void load_run(const T* __restrict__ p, int nv, A (&o)[VEC]) {
  if (VL) ldv<T, VEC, POL>(p, o);
  else lds<T, VEC>(p, nv, o);
}
template <class T, int VEC, bool VL, bool STREAM = false, class A>
__device__ __forceinline__ void store_run(T* __restrict__ p, int nv, const A (&v)[VEC]) {
  if (VL) stv<T, VEC, STREAM>(p, v);
  else sts<T, VEC>(p, nv, v);
}

// Value as it is after a round trip through storage type T.
template <class T, class A> __device__ __forceinline__ A as_stored(A v) {
  return to_acc<A>(from_acc<T>(v));
}

template <class A, int VEC> __device__ __forceinline__ void zero(A (&v)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; ++k) v[k] = A(0);
}

// Shared-memory run of VEC values at `p` (aligned to VEC elements): vector
// accesses of up to 16 bytes.
template <class A, int VEC> __device__ __forceinline__ void sm_load(const A* p, A (&o)[VEC]) {
  ldv<A, VEC>(p, o);
}
template <class A, int VEC> __device__ __forceinline__ void sm_store(A* p, const A (&v)[VEC]) {
  stv<A, VEC>(p, v);
}

// ---------------------------------------------------------------------------
// L2 prefetch of the coefficient planes ahead of the z march
// ---------------------------------------------------------------------------
// The register sweeps load each plane's coefficients when they reach it and
// wait for DRAM at that point unless other warps cover the wait.  Each thread
// asks for the lines of its own cells' coefficients a few planes ahead to be
// brought into L2 (`prefetch.global.L2`, a hint nothing waits on), so that
// those loads find them there.  The addresses are always cells of the mesh.
// Only the batched sweeps take it (sweep_body's PF): on 512 mixed systems in
// the persistent launch 4.66 -> 4.78e10 cell-iters/s, while the single-system
// q/y sweep in registers lost occupancy to it (3.18 -> 3.48 ms at
// 600x595x1536).
constexpr int kCoefPrefetchPlanes = 2;

template <class T> __device__ __forceinline__ void l2_prefetch(const T* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <class CT, class A>
__device__ __forceinline__ void prefetch_coef(const CoefView<CT, A>& cf, long long i) {
#pragma unroll
  for (int d = 0; d < 6; ++d) l2_prefetch(cf.c[d] + i);
  if (cf.diag) l2_prefetch(cf.diag + i);
}

// ---------------------------------------------------------------------------
// the sweep kernel
// ---------------------------------------------------------------------------
// Template parameters: CT coefficient type, A arithmetic type, VEC cells per
// thread, VL vector loads (nx % VEC == 0 and aligned buffers), Src / Epi the
// policies.  blockDim.x = roundup(bx*by, 32); threads past bx*by own no
// cells but take part in barriers and reductions.
// The body of one sweep block: block `bid` of the `nblocks` blocks of the
// sweep over the mesh `g`.  `sm` is the dynamic shared memory (three plane
// buffers), `red` 128 doubles of reduction scratch.
template <class CT, class A, int VEC, bool VL, bool PF = false, class Src, class Epi>
__device__ __forceinline__ void sweep_body(const Geom& g, const CoefView<CT, A>& cf, Src& src,
                                           Epi& epi, Scalars* sc, int bid, int nblocks, A* sm,
                                           double* red) {
  src.setup(sc);
  epi.setup(sc);

  const int t = threadIdx.x;
  const bool has_cell = t < g.bx * g.by;
  const int tx = has_cell ? t % g.bx : 0;
  const int ty = has_cell ? t / g.bx : 0;
  const int tile_x = bid % g.tiles_x;
  const int rest = bid / g.tiles_x;
  const int tile_y = rest % g.tiles_y;
  const int chunk = rest / g.tiles_y;
  const int x0 = tile_x * g.bx * VEC;
  const int y0 = tile_y * g.by;
  const int z0 = chunk * g.zchunk;
  const int z1 = min(z0 + g.zchunk, g.nz);
  const int x = x0 + tx * VEC;
  const int y = y0 + ty;
  const int W = g.bx * VEC + 2 * VEC;     // smem row pitch (VEC pad each side)
  const int PL = (g.by + 2) * W;          // one plane buffer
  const int so = (ty + 1) * W + VEC + tx * VEC;  // own element 0 in a buffer

  auto run_len = [&](int yy) -> int {
    if (!has_cell || yy < 0 || yy >= g.ny) return 0;
    int r = g.nx - x;
    return r <= 0 ? 0 : (r < VEC ? r : VEC);
  };
  const int nv = run_len(y);
  const int nv_top = (has_cell && ty == 0) ? run_len(y - 1) : 0;
  const int nv_bot = (has_cell && ty == g.by - 1) ? run_len(y + 1) : 0;
  const bool is_top = has_cell && ty == 0;
  const bool is_bot = has_cell && ty == g.by - 1;
  const bool is_lft = has_cell && tx == 0;
  const bool is_rgt = has_cell && tx == g.bx - 1;
  const bool ok_l = is_lft && x0 > 0 && y < g.ny;
  const bool ok_r = is_rgt && (x0 + g.bx * VEC) < g.nx && y < g.ny;
  const long long row = (long long)y * g.nx + x;   // + z * plane

  // Form the input vector on plane zp: own run into `own`, and (if `ring`)
  // own run plus halo ring into shared buffer `buf`.  Own cells inside the
  // block's z range are written out by the Src if it stores its input.
  auto produce = [&](int zp, A* buf, A (&own)[VEC], bool ring, bool write_own) {
    const long long base = (long long)zp * g.plane + row;
    if (nv > 0) src.template produce<VEC, VL>(base, nv, own, write_own);
    else zero(own);
    if (!ring || !has_cell) return;
    sm_store<A, VEC>(buf + so, own);
    if (is_top) {
      A h[VEC];
      if (nv_top > 0) src.template produce<VEC, VL>(base - g.nx, nv_top, h, false);
      else zero(h);
      sm_store<A, VEC>(buf + so - W, h);
    }
    if (is_bot) {
      A h[VEC];
      if (nv_bot > 0) src.template produce<VEC, VL>(base + g.nx, nv_bot, h, false);
      else zero(h);
      sm_store<A, VEC>(buf + so + W, h);
    }
    if (is_lft) buf[so - 1] = ok_l ? src.produce1(base - 1) : A(0);
    if (is_rgt) buf[so + VEC] = ok_r ? src.produce1(base + VEC) : A(0);
  };

  if (PF && !cf.constant && nv > 0)
    for (int zp = z0 + 1; zp < z0 + kCoefPrefetchPlanes && zp < z1; ++zp)
      prefetch_coef(cf, (long long)zp * g.plane + row);
  A vm[VEC], vc[VEC], vp[VEC];
  if (z0 > 0) produce(z0 - 1, nullptr, vm, false, false);
  else zero(vm);
  produce(z0, sm, vc, true, true);

  for (int z = z0, k = 0; z < z1; ++z, ++k) {
    const long long ib = (long long)z * g.plane + row;
    if (PF && !cf.constant && nv > 0 && z + kCoefPrefetchPlanes < z1)
      prefetch_coef(cf, ib + kCoefPrefetchPlanes * g.plane);
    // coefficients of plane z (streamed: no other block reads them)
    typename CoefOf<A>::t c[6][VEC], dg[VEC];
    if (cf.constant) {
#pragma unroll
      for (int d = 0; d < 6; ++d)
#pragma unroll
        for (int j = 0; j < VEC; ++j) c[d][j] = cf.cc[d];
#pragma unroll
      for (int j = 0; j < VEC; ++j) dg[j] = cf.cdiag;
    } else if (nv > 0) {
#pragma unroll
      for (int d = 0; d < 6; ++d) load_run<CT, VEC, VL, LD_STREAM>(cf.c[d] + ib, nv, c[d]);
      if (cf.diag) load_run<CT, VEC, VL, LD_STREAM>(cf.diag + ib, nv, dg);
      else
#pragma unroll
        for (int j = 0; j < VEC; ++j) dg[j] = cf.cdiag;
    } else {
#pragma unroll
      for (int d = 0; d < 6; ++d) zero(c[d]);
      zero(dg);
    }
    epi.template load<VEC, VL>(ib, nv);

    A* nb = sm + ((k + 1) % 3) * PL;
    if (z + 1 < g.nz) produce(z + 1, nb, vp, z + 1 < z1, z + 1 < z1);
    else zero(vp);
    __syncthreads();

    if (nv > 0) {
      const A* cb = sm + (k % 3) * PL;
      A up[VEC], dn[VEC];
      sm_load<A, VEC>(cb + so - W, up);
      sm_load<A, VEC>(cb + so + W, dn);
      const A lf = cb[so - 1];
      const A rt = cb[so + VEC];
      A out[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const A l = (j == 0) ? lf : vc[j - 1];
        const A r = (j == VEC - 1) ? rt : vc[j + 1];
        A acc = dg[j] * vc[j];
        acc = fma(c[0][j], l, acc);
        acc = fma(c[1][j], r, acc);
        acc = fma(c[2][j], up[j], acc);
        acc = fma(c[3][j], dn[j], acc);
        acc = fma(c[4][j], vm[j], acc);
        acc = fma(c[5][j], vp[j], acc);
        out[j] = settle(acc);
      }
      epi.template consume<VEC, VL>(ib, nv, out, vc);
    }
    epi.step_end(k);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      vm[j] = vc[j];
      vc[j] = vp[j];
    }
  }
  epi.finish(sc, nblocks, bid, red);
}

// One policy object in both roles (its producer and epilogue share state).
template <class CT, class A, int VEC, bool VL, class P>
__global__ void __launch_bounds__(512) k_sweep1(Geom g, CoefView<CT, A> cf, P p_in, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  if (sc != nullptr && P::kSkipWhenDone && *((volatile int*)&sc->done)) return;
  P pol = p_in;
  sweep_body<CT, A, VEC, VL>(g, cf, pol, pol, sc, blockIdx.x, s7_nblocks(g),
                             reinterpret_cast<A*>(s7_smem), red);
}

template <class CT, class A, int VEC, bool VL, class Src, class Epi>
__global__ void __launch_bounds__(512) k_sweep(Geom g, CoefView<CT, A> cf, Src src_in, Epi epi_in,
                                               Scalars* sc) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  if (sc != nullptr && Epi::kSkipWhenDone && *((volatile int*)&sc->done)) return;
  Src src = src_in;
  Epi epi = epi_in;
  sweep_body<CT, A, VEC, VL>(g, cf, src, epi, sc, blockIdx.x, s7_nblocks(g),
                             reinterpret_cast<A*>(s7_smem), red);
}

// ---------------------------------------------------------------------------
// Src policies: the SpMV input formed on the fly
// ---------------------------------------------------------------------------

// v = x (a stored vector).
template <class T, class A>
struct SrcPlain {
  const T* x;
  __device__ void setup(const Scalars*) {}
  template <int VEC, bool VL>
  __device__ __forceinline__ void produce(long long i, int nv, A (&v)[VEC], bool) {
    load_run<T, VEC, VL>(x + i, nv, v);
  }
  __device__ __forceinline__ A produce1(long long i) { return to_acc<A>(x[i]); }
};

// p_i = r_i + beta (p_{i-1} - omega s_{i-1}), or p_0 = r_0 (Algorithm 1,
// last line of the loop body, moved to the start of the next step so that
// it fuses with s = A p).  The block's own cells are written to p_i.  p and s
// are double-buffered by step parity: neighbouring blocks still read
// p_{i-1}, s_{i-1} as halo while p_i, s_i are written.
template <class T, class A>
struct SrcPUpdate {
  const T* r;
  T* pbuf[2];
  T* sbuf[2];
  const T* p_old;
  const T* s_old;
  T* p_out;
  A beta, omega;
  int first;
  __device__ void setup(const Scalars* sc) {
    const int it = sc->iter;
    first = (it == 0);
    beta = (A)sc->beta;
    omega = (A)sc->omega;
    const bool odd = (it & 1) != 0;
    p_out = odd ? pbuf[1] : pbuf[0];
    p_old = odd ? pbuf[0] : pbuf[1];
    s_old = odd ? sbuf[0] : sbuf[1];
  }
  __device__ __forceinline__ A upd(A rv, A pv, A sv) const {
    return as_stored<T>(fma(beta, fma(-omega, sv, pv), rv));
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void produce(long long i, int nv, A (&v)[VEC], bool write) {
    load_run<T, VEC, VL>(r + i, nv, v);
    if (!first) {
      A pv[VEC], sv[VEC];
      load_run<T, VEC, VL>(p_old + i, nv, pv);
      load_run<T, VEC, VL>(s_old + i, nv, sv);
#pragma unroll
      for (int k = 0; k < VEC; ++k) v[k] = upd(v[k], pv[k], sv[k]);
    }
    if (write) store_run<T, VEC, VL, true>(p_out + i, nv, v);
  }
  __device__ __forceinline__ A produce1(long long i) {
    A rv = to_acc<A>(r[i]);
    if (first) return rv;
    return upd(rv, to_acc<A>(p_old[i]), to_acc<A>(s_old[i]));
  }
};

// q_i = r_i - alpha_i s_i, rounded to the storage type like every other
// Krylov vector (a no-op for float32 and float64 storage).  It is not
// stored: the SpMV sweep, the update and the fused pass each form it with
// these operations, so all of them see identical values.
template <class T, class A> __device__ __forceinline__ A q_of(A r, A s, A alpha) {
  return as_stored<T>(fma(-alpha, s, r));
}

template <class T, class A>
struct SrcQ {
  const T* r;
  T* sbuf[2];
  const T* s;
  A alpha;
  __device__ void setup(const Scalars* sc) {
    alpha = (A)sc->alpha;
    s = (sc->iter & 1) ? sbuf[1] : sbuf[0];
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void produce(long long i, int nv, A (&v)[VEC], bool) {
    A sv[VEC];
    load_run<T, VEC, VL>(r + i, nv, v);
    load_run<T, VEC, VL>(s + i, nv, sv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = q_of<T>(v[k], sv[k], alpha);
  }
  __device__ __forceinline__ A produce1(long long i) {
    return q_of<T>(to_acc<A>(r[i]), to_acc<A>(s[i]), alpha);
  }
};

// ---------------------------------------------------------------------------
// Epi policies
// ---------------------------------------------------------------------------

// Per-thread inner-product accumulator: terms are summed in A over a few
// planes, then folded into a float64 total (bounds the float32 error of long
// per-thread sums at a small cost in float64 adds).
template <class A, int NV>
struct DotAcc {
  A part[NV];
  double tot[NV];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { part[j] = A(0); tot[j] = 0.0; }
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { tot[j] += (double)part[j]; part[j] = A(0); }
  }
};

// y = A v, stored.
template <class T, class A>
struct EpiStore {
  static constexpr bool kSkipWhenDone = false;
  T* y;
  __device__ void setup(const Scalars*) {}
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long, int) {}
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&)[VEC]) {
    store_run<T, VEC, VL, true>(y + i, nv, out);
  }
  __device__ __forceinline__ void step_end(int) {}
  __device__ __forceinline__ void finish(Scalars*, int, int, double*) {}
};

// s_i = A p_i stored; (r0, s_i) reduced; alpha_i = (r0, r_i) / (r0, s_i).
template <class T, class A>
struct EpiS {
  static constexpr bool kSkipWhenDone = true;
  T* sbuf[2];
  T* s_out;
  const T* rh;
  double* parts;
  DotAcc<A, 1> acc;
  A rh_v[8];
  __device__ void setup(const Scalars* sc) {
    acc.init();
    s_out = (sc->iter & 1) ? sbuf[1] : sbuf[0];
  }
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long i, int nv) {
    static_assert(VEC <= 8, "run too long");
    if (nv > 0) {
      A t[VEC];
      load_run<T, VEC, VL>(rh + i, nv, t);
#pragma unroll
      for (int k = 0; k < VEC; ++k) rh_v[k] = t[k];
    }
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&)[VEC]) {
    A sv[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) sv[k] = as_stored<T>(out[k]);
    store_run<T, VEC, VL, true>(s_out + i, nv, sv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc.part[0] = fma(rh_v[k], sv[k], acc.part[0]);
  }
  __device__ __forceinline__ void step_end(int k) { if ((k & 7) == 7) acc.fold(); }
  __device__ void finish(Scalars* sc, int nblocks, int bid, double* red) {
    acc.fold();
    double v[1] = {acc.tot[0]}, tot[1];
    block_sum<1>(v, red);
    if (grid_combine<1>(parts, &sc->counter[CNT_A], nblocks, bid, v, tot, red) && threadIdx.x == 0) {
      const double sigma = tot[0];
      if (sigma == 0.0 || !isfinite(sigma) || !isfinite(sc->rho)) {
        sc->status = 3;  // S7_EBREAKDOWN
        sc->done = 1;
      } else {
        sc->alpha = sc->rho / sigma;
        sc->res[3] = sigma;
      }
    }
  }
};

// y_i = A q_i stored; (q, y) and (y, y) reduced; omega_i = (q,y)/(y,y).
template <class T, class A>
struct EpiY {
  static constexpr bool kSkipWhenDone = true;
  T* y_out;
  double* parts;
  DotAcc<A, 2> acc;
  __device__ void setup(const Scalars*) { acc.init(); }
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long, int) {}
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&q)[VEC]) {
    A yv[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) yv[k] = as_stored<T>(out[k]);
    store_run<T, VEC, VL, true>(y_out + i, nv, yv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      acc.part[0] = fma(q[k], yv[k], acc.part[0]);
      acc.part[1] = fma(yv[k], yv[k], acc.part[1]);
    }
  }
  __device__ __forceinline__ void step_end(int k) { if ((k & 7) == 7) acc.fold(); }
  __device__ void finish(Scalars* sc, int nblocks, int bid, double* red) {
    acc.fold();
    double v[2] = {acc.tot[0], acc.tot[1]}, tot[2];
    block_sum<2>(v, red);
    if (grid_combine<2>(parts, &sc->counter[CNT_B], nblocks, bid, v, tot, red) && threadIdx.x == 0) {
      const double qy = tot[0], yy = tot[1];
      if (yy == 0.0) {
        sc->special = 1;   // q = 0: half step x += alpha p, then stop
        sc->omega = 0.0;
      } else {
        const double om = qy / yy;
        if (om == 0.0 || !isfinite(om)) {
          sc->status = 3;
          sc->done = 1;
        } else {
          sc->omega = om;
        }
      }
    }
  }
};

// Residual r = rhs - (A v) with rhs = b (or D^-1 b, or b with A v scaled by
// d): used for the start residual r_0 = b~ - A~ x_0 (stored to r and r0_hat)
// and for true residuals.  Reduces (r, r) and (rhs, rhs).
template <class XT, class T, class DT, class A>
struct EpiResid {
  static constexpr bool kSkipWhenDone = false;
  const XT* b;
  const DT* dinv;    // non-NULL: rhs = b / d   (Jacobi-scaled system)
  const DT* dmul;    // non-NULL: r = b - d * (A v)   (raw system from A~)
  A dc;              // used when dinv is NULL: rhs = b / dc (1: no scaling)
  A dmc;             // used when dmul is NULL: r = b - dmc * (A v)
  T* r_out;          // may be NULL
  T* rh_out;         // may be NULL
  double* parts;
  int counter;       // which Scalars counter
  int mode;          // 0: start of a solve (sets scalars); 1: stores totals in res[0..1]
  SqAcc<A, 2> acc;
  A bv[8];
  A dv[8];
  __device__ void setup(const Scalars*) { acc.init(); }
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long i, int nv) {
    if (nv <= 0) return;
    A t[VEC];
    load_run<XT, VEC, VL>(b + i, nv, t);
#pragma unroll
    for (int k = 0; k < VEC; ++k) bv[k] = t[k];
    if (dinv || dmul) {
      load_run<DT, VEC, VL>((dinv ? dinv : dmul) + i, nv, t);
#pragma unroll
      for (int k = 0; k < VEC; ++k) dv[k] = t[k];
    }
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&)[VEC]) {
    A rv[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      A rhs = bv[k];
      A av = out[k];
      // unit scales (no Jacobi scaling, or a raw residual) skip the
      // division and multiplication: float64 division is costly here
      if (dinv) rhs = rhs / dv[k];
      else if (dc != A(1)) rhs = rhs / dc;
      if (dmul) av = av * dv[k];
      else if (dmc != A(1)) av = av * dmc;
      const A rk = rhs - av;
      rv[k] = as_stored<T>(rk);
      // a solve's start residual enters the recurrence as stored; a reported
      // residual's norm is that of the unrounded value
      if (k < nv) {
        acc.add_sq(0, mode == 0 ? rv[k] : rk);
        acc.add_sq(1, rhs);
      }
    }
    if (r_out) store_run<T, VEC, VL>(r_out + i, nv, rv);
    if (rh_out) store_run<T, VEC, VL>(rh_out + i, nv, rv);
  }
  __device__ __forceinline__ void step_end(int k) { if ((k & 7) == 7) acc.fold(); }
  __device__ void finish(Scalars* sc, int nblocks, int bid, double* red) {
    acc.fold();
    double v[2] = {acc.tot[0], acc.tot[1]}, tot[2];
    block_sum<2>(v, red);
    if (grid_combine<2>(parts, &sc->counter[counter], nblocks, bid, v, tot, red) && threadIdx.x == 0) {
      sc->res[0] = tot[0];
      sc->res[1] = tot[1];
      if (mode == 0) {
        // start of a solve: r0_hat = r_0, rho_0 = (r0_hat, r_0) = (r_0, r_0)
        const double bn = sqrt(tot[1]);
        sc->bnorm = bn;
        sc->rho = tot[0];
        sc->iter = 0;
        sc->special = 0;
        sc->alpha = sc->omega = sc->beta = 0.0;
        if (bn == 0.0) {
          sc->status = 0;
          sc->done = 1;
          sc->res[2] = 0.0;
        } else {
          const double h0 = sqrt(tot[0]) / bn;
          sc->res[2] = h0;
          if (h0 <= sc->tol) { sc->status = 0; sc->done = 1; }
          else if (sc->maxit <= 0) { sc->status = 4; sc->done = 1; }
          else if (!isfinite(h0)) { sc->status = 3; sc->done = 1; }
          else { sc->done = 0; sc->status = 4; }
        }
      }
    }
  }
};

}  // namespace s7

namespace s7 {

// ---------------------------------------------------------------------------
// Two reductions per step (the merged variant).  (r0, r_{i+1}) follows from
// (r0, r_i) - alpha (r0, s_i) - omega (r0, y_i), so beta_i is known after the
// y pass, and the x, r updates of step i fuse with the p update and SpMV of
// step i+1.  r, p and s are double-buffered by step parity.
// ---------------------------------------------------------------------------

// q_i = r_i - alpha s_i formed on the fly, with r double-buffered.
template <class T, class A>
struct SrcQ2 {
  T* rbuf[2];
  T* sbuf[2];
  const T* r;
  const T* s;
  A alpha;
  __device__ void setup(const Scalars* sc) {
    alpha = (A)sc->alpha;
    const bool odd = (sc->iter & 1) != 0;
    r = odd ? rbuf[1] : rbuf[0];
    s = odd ? sbuf[1] : sbuf[0];
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void produce(long long i, int nv, A (&v)[VEC], bool) {
    A sv[VEC];
    load_run<T, VEC, VL>(r + i, nv, v);
    load_run<T, VEC, VL>(s + i, nv, sv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = q_of<T>(v[k], sv[k], alpha);
  }
  __device__ __forceinline__ A produce1(long long i) {
    return q_of<T>(to_acc<A>(r[i]), to_acc<A>(s[i]), alpha);
  }
};

// Scalars after the q/y pass of the two-reduction variant: omega_i, and
// beta_i from the recurrence (r0, r_{i+1}) = (r0, r_i) - alpha (r0, s_i) -
// omega (r0, y_i); sigma = (r0, s_i) is in res[3].  Last block, thread 0.
__device__ inline void merged_q_finish(Scalars* sc, double qy, double yy, double ry) {
  if (yy == 0.0) {
    sc->special = 1;
    sc->omega = 0.0;
    sc->beta = 0.0;
    sc->rho_next = 0.0;
    return;
  }
  const double om = qy / yy;
  if (om == 0.0 || !isfinite(om)) {
    sc->status = 3;
    sc->done = 1;
    return;
  }
  sc->omega = om;
  const double rn = sc->rho - sc->alpha * sc->res[3] - om * ry;
  sc->rho_next = rn;
  sc->beta = (sc->alpha / om) * (rn / sc->rho);
}

// Scalars after the fused pass: history, stopping test, breakdown on the
// directly reduced (r0, r_{i+1}), which becomes rho for alpha_{i+1}.
__device__ inline void merged_pass_finish(Scalars* sc, double* hist, double sigma, double rr,
                                          double rho_direct) {
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
  } else if (rho_direct == 0.0 || !isfinite(rho_direct) || sigma == 0.0 || !isfinite(sigma)) {
    sc->status = 3;
    sc->done = 1;
  } else {
    sc->rho = rho_direct;
    sc->alpha = rho_direct / sigma;
    sc->res[3] = sigma;
    if (it >= sc->maxit) {
      sc->status = 4;
      sc->done = 1;
    }
  }
}

// y_i = A q_i stored; (q,y), (y,y), (r0,y) reduced; omega_i, rho_{i+1}, beta_i.
template <class T, class A>
struct EpiYMerged {
  static constexpr bool kSkipWhenDone = true;
  T* y_out;
  const T* rh;
  double* parts;
  DotAcc<A, 3> acc;
  A rh_v[8];
  __device__ void setup(const Scalars*) { acc.init(); }
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long i, int nv) {
    if (nv > 0) {
      A t[VEC];
      load_run<T, VEC, VL>(rh + i, nv, t);
#pragma unroll
      for (int k = 0; k < VEC; ++k) rh_v[k] = t[k];
    }
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&q)[VEC]) {
    A yv[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) yv[k] = as_stored<T>(out[k]);
    store_run<T, VEC, VL, true>(y_out + i, nv, yv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      acc.part[0] = fma(q[k], yv[k], acc.part[0]);
      acc.part[1] = fma(yv[k], yv[k], acc.part[1]);
      acc.part[2] = fma(rh_v[k], yv[k], acc.part[2]);
    }
  }
  __device__ __forceinline__ void step_end(int k) { if ((k & 7) == 7) acc.fold(); }
  __device__ void finish(Scalars* sc, int nblocks, int bid, double* red) {
    acc.fold();
    double v[3] = {acc.tot[0], acc.tot[1], acc.tot[2]}, tot[3];
    block_sum<3>(v, red);
    if (grid_combine<3>(parts, &sc->counter[CNT_B], nblocks, bid, v, tot, red) && threadIdx.x == 0)
      merged_q_finish(sc, tot[0], tot[1], tot[2]);
  }
};

// The fused pass: on every cell of the march (own and halo) it forms
// r_{i+1} = (r_i - alpha s_i) - omega y_i and p_{i+1} = r_{i+1} + beta (p_i -
// omega s_i); on the block's own cells it also updates x (x += alpha p_i +
// omega q_i) and stores r_{i+1}, p_{i+1}.  As the epilogue it stores
// s_{i+1} = A p_{i+1} and reduces (r0, s_{i+1}), (r_{i+1}, r_{i+1}) and
// (r0, r_{i+1}): the recurrence value of the latter only predicted beta_i;
// alpha_{i+1} and the next prediction use the reduced one.  One object serves
// as both producer and epilogue (k_sweep1): r_{i+1} of the block's own cells
// waits in a two-plane register ring between the two.
template <class T, class X, class A>
struct MergedPass {
  static constexpr bool kSkipWhenDone = true;
  T* rbuf[2];
  T* pbuf[2];
  T* sbuf[2];
  const T* y;
  const T* rh;
  X* x;
  double* parts;
  double* hist;
  // set up per launch
  const T *r_in, *p_in, *s_in;
  T *r_out, *p_out, *s_out;
  A alpha, omega, beta;
  DotAcc<A, 3> acc;  // (r0, s_{i+1}), (r_{i+1}, r_{i+1}), (r0, r_{i+1})
  A rh_v[8];
  A ring0[8], ring1[8];  // r_{i+1} of own cells, by plane parity
  int pw, pc;
  __device__ void setup(const Scalars* sc) {
    const bool odd = (sc->iter & 1) != 0;
    r_in = odd ? rbuf[1] : rbuf[0];
    r_out = odd ? rbuf[0] : rbuf[1];
    p_in = odd ? pbuf[1] : pbuf[0];
    p_out = odd ? pbuf[0] : pbuf[1];
    s_in = odd ? sbuf[1] : sbuf[0];
    s_out = odd ? sbuf[0] : sbuf[1];
    alpha = (A)sc->alpha;
    omega = (A)sc->omega;
    beta = (A)sc->beta;
    acc.init();
    pw = pc = 0;
  }
  __device__ __forceinline__ void form(A rv, A sv, A yv, A pv, A& q, A& rn, A& pn) const {
    q = q_of<T>(rv, sv, alpha);
    rn = as_stored<T>(fma(-omega, yv, q));
    pn = as_stored<T>(fma(beta, fma(-omega, sv, pv), rn));
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void produce(long long i, int nv, A (&v)[VEC], bool write) {
    static_assert(VEC <= 8, "run too long");
    A rv[VEC], sv[VEC], yv[VEC], pv[VEC];
    load_run<T, VEC, VL>(r_in + i, nv, rv);
    load_run<T, VEC, VL>(s_in + i, nv, sv);
    load_run<T, VEC, VL>(y + i, nv, yv);
    load_run<T, VEC, VL>(p_in + i, nv, pv);
    A rn[VEC], q[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) form(rv[k], sv[k], yv[k], pv[k], q[k], rn[k], v[k]);
    if (write) {
      A xv[VEC];
      load_run<X, VEC, VL>(x + i, nv, xv);
#pragma unroll
      for (int k = 0; k < VEC; ++k) xv[k] = fma(omega, q[k], fma(alpha, pv[k], xv[k]));
      store_run<X, VEC, VL, true>(x + i, nv, xv);
      store_run<T, VEC, VL, true>(r_out + i, nv, rn);
      store_run<T, VEC, VL, true>(p_out + i, nv, v);
      if (pw) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) ring1[k] = (k < nv) ? rn[k] : A(0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) ring0[k] = (k < nv) ? rn[k] : A(0);
      }
      pw ^= 1;
    }
  }
  __device__ __forceinline__ A produce1(long long i) {
    A q, rn, pn;
    form(to_acc<A>(r_in[i]), to_acc<A>(s_in[i]), to_acc<A>(y[i]), to_acc<A>(p_in[i]), q, rn, pn);
    return pn;
  }
  template <int VEC, bool VL> __device__ __forceinline__ void load(long long i, int nv) {
    if (nv > 0) {
      A t[VEC];
      load_run<T, VEC, VL>(rh + i, nv, t);
#pragma unroll
      for (int k = 0; k < VEC; ++k) rh_v[k] = t[k];
    }
  }
  template <int VEC, bool VL>
  __device__ __forceinline__ void consume(long long i, int nv, const A (&out)[VEC], const A (&)[VEC]) {
    A sv[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) sv[k] = as_stored<T>(out[k]);
    store_run<T, VEC, VL, true>(s_out + i, nv, sv);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const A rn = pc ? ring1[k] : ring0[k];
      acc.part[0] = fma(rh_v[k], sv[k], acc.part[0]);
      acc.part[1] = fma(rn, rn, acc.part[1]);
      acc.part[2] = fma(rh_v[k], rn, acc.part[2]);
    }
    pc ^= 1;
  }
  __device__ __forceinline__ void step_end(int k) { if ((k & 7) == 7) acc.fold(); }
  __device__ void finish(Scalars* sc, int nblocks, int bid, double* red) {
    acc.fold();
    double v[3] = {acc.tot[0], acc.tot[1], acc.tot[2]}, tot[3];
    block_sum<3>(v, red);
    if (grid_combine<3>(parts, &sc->counter[CNT_C], nblocks, bid, v, tot, red) && threadIdx.x == 0)
      merged_pass_finish(sc, hist, tot[0], tot[1], tot[2]);
  }
};

}  // namespace s7
