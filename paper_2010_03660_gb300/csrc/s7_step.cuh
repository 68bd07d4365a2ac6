// Pipelined step sweeps: the two SpMV kernels of a BiCGStab step with their
// inputs staged through shared memory by asynchronous copies.
//
// Same arithmetic and the same z march as k_sweep (s7_sweep.cuh), but every
// global read of plane z+1 (the six coefficient tiles, r0_hat, and the
// inputs of the on-the-fly vector with a one-cell halo ring) is issued with
// cp.async into a STAGES-deep ring of shared-memory stages while plane z is
// computed.  No register holds an in-flight load, so a block keeps whole
// planes of loads in flight at modest register use.
//
// Stage k (for output plane z = z0 + k) holds: coef(z), r0_hat(z) and the
// inputs at plane z+1 (rows y0-1 .. y0+by, each the aligned span
// [x0-VEC, x0+bx*VEC+VEC), so the x halo cells come from the neighbouring
// 16-byte vectors), and for the fused pass of the two-reduction variant the
// iterate x of the block's own cells at plane z+1.  Cells outside the mesh
// are zero-filled by the copy.
//
// Kinds: 0 = p update + s = A p + (r0,s); 1 = q + y = A q + (q,y),(y,y);
// two-reduction variant: 2 = q + y = A q + (q,y),(y,y),(r0,y); 3 = the fused
// pass (x, r updates of step i, p_{i+1}, s_{i+1} = A p_{i+1}, (r0,s),
// (r,r), (r0,r)).  Kinds 2 and 3 compute exactly what the register sweeps
// with SrcQ2/EpiYMerged and MergedPass compute, in the same order.
//
// Barriers: one per plane.  At step k a thread waits for its own copies of
// stage k, then __syncthreads() makes all of stage k and the vector plane z
// (produced at step k-1) visible; it then refills the stage buffer that
// held stage k-1 (fully consumed before the barrier), forms plane z+1 into
// one buffer of a 2-buffer vector ring, and computes plane z from the other
// (written at step k-1).  Two buffers suffice because plane z+1 is written
// after the barrier: the buffer it overwrites held plane z-1, which every
// thread finished reading at step k-1 (the plane z-1 values a thread keeps
// for its own cells live in registers).
//
// Staging engine.  With tensor maps of the handle's arrays (StepArgs::maps,
// a kernel parameter of the single-system sweeps), the first warp stages
// each plane with TMA tensor copies (cp.async.bulk.tensor, one box per
// lane: the six coefficient tiles, r0_hat, the inputs with their halo, the
// iterate tile), completing on a per-stage mbarrier; boxes reaching past
// the mesh are zero-filled by the copy engine.  Otherwise every thread
// issues cp.async copies of its own vectors and halo.  Both fill the same
// shared-memory layout with the same values, so the two give identical
// results; TMA takes the per-thread address, predicate and copy
// instructions off the critical path.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "s7_sweep.cuh"

namespace s7 {

// Tensor maps of one handle's arrays for one tile shape (a kernel
// parameter): coefficient and r0_hat tiles (box TW x by x 1), the
// SpMV inputs with a one-cell halo ring (box (TW + 2 VEC) x (by + 2) x 1,
// started one vector left of and one row below the tile), the iterate tile.
enum { MAP_R = 0, MAP_R2, MAP_P0, MAP_P1, MAP_S0, MAP_S1, MAP_Y, MAP_NIN };
struct StepMaps {
  CUtensorMap c[6];
  CUtensorMap rh;
  CUtensorMap in[MAP_NIN];
  CUtensorMap x;
};

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the mbarrier, at most about two seconds of SM
// clock; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 32)) return false;
  return true;
}
// Order this thread's earlier shared-memory accesses before later
// asynchronous-proxy (TMA) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// 3D tile load of the box at (x, y, z) of `map` into shared memory at `dst`
// (128-byte aligned), completing on the mbarrier `bar`.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Asynchronous global->shared copy of B bytes (16, 8 or 4); `bytes` = B
// copies, 0 zero-fills.  16-byte copies bypass L1 (.cg); smaller ones must
// use .ca.
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes) {
  if (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
  else if (B == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}


// Pointers of one pipelined sweep.  KIND 0: p_i = r + beta (p_{i-1} - omega
// s_{i-1}) formed on the fly, s_i = A p_i, (r0,s_i).  KIND 1: q = r - alpha s
// formed on the fly, y = A q, (q,y), (y,y).  Kinds 2 and 3 read r from rbuf
// by step parity; kind 3 also updates x and writes the history.
template <class T>
struct StepArgs {
  const T* c[6];
  const T* r;
  const T* rh;
  T* pbuf[2];
  T* sbuf[2];
  T* y;
  double* parts;
  T* rbuf[2];
  void* x;
  double* hist;
  const StepMaps* maps;   // tensor maps for this tile shape (kernel parameter space), or
                          // NULL: cp.async staging
};

// The iterate's type for storage type T (float64 for float64 storage).
template <class T> struct IterOf { typedef float t; };
template <> struct IterOf<double> { typedef double t; };

// Staged arrays per kind: inputs with halo, r0_hat tile, x tile.
template <int KIND> struct KindShape {
  static constexpr int nin = KIND == 0 ? 3 : (KIND == 3 ? 4 : 2);
  static constexpr bool rh = KIND != 1;
  static constexpr bool x = KIND == 3;
};

// The register-form producer of each kind: it forms the two planes before
// the pipeline starts (and, for the block's own cells of its first plane,
// writes what that kind writes).
template <int KIND, class T, class X, class A> struct KindSrc;
template <class T, class X, class A> struct KindSrc<0, T, X, A> { typedef SrcPUpdate<T, A> type; };
template <class T, class X, class A> struct KindSrc<1, T, X, A> { typedef SrcQ<T, A> type; };
template <class T, class X, class A> struct KindSrc<2, T, X, A> { typedef SrcQ2<T, A> type; };
template <class T, class X, class A> struct KindSrc<3, T, X, A> { typedef MergedPass<T, X, A> type; };

template <class T, class X, class A>
__device__ __forceinline__ void init_src(SrcPUpdate<T, A>& p, const StepArgs<T>& a, X*) {
  p.r = a.r;
  p.pbuf[0] = a.pbuf[0];
  p.pbuf[1] = a.pbuf[1];
  p.sbuf[0] = a.sbuf[0];
  p.sbuf[1] = a.sbuf[1];
}
template <class T, class X, class A>
__device__ __forceinline__ void init_src(SrcQ<T, A>& p, const StepArgs<T>& a, X*) {
  p.r = a.r;
  p.sbuf[0] = a.sbuf[0];
  p.sbuf[1] = a.sbuf[1];
}
template <class T, class X, class A>
__device__ __forceinline__ void init_src(SrcQ2<T, A>& p, const StepArgs<T>& a, X*) {
  p.rbuf[0] = a.rbuf[0];
  p.rbuf[1] = a.rbuf[1];
  p.sbuf[0] = a.sbuf[0];
  p.sbuf[1] = a.sbuf[1];
}
template <class T, class X, class A>
__device__ __forceinline__ void init_src(MergedPass<T, X, A>& p, const StepArgs<T>& a, X* x) {
  for (int k = 0; k < 2; ++k) {
    p.rbuf[k] = a.rbuf[k];
    p.pbuf[k] = a.pbuf[k];
    p.sbuf[k] = a.sbuf[k];
  }
  p.y = a.y;
  p.rh = a.rh;
  p.x = x;
  p.parts = a.parts;
  p.hist = a.hist;
}

// Every staged array of a stage starts on a 128-byte boundary (the
// alignment of a TMA destination), so it is one dense box of a tensor copy.
__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) / 128 * 128; }

template <class T, int VEC>
struct StepLayout {
  int TW, W, rows;     // tile width (elements), padded row pitch, rows incl. halo
  int cs;              // elements from one coefficient tile to the next (r0_hat: one more)
  int PL;              // elements from one staged input plane to the next
  int coef_sz, rh_sz, in_sz, stage_sz;  // in elements of T
};

template <class T, int VEC>
__host__ __device__ inline StepLayout<T, VEC> step_layout(int bx, int by, int nin, bool rh) {
  StepLayout<T, VEC> L;
  L.TW = bx * VEC;
  L.W = L.TW + 2 * VEC;
  L.rows = by + 2;
  L.cs = (int)(round128((size_t)by * L.TW * sizeof(T)) / sizeof(T));
  L.PL = (int)(round128((size_t)L.rows * L.W * sizeof(T)) / sizeof(T));
  L.coef_sz = 6 * L.cs;
  L.rh_sz = rh ? L.cs : 0;
  L.in_sz = nin * L.PL;
  L.stage_sz = L.coef_sz + L.rh_sz + L.in_sz;
  return L;
}

// Bytes of the staged T arrays of one stage (a multiple of 128, so the
// iterate tile after them, the next stage and the ring after the stages
// stay 128-byte aligned).
template <class T, int VEC>
__host__ __device__ inline size_t stage_stride_bytes(const StepLayout<T, VEC>& L) {
  return round128((size_t)L.stage_sz * sizeof(T));
}

// Bytes of one stage of kind KIND: the T arrays, then (kind 3) the tile of
// the iterate x.
template <class T, int VEC, int KIND>
__host__ __device__ inline size_t kind_stride_bytes(const StepLayout<T, VEC>& L) {
  if (!KindShape<KIND>::x) return stage_stride_bytes(L);
  return stage_stride_bytes(L) +
         round128(sizeof(typename IterOf<T>::t) * L.TW * (size_t)(L.rows - 2));
}

template <class T, int VEC, int KIND>
__host__ __device__ inline StepLayout<T, VEC> kind_layout(int bx, int by) {
  return step_layout<T, VEC>(bx, by, KindShape<KIND>::nin, KindShape<KIND>::rh);
}

// Element type of the ring of the on-the-fly vector (p or q): the storage
// type, which holds it exactly (both are rounded to storage when formed),
// in half the bytes of the arithmetic type for 16-bit storage.
template <class T, class A, int KIND> struct RingOf {
  typedef T t;
};

// Dynamic shared memory of a block: the stages, the 2-plane ring of the
// on-the-fly vector, and 128 bytes to align the start.
template <class T, class A, int VEC, int KIND>
__host__ __device__ inline size_t kind_smem_bytes(int bx, int by, int stages) {
  const StepLayout<T, VEC> L = kind_layout<T, VEC, KIND>(bx, by);
  const size_t ring = (size_t)2 * L.rows * L.W * sizeof(typename RingOf<T, A, KIND>::t);
  return (size_t)stages * kind_stride_bytes<T, VEC, KIND>(L) + ring + 128;
}

template <class T, class A, int VEC>
__host__ __device__ inline size_t step_smem_bytes(int bx, int by, int stages, int kind) {
  switch (kind) {
    case 0: return kind_smem_bytes<T, A, VEC, 0>(bx, by, stages);
    case 1: return kind_smem_bytes<T, A, VEC, 1>(bx, by, stages);
    case 2: return kind_smem_bytes<T, A, VEC, 2>(bx, by, stages);
    default: return kind_smem_bytes<T, A, VEC, 3>(bx, by, stages);
  }
}

// Block `bid` of the `nblocks` blocks of one pipelined sweep over the mesh
// `g` (s7_smem: the dynamic shared memory; red: 128 doubles of reduction
// scratch; bars: STAGES mbarriers for the TMA staging).  The caller has
// checked the stop flag.
template <class T, class A, int VEC, int KIND, int STAGES>
__device__ __forceinline__ void step_body(const Geom& g, const StepArgs<T>& a, Scalars* sc,
                                          int bid, int nb_total, unsigned char* s7_smem,
                                          double* red, unsigned long long* bars) {
  typedef typename IterOf<T>::t X;
  const int it = sc->iter;
  const bool odd = (it & 1) != 0;
  const bool first = (KIND == 0) && it == 0;
  const A beta = (A)sc->beta, omega = (A)sc->omega, alpha = (A)sc->alpha;
  // inputs of the on-the-fly vector
  const T* in0 = KIND >= 2 ? (odd ? a.rbuf[1] : a.rbuf[0]) : a.r;
  const T* in1 = (KIND == 0) ? (odd ? a.pbuf[0] : a.pbuf[1]) : (odd ? a.sbuf[1] : a.sbuf[0]);
  const T* in2 = (KIND == 0) ? (odd ? a.sbuf[0] : a.sbuf[1]) : (KIND == 3 ? a.y : nullptr);
  const T* in3 = (KIND == 3) ? (odd ? a.pbuf[1] : a.pbuf[0]) : nullptr;
  const int nin = (KIND == 0) ? (first ? 1 : 3) : KindShape<KIND>::nin;
  // kind 0 writes p_i; kind 3 writes p_{i+1}, r_{i+1} (the other parity)
  T* p_out = (KIND == 3) ? (odd ? a.pbuf[0] : a.pbuf[1]) : (odd ? a.pbuf[1] : a.pbuf[0]);
  T* r_out = odd ? a.rbuf[0] : a.rbuf[1];
  X* xg = reinterpret_cast<X*>(a.x);
  T* out = (KIND == 0) ? (odd ? a.sbuf[1] : a.sbuf[0])
         : (KIND == 3) ? (odd ? a.sbuf[0] : a.sbuf[1]) : a.y;

  const StepLayout<T, VEC> L = kind_layout<T, VEC, KIND>(g.bx, g.by);
  const size_t sstride = kind_stride_bytes<T, VEC, KIND>(L);
  // the stages start on a 128-byte boundary (the dynamic area has 128 bytes to spare)
  unsigned char* sm = s7_smem + ((128u - (smem_u32(s7_smem) & 127u)) & 127u);
  auto stage_buf = [&](int k) { return reinterpret_cast<T*>(sm + (size_t)k * sstride); };
  typedef typename RingOf<T, A, KIND>::t R;
  R* ring = reinterpret_cast<R*>(sm + (size_t)STAGES * sstride);
  const int PL = L.PL;              // staged input planes
  const int RPL = L.rows * L.W;     // ring planes

  const int t = threadIdx.x;
  const bool has_cell = t < g.bx * g.by;
  const int tx = has_cell ? t % g.bx : 0;
  const int ty = has_cell ? t / g.bx : 0;
  const int tile_x = bid % g.tiles_x;
  const int rest = bid / g.tiles_x;
  const int tile_y = rest % g.tiles_y;
  const int chunk = rest / g.tiles_y;
  const int x0 = tile_x * L.TW;
  const int y0 = tile_y * g.by;
  const int z0 = chunk * g.zchunk;
  const int z1 = min(z0 + g.zchunk, g.nz);
  const int x = x0 + tx * VEC;
  const int y = y0 + ty;
  const bool own = has_cell && y < g.ny && x < g.nx;   // full vector (nx % VEC == 0)
  const long long row = (long long)y * g.nx + x;
  const int so = (ty + 1) * L.W + VEC + tx * VEC;     // own element 0 in an input/ring plane
  const int sc_own = ty * L.TW + tx * VEC;            // own element 0 in a coef/rh tile

  // ---- asynchronous copy of stage `k` (output plane z0+k) into buffer `buf`.
  // Each thread copies its own 16-byte vectors; threads on the tile edge also
  // copy the halo vector beside them.  Every staged value a thread later
  // reads is one it copied itself (the barrier orders buffer reuse).
  const bool v_top = has_cell && ty == 0 && y0 > 0 && x < g.nx;
  const bool v_bot = has_cell && ty == g.by - 1 && y + 1 < g.ny && x < g.nx;
  const bool v_lft = has_cell && tx == 0 && x0 > 0 && y < g.ny;
  const bool v_rgt = has_cell && tx == g.bx - 1 && x + VEC < g.nx && y < g.ny;
  constexpr int VB = VEC * (int)sizeof(T);   // bytes per vector copy
  auto issue_stage = [&](int k, T* buf) {
    if (!has_cell) return;
    const int z = z0 + k;
    const long long gi = own ? (long long)z * g.plane + row : 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) cp_async<VB>(buf + d * L.cs + sc_own, a.c[d] + gi, own ? VB : 0);
    if constexpr (KindShape<KIND>::rh) cp_async<VB>(buf + L.coef_sz + sc_own, a.rh + gi, own ? VB : 0);
    const int zi = z + 1;
    if (zi >= g.nz) return;
    const long long gb = (long long)zi * g.plane + row;
    if constexpr (KindShape<KIND>::x) {
      X* xb = reinterpret_cast<X*>(reinterpret_cast<unsigned char*>(buf) +
                                   stage_stride_bytes(L)) + sc_own;
      constexpr int XB = VEC * (int)sizeof(X);
      constexpr int XC = XB > 16 ? 16 : XB;      // bytes per copy
      constexpr int XE = XC / (int)sizeof(X);    // elements per copy
#pragma unroll
      for (int c = 0; c < XB / XC; ++c)
        cp_async<XC>(xb + c * XE, xg + (own ? gb + c * XE : 0), own ? XC : 0);
    }
    T* ib = buf + L.coef_sz + L.rh_sz + so;
    for (int sidx = 0; sidx < nin; ++sidx) {
      const T* base =
          sidx == 0 ? in0 : (sidx == 1 ? in1 : ((KIND == 3 && sidx == 3) ? in3 : in2));
      T* d = ib + sidx * PL;
      cp_async<VB>(d, base + (own ? gb : 0), own ? VB : 0);
      if (ty == 0) cp_async<VB>(d - L.W, base + (v_top ? gb - g.nx : 0), v_top ? VB : 0);
      if (ty == g.by - 1) cp_async<VB>(d + L.W, base + (v_bot ? gb + g.nx : 0), v_bot ? VB : 0);
      if (tx == 0) cp_async<VB>(d - VEC, base + (v_lft ? gb - VEC : 0), v_lft ? VB : 0);
      if (tx == g.bx - 1) cp_async<VB>(d + VEC, base + (v_rgt ? gb + VEC : 0), v_rgt ? VB : 0);
    }
  };

  // ---- the same stage as TMA tensor copies, issued by the first warp, one
  // box per lane: every array of the stage is one box at the tile's origin
  // (inputs: one vector left and one row below it, with the halo ring);
  // lane 0 first sets the buffer's mbarrier to expect the bytes of every
  // box, cells past the mesh included (the copy engine fills them with
  // zeros).
  const StepMaps* maps = a.maps;
  const int m_in0 = KIND >= 2 ? (odd ? MAP_R2 : MAP_R) : MAP_R;
  const int m_in1 = (KIND == 0) ? (odd ? MAP_P0 : MAP_P1) : (odd ? MAP_S1 : MAP_S0);
  const int m_in2 = (KIND == 0) ? (odd ? MAP_S0 : MAP_S1) : MAP_Y;
  const int m_in3 = odd ? MAP_P1 : MAP_P0;
  constexpr int NT = 6 + (KindShape<KIND>::rh ? 1 : 0);   // tile boxes of a plane
  auto issue_stage_tma = [&](int k, T* buf) {   // called by the 32 lanes of warp 0
    const int lane = t & 31;
    const int z = z0 + k;
    const int zi = z + 1;
    const unsigned bar = smem_u32(bars + (k % STAGES));
    const unsigned tile_b = (unsigned)(L.TW * g.by * sizeof(T));
    const unsigned in_b = (unsigned)(L.W * L.rows * sizeof(T));
    const int nxb = (zi < g.nz && KindShape<KIND>::x) ? 1 : 0;   // iterate tile box
    const int nib = zi < g.nz ? nin : 0;                           // input boxes
    if (lane == 0)
      mbar_expect_tx(bar, NT * tile_b + nib * in_b + nxb * (unsigned)(L.TW * g.by * sizeof(X)));
    __syncwarp();
    const unsigned b0 = smem_u32(buf);
    if (lane < 6) {
      tma_load_3d(b0 + (unsigned)(lane * L.cs * sizeof(T)), &maps->c[lane], x0, y0, z, bar);
    } else if (KindShape<KIND>::rh && lane == 6) {
      tma_load_3d(b0 + (unsigned)(L.coef_sz * sizeof(T)), &maps->rh, x0, y0, z, bar);
    } else if (lane == NT && nxb) {
      tma_load_3d(b0 + (unsigned)stage_stride_bytes(L), &maps->x, x0, y0, zi, bar);
    } else if (lane >= NT + nxb && lane < NT + nxb + nib) {
      const int sidx = lane - NT - nxb;
      const int m = sidx == 0 ? m_in0 : (sidx == 1 ? m_in1 : ((KIND == 3 && sidx == 3) ? m_in3 : m_in2));
      tma_load_3d(b0 + (unsigned)((L.coef_sz + L.rh_sz + sidx * PL) * sizeof(T)), &maps->in[m],
                  x0 - VEC, y0 - 1, zi, bar);
    }
  };
  // A wait that gave up (about two seconds) marks the solve timed out
  // (status 5, S7_ETIMEOUT) and stops waiting: every thread still reaches
  // every barrier, the block ends, and the host reads the status.
  __shared__ int s_timed_out;
  // The mbarriers of the stage buffers: one arrival (the issuing thread's,
  // with the byte count) per phase.
  if (maps) {
    if (t == 0) {
      s_timed_out = 0;
      for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(bars + k), 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  auto wait_stage = [&](int k) {
    if (maps) {
      if (!*((volatile int*)&s_timed_out) &&
          !mbar_wait_bounded(smem_u32(bars + (k % STAGES)), (unsigned)((k / STAGES) & 1))) {
        s_timed_out = 1;
        sc->status = 5;
        sc->done = 1;
      }
    } else {
      cp_async_wait<STAGES - 2>();
    }
  };

  // p_{i+1} of the fused pass from r_i, s_i, y_i, p_i (as MergedPass forms it)
  auto form_merged = [&](A rv, A sv, A yv, A pv, A& q, A& rn) -> A {
    q = q_of<T>(rv, sv, alpha);
    rn = as_stored<T>(fma(-omega, yv, q));
    return as_stored<T>(fma(beta, fma(-omega, sv, pv), rn));
  };
  // value of the on-the-fly vector from staged inputs (index e in a plane)
  auto form = [&](const T* inb, int e) -> A {
    const A rv = to_acc<A>(inb[e]);
    if constexpr (KIND == 1 || KIND == 2) return q_of<T>(rv, to_acc<A>(inb[PL + e]), alpha);
    if constexpr (KIND == 3) {
      A q, rn;
      return form_merged(rv, to_acc<A>(inb[PL + e]), to_acc<A>(inb[2 * PL + e]),
                         to_acc<A>(inb[3 * PL + e]), q, rn);
    }
    if (first) return rv;
    return as_stored<T>(fma(beta, fma(-omega, to_acc<A>(inb[2 * PL + e]), to_acc<A>(inb[PL + e])), rv));
  };
  // the same for a run of VEC cells starting at e (one vector load per input)
  auto form_run = [&](const T* inb, int e, A (&v)[VEC]) {
    ldv<T, VEC>(inb + e, v);
    if constexpr (KIND == 1 || KIND == 2) {
      A sv[VEC];
      ldv<T, VEC>(inb + PL + e, sv);
#pragma unroll
      for (int j = 0; j < VEC; ++j) v[j] = q_of<T>(v[j], sv[j], alpha);
    } else if constexpr (KIND == 3) {
      A sv[VEC], yv[VEC], pv[VEC];
      ldv<T, VEC>(inb + PL + e, sv);
      ldv<T, VEC>(inb + 2 * PL + e, yv);
      ldv<T, VEC>(inb + 3 * PL + e, pv);
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        A q, rn;
        v[j] = form_merged(v[j], sv[j], yv[j], pv[j], q, rn);
      }
    } else if (!first) {
      A pv[VEC], sv[VEC];
      ldv<T, VEC>(inb + PL + e, pv);
      ldv<T, VEC>(inb + 2 * PL + e, sv);
#pragma unroll
      for (int j = 0; j < VEC; ++j) v[j] = as_stored<T>(fma(beta, fma(-omega, sv[j], pv[j]), v[j]));
    }
  };

  // prologue: the vector at z0-1 (own) and z0 (own + ring) from global memory,
  // then the first STAGES-1 stages in flight
  A vm[VEC], vc[VEC], vp[VEC];
  A rn_c[VEC], rn_p[VEC];   // kind 3: r_{i+1} of own cells at planes z, z+1
  zero(rn_c);
  zero(rn_p);
  {
    typename KindSrc<KIND, T, X, A>::type src;
    init_src(src, a, xg);
    src.setup(sc);
    auto prod = [&](long long i, int nv, A (&v)[VEC], bool write) {
      src.template produce<VEC, true>(i, nv, v, write);
    };
    auto prod1 = [&](long long i) -> A { return src.produce1(i); };
    if (z0 > 0 && own) prod((long long)(z0 - 1) * g.plane + row, VEC, vm, false);
    else zero(vm);
    R* rb = ring;
    if (has_cell) {
      const long long base = (long long)z0 * g.plane + row;
      if (own) {
        prod(base, VEC, vc, true);
        // the fused pass keeps r_{i+1} of its own cells for the epilogue
        if constexpr (KIND == 3) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) rn_c[j] = src.ring0[j];
        }
      } else {
        zero(vc);
      }
      stv<R, VEC>(rb + so, vc);
      if (ty == 0) {
        A h[VEC];
        if (y0 > 0 && x < g.nx) prod(base - g.nx, VEC, h, false);
        else zero(h);
        stv<R, VEC>(rb + so - L.W, h);
      }
      if (ty == g.by - 1) {
        A h[VEC];
        if (y + 1 < g.ny && x < g.nx) prod(base + g.nx, VEC, h, false);
        else zero(h);
        stv<R, VEC>(rb + so + L.W, h);
      }
      if (tx == 0) rb[so - 1] = from_acc<R>((x0 > 0 && y < g.ny) ? prod1(base - 1) : A(0));
      if (tx == g.bx - 1)
        rb[so + VEC] = from_acc<R>((x + VEC < g.nx && y < g.ny) ? prod1(base + VEC) : A(0));
    } else {
      zero(vc);
    }
  }
  const int nsteps = z1 - z0;
  if (maps) {
    if (t < 32)
      for (int k = 0; k < STAGES - 1 && k < nsteps; ++k) issue_stage_tma(k, stage_buf(k));
  } else {
#pragma unroll
    for (int k = 0; k < STAGES - 1; ++k) {
      if (k < nsteps) issue_stage(k, stage_buf(k));
      cp_async_commit();
    }
  }

  DotAcc<A, (KIND >= 2 ? 3 : 2)> acc;
  constexpr int I2 = KIND >= 2 ? 2 : 1;   // third sum (kinds 2, 3 only)
  acc.init();
  for (int k = 0; k < nsteps; ++k) {
    const int z = z0 + k;
    wait_stage(k);
    __syncthreads();
    // refill the buffer of stage k-1 with stage k+STAGES-1
    {
      const int kn = k + STAGES - 1;
      if (maps) {
        if (t < 32 && kn < nsteps) {
          fence_proxy_async_smem();   // this block's reads of the buffer came first
          issue_stage_tma(kn, stage_buf(kn % STAGES));
        }
      } else {
        if (kn < nsteps) issue_stage(kn, stage_buf(kn % STAGES));
        cp_async_commit();
      }
    }
    const T* st = stage_buf(k % STAGES);
    const T* inb = st + L.coef_sz + L.rh_sz;
    // form plane z+1: own cells (+ ring if the next step needs it)
    R* nb = ring + ((k + 1) & 1) * RPL;
    if (z + 1 < g.nz) {
      const bool ring_needed = z + 1 < z1;
      if (has_cell) {
        bool formed = false;
        if constexpr (KIND == 3) {
          if (own && ring_needed) {
            // own cells of plane z+1: x and r updates of step i, p_{i+1}
            A rv[VEC], sv[VEC], yv[VEC], pv[VEC], xv[VEC], q[VEC];
            ldv<T, VEC>(inb + so, rv);
            ldv<T, VEC>(inb + PL + so, sv);
            ldv<T, VEC>(inb + 2 * PL + so, yv);
            ldv<T, VEC>(inb + 3 * PL + so, pv);
            ldv<X, VEC>(reinterpret_cast<const X*>(reinterpret_cast<const unsigned char*>(st) +
                                                   stage_stride_bytes(L)) + sc_own, xv);
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
              vp[j] = form_merged(rv[j], sv[j], yv[j], pv[j], q[j], rn_p[j]);
              xv[j] = fma(omega, q[j], fma(alpha, pv[j], xv[j]));
            }
            const long long gz = (long long)(z + 1) * g.plane + row;
            store_run<X, VEC, true, true>(xg + gz, VEC, xv);
            store_run<T, VEC, true, true>(r_out + gz, VEC, rn_p);
            store_run<T, VEC, true, true>(p_out + gz, VEC, vp);
            formed = true;
          }
        }
        if (!formed) {
          if (own) form_run(inb, so, vp);
          else zero(vp);
        }
        if (ring_needed) {
          stv<R, VEC>(nb + so, vp);
          if (KIND == 0 && own) store_run<T, VEC, true, true>(p_out + (long long)(z + 1) * g.plane + row, VEC, vp);
          if (ty == 0) {
            A h[VEC];
            form_run(inb, so - L.W, h);
            stv<R, VEC>(nb + so - L.W, h);
          }
          if (ty == g.by - 1) {
            A h[VEC];
            form_run(inb, so + L.W, h);
            stv<R, VEC>(nb + so + L.W, h);
          }
          if (tx == 0) nb[so - 1] = from_acc<R>(form(inb, so - 1));
          if (tx == g.bx - 1) nb[so + VEC] = from_acc<R>(form(inb, so + VEC));
        }
      }
    } else {
      zero(vp);
    }
    // stencil on plane z
    if (own) {
      const R* cb = ring + (k & 1) * RPL;
      A up[VEC], dn[VEC], c[6][VEC];
      ldv<R, VEC>(cb + so - L.W, up);
      ldv<R, VEC>(cb + so + L.W, dn);
      const A lf = to_acc<A>(cb[so - 1]);
      const A rt = to_acc<A>(cb[so + VEC]);
#pragma unroll
      for (int d = 0; d < 6; ++d) ldv<T, VEC>(st + d * L.cs + sc_own, c[d]);
      A o[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const A l = (j == 0) ? lf : vc[j - 1];
        const A r = (j == VEC - 1) ? rt : vc[j + 1];
        A s = vc[j];
        s = fma(c[0][j], l, s);
        s = fma(c[1][j], r, s);
        s = fma(c[2][j], up[j], s);
        s = fma(c[3][j], dn[j], s);
        s = fma(c[4][j], vm[j], s);
        s = fma(c[5][j], vp[j], s);
        o[j] = as_stored<T>(s);
      }
      store_run<T, VEC, true, true>(out + (long long)z * g.plane + row, VEC, o);
      if constexpr (KIND == 0) {
        A hv[VEC];
        ldv<T, VEC>(st + L.coef_sz + sc_own, hv);
#pragma unroll
        for (int j = 0; j < VEC; ++j) acc.part[0] = fma(hv[j], o[j], acc.part[0]);
      } else if constexpr (KIND == 1) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          acc.part[0] = fma(vc[j], o[j], acc.part[0]);
          acc.part[1] = fma(o[j], o[j], acc.part[1]);
        }
      } else if constexpr (KIND == 2) {
        A hv[VEC];
        ldv<T, VEC>(st + L.coef_sz + sc_own, hv);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          acc.part[0] = fma(vc[j], o[j], acc.part[0]);
          acc.part[1] = fma(o[j], o[j], acc.part[1]);
          acc.part[I2] = fma(hv[j], o[j], acc.part[I2]);
        }
      } else {
        A hv[VEC];
        ldv<T, VEC>(st + L.coef_sz + sc_own, hv);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          acc.part[0] = fma(hv[j], o[j], acc.part[0]);
          acc.part[1] = fma(rn_c[j], rn_c[j], acc.part[1]);
          acc.part[I2] = fma(hv[j], rn_c[j], acc.part[I2]);
        }
      }
    }
    if ((k & 7) == 7) acc.fold();
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      vm[j] = vc[j];
      vc[j] = vp[j];
      if constexpr (KIND == 3) rn_c[j] = rn_p[j];
    }
  }
  if (!maps) cp_async_wait<0>();
  acc.fold();
  if constexpr (KIND >= 2) {
    double v[3] = {acc.tot[0], acc.tot[1], acc.tot[I2]}, tot[3];
    block_sum<3>(v, red);
    if (grid_combine<3>(a.parts, &sc->counter[KIND == 2 ? CNT_B : CNT_C], nb_total, bid, v, tot,
                        red) && t == 0) {
      if (KIND == 2) merged_q_finish(sc, tot[0], tot[1], tot[2]);
      else merged_pass_finish(sc, a.hist, tot[0], tot[1], tot[2]);
    }
  } else if constexpr (KIND == 0) {
    double v[1] = {acc.tot[0]}, tot[1];
    block_sum<1>(v, red);
    if (grid_combine<1>(a.parts, &sc->counter[CNT_A], nb_total, bid, v, tot, red) && t == 0) {
      const double sigma = tot[0];
      if (sigma == 0.0 || !isfinite(sigma) || !isfinite(sc->rho)) {
        sc->status = 3;
        sc->done = 1;
      } else {
        sc->alpha = sc->rho / sigma;
        sc->res[3] = sigma;
      }
    }
  } else {
    double v[2] = {acc.tot[0], acc.tot[1]}, tot[2];
    block_sum<2>(v, red);
    if (grid_combine<2>(a.parts, &sc->counter[CNT_B], nb_total, bid, v, tot, red) && t == 0) {
      const double qy = tot[0], yy = tot[1];
      if (yy == 0.0) {
        sc->special = 1;
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
}

// maps: the tensor maps of the tile (used when use_maps is 1), passed by
// value so they sit in kernel parameter space.
template <class T, class A, int VEC, int KIND, int STAGES>
__global__ void __launch_bounds__(256) k_step(Geom g, StepArgs<T> a, Scalars* sc,
                                              const __grid_constant__ StepMaps maps,
                                              int use_maps) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  if (*((volatile int*)&sc->done)) return;
  a.maps = use_maps ? &maps : nullptr;
  step_body<T, A, VEC, KIND, STAGES>(g, a, sc, blockIdx.x, s7_nblocks(g), s7_smem, red, bars);
}

}  // namespace s7
