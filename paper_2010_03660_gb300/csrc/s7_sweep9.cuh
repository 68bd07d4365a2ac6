// The y-marching 9-point stencil sweep on a 2D mesh (Sec. IV-A, "SpMV (2D)").
//
// The paper keeps a rectangular sub-block of the 2D mesh per core and adds
// the products of the block's columns into an output halo exchanged with
// the neighbouring cores, one direction at a time.  The GB300 analogue reads
// instead of scatters: a thread block owns a strip of bx*VEC columns and a
// chunk of rows, and marches along y.  Each thread owns VEC consecutive x
// cells of the current row and keeps the input vector at rows y-1, y, y+1 for
// them in registers, so the ym/yp terms and the inner parts of the four
// diagonal terms cost no extra traffic.  Only the values one cell left and
// right of each thread's run cross thread boundaries; each thread publishes
// its run of row y+1 in a shared-memory row ring, and after the row's
// barrier reads the two values beside it.  The x halo of row y-1 is carried
// in registers from the previous step, so every step reads only the ring
// buffers of rows y and y+1, and three buffers with one barrier per row are
// race free: step k writes buffer (k+1)%3, which steps k-1 and k do not read.
//
// Geometry: the 2D mesh is a Geom with ny = 1, nz = number of rows and
// plane = nx; a block is tile (bid % tiles_x) of row chunk (bid / tiles_x).
// The same Src / Epi policies as the 3D sweep form the input on the fly and
// consume the output.
#pragma once

#include "s7_sweep.cuh"

namespace s7 {

// Coefficients of a stored 9-point operator: xm xp ym yp xmym xpym xmyp xpyp.
template <class CT, class A>
struct CoefView9 {
  const CT* c[8];
  const CT* diag;    // NULL: unit diagonal
  typename CoefOf<A>::t cdiag;
};

template <class CT, class A, int VEC, bool VL, class Src, class Epi>
__device__ __forceinline__ void sweep9_body(const Geom& g, const CoefView9<CT, A>& cf, Src& src,
                                            Epi& epi, Scalars* sc, int bid, int nblocks, A* sm,
                                            double* red) {
  src.setup(sc);
  epi.setup(sc);

  const int nx = g.nx, nrows = g.nz;
  const int t = threadIdx.x;
  const bool has_cell = t < g.bx;
  const int tx = has_cell ? t : 0;
  const int tile_x = bid % g.tiles_x;
  const int chunk = bid / g.tiles_x;
  const int x0 = tile_x * g.bx * VEC;
  const int y0 = chunk * g.zchunk;
  const int y1 = min(y0 + g.zchunk, nrows);
  const int x = x0 + tx * VEC;
  const int W = g.bx * VEC + 2 * VEC;     // ring row pitch (VEC pad each side)
  const int so = VEC + tx * VEC;          // own element 0 in a ring row
  const int nv = (has_cell && x < nx) ? min(VEC, nx - x) : 0;
  const bool is_lft = has_cell && tx == 0;
  const bool is_rgt = has_cell && tx == g.bx - 1;
  const bool ok_l = is_lft && x0 > 0;
  const bool ok_r = is_rgt && x0 + g.bx * VEC < nx;

  // Form the input on row yy: own run into `own`; if `buf`, also publish it
  // (and, at the tile edges, the cell beside the tile) in that ring row.
  auto produce = [&](int yy, A* buf, A (&own)[VEC], bool write_own) {
    const long long base = (long long)yy * nx + x;
    if (nv > 0) src.template produce<VEC, VL>(base, nv, own, write_own);
    else zero(own);
    if (!buf || !has_cell) return;
    sm_store<A, VEC>(buf + so, own);
    if (is_lft) buf[so - 1] = ok_l ? src.produce1(base - 1) : A(0);
    if (is_rgt) buf[so + VEC] = ok_r ? src.produce1(base + VEC) : A(0);
  };

  A vm[VEC], vc[VEC], vp[VEC];
  A lm = A(0), rm = A(0);   // input one cell left / right of the run, row y-1
  // prologue: rows y0-1 (ring buffer 2) and y0 (ring buffer 0)
  if (y0 > 0) produce(y0 - 1, sm + 2 * W, vm, false);
  else zero(vm);
  produce(y0, sm, vc, true);
  __syncthreads();
  if (y0 > 0 && has_cell) {
    lm = sm[2 * W + so - 1];
    rm = sm[2 * W + so + VEC];
  }
  A lc = has_cell ? sm[so - 1] : A(0);
  A rc = has_cell ? sm[so + VEC] : A(0);

  for (int y = y0, k = 0; y < y1; ++y, ++k) {
    const long long ib = (long long)y * nx + x;
    typename CoefOf<A>::t c[8][VEC], dg[VEC];
    if (nv > 0) {
#pragma unroll
      for (int d = 0; d < 8; ++d) load_run<CT, VEC, VL, LD_STREAM>(cf.c[d] + ib, nv, c[d]);
      if (cf.diag) load_run<CT, VEC, VL, LD_STREAM>(cf.diag + ib, nv, dg);
      else
#pragma unroll
        for (int j = 0; j < VEC; ++j) dg[j] = cf.cdiag;
    } else {
#pragma unroll
      for (int d = 0; d < 8; ++d) zero(c[d]);
      zero(dg);
    }
    epi.template load<VEC, VL>(ib, nv);

    // row y+1 into ring buffer (k+1)%3 (the halo is needed even past the
    // chunk's last row; own cells are written only inside the chunk)
    A* nb = sm + ((k + 1) % 3) * W;
    const bool next = y + 1 < nrows;
    if (next) produce(y + 1, nb, vp, y + 1 < y1);
    else zero(vp);
    __syncthreads();
    A lp = A(0), rp = A(0);
    if (next && has_cell) {
      lp = nb[so - 1];
      rp = nb[so + VEC];
    }

    if (nv > 0) {
      A out[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const A l = (j == 0) ? lc : vc[j - 1];
        const A r = (j == VEC - 1) ? rc : vc[j + 1];
        const A l_m = (j == 0) ? lm : vm[j - 1];
        const A r_m = (j == VEC - 1) ? rm : vm[j + 1];
        const A l_p = (j == 0) ? lp : vp[j - 1];
        const A r_p = (j == VEC - 1) ? rp : vp[j + 1];
        A acc = dg[j] * vc[j];
        acc = fma(c[0][j], l, acc);
        acc = fma(c[1][j], r, acc);
        acc = fma(c[2][j], vm[j], acc);
        acc = fma(c[3][j], vp[j], acc);
        acc = fma(c[4][j], l_m, acc);
        acc = fma(c[5][j], r_m, acc);
        acc = fma(c[6][j], l_p, acc);
        acc = fma(c[7][j], r_p, acc);
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
    lm = lc;
    rm = rc;
    lc = lp;
    rc = rp;
  }
  epi.finish(sc, nblocks, bid, red);
}

template <class CT, class A, int VEC, bool VL, class Src, class Epi>
__global__ void __launch_bounds__(512) k_sweep9(Geom g, CoefView9<CT, A> cf, Src src_in,
                                                Epi epi_in, Scalars* sc) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  if (sc != nullptr && Epi::kSkipWhenDone && *((volatile int*)&sc->done)) return;
  Src src = src_in;
  Epi epi = epi_in;
  sweep9_body<CT, A, VEC, VL>(g, cf, src, epi, sc, blockIdx.x, s7_nblocks(g),
                              reinterpret_cast<A*>(s7_smem), red);
}

// One policy object in both roles (see k_sweep1).
template <class CT, class A, int VEC, bool VL, class P>
__global__ void __launch_bounds__(512) k_sweep9_1(Geom g, CoefView9<CT, A> cf, P p_in,
                                                  Scalars* sc) {
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  if (sc != nullptr && P::kSkipWhenDone && *((volatile int*)&sc->done)) return;
  P pol = p_in;
  sweep9_body<CT, A, VEC, VL>(g, cf, pol, pol, sc, blockIdx.x, s7_nblocks(g),
                              reinterpret_cast<A*>(s7_smem), red);
}

// Dynamic shared memory of a 9-point sweep: three ring rows.
template <class A, int VEC>
__host__ __device__ inline size_t sweep9_smem(const Geom& g) {
  return (size_t)3 * (g.bx * VEC + 2 * VEC) * sizeof(A);
}

// ---------------------------------------------------------------------------
// Stored 9-point coefficients from the caller's raw arrays (row or column
// layout), scaled to a unit diagonal.  Row layout: out_e[i] = raw_e[i] / d_i.
// Column layout (the paper's 2D storage: raw_e[j] = A_{j+e, j}): row i's
// entry towards i+e is A_{i, i+e} = raw_{-e}[i+e], zero where i+e is
// off-mesh; `src` is then the array of the opposite direction.
// ---------------------------------------------------------------------------
template <class RT, class T>
__global__ void k_scale9(long long n, int nx, int ny, const RT* __restrict__ src, int dx, int dy,
                         int columns, const RT* __restrict__ diag, T* __restrict__ out,
                         int jacobi) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double v;
    if (columns) {
      const int x = (int)(i % nx), y = (int)(i / nx);
      const bool in = x + dx >= 0 && x + dx < nx && y + dy >= 0 && y + dy < ny;
      v = in ? (double)src[i + dx + (long long)nx * dy] : 0.0;
    } else {
      v = (double)src[i];
    }
    out[i] = from_acc<T>(jacobi ? v / (double)diag[i] : v);
  }
}

}  // namespace s7
