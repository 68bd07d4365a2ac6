// Residual sweep of float64 accuracy, specialised: r = rhs - A x for a
// 7-point operator with per-cell binary32 (or 16-bit) coefficients, in
// double words (pairs of binary32 numbers, about 48 significant bits).
//
// It computes what the generic sweep with the double-word arithmetic type
// computes (s7_sweep.cuh, EpiResid in mode 1) in fewer operations:
//
// * the right-hand side seeds the compensated dot product and the seven
//   products are subtracted from it (Ogita, Rump and Oishi's Dot2 with
//   products made exact by FMA), so the residual comes out of one
//   normalisation instead of a product sum followed by an accurate
//   double-word subtraction;
// * with a unit diagonal (the Jacobi-scaled operator) rhs = b / d is one
//   correctly rounded reciprocal, a product and one exact FMA remainder
//   (b - th d), the remainder scaled by the reciprocal as the low word;
// * a binary32 iterate stays binary32 in the shared-memory ring (its low
//   word is zero); a binary64 iterate is split into a double word with
//   integer operations (the high word its leading 24 significant bits, the
//   low word the next 24, rounded), keeping the float64 pipe off the
//   per-cell path;
// * the squared norms accumulate as compensated sums (exact squares, the
//   errors summed apart) folded into binary64 every eight planes.
//
// Error: below about n^2 u^2 (u = 2^-24, n = 8 terms) of the magnitude of
// the terms that cancel, plus the 2^-48 relative split of a binary64 iterate.
#pragma once

#include "s7_sweep.cuh"

namespace s7 {

// A binary64 value as a double word: the leading 24 significant bits exactly
// (hi, truncated) and the rest rounded to binary32 (lo).  Integer operations
// only, for values whose hi and lo are normal binary32 numbers; zero, values
// outside that range, infinities and NaN take the hardware conversions.
__device__ __forceinline__ dfl d2dw(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7ffull) - 1023;
  if (__builtin_expect(e < -70 || e > 126, 0)) {
    const float h = (float)v;
    return dfl(h, (float)(v - (double)h));
  }
  const unsigned int sign = (unsigned int)(u >> 63) << 31;
  const unsigned long long m = u & 0xfffffffffffffull;          // 52 fraction bits
  const float hi = __uint_as_float(sign | ((unsigned int)(e + 127) << 23) |
                                   (unsigned int)(m >> 29));      // top 23 fraction bits
  // the remaining 29 bits, worth 2^(e-52) each: an exact integer rounded once
  const long long rest = (long long)(m & 0x1fffffffull);
  float lo = __ll2float_rn(rest) * __uint_as_float((unsigned int)(e - 52 + 127) << 23);
  if (sign) lo = -lo;
  return dfl(hi, lo);
}

// Compensated accumulation of the squares of double words (binary64 totals
// folded every few steps): in binary32 pairs while |hi| lies in
// [2^-50, 2^50] (squares and partial sums stay normal binary32 numbers), in
// binary64 otherwise (rare; infinities and NaN propagate there).
template <int NV>
struct SqDw {
  float hi[NV], lo[NV];
  double tot[NV];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      hi[j] = lo[j] = 0.f;
      tot[j] = 0.0;
    }
  }
  __device__ __forceinline__ void add(int j, dfl v) {
    const float a = fabsf(v.hi);
    if (__builtin_expect(a >= 0x1p-50f && a <= 0x1p50f, 1)) {
      const float p = v.hi * v.hi;
      const float e = fmaf(2.0f * v.hi, v.lo, fmaf(v.hi, v.hi, -p));
      const dfl s = dw::two_sum(hi[j], p);
      hi[j] = s.hi;
      lo[j] += s.lo + e;
    } else if (v.hi != 0.f) {
      const double d = f2d_exact(v.hi) + f2d_exact(v.lo);
      tot[j] = fma(d, d, tot[j]);
    }
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      tot[j] += f2d_exact(hi[j]) + f2d_exact(lo[j]);
      hi[j] = lo[j] = 0.f;
    }
  }
};

// Pointers of one residual sweep.  UNIT: the stored operator has a unit
// diagonal and rhs = b / dinv (dinv: the kept diagonal); otherwise diag is
// the operator's diagonal and rhs = b.  CT: coefficient type; XT: iterate
// and right-hand-side type (binary32 or binary64); DTT: kept-diagonal type.
template <class CT, class XT, class DTT>
struct ResidArgs {
  const CT* c[6];
  const CT* diag;
  const DTT* dinv;
  const XT* x;
  const XT* b;
  XT* r;            // residual out (may be NULL)
  double* parts;
  int counter;
};

template <class XT> struct RingOfX { typedef float t; };
template <> struct RingOfX<double> { typedef dfl t; };

__device__ __forceinline__ dfl to_dw(float v) { return dfl(v, 0.f); }
__device__ __forceinline__ dfl to_dw(dfl v) { return v; }
__device__ __forceinline__ float hi_of(float v) { return v; }
__device__ __forceinline__ float hi_of(dfl v) { return v.hi; }
__device__ __forceinline__ float lo_of(float) { return 0.f; }
__device__ __forceinline__ float lo_of(dfl v) { return v.lo; }

// acc - c * v (Dot2 step: the product's leading part exact by FMA, its
// rounding error and the low word's product carried in acc.lo)
__device__ __forceinline__ void sub_term(dfl& acc, float c, float v) {
  const float p = c * v;
  const float pe = fmaf(c, v, -p);
  const dfl s = dw::two_sum(acc.hi, -p);
  acc = dfl(s.hi, acc.lo + (s.lo - pe));
}
__device__ __forceinline__ void sub_term(dfl& acc, float c, dfl v) {
  const float p = c * v.hi;
  const float pe = fmaf(c, v.lo, fmaf(c, v.hi, -p));
  const dfl s = dw::two_sum(acc.hi, -p);
  acc = dfl(s.hi, acc.lo + (s.lo - pe));
}
// acc - v (unit coefficient: no product)
__device__ __forceinline__ void sub_unit(dfl& acc, float v) {
  const dfl s = dw::two_sum(acc.hi, -v);
  acc = dfl(s.hi, acc.lo + s.lo);
}
__device__ __forceinline__ void sub_unit(dfl& acc, dfl v) {
  const dfl s = dw::two_sum(acc.hi, -v.hi);
  acc = dfl(s.hi, acc.lo + (s.lo - v.lo));
}

template <class XT> __device__ __forceinline__ void ld_x4(const XT* p, typename RingOfX<XT>::t (&o)[4]);
template <> __device__ __forceinline__ void ld_x4<float>(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <> __device__ __forceinline__ void ld_x4<double>(const double* p, dfl (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = d2dw(a.x);
  o[1] = d2dw(a.y);
  o[2] = d2dw(b.x);
  o[3] = d2dw(b.y);
}
template <class XT> __device__ __forceinline__ typename RingOfX<XT>::t ld_x1(const XT* p);
template <> __device__ __forceinline__ float ld_x1<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ dfl ld_x1<double>(const double* p) { return d2dw(*p); }

template <class T> __device__ __forceinline__ void ld_c4(const T* p, float (&o)[4]) {
  ldv<T, 4, LD_STREAM>(p, o);
}

// The residual out: binary32 gets the normalised high word, binary64 the
// exact sum of the two words.
__device__ __forceinline__ void st_r4(float* p, const dfl (&r)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0].hi, r[1].hi, r[2].hi, r[3].hi);
}
__device__ __forceinline__ void st_r4(double* p, const dfl (&r)[4]) {
  *reinterpret_cast<double2*>(p) =
      make_double2(f2d_exact(r[0].hi) + f2d_exact(r[0].lo), f2d_exact(r[1].hi) + f2d_exact(r[1].lo));
  *reinterpret_cast<double2*>(p + 2) =
      make_double2(f2d_exact(r[2].hi) + f2d_exact(r[2].lo), f2d_exact(r[3].hi) + f2d_exact(r[3].lo));
}

// 4 cells per thread; rows of whole 4-cell vectors, 16-byte aligned arrays
// (the host checks).  Block shape and z march as in sweep_body; the ring
// holds the iterate (binary32, or double words for a binary64 iterate).
// Leaves ||r||^2 in res[0] and ||rhs||^2 in res[1].
template <class CT, class XT, class DTT, bool UNIT>
__global__ void __launch_bounds__(256) k_resid_dw(Geom g, ResidArgs<CT, XT, DTT> a, Scalars* sc) {
  typedef typename RingOfX<XT>::t RX;
  extern __shared__ __align__(16) unsigned char s7_smem[];
  __shared__ double red[32 * 4];
  RX* sm = reinterpret_cast<RX*>(s7_smem);
  constexpr int VEC = 4;
  const int t = threadIdx.x;
  const bool has_cell = t < g.bx * g.by;
  const int tx = has_cell ? t % g.bx : 0;
  const int ty = has_cell ? t / g.bx : 0;
  const int bid = blockIdx.x;
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
  const int W = g.bx * VEC + 2 * VEC;
  const int PL = (g.by + 2) * W;
  const int so = (ty + 1) * W + VEC + tx * VEC;
  const bool own = has_cell && y < g.ny && x < g.nx;
  const bool top = has_cell && ty == 0 && y0 > 0 && x < g.nx;
  const bool bot = has_cell && ty == g.by - 1 && y + 1 < g.ny && x < g.nx;
  const bool lft = has_cell && tx == 0 && x0 > 0 && y < g.ny;
  const bool rgt = has_cell && tx == g.bx - 1 && x + VEC < g.nx && y < g.ny;
  const long long row = (long long)y * g.nx + x;
  const RX zero = RX(0.f);

  // plane zp of the iterate: own run into v (and into the ring buffer buf
  // with its halo when `ring`)
  auto produce = [&](int zp, RX* buf, RX (&v)[VEC], bool ring) {
    const long long base = (long long)zp * g.plane + row;
    if (own) ld_x4<XT>(a.x + base, v);
    else
#pragma unroll
      for (int j = 0; j < VEC; ++j) v[j] = zero;
    if (!ring || !has_cell) return;
#pragma unroll
    for (int j = 0; j < VEC; ++j) buf[so + j] = v[j];
    if (ty == 0) {
      RX h[VEC];
      if (top) ld_x4<XT>(a.x + base - g.nx, h);
      else
#pragma unroll
        for (int j = 0; j < VEC; ++j) h[j] = zero;
#pragma unroll
      for (int j = 0; j < VEC; ++j) buf[so - W + j] = h[j];
    }
    if (ty == g.by - 1) {
      RX h[VEC];
      if (bot) ld_x4<XT>(a.x + base + g.nx, h);
      else
#pragma unroll
        for (int j = 0; j < VEC; ++j) h[j] = zero;
#pragma unroll
      for (int j = 0; j < VEC; ++j) buf[so + W + j] = h[j];
    }
    if (tx == 0) buf[so - 1] = lft ? ld_x1<XT>(a.x + base - 1) : zero;
    if (tx == g.bx - 1) buf[so + VEC] = rgt ? ld_x1<XT>(a.x + base + VEC) : zero;
  };

  SqDw<2> acc;
  acc.init();
  RX vm[VEC], vc[VEC], vp[VEC];
  if (z0 > 0) produce(z0 - 1, nullptr, vm, false);
  else
#pragma unroll
    for (int j = 0; j < VEC; ++j) vm[j] = zero;
  produce(z0, sm, vc, true);
  for (int z = z0, k = 0; z < z1; ++z, ++k) {
    const long long ib = (long long)z * g.plane + row;
    float c[6][VEC], dg[VEC];
    RX bv[VEC];
    if (own) {
#pragma unroll
      for (int d = 0; d < 6; ++d) ld_c4<CT>(a.c[d] + ib, c[d]);
      if (UNIT) ld_c4<DTT>(a.dinv + ib, dg);
      else ld_c4<CT>(a.diag + ib, dg);
      ld_x4<XT>(a.b + ib, bv);
    }
    RX* nb = sm + ((k + 1) % 3) * PL;
    if (z + 1 < g.nz) produce(z + 1, nb, vp, z + 1 < z1);
    else
#pragma unroll
      for (int j = 0; j < VEC; ++j) vp[j] = zero;
    __syncthreads();
    if (own) {
      const RX* cb = sm + (k % 3) * PL;
      dfl r[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const RX l = (j == 0) ? cb[so - 1] : vc[j - 1];
        const RX rr = (j == VEC - 1) ? cb[so + VEC] : vc[j + 1];
        const RX up = cb[so - W + j];
        const RX dn = cb[so + W + j];
        dfl s;
        if (UNIT) {
          // rhs = b / d as a double word: th = b * (1/d) (correctly rounded
          // reciprocal), the exact remainder b - th d, scaled by 1/d
          const float rc = __frcp_rn(dg[j]);
          const float th = hi_of(bv[j]) * rc;
          const float rem = fmaf(-th, dg[j], hi_of(bv[j])) + lo_of(bv[j]);
          s = dw::fast_two_sum(th, rem * rc);
          acc.add(1, s);
          sub_unit(s, vc[j]);
        } else {
          s = to_dw(bv[j]);
          acc.add(1, s);
          sub_term(s, dg[j], vc[j]);
        }
        sub_term(s, c[0][j], l);
        sub_term(s, c[1][j], rr);
        sub_term(s, c[2][j], up);
        sub_term(s, c[3][j], dn);
        sub_term(s, c[4][j], vm[j]);
        sub_term(s, c[5][j], vp[j]);
        r[j] = dw::two_sum(s.hi, s.lo);
        acc.add(0, r[j]);
      }
      if (a.r) st_r4(a.r + ib, r);
    }
    if ((k & 7) == 7) acc.fold();
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      vm[j] = vc[j];
      vc[j] = vp[j];
    }
  }
  acc.fold();
  double v[2] = {acc.tot[0], acc.tot[1]}, tot[2];
  block_sum<2>(v, red);
  if (grid_combine<2>(a.parts, &sc->counter[a.counter], s7_nblocks(g), bid, v, tot, red) &&
      t == 0) {
    sc->res[0] = tot[0];
    sc->res[1] = tot[1];
  }
}

// Dynamic shared memory of k_resid_dw for geometry g.
template <class XT>
inline size_t resid_dw_smem(const Geom& g) {
  return (size_t)3 * (g.by + 2) * (g.bx * 4 + 8) * sizeof(typename RingOfX<XT>::t);
}

}  // namespace s7
