// Device helpers shared by the stencil sweeps and the pointwise kernels:
// element types and conversions, 16-byte vector loads/stores, deterministic
// block reductions and the last-block grid combine that stands in for the
// paper's AllReduce (Sec. IV-C): per-block partial sums written to global
// memory, then summed in a fixed order in float64 by whichever block
// finishes last.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace s7 {

typedef __nv_bfloat16 bf16;
typedef __half f16;

// ---------------------------------------------------------------------------
// conversions (all rounding is round-to-nearest-even)
// ---------------------------------------------------------------------------
// binary32 -> binary64 is exact: for normal numbers it only re-biases the
// exponent (127 -> 1023) and widens the significand, and a signed zero keeps
// its sign bit alone, which integer instructions do at full rate; only
// subnormals, infinities and NaN take the hardware conversion, on a branch
// kept out of the common path.  GB300 runs float64 arithmetic (conversions
// included) at a small fraction of its float32 rate, and the float64
// residual sweeps convert seven coefficients per cell.
__device__ __forceinline__ double f2d_exact(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned int m = u & 0x7fffffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (__builtin_expect((e == 0u && m != 0u) || e == 0xffu, 0)) return (double)v;
  const unsigned long long bits =
      e == 0u ? sign
              : sign | ((unsigned long long)(e + (1023u - 127u)) << 52) |
                    ((unsigned long long)m << 29);
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// double-word arithmetic: a value held as the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi)/2 (about 48 significant bits).
// GB300 runs float64 at a small fraction of its float32 rate, so the
// residual sweeps that want more than float32 accuracy sum their stencil
// terms in double words on the float32 pipes.  The building blocks are the
// error-free transformations of Dekker and Knuth (the exact error of a sum
// from six additions, of a product from one FMA) and the double-word
// algorithms of Joldes, Muller and Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic" (ACM TOMS 44, 2017):
// the accurate sum of two double words, the products of a double word by a
// binary32 number and by a double word, and the quotient of two double
// words, each with a proven relative error of a small multiple of u^2
// (u = 2^-24).  The operations live in their own namespace and are found by
// argument-dependent lookup, so the binary32 / binary64 overloads of fma
// stay visible.
// ---------------------------------------------------------------------------
namespace dw {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfl(float v) : hi(v), lo(0.f) {}
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // nearest double word of a binary64 value (exact for |v| in binary32
  // range with at most 48 significant bits)
  __host__ __device__ dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const {
#ifdef __CUDA_ARCH__
    return f2d_exact(hi) + f2d_exact(lo);
#else
    return (double)hi + (double)lo;
#endif
  }
};

// s + e = a + b exactly (any a, b).
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl(s, (a - (s - bb)) + (b - bb));
}
// s + e = a + b exactly, provided |a| >= |b| (or a == 0).
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfl(s, b - (s - a));
}
// p + e = a * b exactly (barring underflow).
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = a * b;
  return dfl(p, fmaf(a, b, -p));
}

__device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }

__device__ __forceinline__ dfl operator+(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  const dfl v = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(v.hi, t.lo + v.lo);
}
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }

__device__ __forceinline__ dfl operator*(dfl x, float y) {
  const dfl c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, fmaf(x.lo, y, c.lo));
}
__device__ __forceinline__ dfl operator*(float y, dfl x) { return x * y; }

__device__ __forceinline__ dfl operator*(dfl x, dfl y) {
  const dfl c = two_prod(x.hi, y.hi);
  const float t = fmaf(x.hi, y.lo, x.lo * y.lo);
  return fast_two_sum(c.hi, c.lo + fmaf(x.lo, y.hi, t));
}

__device__ __forceinline__ dfl operator/(dfl x, dfl y) {
  const float th = x.hi / y.hi;
  const dfl r = y * th;
  const float d = (x.hi - r.hi) + (x.lo - r.lo);
  return fast_two_sum(th, d / y.hi);
}

// One step of a compensated dot product (the "Dot2" scheme of Ogita, Rump and
// Oishi, with the products made exact by FMA): acc.hi carries the running
// binary32 sum of the products' leading parts, acc.lo the sum of every
// rounding error and product tail.  The pair is left unnormalised; settle()
// turns it into a double word.  About 11 operations against 26 for a product
// followed by an accurate double-word sum; for n terms the error stays below
// about n^2 u^2 times the sum of their magnitudes.
__device__ __forceinline__ dfl fma(float a, dfl x, dfl acc) {
  const dfl p = two_prod(a, x.hi);
  const dfl s = two_sum(acc.hi, p.hi);
  return dfl(s.hi, acc.lo + (s.lo + fmaf(a, x.lo, p.lo)));
}
__device__ __forceinline__ dfl settle(dfl v) { return two_sum(v.hi, v.lo); }

__host__ __device__ __forceinline__ bool operator==(dfl x, dfl y) {
  return x.hi == y.hi && x.lo == y.lo;
}
__host__ __device__ __forceinline__ bool operator!=(dfl x, dfl y) { return !(x == y); }

// hi + lo rounded to odd in binary32: hi when hi is odd (or the pair is
// exact), else hi's neighbour towards lo.  Rounding that value to nearest in
// a format of at most 22 bits gives the correctly rounded hi + lo.
__device__ __forceinline__ float round_odd(dfl x) {
  unsigned int u = __float_as_uint(x.hi);
  if (x.lo != 0.f && (u & 1u) == 0u && isfinite(x.hi))
    u += ((x.lo > 0.f) == (x.hi > 0.f)) ? 1u : 0xffffffffu;
  return __uint_as_float(u);
}

}  // namespace dw
using dw::dfl;

template <class A> __device__ __forceinline__ A to_acc(float v);
template <> __device__ __forceinline__ float to_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ dfl to_acc<dfl>(float v) { return dfl(v); }
template <> __device__ __forceinline__ double to_acc<double>(float v) { return f2d_exact(v); }

template <class A> __device__ __forceinline__ A to_acc(double v);
template <> __device__ __forceinline__ double to_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_acc<float>(double v) { return (float)v; }

template <class A> __device__ __forceinline__ A to_acc(bf16 v) { return (A)__bfloat162float(v); }
template <class A> __device__ __forceinline__ A to_acc(f16 v) { return (A)__half2float(v); }

template <class T> __device__ __forceinline__ T from_acc(float v);
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_acc<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ bf16 from_acc<bf16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ f16 from_acc<f16>(float v) { return __float2half_rn(v); }

template <class T> __device__ __forceinline__ T from_acc(double v);
template <> __device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_acc<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ bf16 from_acc<bf16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ f16 from_acc<f16>(double v) { return __double2half(v); }

template <> __device__ __forceinline__ dfl to_acc<dfl>(double v) { return dfl(v); }
template <class A> __device__ __forceinline__ A to_acc(dfl v);
template <> __device__ __forceinline__ dfl to_acc<dfl>(dfl v) { return v; }
// a double word to storage: binary32 takes hi (the pair is normalised, so hi
// is hi + lo rounded to nearest); binary64 the exact sum; the 16-bit types
// round the round-to-odd binary32 value, which rounds hi + lo correctly
template <class T> __device__ __forceinline__ T from_acc(dfl v);
template <> __device__ __forceinline__ dfl from_acc<dfl>(dfl v) { return v; }
template <> __device__ __forceinline__ float from_acc<float>(dfl v) { return v.hi; }
template <> __device__ __forceinline__ double from_acc<double>(dfl v) { return (double)v; }
template <> __device__ __forceinline__ bf16 from_acc<bf16>(dfl v) {
  return __float2bfloat16_rn(dw::round_odd(v));
}
template <> __device__ __forceinline__ f16 from_acc<f16>(dfl v) {
  return __float2half_rn(dw::round_odd(v));
}

// Element type of the stored coefficients inside a sweep of arithmetic type
// A (binary32 for double-word sweeps: coefficient times input is then a
// double word from one product and one FMA), and the type the inner
// products of the residual norms accumulate in (binary64 for double words:
// squares of binary32-range values can overflow binary32).
template <class A> struct CoefOf { typedef A t; };
template <> struct CoefOf<dfl> { typedef float t; };
template <class A> struct NormOf { typedef A t; };
template <> struct NormOf<dfl> { typedef double t; };
template <class N, class A> __device__ __forceinline__ N to_norm(A v) { return (N)v; }

// An accumulator value ready for use (double words: normalised).
__device__ __forceinline__ float settle(float v) { return v; }
__device__ __forceinline__ double settle(double v) { return v; }

// Per-thread sums of squares, folded into binary64 totals every few steps.
template <class A, int NV>
struct SqAcc {
  typedef typename NormOf<A>::t N;
  N part[NV];
  double tot[NV];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { part[j] = N(0); tot[j] = 0.0; }
  }
  __device__ __forceinline__ void add_sq(int j, A v) {
    const N t = to_norm<N>(v);
    part[j] = fma(t, t, part[j]);
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { tot[j] += (double)part[j]; part[j] = N(0); }
  }
};

// Double words: squares in double words while |hi| lies in [2^-50, 2^50]
// (square and partial sums stay normal binary32 numbers), in binary64
// otherwise (rare; infinities and NaN propagate there).
template <int NV>
struct SqAcc<dfl, NV> {
  dfl part[NV];
  double tot[NV];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { part[j] = dfl(0); tot[j] = 0.0; }
  }
  __device__ __forceinline__ void add_sq(int j, dfl v) {
    const float a = fabsf(v.hi);
    if (a >= 0x1p-50f && a <= 0x1p50f) {
      const dfl p = dw::two_prod(v.hi, v.hi);
      part[j] = part[j] + dw::fast_two_sum(p.hi, fmaf(2.0f * v.hi, v.lo, p.lo));
    } else if (v.hi != 0.f) {
      const double d = (double)v;
      tot[j] = fma(d, d, tot[j]);
    }
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int j = 0; j < NV; ++j) { tot[j] += (double)part[j]; part[j] = dfl(0); }
  }
};

// ---------------------------------------------------------------------------
// vector loads / stores of VEC consecutive elements (VEC*sizeof(T) <= 16 B,
// address aligned to that size)
// ---------------------------------------------------------------------------
template <int BYTES> struct Raw;
template <> struct Raw<16> { typedef uint4 t; };
template <> struct Raw<8> { typedef uint2 t; };
template <> struct Raw<4> { typedef unsigned int t; };
template <> struct Raw<2> { typedef unsigned short t; };

template <class T> struct Bits { typedef T t; };
template <> struct Bits<bf16> { typedef unsigned short t; };
template <> struct Bits<f16> { typedef unsigned short t; };

template <class T, class B> __device__ __forceinline__ T from_bits(B b) { return b; }
template <> __device__ __forceinline__ bf16 from_bits<bf16, unsigned short>(unsigned short b) {
  return __ushort_as_bfloat16(b);
}
template <> __device__ __forceinline__ f16 from_bits<f16, unsigned short>(unsigned short b) {
  return __ushort_as_half(b);
}
template <class T> __device__ __forceinline__ typename Bits<T>::t to_bits(T v) { return v; }
template <> __device__ __forceinline__ unsigned short to_bits<bf16>(bf16 v) { return __bfloat16_as_ushort(v); }
template <> __device__ __forceinline__ unsigned short to_bits<f16>(f16 v) { return __half_as_ushort(v); }

// Cache policy of a load: default (L1+L2), or streaming (read once, evict
// first) for coefficient arrays that no other block reads.
enum { LD_DEFAULT = 0, LD_STREAM = 1 };

template <int POL, class R> __device__ __forceinline__ R ld_raw(const R* p) {
  if (POL == LD_STREAM) return __ldcs(p);
  return *p;
}

// Elements per memory transaction: at most 16 bytes.
template <class T, int VEC> struct Chunk {
  static constexpr int n = (VEC * (int)sizeof(T) > 16) ? (16 / (int)sizeof(T)) : VEC;
};

template <class T, int VEC, int POL = LD_DEFAULT, class A>
__device__ __forceinline__ void ldv(const T* __restrict__ p, A (&o)[VEC]) {
  constexpr int CH = Chunk<T, VEC>::n;
  typedef typename Raw<CH * sizeof(T)>::t R;
  typedef typename Bits<T>::t B;
#pragma unroll
  for (int c = 0; c < VEC / CH; ++c) {
    union { R r; B b[CH]; } u;
    u.r = ld_raw<POL>(reinterpret_cast<const R*>(p + c * CH));
#pragma unroll
    for (int k = 0; k < CH; ++k) o[c * CH + k] = to_acc<A>(from_bits<T>(u.b[k]));
  }
}

template <class T, int VEC, bool STREAM = false, class A>
__device__ __forceinline__ void stv(T* __restrict__ p, const A (&v)[VEC]) {
  constexpr int CH = Chunk<T, VEC>::n;
  typedef typename Raw<CH * sizeof(T)>::t R;
  typedef typename Bits<T>::t B;
#pragma unroll
  for (int c = 0; c < VEC / CH; ++c) {
    union { R r; B b[CH]; } u;
#pragma unroll
    for (int k = 0; k < CH; ++k) u.b[k] = to_bits<T>(from_acc<T>(v[c * CH + k]));
    if (STREAM) __stcs(reinterpret_cast<R*>(p + c * CH), u.r);
    else *reinterpret_cast<R*>(p + c * CH) = u.r;
  }
}

// Element-wise masked variants for rows whose start is not vector aligned.
template <class T, int VEC, class A>
__device__ __forceinline__ void lds(const T* __restrict__ p, int nvalid, A (&o)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; ++k) o[k] = (k < nvalid) ? to_acc<A>(p[k]) : A(0);
}
template <class T, int VEC, class A>
__device__ __forceinline__ void sts(T* __restrict__ p, int nvalid, const A (&v)[VEC]) {
#pragma unroll
  for (int k = 0; k < VEC; ++k)
    if (k < nvalid) p[k] = from_acc<T>(v[k]);
}

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the block in a fixed order (float64).  `sh` needs
// NV * 32 doubles.  The result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  __syncthreads();  // sh may alias memory used just before
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j * 32 + warp] = v[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = lane < nw ? sh[j * 32 + lane] : 0.0;
      v[j] = warp_sum(t);
    }
  }
}

// Last-block grid combine.  Every block calls this once with its block sums
// (valid in thread 0).  Block `bid` of `nblocks` stores them to
// parts[j*nblocks + bid]; the block that arrives last sums all partials in a
// fixed order (so the totals do not depend on which block is last) and gets
// true back, with the totals in thread 0's `tot`.  The counter is reset for
// the next use.  `sh` needs NV * 32 doubles.
template <int NV>
__device__ __forceinline__ bool grid_combine(double* parts, unsigned int* counter, int nblocks,
                                             int bid, const double (&v)[NV], double (&tot)[NV],
                                             double* sh) {
  __shared__ int s_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) parts[(size_t)j * nblocks + bid] = v[j];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == (unsigned int)nblocks - 1u);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    acc[j] = 0.0;
    for (int i = tid; i < nblocks; i += nt) acc[j] += __ldcg(parts + (size_t)j * nblocks + i);
  }
  block_sum<NV>(acc, sh);
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = acc[j];
    *counter = 0u;
  }
  return true;
}

}  // namespace s7
