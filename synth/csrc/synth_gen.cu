// Device-side generator of the seeded synthetic systems of the `synth`
// package: the variable-coefficient 7-point recipe (per-cell off-diagonals
// -U[0.5,1.5], diagonal = sum |off| + U[0.01,0.1], b ~ N(0,1)) drawn from the
// same counter-based SplitMix64 streams as the host generator (Steele, Lea
// and Flood, OOPSLA 2014), so that long request streams can be generated
// where they are used.  It produces inputs only: no operator application,
// scaling or solver arithmetic.
//
// The off-diagonals and the diagonal are formed with the host generator's
// operations in its order (each IEEE operation rounded alone, no fused
// multiply-add), so they equal the host values bit for bit.  b goes through
// log, sqrt and cos, whose last bit may differ from the host's libm; after
// rounding to float32 it agrees with the host value except in rare cells,
// where it is one unit in the last place away.
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// U[0,1) with 53 random bits at counter c of the stream with start `key`.
__device__ __forceinline__ double uniform_at(uint64_t key, uint64_t c) {
  const uint64_t w = mix64(key + (c + 1) * kGamma);
  return __dmul_rn((double)(w >> 11), 1.1102230246251565e-16);   // 2^-53
}

__global__ void k_varcoef(long long n, uint64_t kc, uint64_t kb, float* xm, float* xp, float* ym,
                          float* yp, float* zm, float* zp, float* diag, float* b32, double* b64) {
  float* off[6] = {xm, xp, ym, yp, zm, zp};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double u = uniform_at(kc, (uint64_t)k * n + i);
      const float v = (float)(-__dadd_rn(0.5, u));
      off[k][i] = v;
      acc = __dadd_rn(acc, fabs((double)v));
    }
    const double m = __dadd_rn(0.01, __dmul_rn(0.09, uniform_at(kc, 6ull * n + i)));
    diag[i] = (float)__dadd_rn(acc, m);
    const double u1 = __dadd_rn(1.0, -uniform_at(kb, 2ull * i));
    const double u2 = uniform_at(kb, 2ull * i + 1);
    const double r = sqrt(__dmul_rn(-2.0, log(u1)));
    const float bv = (float)__dmul_rn(r, cos(__dmul_rn(6.283185307179586, u2)));
    if (b32) b32[i] = bv;
    if (b64) b64[i] = (double)bv;
  }
}

}  // namespace

// Fills the seven coefficient arrays (float32, n = nx*ny*nz each, device
// memory) and b (float32 and/or float64 as the value rounded to float32; either
// pointer may be NULL) of synth.varcoef(nx, ny, nz, seed) with float32 raw
// values.  key_coef / key_rhs are the stream start states of the coefficient
// and right-hand-side streams (synth.stream_key).  Asynchronous on `stream`;
// returns the launch's cudaError_t.
extern "C" int synth_varcoef_device(long long n, uint64_t key_coef, uint64_t key_rhs, float* xm,
                                    float* xp, float* ym, float* yp, float* zm, float* zp,
                                    float* diag, float* b32, double* b64, void* stream) {
  if (n <= 0) return 0;
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 152LL * 32 ? want : 152LL * 32);
  k_varcoef<<<grid, 256, 0, (cudaStream_t)stream>>>(n, key_coef, key_rhs, xm, xp, ym, yp, zm, zp,
                                                    diag, b32, b64);
  return (int)cudaGetLastError();
}
