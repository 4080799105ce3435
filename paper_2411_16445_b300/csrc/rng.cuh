// rng.cuh -- the model's counter-based random numbers on the device
// (Sec. "Computation with stochastic differential equations"):
// Threefry-4x64-12 uniforms (Poisson drive, plasticity noise) and normal
// deviates by the Box-Muller method, with the model's own logarithm and
// circular functions so that the deviates are reproducible to the last bit.
// Written with explicitly rounded operations (never contracted), whatever the
// translation unit's contraction setting.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pa {

// Threefry-4x64-12 (Salmon et al. 2011): Threefish-256 rotations, key parity
// 0x1BD11BDAA9FC1A22, key injection after every fourth round.
__device__ __forceinline__ uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__device__ __forceinline__ void threefry4x64_12(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1, uint64_t k2, uint64_t k3,
                                                uint64_t out[4]) {
  const int R0[8] = {14, 52, 23, 5, 25, 46, 58, 32};
  const int R1[8] = {16, 57, 40, 37, 33, 12, 22, 32};
  uint64_t ks[5] = {k0, k1, k2, k3, 0x1BD11BDAA9FC1A22ULL ^ k0 ^ k1 ^ k2 ^ k3};
  uint64_t x0 = c0 + ks[0], x1 = c1 + ks[1], x2 = c2 + ks[2], x3 = c3 + ks[3];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    if ((r & 1) == 0) {
      x0 += x1; x1 = rotl(x1, R0[r & 7]); x1 ^= x0;
      x2 += x3; x3 = rotl(x3, R1[r & 7]); x3 ^= x2;
    } else {
      x0 += x3; x3 = rotl(x3, R0[r & 7]); x3 ^= x0;
      x2 += x1; x1 = rotl(x1, R1[r & 7]); x1 ^= x2;
    }
    if ((r & 3) == 3) {
      const int s = (r >> 2) + 1;
      x0 += ks[s % 5];
      x1 += ks[(s + 1) % 5];
      x2 += ks[(s + 2) % 5];
      x3 += ks[(s + 3) % 5] + (uint64_t)s;
    }
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// The model's natural logarithm of a positive normal x: x = m 2^e with m in
// [sqrt(1/2), sqrt(2)); log m = 2 atanh(s), s = (m - 1)/(m + 1), by the odd
// series s + s^3/3 + ... + s^23/23 (Horner, fused multiply-adds; |s| < 0.172);
// e ln2 added with ln2 split into a 32-bit head and a tail.  Coefficients: 1/k
// rounded to double.
__device__ __forceinline__ double model_log(double x) {
  const double c[12] = {0.043478260869565216, 0.047619047619047616, 0.05263157894736842,
                        0.058823529411764705, 0.06666666666666667, 0.07692307692307693,
                        0.09090909090909091, 0.1111111111111111, 0.14285714285714285,
                        0.2, 0.3333333333333333, 1.0};
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7ff) - 1022;
  double m = __longlong_as_double((long long)((b & 0x800fffffffffffffULL) | (1022ULL << 52)));
  if (m < 0.70710678118654752440) {
    m = __dmul_rn(m, 2.0);
    e = e - 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double p = c[0];
#pragma unroll
  for (int i = 1; i < 12; ++i) p = __fma_rn(p, s2, c[i]);
  const double t = __dmul_rn(s, p);
  const double lm = __dadd_rn(t, t);
  const double ed = (double)e;
  const double hi = __dmul_rn(ed, 6.93147180369123816490e-01);
  return __dadd_rn(hi, __fma_rn(ed, 1.9082149292705877e-10, lm));
}

// cos(2 pi v) (which = 0) or sin(2 pi v) (which = 1) for v in [0, 1): quadrant
// q = rint(4v) and remainder r = v - q/4 (|r| <= 1/8), both exact; t = 2 pi r
// by one rounded product; Taylor series of sin t (to t^21) or cos t (to t^22),
// Horner with fused multiply-adds; coefficients (-1)^k / n! rounded to double.
__device__ __forceinline__ double model_cis2pi(double v, int which) {
  const double sc[10] = {1.9572941063391263e-20, -8.22063524662433e-18, 2.8114572543455206e-15,
                         -7.647163731819816e-13, 1.6059043836821613e-10, -2.505210838544172e-08,
                         2.7557319223985893e-06, -0.0001984126984126984, 0.008333333333333333,
                         -0.16666666666666666};
  const double cc[11] = {-8.896791392450574e-22, 4.110317623312165e-19, -1.5619206968586225e-16,
                         4.779477332387385e-14, -1.1470745597729725e-11, 2.08767569878681e-09,
                         -2.755731922398589e-07, 2.48015873015873e-05, -0.001388888888888889,
                         0.041666666666666664, -0.5};
  const double q = rint(__dmul_rn(4.0, v));
  const double r = __dsub_rn(v, __dmul_rn(0.25, q));
  const double t = __dmul_rn(r, 6.283185307179586);
  const double t2 = __dmul_rn(t, t);
  const int quad = ((int)q) & 3;
  const bool want_sin = which ? (quad == 0 || quad == 2) : (quad == 1 || quad == 3);
  double val;
  if (want_sin) {
    double sp = sc[0];
#pragma unroll
    for (int i = 1; i < 10; ++i) sp = __fma_rn(sp, t2, sc[i]);
    val = __fma_rn(__dmul_rn(sp, t2), t, t);
  } else {
    double cp = cc[0];
#pragma unroll
    for (int i = 1; i < 11; ++i) cp = __fma_rn(cp, t2, cc[i]);
    val = __fma_rn(cp, t2, 1.0);
  }
  const bool neg = which ? (quad >= 2) : (quad == 1 || quad == 2);
  return neg ? -val : val;
}

// Normal deviate of noise source `id` at step `step` (plasticity noise,
// Eqs. plasticity_noise_1-2): one Threefry call, key = (seed, 0, 0, 0),
// counter = (id, step / 4, 2, 0), serves four steps; step mod 4 = 2p + j takes
// the Box-Muller pair of output words 2p and 2p+1 as 53-bit uniforms u1, u2 in
// [0, 1): sqrt(-2 log(1 - u1)) times cos (j = 0) or sin (j = 1) of 2 pi u2.
__device__ __forceinline__ double model_normal(uint64_t seed, uint64_t id, int64_t step) {
  uint64_t w[4];
  threefry4x64_12(id, (uint64_t)step >> 2, 2, 0, seed, 0, 0, 0, w);
  const int j = (int)(step & 3);
  const double u1 = __dmul_rn(__ull2double_rn(w[j & 2] >> 11), 0x1p-53);
  const double u2 = __dmul_rn(__ull2double_rn(w[(j & 2) + 1] >> 11), 0x1p-53);
  const double rad = __dsqrt_rn(__dmul_rn(-2.0, model_log(__dsub_rn(1.0, u1))));
  return __dmul_rn(rad, model_cis2pi(u2, j & 1));
}

}  // namespace pa
