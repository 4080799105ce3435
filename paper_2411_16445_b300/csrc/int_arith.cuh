// int_arith.cuh -- FP64 operations rebuilt from integer arithmetic, for a GPU
// whose FP64 pipe issues about 1.5 thread operations per clock and SM while its
// integer pipes issue 64.  Both routines return exactly the IEEE result of the
// operation they replace (round to nearest even), so the FP64 path stays
// identical, bit for bit, to the plain definition.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pa {

// Correctly rounded 1/d for a positive normal double d (other inputs take the
// IEEE division).  A hardware-sequenced FP64 division costs about 6.5 FP64
// FMAs of issue time on this GPU; this routine spends one single-precision
// MUFU op and about forty-five integer ops, mostly 32-bit.
//
// Method: a third-order Newton-Raphson step from a single-precision seed,
// then an exact remainder test that decides the rounding (the classic
// correct-rounding argument for division; Muller et al., Handbook of
// Floating-Point Arithmetic, division by Newton-Raphson iteration):
//   d = M 2^(ex-1023), M = m 2^-52 in [1, 2), m a 53-bit integer;
//   seed y0 ~ 1/M from rcp.approx.f32 of M truncated to 24 bits, held as
//     the integer y24 = y0 2^24 (relative error about 2^-22);
//   E = eps 2^76 with eps = 1 - M y0, exactly: -(m y24) modulo 2^64, since
//     2^76 vanishes modulo 2^64 and |E| < 2^57;
//   S = (eps + eps^2) 2^76, the square from the top 32 bits of E (S is
//     needed to about 2^22 only);
//   Y1 = y0 (1 + eps + eps^2) 2^63 = (1 - eps^3) 2^63 / M, relative error
//     below 2^-59, from y24 2^39 + y24 S 2^-37 (two 32x32 products);
//   Q0 = round(Y1 2^-10) is then within 1 of Q = round(2^105 / m) (Q = 2^53
//     for M = 1, whose exponent carry the final addition absorbs);
//   with D = (2 Q0 + 1) m - 2^106 (exact modulo 2^64, |D| < 2^56):
//     D < 0 -> Q = Q0 + 1;  D - 2m > 0 -> Q = Q0 - 1;  else Q = Q0.
//   No tie exists: 2^106 = (2Q0 +- 1) m would make m a power of two, and the
//   one power of two, m = 2^52, gives D = 2^52 (no change).
//   1/d = (2/M) 2^(1022-ex) and 2/M = Q 2^-52.
// The seed's error may reach about 2^-19 before Q0 can miss by more than 1;
// rcp.approx.f32 errs by at most about 2^-23.
// The IEEE division for the inputs outside rcp_rn_pos's domain, behind a call so
// that the compiler cannot turn the rare branch into predicated FP64 work on
// every row.
static __device__ __noinline__ double rcp_ieee(double d) { return 1.0 / d; }

__device__ __forceinline__ double rcp_rn_pos(double d) {
  const uint64_t x = (uint64_t)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(x >> 32), lo = (uint32_t)x;
  const uint32_t ex = hi >> 20;          // includes the sign bit: d < 0 -> ex >= 2048
  if (ex - 1u >= 2044u) return rcp_ieee(d);  // zero, subnormal, huge, negative, inf, nan
  const uint64_t m = (x & 0x000fffffffffffffULL) | 0x0010000000000000ULL;
  const float mh = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
  float y0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(mh));
  const uint32_t y24 = __float2uint_rz(y0 * 16777216.0f);
  const int64_t e = (int64_t)(0ull - m * (uint64_t)y24);
  const int32_t eh = (int32_t)(e >> 32);
  const int64_t s = e + (((int64_t)eh * eh) >> 12);
  const int32_t sh = (int32_t)(s >> 32);
  const uint32_t sl = (uint32_t)s;
  const int64_t t = (((int64_t)y24 * sh) >> 5) + (int64_t)(((uint64_t)y24 * sl) >> 37);
  const uint64_t y1 = ((uint64_t)y24 << 39) + (uint64_t)t;  // ~ 2^63 / M
  uint64_t q = (y1 + 512u) >> 10;
  const int64_t r = (int64_t)((2 * q + 1) * m);
  if (r < 0) {
    q += 1;
  } else if (r - (int64_t)(2 * m) > 0) {
    q -= 1;
  }
  return __longlong_as_double((long long)(((uint64_t)(2044u - ex) << 52) + q));
}

// Exact widening of a float to double by moving its fields (sign; exponent
// rebiased from 127 to 1023; fraction shifted from 23 to 52 bits), without a
// branch: the hardware conversion issues on the FP64-rate pipe of this GPU,
// and a rarely taken branch to it may be turned into a predicated conversion
// on every call.  A subnormal is first scaled by 2^24 in FP32 (exact) and
// rebiased 24 lower; infinities and NaNs keep exponent 2047 and their
// fraction; zeros keep their sign.
__device__ __forceinline__ double widen_f32(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t s = u & 0x80000000u, a0 = u & 0x7fffffffu;
  const bool sub = a0 < 0x00800000u;
  const uint32_t as = __float_as_uint(__fmul_rn(__uint_as_float(a0), 16777216.0f));
  const uint32_t a = sub ? as : a0;
  uint32_t hi = (a >> 3) + ((sub ? (1023u - 127u - 24u) : (1023u - 127u)) << 20);
  hi = a0 >= 0x7f800000u ? ((a0 >> 3) | 0x7ff00000u) : hi;
  hi = a0 == 0u ? 0u : hi;
  return __hiloint2double((int)(hi | s), (int)(a << 29));
}
__device__ __forceinline__ double widen_f32(double v) { return v; }

}  // namespace pa
