// precision.cuh -- the arithmetic policies of the time-step kernels.
//
// A policy fixes how the synaptic conductances g (the exponential synapse's
// state, decayed every step by the exact factor exp(-dt/tau)), the event
// weights, the STDP traces, the per-CV synaptic sums (the synapses' share of
// the backward-Euler row of Eq. cable) and the cable solve itself are stored
// and computed.  HH, calcium and the slow plasticity state (GB w, STC h/z/p,
// STDP w) are FP64 in PA_FP64 and PA_MIXED.
//
//   PrecF64  (PA_FP64)  everything FP64, operation for operation the plain
//                       definition (bit-identical to the FP64 oracle);
//   PrecMix  (PA_MIXED) g is an unevaluated sum of two floats (float-float,
//                       about 48 significand bits) decayed and summed on the
//                       FP32 pipes; STDP traces FP32; event weights FP64 (read
//                       at events only); the per-CV sums, V, the cable
//                       coefficients and the elimination scratch are
//                       float-float pairs too, and the row's assembly,
//                       elimination and back substitution run in float-float
//                       on the FP32 pipes (RowFF);
//   PrecF32  (PA_FP32)  g, weights, traces and the per-CV sums plain FP32, and
//                       the mechanisms in FP32: HH rates and gates, calcium,
//                       the GB / STC / STDP increments (the slow state they
//                       accumulate into stays FP64); the cable solve FP64.
//
// Why the conductance path needs more than FP32 in PA_MIXED (measured with a
// CPU emulation of each variant against the FP64 oracle, recurrent tagging-
// and-capture network at dt = 0.2 ms, open loop): a stored FP32 conductance
// is re-rounded every step, and those errors random-walk over the hundreds of
// steps a conductance lives; on an HH soma near threshold the resulting
// voltage noise moves interpolated crossings by up to 7e-3 ms.  Even a single
// static rounding of every event weight to FP32 moves them by 2e-3 ms, and
// per-CV sums rounded to FP32 each step by up to 1e-3 ms.  Float-float keeps
// the per-step rounding near 2^-47 while the work stays off the FP64 pipe,
// where every warp instruction holds its scheduler's FP64 unit for 64 cycles
// on this GPU (an FP32 addition chains at 4.5).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "int_arith.cuh"

namespace pa {

// ---------------------------------------------------------------------------
// Float-float arithmetic.  Error-free transformations: TwoSum (Knuth), Fast2Sum
// (Dekker; needs |a| >= |b| or a = 0) and the FMA-based exact product.  Spelled
// with explicitly rounded intrinsics so that no contraction alters them.
__device__ __forceinline__ float2 ff_fast2sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_twosum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, err);
}
// a + b of two normalised float-float values
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = ff_twosum(a.x, b.x);
  return ff_fast2sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
// a + b without the final normalisation (a running sum over a short run of
// synapses: lo collects the exact rounding errors of the hi additions and the
// lo parts; it is normalised once, when the run is turned into FP64)
__device__ __forceinline__ float2 ff_add_acc(float2 a, float2 b) {
  const float2 s = ff_twosum(a.x, b.x);
  return make_float2(s.x, __fadd_rn(a.y, __fadd_rn(b.y, s.y)));
}
// a * c with the constant c = ch + cl given as two floats
__device__ __forceinline__ float2 ff_mul(float2 a, float ch, float cl) {
  const float p = __fmul_rn(a.x, ch);
  float e = __fmaf_rn(a.x, ch, -p);
  e = __fmaf_rn(a.x, cl, e);
  e = __fmaf_rn(a.y, ch, e);
  return ff_fast2sum(p, e);
}
// a double split into the nearest float and the float nearest the remainder
__device__ __forceinline__ float2 ff_from_d(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
}
// hi + lo in FP64: exact widening of both parts on the integer pipes, one FP64
// addition (exact while the parts' exponents differ by at most 29)
__device__ __forceinline__ double ff_to_d(float2 a) {
  return __dadd_rn(widen_f32(a.x), widen_f32(a.y));
}

// Sums of plain numbers, never contracted: both cell bins (and any compiler
// schedule) produce the same values.
__device__ __forceinline__ float tm_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float tm_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double tm_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double tm_add(double a, double b) { return __dadd_rn(a, b); }

// ---------------------------------------------------------------------------
// Row arithmetic of the cable solve (assembly, elimination, back
// substitution).  RowD: FP64, the plain operations (PA_FP64, where they are the
// oracle's operation for operation, and PA_FP32).  RowFF (PA_MIXED): values as
// float-float pairs (hi + lo, about 48 significand bits) on the FP32 pipes:
// additions by TwoSum, products by the FMA-exact product, the reciprocal by
// one Newton step from the FP32 approximation (relative error about 2^-45).
// Voltages, cable coefficients, per-CV sums and the elimination scratch are
// stored in the row's own form, so the solve needs no conversion.
struct RowD {
  using R = double;
  __device__ static __forceinline__ R add(R a, R b) { return a + b; }
  __device__ static __forceinline__ R mul(R a, R b) { return a * b; }
  __device__ static __forceinline__ R fma(R a, R b, R c) { return ::fma(a, b, c); }
  // c - a b
  __device__ static __forceinline__ R fnma(R a, R b, R c) { return ::fma(-a, b, c); }
  // a non-first child enters its parent's row by fused multiply-adds (the
  // oracle's operations); its fork-stack entry holds (f, x', coupling)
  static constexpr bool kProdStack = false;
  __device__ static __forceinline__ R rcp(R d) { return rcp_rn_pos(d); }
  __device__ static __forceinline__ double to_d(R a) { return a; }
  __device__ static __forceinline__ R from_d(double x) { return x; }
  __device__ static __forceinline__ R zero() { return 0.0; }
};
struct RowFF {
  using R = float2;
  __device__ static __forceinline__ R add(R a, R b) { return ff_add(a, b); }
  __device__ static __forceinline__ R mul(R a, R b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_fast2sum(p, e);
  }
  // a b + c and c - a b: the product (ph, pl) exact in ph and FMA-formed in pl,
  // folded into c by TwoSum without normalising the product first (a shorter
  // dependent chain than a product followed by an addition)
  __device__ static __forceinline__ R fma(R a, R b, R c) { return fold(a, b, c, 1.0f); }
  __device__ static __forceinline__ R fnma(R a, R b, R c) { return fold(a, b, c, -1.0f); }
  // a non-first child enters its parent's row as the normalised products
  // (coupling f, coupling x') subtracted, so that a fork-stack entry holds the
  // two products (16 bytes) instead of f, x' and the coupling
  static constexpr bool kProdStack = true;
  __device__ static __forceinline__ R sub(R c, R p) {
    return ff_add(c, make_float2(-p.x, -p.y));
  }
  __device__ static __forceinline__ R fold(R a, R b, R c, float sg) {
    const float ph = __fmul_rn(a.x, b.x);
    float pl = __fmaf_rn(a.x, b.x, -ph);
    pl = __fmaf_rn(a.x, b.y, pl);
    pl = __fmaf_rn(a.y, b.x, pl);
    const float2 s = ff_twosum(c.x, sg * ph);  // (sg = +-1: exact)
    return ff_fast2sum(s.x, __fadd_rn(s.y, __fmaf_rn(sg, pl, c.y)));
  }
  // 1/d for d > 0: y0 = rcp.approx(hi), then y0 + y0 (1 - d y0) with the
  // residual formed by FMAs
  __device__ static __forceinline__ R rcp(R d) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d.x));
    float e = __fmaf_rn(-d.x, y, 1.0f);
    e = __fmaf_rn(-d.y, y, e);
    return ff_fast2sum(y, __fmul_rn(y, e));
  }
  __device__ static __forceinline__ double to_d(R a) { return ff_to_d(a); }
  __device__ static __forceinline__ R from_d(double x) { return ff_from_d(x); }
  __device__ static __forceinline__ R zero() { return make_float2(0.0f, 0.0f); }
};

// ---------------------------------------------------------------------------
// Reversal potentials of exactly +0 (EZ).  For a finite g, g (+0) is the zero
// with g's sign, and a sum of signed zeros is -0 exactly when every term is
// -0: the IEEE results follow from the sign bits alone, so a model whose every
// stream has E = +0 forms its per-CV g E sums on the integer pipes.
__device__ __forceinline__ double zero_of(double g) {
  return __longlong_as_double(__double_as_longlong(g) & (long long)0x8000000000000000ull);
}
__device__ __forceinline__ float zero_of(float g) {
  return __uint_as_float(__float_as_uint(g) & 0x80000000u);
}
// a + b for signed zeros a, b
__device__ __forceinline__ double zsum(double a, double b) {
  return __longlong_as_double(__double_as_longlong(a) & __double_as_longlong(b));
}
__device__ __forceinline__ float zsum(float a, float b) {
  return __uint_as_float(__float_as_uint(a) & __float_as_uint(b));
}

// ---------------------------------------------------------------------------
// Per-CV sum accumulators over one run of same-CV synapses of a stream, in the
// canonical synapse order.  start() opens the run with its first synapse (from
// zero on the CV's first run of the step, else continuing the sums an earlier
// stream left); add() takes the next synapse; store() writes the CV's sums.
// A synapse's contribution C is formed once, on its own lane (contrib); the
// wide kernel hands contributions to other lanes by shuffle (shfl_c).  With
// EZ (every stream's E is +0) the g E sums are signed zeros (zero_of, zsum).
__device__ __forceinline__ bool is_zero_bits(double x) {
  return (__double_as_longlong(x) << 1) == 0;
}
__device__ __forceinline__ bool is_zero_bits(float x) { return (__float_as_uint(x) << 1) == 0u; }
__device__ __forceinline__ bool is_pos_zero_bits(double x) { return __double_as_longlong(x) == 0; }
__device__ __forceinline__ bool is_pos_zero_bits(float x) { return __float_as_uint(x) == 0u; }
// a + (a run of exact zeros, any_pos: one of them is +0): a nonzero a is
// unchanged, a zero a becomes +0 when any term is +0 (the IEEE sum of zeros,
// -0 only when every term is -0)
__device__ __forceinline__ double zero_join(double a, bool any_pos) {
  return (any_pos && is_zero_bits(a)) ? __longlong_as_double(0) : a;
}
__device__ __forceinline__ float zero_join(float a, bool any_pos) {
  return (any_pos && is_zero_bits(a)) ? __uint_as_float(0u) : a;
}

template <class T>
struct AccPlain {  // FP64 / FP32: gs = gs + g, es = es + g E per synapse
  struct C {
    T g, ge;
  };
  // a run of contributions that are all exact zeros folds on the integer
  // pipes (add_zeros): the result of the in-order sum follows from the signs
  static constexpr bool kZeroRuns = true;
  __device__ static __forceinline__ bool zero_c(C c) { return is_zero_bits(c.g) && is_zero_bits(c.ge); }
  __device__ static __forceinline__ bool pos_zero_g(C c) { return is_pos_zero_bits(c.g); }
  __device__ static __forceinline__ bool pos_zero_e(C c) { return is_pos_zero_bits(c.ge); }
  __device__ __forceinline__ void add_zeros(bool any_pos_g, bool any_pos_e) {
    g = zero_join(g, any_pos_g);
    e = zero_join(e, any_pos_e);
  }
  template <bool EZ>
  __device__ static __forceinline__ T ge_of(T gv, T E) {
    return EZ ? zero_of(gv) : tm_mul(gv, E);
  }
  template <bool EZ>
  __device__ static __forceinline__ T e_add(T a, T b) {
    return EZ ? zsum(a, b) : tm_add(a, b);
  }
  template <bool EZ>
  __device__ static __forceinline__ C contrib(T gv, T E) { return C{gv, ge_of<EZ>(gv, E)}; }
  __device__ static __forceinline__ C shfl_c(C c, int src) {
    return C{__shfl_sync(0xffffffffu, c.g, src), __shfl_sync(0xffffffffu, c.ge, src)};
  }
  template <bool EZ>
  __device__ __forceinline__ void start_c(C c, bool first, const T* gs, const T* es,
                                          uint32_t ce) {
    if (first) {
      g = c.g;
      e = c.ge;
    } else {
      g = tm_add(gs[ce], c.g);
      e = e_add<EZ>(es[ce], c.ge);
    }
  }
  template <bool EZ>
  __device__ __forceinline__ void add_c(C c) {
    g = tm_add(g, c.g);
    e = e_add<EZ>(e, c.ge);
  }
  T g, e;
  template <bool EZ>
  __device__ __forceinline__ void start(T gv, T E, bool first, const T* gs, const T* es,
                                        uint32_t ce) {
    const T ge = ge_of<EZ>(gv, E);
    if (first) {
      g = gv;
      e = ge;
    } else {
      g = tm_add(gs[ce], gv);
      e = e_add<EZ>(es[ce], ge);
    }
  }
  template <bool EZ>
  __device__ __forceinline__ void add(T gv, T E) {
    const T ge = ge_of<EZ>(gv, E);
    g = tm_add(g, gv);
    e = e_add<EZ>(e, ge);
  }
  template <bool EZ>
  __device__ __forceinline__ void store(T* gs, T* es, uint32_t ce, T) const {
    gs[ce] = g;
    es[ce] = e;
  }
  __device__ __forceinline__ AccPlain shfl(int src) const {
    AccPlain r;
    r.g = __shfl_sync(0xffffffffu, g, src);
    r.e = __shfl_sync(0xffffffffu, e, src);
    return r;
  }
};

struct AccFF {  // mixed: the run's conductance in float-float, stored as a normalised pair
  using C = float2;
  static constexpr bool kZeroRuns = false;
  template <bool EZ>
  __device__ static __forceinline__ C contrib(float2 gv, float2) { return gv; }
  __device__ static __forceinline__ C shfl_c(C c, int src) {
    return make_float2(__shfl_sync(0xffffffffu, c.x, src), __shfl_sync(0xffffffffu, c.y, src));
  }
  template <bool EZ>
  __device__ __forceinline__ void start_c(C c, bool first_on_cv, const float2*, const float2*,
                                          uint32_t) {
    g = c;
    first = first_on_cv;
  }
  template <bool EZ>
  __device__ __forceinline__ void add_c(C c) { g = ff_add_acc(g, c); }
  float2 g;
  bool first;
  template <bool EZ>
  __device__ __forceinline__ void start(float2 gv, float2, bool first_on_cv, const float2*,
                                        const float2*, uint32_t) {
    g = gv;
    first = first_on_cv;
  }
  template <bool EZ>
  __device__ __forceinline__ void add(float2 gv, float2) { g = ff_add_acc(g, gv); }
  template <bool EZ>
  __device__ __forceinline__ void store(float2* gs, float2* es, uint32_t ce, float2 E) const {
    const float2 s = ff_fast2sum(g.x, g.y);
    // (EZ: the g E sums are zeros the row never reads; written as zeros)
    const float2 se = EZ ? make_float2(zero_of(s.x), 0.0f) : ff_mul(s, E.x, E.y);
    if (first) {
      gs[ce] = s;
      es[ce] = se;
    } else {
      gs[ce] = ff_add(gs[ce], s);
      es[ce] = EZ ? se : ff_add(es[ce], se);
    }
  }
  __device__ __forceinline__ AccFF shfl(int src) const {
    AccFF r;
    r.g.x = __shfl_sync(0xffffffffu, g.x, src);
    r.g.y = __shfl_sync(0xffffffffu, g.y, src);
    r.first = __shfl_sync(0xffffffffu, (int)first, src) != 0;
    return r;
  }
};

// A double narrowed to a float by truncation on the integer pipes (sign,
// exponent rebiased, the top 23 fraction bits); values below the float range
// flush to zero.  The FP32-mechanism policy reads its FP64 slow state this way
// (the variables it narrows are bounded: calcium, weights, tags, voltages).
__device__ __forceinline__ float narrow_rz(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const uint32_t f = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t s = hi & 0x80000000u;
  return __uint_as_float(e <= 0 ? s : (s | ((uint32_t)e << 23) | f));
}

// ---------------------------------------------------------------------------
// The policies.  G: conductance element; W: event weight element; T: STDP
// trace element; S: per-CV sum element; Ec / Dc: the stream's reversal
// potential and decay factor as the policy uses them.
struct PrecF64 {
  using G = double;
  using W = double;
  using T = double;
  using S = double;
  using Ec = double;
  using Dc = double;
  using Acc = AccPlain<double>;
  using Row = RowD;
  static constexpr bool kDeriveEM = false;  // the leak E-term row is read (the oracle's value)
  static constexpr int kId = 0;
  static constexpr bool kMech32 = false;  // HH, calcium, plasticity increments in FP64
  __device__ static __forceinline__ Ec e_const(double e) { return e; }
  __device__ static __forceinline__ Dc d_const(double d) { return d; }
  __device__ static __forceinline__ G add_w(G g, W w) { return g + w; }
  __device__ static __forceinline__ G add_d(G g, double x) { return g + x; }
  __device__ static __forceinline__ G decay(G g, Dc d) { return g * d; }
  __device__ static __forceinline__ G zero() { return 0.0; }
  __device__ static __forceinline__ G shfl(G g, int src) { return __shfl_sync(0xffffffffu, g, src); }
  __device__ static __forceinline__ Row::R sum_r(S s) { return s; }
  __device__ static __forceinline__ S s_zero() { return 0.0; }
};

struct PrecMix {
  using G = float2;
  using W = double;
  using T = float;
  using S = float2;   // per-CV sums as float-float pairs
  using Ec = float2;  // E as hi + lo
  using Dc = float2;  // exp(-dt/tau) as hi + lo
  using Acc = AccFF;
  using Row = RowFF;
  // a passive dendrite row's leak E-term formed as (C/dt) k where the model
  // allows it (EpochArgs::em_derived), instead of read
  static constexpr bool kDeriveEM = true;
  static constexpr int kId = 1;
  static constexpr bool kMech32 = false;
  __device__ static __forceinline__ Ec e_const(double e) { return ff_from_d(e); }
  __device__ static __forceinline__ Dc d_const(double d) { return ff_from_d(d); }
  __device__ static __forceinline__ G add_w(G g, W w) { return ff_add(g, ff_from_d(w)); }
  __device__ static __forceinline__ G add_d(G g, double x) { return ff_add(g, ff_from_d(x)); }
  __device__ static __forceinline__ G decay(G g, Dc d) { return ff_mul(g, d.x, d.y); }
  __device__ static __forceinline__ G zero() { return make_float2(0.0f, 0.0f); }
  __device__ static __forceinline__ G shfl(G g, int src) {
    return make_float2(__shfl_sync(0xffffffffu, g.x, src), __shfl_sync(0xffffffffu, g.y, src));
  }
  __device__ static __forceinline__ Row::R sum_r(S s) { return s; }
  __device__ static __forceinline__ S s_zero() { return make_float2(0.0f, 0.0f); }
};

struct PrecF32 {
  using G = float;
  using W = float;
  using T = float;
  using S = float;
  using Ec = float;
  using Dc = float;
  using Acc = AccPlain<float>;
  using Row = RowD;
  static constexpr bool kDeriveEM = false;
  static constexpr int kId = 2;
  // HH rates and gates, calcium and the GB / STC / STDP increments in FP32
  // (exponential integration with CUDA's expf); the slow state w, h, z, p
  // accumulates the increments in FP64
  static constexpr bool kMech32 = true;
  __device__ static __forceinline__ Ec e_const(double e) { return (float)e; }
  __device__ static __forceinline__ Dc d_const(double d) { return (float)d; }
  __device__ static __forceinline__ G add_w(G g, W w) { return __fadd_rn(g, w); }
  __device__ static __forceinline__ G add_d(G g, double x) { return __fadd_rn(g, (float)x); }
  __device__ static __forceinline__ G decay(G g, Dc d) { return __fmul_rn(g, d); }
  __device__ static __forceinline__ G zero() { return 0.0f; }
  __device__ static __forceinline__ G shfl(G g, int src) { return __shfl_sync(0xffffffffu, g, src); }
  __device__ static __forceinline__ Row::R sum_r(S s) { return widen_f32(s); }
  __device__ static __forceinline__ S s_zero() { return 0.0f; }
};

}  // namespace pa
