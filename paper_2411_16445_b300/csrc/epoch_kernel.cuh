// epoch_kernel.cuh -- the fused per-epoch time-step kernel.
//
// One warp advances one group of 32 cells (one thread per cell) through the
// steps [k_begin, k_end) of one min-delay epoch.  Cells do not interact inside
// an epoch: every synaptic event produced by a spike in this epoch is due at
// least one epoch later, and the POST_EVENT hook only touches the spiking
// cell's own synapses.  So the launch needs no inter-block synchronisation and
// contains no waits.
//
// Per step and cell (Sec. "Design and Implementation" of arXiv 2411.16445):
//   a. synapse streams: deliver this step's pre / delayed-calcium events (bit
//      (k - k0) of the synapse's epoch mask), the POST_EVENT of a spike in the
//      previous step, scatter g and g*E into the per-CV accumulators, then
//      decay g, calcium and STDP traces and take the forward-Euler step of the
//      plasticity ODEs (Eqs. weight_graupner_brunel, early_phase_weight,
//      late_phase_weight, prp_single_comp);
//   b. backward pass over rows n-1..0: assemble the backward-Euler row of the
//      cable equation (Eq. cable) and eliminate it into its parent (Hines);
//   c. forward pass over rows 0..n-1: back substitution -> V^{k+1};
//   d. soma: HH gates by exponential integration at V^{k+1}; threshold
//      detection; warp-ballot compaction of the spikes.
//
// Arithmetic: the FP64 instantiation is compiled without contraction so that
// every operation and its order equal the plain definition (one correctly
// rounded reciprocal per row, computed on the integer pipes by rcp_rn_pos;
// fused multiply-adds only where written as fma), and the
// model's exponential is the Cody-Waite + degree-13 Taylor function below.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "engine.h"
#include "int_arith.cuh"
#include "precision.cuh"
#include "prp_field.cuh"
#include "rng.cuh"

namespace pa {

// ---------------------------------------------------------------------------
// The model's exponential (the FP64 path): x = k ln2 + r with ln2 split into a
// 32-bit head (ln2 rounded to a double with its low 21 mantissa bits cleared)
// and a tail; exp(r) by the degree-13 Taylor polynomial sum r^j / j! in
// Horner form with fused multiply-adds; scaling by 2^k through the exponent
// field.  |r| <= ln2/2, so the truncation error is below r^14/14! < 5e-18.
__device__ __forceinline__ double model_exp(double x) {
  const double ln2_hi = 6.93147180369123816490e-01;
  const double ln2_lo = 1.9082149292705877e-10;
  const double inv_ln2 = 1.4426950408889634;
  if (x != x) return x;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
  if (x < -708.0) return 0.0;
  double kd = rint(x * inv_ln2);
  double r = (x - kd * ln2_hi) - kd * ln2_lo;
  double p = 1.6059043836821613e-10;            // 1/13!
  p = fma(p, r, 2.08767569878681e-09);           // 1/12!
  p = fma(p, r, 2.505210838544172e-08);          // 1/11!
  p = fma(p, r, 2.755731922398589e-07);          // 1/10!
  p = fma(p, r, 2.7557319223985893e-06);         // 1/9!
  p = fma(p, r, 2.48015873015873e-05);           // 1/8!
  p = fma(p, r, 0.0001984126984126984);          // 1/7!
  p = fma(p, r, 0.001388888888888889);           // 1/6!
  p = fma(p, r, 0.008333333333333333);           // 1/5!
  p = fma(p, r, 0.041666666666666664);           // 1/4!
  p = fma(p, r, 0.16666666666666666);            // 1/3!
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  long long k = (long long)kd;
  return p * __longlong_as_double((k + 1023LL) << 52);
}

// Hodgkin-Huxley kinetics (textbook, rest -65 mV, 6.3 C) with the model's
// exponential, in FP64 in both precisions: FP32 rate functions (CUDA's expf)
// shift the phase of tonic firing by ~2e-5 V within a second, twice the mixed
// path's tolerance, while the soma is one CV of hundreds.
struct HH64 {
  __device__ static __forceinline__ double vtrap(double x, double y) {
    double u = x / y;
    if (fabs(u) < 1e-6) return y * (1.0 - 0.5 * u);
    return x / (model_exp(u) - 1.0);
  }
  __device__ static __forceinline__ void rates(double v, double& am, double& bm, double& ah,
                                               double& bh, double& an, double& bn) {
    am = 0.1 * vtrap(-(v + 40.0), 10.0);
    bm = 4.0 * model_exp(-(v + 65.0) / 18.0);
    ah = 0.07 * model_exp(-(v + 65.0) / 20.0);
    bh = 1.0 / (model_exp(-(v + 35.0) / 10.0) + 1.0);
    an = 0.01 * vtrap(-(v + 55.0), 10.0);
    bn = 0.125 * model_exp(-(v + 65.0) / 80.0);
  }
  __device__ static __forceinline__ double gate(double x, double a, double b, double dt) {
    double s = a + b;
    double xinf = a / s;
    return xinf + (x - xinf) * model_exp(-dt * s);
  }
};

// The same kinetics in FP32 with CUDA's expf (the FP32-mechanism policy).
struct HH32 {
  __device__ static __forceinline__ float vtrap(float x, float y) {
    const float u = x / y;
    if (fabsf(u) < 1e-6f) return y * (1.0f - 0.5f * u);
    return x / (expf(u) - 1.0f);
  }
  __device__ static __forceinline__ void rates(float v, float& am, float& bm, float& ah,
                                               float& bh, float& an, float& bn) {
    am = 0.1f * vtrap(-(v + 40.0f), 10.0f);
    bm = 4.0f * expf(-(v + 65.0f) / 18.0f);
    ah = 0.07f * expf(-(v + 65.0f) / 20.0f);
    bh = 1.0f / (expf(-(v + 35.0f) / 10.0f) + 1.0f);
    an = 0.01f * vtrap(-(v + 55.0f), 10.0f);
    bn = 0.125f * expf(-(v + 65.0f) / 80.0f);
  }
  __device__ static __forceinline__ float gate(float x, float a, float b, float dt) {
    const float s = a + b;
    const float xinf = a / s;
    return xinf + (x - xinf) * expf(-dt * s);
  }
};

// An HH soma's gates m, h, n: loaded at the start of a launch, the membrane
// conductance and E-weighted sum the assembly takes at V^k, the exponential
// update at V^{k+1}, stored at the end.  FP64 (HH64) or, for the
// FP32-mechanism policy, FP32 (HH32) with the results widened for the FP64
// assembly; the gate array holds doubles in both.
template <bool kF32>
struct SomaHH {
  double m = 0, h = 0, n = 0;
  __device__ __forceinline__ void load(const double* gate, int64_t nl, int64_t L) {
    m = gate[L]; h = gate[nl + L]; n = gate[2 * nl + L];
  }
  __device__ __forceinline__ void store(double* gate, int64_t nl, int64_t L) const {
    gate[L] = m; gate[nl + L] = h; gate[2 * nl + L] = n;
  }
  // per-soma constants are reloaded here rather than kept live
  __device__ __forceinline__ void currents(const EpochArgs& A, int64_t L, double& gmt,
                                           double& emt) const {
    const double gna = __ldg(&A.hh_g[L]), gk = __ldg(&A.hh_g[A.n_lanes + L]),
                 gl = __ldg(&A.hh_g[2 * A.n_lanes + L]);
    const double ena = __ldg(&A.hh_e[L]), ek = __ldg(&A.hh_e[A.n_lanes + L]),
                 el = __ldg(&A.hh_e[2 * A.n_lanes + L]);
    const double mmmh = ((m * m) * m) * h;
    const double nnnn = ((n * n) * n) * n;
    const double g1 = gna * mmmh;
    const double g2 = gk * nnnn;
    gmt = (g1 + g2) + gl;
    emt = ((g1 * ena) + (g2 * ek)) + (gl * el);
  }
  __device__ __forceinline__ void update(double v, double dt) {
    double am, bm, ah, bh, an, bn;
    HH64::rates(v, am, bm, ah, bh, an, bn);
    m = HH64::gate(m, am, bm, dt);
    h = HH64::gate(h, ah, bh, dt);
    n = HH64::gate(n, an, bn, dt);
  }
};
template <>
struct SomaHH<true> {
  float m = 0, h = 0, n = 0;
  __device__ __forceinline__ void load(const double* gate, int64_t nl, int64_t L) {
    m = narrow_rz(gate[L]); h = narrow_rz(gate[nl + L]); n = narrow_rz(gate[2 * nl + L]);
  }
  __device__ __forceinline__ void store(double* gate, int64_t nl, int64_t L) const {
    gate[L] = widen_f32(m); gate[nl + L] = widen_f32(h); gate[2 * nl + L] = widen_f32(n);
  }
  __device__ __forceinline__ void currents(const EpochArgs& A, int64_t L, double& gmt,
                                           double& emt) const {
    const float gna = narrow_rz(__ldg(&A.hh_g[L])), gk = narrow_rz(__ldg(&A.hh_g[A.n_lanes + L])),
                gl = narrow_rz(__ldg(&A.hh_g[2 * A.n_lanes + L]));
    const float ena = narrow_rz(__ldg(&A.hh_e[L])), ek = narrow_rz(__ldg(&A.hh_e[A.n_lanes + L])),
                el = narrow_rz(__ldg(&A.hh_e[2 * A.n_lanes + L]));
    const float mmmh = ((m * m) * m) * h;
    const float nnnn = ((n * n) * n) * n;
    const float g1 = gna * mmmh;
    const float g2 = gk * nnnn;
    gmt = widen_f32((g1 + g2) + gl);
    emt = widen_f32(((g1 * ena) + (g2 * ek)) + (gl * el));
  }
  __device__ __forceinline__ void update(double v, double dt) {
    float am, bm, ah, bh, an, bn;
    const float vf = narrow_rz(v), dtf = narrow_rz(dt);
    HH32::rates(vf, am, bm, ah, bh, an, bn);
    m = HH32::gate(m, am, bm, dtf);
    h = HH32::gate(h, ah, bh, dtf);
    n = HH32::gate(n, an, bn, dtf);
  }
};

// Bounds checks of the checked build (compiled with -DPA_CHECKED, for the
// small parity cases): an index outside its array sets bit 3 of the model's
// error word (reported by the next pa_sync) and the access is skipped.  In the
// normal build PA_IN is the constant true.
#ifdef PA_CHECKED
__device__ __forceinline__ bool pa_in_range(int32_t* flags, int64_t i, int64_t n) {
  if (i >= 0 && i < n) return true;
  atomicOr(flags, 8);
  return false;
}
#define PA_IN(A, i, n) pa_in_range((A).err_flags, (int64_t)(i), (int64_t)(n))
#else
#define PA_IN(A, i, n) true
#endif

__device__ __forceinline__ uint32_t elem_of(int32_t row_base, int32_t row, int lane) {
  return ((uint32_t)(row_base + row) << 5) | (uint32_t)lane;
}


// ---------------------------------------------------------------------------
// Bulk TMA row staging.  Each warp owns a ring of kStages shared-memory stages;
// the chunk sizes (rows per copy in the backward and forward passes) and the
// register budget form the kernel's "shape", chosen per model (autotuned);
// one elected lane issues one-dimensional bulk copies (cp.async.bulk, TMA) of
// the next chunk of rows of every array the pass reads -- a group's rows are
// contiguous in HBM, 32 lanes per row -- and arms the stage's mbarrier with the
// byte count; all lanes wait on the barrier (bounded) before reading.
constexpr int kStages = 2;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking test of the phase
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the phase did not complete within `limit` polls (the
// first a non-blocking test, the others potentially blocking try_waits)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t limit = kSpinLimit) {
  if (mbar_test(bar, parity)) return true;
  for (uint32_t it = 1; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// generic-proxy global writes of this thread become visible to later TMA reads
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// generic-proxy shared reads of this thread are ordered before later TMA writes
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory layout of one warp's stages for a given precision / tree flag.
template <class PR, bool TREE, int kRowsBack, int kRowsFwd, int kStackDepth, bool EZ>
struct Stage {
  // bytes per row (32 lanes) of each staged array.  With fork stacks a tree
  // stages one flag byte per row (fork push / pop, parent = previous row,
  // children through the list); without them, the parent and first-other-child
  // rows.
  static constexpr bool kStacks = TREE && kStackDepth > 0;  // fork stacks in use
  // kE: the leak E-term row, not staged by policies that form it from C/dt
  // (their rare groups that cannot read it from memory)
  static constexpr int kD = 32 * 8, kE = PR::kDeriveEM ? 0 : kD,
                       kM = 32 * (int)sizeof(typename PR::S),
                       kMES = EZ ? 0 : kM,  // the g E sums (not staged with every E = +0)
                       kI = (TREE && !kStacks) ? 32 * 2 : 0, kT = kStacks ? 32 : 0;
  // backward pass: V, C/dt, diagonal, leak E term, axial coupling, synaptic sums,
  // tree rows
  static constexpr int oV = 0, oCDT = oV + kRowsBack * kD, oDC = oCDT + kRowsBack * kD,
                       oEM = oDC + kRowsBack * kD, oA = oEM + kRowsBack * kE,
                       oGS = oA + kRowsBack * kD, oES = oGS + kRowsBack * kM,
                       oPAR = oES + kRowsBack * kMES, oOCH = oPAR + kRowsBack * kI,
                       oTF = oOCH + kRowsBack * kI, kBackBytes = oTF + kRowsBack * kT;
  static constexpr int kBackRow = 4 * kD + kE + kM + kMES + 2 * kI + kT;
  // forward pass: f, x', tree rows
  static constexpr int fF = 0, fXP = fF + kRowsFwd * kD, fPAR = fXP + kRowsFwd * kD,
                       fTF = fPAR + kRowsFwd * kI, kFwdBytes = fTF + kRowsFwd * kT;
  static constexpr int kFwdRow = 2 * kD + kI + kT;
  static constexpr int kBytes = (kBackBytes > kFwdBytes ? kBackBytes : kFwdBytes);
  // fork stacks (trees): the backward pass keeps (f, x', coupling) of up to
  // kStackB pending one-other-children per lane, the forward pass V of up to
  // kStackF pending forks; deeper entries are read back from global memory
  // (the depth is part of the kernel shape: deep stacks where many forks nest,
  // shallow ones where longer backward chunks take the shared memory)
  static constexpr int kStackB = kStackDepth, kStackF = 2 * kStackDepth;
  // a backward entry: (f, x', coupling), or the two products (16 bytes)
  static constexpr int kSE = PR::Row::kProdStack ? 16 : 24;
  static constexpr int kStackBytes = kStacks ? 32 * kStackB * kSE : 0;
  static_assert(32 * kStackF * 8 <= 32 * kStackB * kSE, "forward stack fits the region");
  static constexpr int kWarpBytes = kStages * kBytes + 64 + kStackBytes;  // + mbarriers
};

// A non-first child entering its parent's row: d - f a, b - a x' (by fused
// multiply-adds, or as subtracted products where the row form keeps them)
template <class RW>
__device__ __forceinline__ void other_child(typename RW::R a, typename RW::R f,
                                            typename RW::R x, typename RW::R& d,
                                            typename RW::R& b) {
  if constexpr (RW::kProdStack) {
    d = RW::sub(d, RW::mul(a, f));
    b = RW::sub(b, RW::mul(a, x));
  } else {
    d = RW::fnma(f, a, d);
    b = RW::fnma(a, x, b);
  }
}

// b + es for a CV whose g E sum es is a signed zero (every stream's E is +0):
// b itself unless b is -0, when the stored es decides (a call, so that the
// compiler cannot turn the rare branch into FP64 work on every row).
template <class TS>
__device__ __noinline__ double ez_fix(double b, const TS* es, uint32_t e) {
  return b + widen_f32(es[e]);
}
template <class TS>
__device__ __forceinline__ double ez_add(double b, const TS* es, uint32_t e) {
  return __double_as_longlong(b) == (long long)0x8000000000000000ull ? ez_fix(b, es, e) : b;
}

// One synapse's step (rows a1, a2, a4): this step's conductance event, the
// delayed calcium event and the POST_EVENT of the cell's spike in the previous
// step, then the plasticity update of its kind (Eqs. weight_graupner_brunel,
// early_phase_weight, late_phase_weight, stdp_ode_1-3); stores the synapse's
// plastic state and returns the conductance entering this step's per-CV sums.
// cc, wv, zv are the synapse's calcium, weight (h for STC) and z as loaded by
// the caller (only those its kind uses); S accumulates |h - h0| (STC).
template <class PR>
__device__ __forceinline__ typename PR::G syn_update(const StreamParams& P, const StreamDev& D,
                                                     uint32_t e, bool pre, bool capre, bool post,
                                                     typename PR::G gv, double cc, double wv,
                                                     double zv, double prp, int64_t k, double dt,
                                                     uint64_t seed, double& S) {
  using TW = typename PR::W;
  if (P.kind == SK_EXPSYN) {
    if (pre) gv = PR::add_w(gv, ((const TW*)D.weight)[e]);
  } else if (P.kind == SK_GB && PR::kMech32) {
    // FP32 mechanism: calcium and the increment of Eq. weight_graupner_brunel
    // in FP32, accumulated into the FP64 w
    if (pre) gv = PR::add_w(gv, ((const TW*)D.weight)[e]);
    const StreamParams::F32& Q = P.f;
    float c = narrow_rz(cc);
    if (capre) c = c + Q.c_pre;
    if (post) c = c + Q.c_post;
    const float w = narrow_rz(wv);
    const float Aw = (w * (1.0f - w)) * (Q.w_star - w);
    const float Pw = (c > Q.theta_p) ? Q.gamma_p * (1.0f - w) : 0.0f;
    const float Dw = (c > Q.theta_d) ? Q.gamma_d * w : 0.0f;
    double wn = wv + widen_f32(Q.rate_w * ((Pw - Aw) - Dw));
    const int nth = (c > Q.theta_p) + (c > Q.theta_d);
    if (P.sigma > 0.0 && nth > 0)
      wn = __dadd_rn(wn, __dmul_rn(P.amp[nth], model_normal(seed, (uint64_t)D.nid[e], k)));
    D.w[e] = wn;
    D.c[e] = widen_f32(c * Q.decay_c);
  } else if (P.kind == SK_GB) {
    if (pre) gv = PR::add_w(gv, ((const TW*)D.weight)[e]);
    if (capre) cc = cc + P.c_pre;
    if (post) cc = cc + P.c_post;
    const double w = wv;
    const double Aw = (w * (1.0 - w)) * (P.w_star - w);
    const double Pw = (cc > P.theta_p) ? P.gamma_p * (1.0 - w) : 0.0;
    const double Dw = (cc > P.theta_d) ? P.gamma_d * w : 0.0;
    double wn = w + P.rate_w * ((Pw - Aw) - Dw);
    // Eq. plasticity_noise_1, Euler-Maruyama, gated by the thresholds crossed
    const int nth = (cc > P.theta_p) + (cc > P.theta_d);
    if (P.sigma > 0.0 && nth > 0)
      wn = __dadd_rn(wn, __dmul_rn(P.amp[nth], model_normal(seed, (uint64_t)D.nid[e], k)));
    D.w[e] = wn;
    D.c[e] = cc * P.decay_c;
  } else if (P.kind == SK_STC && PR::kMech32) {
    // FP32 mechanism: calcium and the increments of Eqs. early_phase_weight and
    // late_phase_weight in FP32, accumulated into the FP64 h and z
    const StreamParams::F32& Q = P.f;
    const float h = narrow_rz(wv), z = narrow_rz(zv), pf = narrow_rz(prp);
    if (pre) gv = PR::add_w(gv, (TW)(((const TW*)D.weight)[e] * ((h + Q.h0 * z) / Q.h0)));
    float c = narrow_rz(cc);
    if (capre) c = c + Q.c_pre;
    if (post) c = c + Q.c_post;
    S = S + widen_f32(fabsf(h - Q.h0));
    const float T1 = ((h - Q.h0) > Q.theta_tag) ? (pf * Q.f_int) * (1.0f - z) : 0.0f;
    const float T2 = ((Q.h0 - h) > Q.theta_tag) ? (pf * Q.f_int) * (z + 0.5f) : 0.0f;
    D.z[e] = zv + widen_f32(Q.rate_z * (T1 - T2));
    const float Ph = (c > Q.theta_p) ? Q.gamma_p * (10.0f - h) : 0.0f;
    const float Dh = (c > Q.theta_d) ? Q.gamma_d * h : 0.0f;
    double hn = wv + widen_f32(Q.rate_h * ((0.1f * (Q.h0 - h) + Ph) - Dh));
    const int nth = (c > Q.theta_p) + (c > Q.theta_d);
    if (P.sigma > 0.0 && nth > 0)
      hn = __dadd_rn(hn, __dmul_rn(P.amp[nth], model_normal(seed, (uint64_t)D.nid[e], k)));
    D.w[e] = hn;
    D.c[e] = widen_f32(c * Q.decay_c);
  } else if (P.kind == SK_STC) {
    const double h = wv, z = zv;
    const double h0 = P.h0;
    if (pre) gv = PR::add_d(gv, (double)((const TW*)D.weight)[e] * ((h + h0 * z) / h0));
    if (capre) cc = cc + P.c_pre;
    if (post) cc = cc + P.c_post;
    S = S + fabs(h - h0);
    const double T1 = ((h - h0) > P.theta_tag) ? (prp * P.f_int) * (1.0 - z) : 0.0;
    const double T2 = ((h0 - h) > P.theta_tag) ? (prp * P.f_int) * (z + 0.5) : 0.0;
    D.z[e] = z + P.rate_z * (T1 - T2);
    const double Ph = (cc > P.theta_p) ? P.gamma_p * (10.0 - h) : 0.0;
    const double Dh = (cc > P.theta_d) ? P.gamma_d * h : 0.0;
    double hn = h + P.rate_h * ((0.1 * (h0 - h) + Ph) - Dh);
    // Eq. plasticity_noise_2
    const int nth = (cc > P.theta_p) + (cc > P.theta_d);
    if (P.sigma > 0.0 && nth > 0)
      hn = __dadd_rn(hn, __dmul_rn(P.amp[nth], model_normal(seed, (uint64_t)D.nid[e], k)));
    D.w[e] = hn;
    D.c[e] = cc * P.decay_c;
  } else if ((pre || post) && PR::kMech32) {  // SK_STDP, FP32 traces and increments
    using TT = typename PR::T;
    TT* AP = (TT*)D.apre;
    TT* AQ = (TT*)D.apost;
    const StreamParams::F32& Q = P.f;
    const float dtf = narrow_rz(dt);
    double w = D.w[e];
    float ap = (float)AP[e] * expf(-((float)(k - D.kpre[e]) * dtf) / Q.tau_pre);
    float aq = (float)AQ[e] * expf(-((float)(k - D.kpost[e]) * dtf) / Q.tau_post);
    if (pre) {
      const double wc = w < 0.0 ? 0.0 : (w > P.w_max ? P.w_max : w);
      gv = PR::add_w(gv, (TW)(((const TW*)D.weight)[e] * narrow_rz(wc)));
      ap = ap + Q.a_pre;
      w = w + widen_f32(aq);
      AP[e] = (TT)ap;
      D.kpre[e] = (int32_t)k;
    }
    if (post) {
      aq = aq + Q.a_post;
      w = w + widen_f32(ap);
      AQ[e] = (TT)aq;
      D.kpost[e] = (int32_t)k;
    }
    D.w[e] = w;
  } else if (pre || post) {  // SK_STDP: traces evaluated in closed form at events only
    using TT = typename PR::T;
    TT* AP = (TT*)D.apre;
    TT* AQ = (TT*)D.apost;
    double w = D.w[e];
    double ap = (double)AP[e] * model_exp(-((double)(k - D.kpre[e]) * dt) / P.tau_pre);
    double aq = (double)AQ[e] * model_exp(-((double)(k - D.kpost[e]) * dt) / P.tau_post);
    if (pre) {
      const double wc = w < 0.0 ? 0.0 : (w > P.w_max ? P.w_max : w);
      gv = PR::add_d(gv, (double)((const TW*)D.weight)[e] * wc);
      ap = ap + P.a_pre;
      w = w + aq;
      AP[e] = (TT)ap;
      D.kpre[e] = (int32_t)k;
    }
    if (post) {
      aq = aq + P.a_post;
      w = w + ap;
      AQ[e] = (TT)aq;
      D.kpost[e] = (int32_t)k;
    }
    D.w[e] = w;
  }
  return gv;
}

// One step of the lane's synapses of the heterosynaptic calcium stream (HCA),
// apart from the TMA-staged loop of the other kinds so that theirs stays as
// small as it is (HCA models are small; plain loads suffice).  Per synapse, in
// canonical order: Eq. ca_injection_current_spine (I jumps by I0 at an event),
// its calcium w gamma I / (2 F) summed per CV over each run into ca_src (the
// source of Eq. ca_diffusion_dendrite), Eq. heterosyn_weight by forward Euler
// with the CV's calcium before this step's field update, then I decays.  The
// synapses carry no conductance: where an HCA run is the first on its CV, the
// per-CV conductance sums start at zero there, as the loop of the other kinds
// would make them.
template <class PR>
__device__ __noinline__ void hca_stream(const EpochArgs& A, int s, int g, int lane, int32_t rb,
                                        int kk, int32_t slot) {
  const StreamParams& P = A.sp[s];
  const StreamDev& D = A.sd[s];
  const int32_t sb = D.sbase[g], nrow = D.sbase[g + 1] - sb;
  const uint64_t* cmg = D.cmask + (int64_t)slot * D.n_elem;
  using TS = typename PR::S;
  TS* GS = (TS*)A.gs;
  TS* ES = (TS*)A.es;
  double accq = 0.0;
  bool zero = false;
  for (int j = 0; j < nrow; ++j) {
    const uint32_t e = ((uint32_t)(sb + j) << 5) | (uint32_t)lane;
    const int32_t cvf = D.cvf[e];
    if (cvf < 0) continue;
    const uint32_t ce = elem_of(rb, cvf >> 3, lane);
    const bool pre = (cmg[e] >> kk) & 1ull;
    double cc = D.c[e];
    const double w = D.w[e], cl = A.ca_cv[ce];
    if (pre) cc = __dadd_rn(cc, P.c_pre);
    const double qv = __dmul_rn(w, __dmul_rn(P.hca_kq, cc));
    const double Pw = (cl > P.theta_p) ? __dmul_rn(P.hca_gpr, __dsub_rn(1.0, w)) : 0.0;
    const double Dw = (cl > P.theta_d) ? __dmul_rn(P.hca_gdr, w) : 0.0;
    D.w[e] = __dadd_rn(w, __dsub_rn(Pw, Dw));
    D.c[e] = __dmul_rn(cc, P.decay_c);
    if (cvf & 2) zero = cvf & 1;  // the run is the first on its CV this step
    accq = (cvf & 2) ? qv : __dadd_rn(accq, qv);
    if (cvf & 4) {
      A.ca_src[ce] = accq;
      if (zero) {
        GS[ce] = PR::s_zero();
        ES[ce] = PR::s_zero();
      }
    }
  }
}

// The launch window of one warp: group g (32 cells, one per lane) of the model
// A, with the warp's shared-memory stages at wbuf.
template <class PR, bool TREE, int kRowsBack, int kRowsFwd, int kStackDepth, bool EZ>
__device__ __forceinline__ void epoch_warp(const EpochArgs& A, const int g, char* wbuf) {
  using ST = Stage<PR, TREE, kRowsBack, kRowsFwd, kStackDepth, EZ>;
  using TS = typename PR::S;
  using TG = typename PR::G;
  const int lane = threadIdx.x & 31;
  if (g >= A.n_narrow) return;  // whole warps only
  uint64_t* bar = (uint64_t*)(wbuf + kStages * ST::kBytes);
  // the fork stack region (trees): (f, x', coupling) of the child (backward),
  // V (forward)
  struct FX {
    typename PR::Row::R f, x, a;
  };
  struct FP {  // (coupling f, coupling x') of the product form
    typename PR::Row::R p, q;
  };
  using SE = typename std::conditional<PR::Row::kProdStack, FP, FX>::type;
  SE* stack2 = (SE*)(wbuf + kStages * ST::kBytes + 64);
  typename PR::Row::R* stack1 = (typename PR::Row::R*)stack2;
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  uint32_t phase = 0;    // expected parity of each stage's barrier
  uint32_t pending = 0;  // stages with a copy issued and not yet waited for
  bool failed = false;
  const uint32_t wait_limit = A.wait_limit ? A.wait_limit : kSpinLimit;
  const int64_t L = (int64_t)g * 32 + lane;
  const int n = A.ncv[L];
  const int32_t rb = A.row_base[g];
  const int rows = A.row_base[g + 1] - rb;
  const double dt = A.dt;

  // the cable rows in the policy's row form (FP64, or float-float pairs in
  // PA_MIXED; 8 bytes per value either way)
  using RW = typename PR::Row;
  using R = typename RW::R;
  R* __restrict__ Vg = (R*)A.V;
  const R* __restrict__ CDT = (const R*)A.cdt;
  const R* __restrict__ DC = (const R*)A.dc;
  const R* __restrict__ EM = (const R*)A.em;
  const R* __restrict__ AA = (const R*)A.a;
  TS* __restrict__ GS = (TS*)A.gs;
  TS* __restrict__ ES = (TS*)A.es;
  R* __restrict__ F = (R*)A.f;
  R* __restrict__ XP = (R*)A.xp;

  const bool hh = n > 0 && A.is_hh[L];
  SomaHH<PR::kMech32> soma;
  if (hh) soma.load(A.gate, A.n_lanes, L);
  // the leak E-term formed from C/dt instead of staged (warp-uniform)
  const bool em_der = PR::kDeriveEM && A.em_derived[g] != 0;
  const R emk = em_der ? RW::from_d(A.em_k[L]) : RW::zero();
  const double iinj_val = n > 0 ? A.iinj[L] : 0.0;
  const int64_t kon = n > 0 ? A.k_on[L] : 0, koff = n > 0 ? A.k_off[L] : 0;
  const double th = n > 0 ? A.thresh[L] : 0.0;
  bool spiked_prev = n > 0 && A.spiked_prev[L];
  double prp = (n > 0 && A.stc_stream >= 0) ? A.prp[L] : 0.0;
  const bool has_stc = n > 0 && A.stc_stream >= 0 && A.has_stc[L];
  const uint64_t rbits = (A.replay && n > 0) ? A.replay_bits[L] : 0ull;
  const int32_t pq0 = n > 0 ? A.probe_ptr[L] : 0, pq1 = n > 0 ? A.probe_ptr[L + 1] : 0;

  // the launch window: from the arguments, or the whole epoch the clock names
  int64_t k_begin = A.k_begin, k_end = A.k_end, k0 = A.k0, probe0 = A.probe_sample0;
  int32_t slot = A.slot;
  if (A.clock) {
    k0 = A.clock->k0;
    k_begin = k0;
    k_end = k0 + A.epoch_len;
    probe0 = A.clock->probe_sample0;
    slot = (int32_t)((k0 / A.epoch_len) % A.n_slots);
  }
  for (int64_t k = k_begin; k < k_end && !failed; ++k) {
    const int kk = (int)(k - k0);
    const bool post = spiked_prev;
    // ---- a. synapse streams, rows staged by TMA ------------------------------
    fence_async_global();  // last step's synapse state and V, written by plain stores
    __syncwarp();
    double S = 0.0, qs_field = 0.0;
    for (int s = 0; s < A.n_streams && !failed; ++s) {
      if (s == A.ca_stream) {
        hca_stream<PR>(A, s, g, lane, rb, kk, slot);
        continue;
      }
      const StreamParams& P = A.sp[s];
      const StreamDev& D = A.sd[s];
      const int32_t sb = D.sbase[g], nrow = D.sbase[g + 1] - sb;
      const bool calc = P.kind == SK_GB || P.kind == SK_STC;
      const bool stc = P.kind == SK_STC;
      constexpr int szm = 32 * (int)sizeof(TG);
      const int rowb = 128 + 256 + szm + (calc ? 768 : 0) + (stc ? 256 : 0);
      int RS = ST::kBytes / rowb;
      if (RS > 16) RS = 16;
      const int o_cm = RS * 128, o_g = o_cm + RS * 256, o_cam = o_g + RS * szm,
                o_c = o_cam + RS * 256, o_w = o_c + RS * 256, o_z = o_w + RS * 256;
      const int nc = (nrow + RS - 1) / RS;
      const uint64_t* cmg = D.cmask + (int64_t)slot * D.n_elem;
      const uint64_t* camg = calc ? D.camask + (int64_t)slot * D.n_elem : nullptr;
      TG* G = (TG*)D.g;
      const typename PR::Ec E = PR::e_const(P.e);
      const typename PR::Dc dg = PR::d_const(P.decay_g);
      auto issue = [&](int c) {
        const int si = c % kStages;
        const int lo = c * RS, cnt = nrow - lo < RS ? nrow - lo : RS;
        pending |= 1u << si;
        if (lane == 0) {
          char* st = wbuf + si * ST::kBytes;
          const size_t r0 = (size_t)(sb + lo) * 32;
          if (!PA_IN(A, r0 + (size_t)cnt * 32 - 1, D.n_elem)) {
            mbar_expect_tx(&bar[si], 0u);  // nothing copied: the phase completes at once
            return;
          }
          mbar_expect_tx(&bar[si], (uint32_t)(cnt * rowb));
          bulk_load(st, D.cvf + r0, cnt * 128, &bar[si]);
          bulk_load(st + o_cm, cmg + r0, cnt * 256, &bar[si]);
          bulk_load(st + o_g, (const TG*)D.g + r0, cnt * szm, &bar[si]);
          if (calc) {
            bulk_load(st + o_cam, camg + r0, cnt * 256, &bar[si]);
            bulk_load(st + o_c, D.c + r0, cnt * 256, &bar[si]);
            bulk_load(st + o_w, D.w + r0, cnt * 256, &bar[si]);
          }
          if (stc) bulk_load(st + o_z, D.z + r0, cnt * 256, &bar[si]);
        }
      };
      if (nc > 0) {
        fence_async_shared();  // lanes are done reading the stages about to be refilled
        __syncwarp();
        issue(0);
      }
      typename PR::Acc acc;
      for (int c = 0; c < nc; ++c) {
        if (c + 1 < nc) {
          fence_async_shared();
          __syncwarp();
          issue(c + 1);
        }
        const int si = c % kStages;
        if (mbar_wait(&bar[si], (phase >> si) & 1u, wait_limit)) {
          phase ^= 1u << si;
          pending &= ~(1u << si);
        } else {
          failed = true;
        }
        if (__any_sync(0xffffffffu, failed)) {
          failed = true;
          break;
        }
        const char* st = wbuf + si * ST::kBytes;
        const int lo = c * RS, cnt = nrow - lo < RS ? nrow - lo : RS;
        for (int jj = 0; jj < cnt; ++jj) {
          const int r = jj * 32 + lane;
          const int32_t cvf = ((const int32_t*)st)[r];
          if (cvf < 0) continue;
          const uint32_t e = ((uint32_t)(sb + lo + jj) << 5) | (uint32_t)lane;
          if (!PA_IN(A, e, D.n_elem) || !PA_IN(A, elem_of(rb, cvf >> 3, lane), A.n_row_elems))
            continue;
          const bool pre = (((const uint64_t*)(st + o_cm))[r] >> kk) & 1ull;
          const bool capre = calc && ((((const uint64_t*)(st + o_cam))[r] >> kk) & 1ull);
          const double cc = calc ? ((const double*)(st + o_c))[r] : 0.0;
          const double wv = calc ? ((const double*)(st + o_w))[r] : 0.0;
          const double zv = stc ? ((const double*)(st + o_z))[r] : 0.0;
          // Eq. late_phase_weight captures the cell's PRP, or that of the
          // synapse's own CV when the PRP diffuses
          const double pz = (stc && A.prp_diff) ? A.prp_cv[elem_of(rb, cvf >> 3, lane)] : prp;
          TG gv = syn_update<PR>(P, D, e, pre, capre, post, ((const TG*)(st + o_g))[r], cc, wv,
                                 zv, pz, k, dt, A.seed, S);
          // per-CV sums over the run of same-CV synapses, in canonical order
          // (cvf = (cv << 3) | first-on-CV (1) | run start (2) | run end (4))
          const uint32_t ce = elem_of(rb, cvf >> 3, lane);
          if (cvf & 2) acc.template start<EZ>(gv, E, (cvf & 1) != 0, GS, ES, ce);
          else acc.template add<EZ>(gv, E);
          if (cvf & 4) acc.template store<EZ>(GS, ES, ce, E);
          G[e] = PR::decay(gv, dg);
        }
      }
      if (s == A.stc_stream && has_stc) {
        const double qs = (S > P.theta_pro) ? P.p_max : 0.0;
        if (A.prp_diff) qs_field = qs;  // the field takes its step after the voltage solve
        else prp = prp + P.rate_p * (qs - prp);
      }
    }
    if (__any_sync(0xffffffffu, failed)) {
      failed = true;
      break;
    }

    // ---- b. backward pass: assembly + elimination ----------------------------
    // rows n-1 .. 0, staged from HBM in chunks of kRowsBack rows.  Every row
    // takes the same operations (the lanes of a warp are different cells, so a
    // per-row shortcut would run both paths).
    double v0_old = 0.0, v0_new = 0.0;
    R x0 = RW::zero();  // the soma's new V in the row form
    const double iinj = (k >= kon && k < koff) ? iinj_val : 0.0;
    fence_async_global();  // this step's synaptic sums, written by plain stores
    __syncwarp();
    {
      const int nc = (rows + kRowsBack - 1) / kRowsBack;
      auto issue = [&](int c) {
        const int s = c % kStages;
        const int hi = rows - kRowsBack * c, lo = hi > kRowsBack ? hi - kRowsBack : 0;
        const uint32_t cnt = (uint32_t)(hi - lo);
        pending |= 1u << s;
        if (lane == 0) {
          char* st = wbuf + s * ST::kBytes;
          const size_t r0 = (size_t)(rb + lo);
          if (!PA_IN(A, (r0 + cnt) * 32 - 1, A.n_row_elems)) {
            mbar_expect_tx(&bar[s], 0u);
            return;
          }
          // with EZ the g E sums are signed zeros: not staged (see ez_add)
          mbar_expect_tx(&bar[s], cnt * ST::kBackRow);
          bulk_load(st + ST::oV, Vg + r0 * 32, cnt * ST::kD, &bar[s]);
          bulk_load(st + ST::oCDT, CDT + r0 * 32, cnt * ST::kD, &bar[s]);
          bulk_load(st + ST::oDC, DC + r0 * 32, cnt * ST::kD, &bar[s]);
          if (ST::kE) bulk_load(st + ST::oEM, EM + r0 * 32, cnt * ST::kE, &bar[s]);
          bulk_load(st + ST::oA, AA + r0 * 32, cnt * ST::kD, &bar[s]);
          bulk_load(st + ST::oGS, GS + r0 * 32, cnt * ST::kM, &bar[s]);
          if (!EZ) bulk_load(st + ST::oES, ES + r0 * 32, cnt * ST::kM, &bar[s]);
          if (TREE && !ST::kStacks) {
            bulk_load(st + ST::oPAR, A.par + r0 * 32, cnt * ST::kI, &bar[s]);
            bulk_load(st + ST::oOCH, A.och_head + r0 * 32, cnt * ST::kI, &bar[s]);
          }
          if (ST::kStacks) bulk_load(st + ST::oTF, A.tflag + r0 * 32, cnt * ST::kT, &bar[s]);
        }
      };
      fence_async_shared();
      __syncwarp();
      for (int c = 0; c < kStages - 1 && c < nc; ++c) issue(c);
      R cf = RW::zero(), ca = RW::zero(), cx = RW::zero();
      bool carry = false;
      int depth = 0;  // fork-stack depth of this lane
      for (int c = 0; c < nc; ++c) {
        if (c + kStages - 1 < nc) {
          fence_async_shared();  // reads of the stage about to be refilled are done
          __syncwarp();
          issue(c + kStages - 1);
        }
        const int s = c % kStages;
        if (mbar_wait(&bar[s], (phase >> s) & 1u, wait_limit)) {
          phase ^= 1u << s;
          pending &= ~(1u << s);
        } else {
          failed = true;
        }
        if (__any_sync(0xffffffffu, failed)) {
          failed = true;
          break;
        }
        const char* st = wbuf + s * ST::kBytes;
        const int hi = rows - kRowsBack * c, lo = hi > kRowsBack ? hi - kRowsBack : 0;
        for (int i = hi - 1; i >= lo; --i) {
          if (i >= n) continue;
          const int r = (i - lo) * 32 + lane;
          const uint32_t e = elem_of(rb, i, lane);
          if (!PA_IN(A, e, A.n_row_elems)) continue;
          const R v = ((const R*)(st + ST::oV))[r];
          const R cdt = ((const R*)(st + ST::oCDT))[r];
          const R dcv = ((const R*)(st + ST::oDC))[r];
          int pi = i - 1;
          if (TREE && !ST::kStacks && i > 0) pi = ((const int16_t*)(st + ST::oPAR))[r];
          const R gsv = PR::sum_r(((const TS*)(st + ST::oGS))[r]);
          R d, b;
          if (i == 0) {
            v0_old = RW::to_d(v);
            if (hh) {
              double gmt, emt;
              soma.currents(A, L, gmt, emt);
              d = RW::add(RW::add(dcv, RW::from_d(gmt)), gsv);
              b = RW::add(RW::fma(cdt, v, RW::from_d(emt)), RW::from_d(iinj));
            } else {
              d = RW::add(dcv, gsv);
              const R emv = em_der    ? RW::from_d(A.em_soma[L])
                            : ST::kE    ? ((const R*)(st + ST::oEM))[r]
                                        : EM[e];
              b = RW::add(RW::fma(cdt, v, emv), RW::from_d(iinj));
            }
          } else {
            d = RW::add(dcv, gsv);
            const R emv = em_der ? RW::mul(cdt, emk)
                          : ST::kE ? ((const R*)(st + ST::oEM))[r]
                                   : EM[e];
            b = RW::fma(cdt, v, emv);
          }
          if constexpr (!EZ) {
            b = RW::add(b, PR::sum_r(((const TS*)(st + ST::oES))[r]));
          } else if constexpr (std::is_same<R, double>::value) {
            b = ez_add(b, (const TS*)ES, e);  // (float-float: the signed zero is not added)
          }
          uint8_t tf = 0;
          if (TREE) {
            if (ST::kStacks) tf = ((const uint8_t*)(st + ST::oTF))[r];
            if (tf & kForkPop) {
              // the one other child: its f, x' and coupling from the top of the
              // fork stack (eliminated earlier in this pass)
              --depth;
              if constexpr (RW::kProdStack) {
                R pc, qc;
                if (depth < ST::kStackB) {
                  const SE t = stack2[depth * 32 + lane];
                  pc = t.p;
                  qc = t.q;
                } else {
                  const uint32_t ec = elem_of(rb, A.och_head[e], lane);
                  const bool ok = PA_IN(A, ec, A.n_row_elems);
                  const R ac = ok ? AA[ec] : RW::zero();
                  pc = RW::mul(ac, ok ? F[ec] : RW::zero());
                  qc = RW::mul(ac, ok ? XP[ec] : RW::zero());
                }
                d = RW::sub(d, pc);
                b = RW::sub(b, qc);
              } else {
                R fc, xc, ac;
                if (depth < ST::kStackB) {
                  const SE t = stack2[depth * 32 + lane];
                  fc = t.f;
                  xc = t.x;
                  ac = t.a;
                } else {
                  const uint32_t ec = elem_of(rb, A.och_head[e], lane);
                  const bool ok = PA_IN(A, ec, A.n_row_elems);
                  fc = ok ? F[ec] : RW::zero();
                  xc = ok ? XP[ec] : RW::zero();
                  ac = ok ? AA[ec] : RW::zero();
                }
                other_child<RW>(ac, fc, xc, d, b);
              }
            } else if (!ST::kStacks || (tf & kOtherList)) {
              // several other children, highest index first, from the scratch arrays
              const int och = ST::kStacks ? A.och_head[e] : ((const int16_t*)(st + ST::oOCH))[r];
              for (int ch = och; ch >= 0;) {
                const uint32_t ec = elem_of(rb, ch, lane);
                if (!PA_IN(A, ec, A.n_row_elems)) break;
                other_child<RW>(AA[ec], F[ec], XP[ec], d, b);
                ch = A.och_next[ec];
              }
            }
          }
          if (carry) {
            d = RW::fnma(cf, ca, d);
            b = RW::fnma(ca, cx, b);
          }
          if (i > 0) {
            const R ai = ((const R*)(st + ST::oA))[r];
            const R rr = RW::rcp(d);
            const R fi = RW::mul(ai, rr);
            const R xi = RW::mul(b, rr);
            F[e] = fi;
            XP[e] = xi;
            if (TREE && (tf & kForkPush)) {
              if (depth < ST::kStackB) {
                if constexpr (RW::kProdStack) stack2[depth * 32 + lane] = SE{RW::mul(ai, fi), RW::mul(ai, xi)};
                else stack2[depth * 32 + lane] = SE{fi, xi, ai};
              }
              ++depth;
            }
            carry = !TREE || (ST::kStacks ? (tf & kParPrev) != 0 : pi == i - 1);
            cf = fi; ca = ai; cx = xi;
          } else {
            x0 = RW::mul(b, RW::rcp(d));
            v0_new = RW::to_d(x0);
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, failed)) {
      failed = true;
      break;
    }
    // ---- c. forward pass: back substitution, rows 0 .. n-1 ------------------
    fence_async_global();  // f and x' of this step, written by plain stores
    __syncwarp();
    {
      const int nc = (rows + kRowsFwd - 1) / kRowsFwd;
      auto issue = [&](int c) {
        const int s = c % kStages;
        const int lo = kRowsFwd * c, hi = lo + kRowsFwd < rows ? lo + kRowsFwd : rows;
        const uint32_t cnt = (uint32_t)(hi - lo);
        pending |= 1u << s;
        if (lane == 0) {
          char* st = wbuf + s * ST::kBytes;
          const size_t r0 = (size_t)(rb + lo);
          if (!PA_IN(A, (r0 + cnt) * 32 - 1, A.n_row_elems)) {
            mbar_expect_tx(&bar[s], 0u);
            return;
          }
          mbar_expect_tx(&bar[s], cnt * ST::kFwdRow);
          bulk_load(st + ST::fF, F + r0 * 32, cnt * ST::kD, &bar[s]);
          bulk_load(st + ST::fXP, XP + r0 * 32, cnt * ST::kD, &bar[s]);
          if (TREE && !ST::kStacks) bulk_load(st + ST::fPAR, A.par + r0 * 32, cnt * ST::kI, &bar[s]);
          if (ST::kStacks) bulk_load(st + ST::fTF, A.tflag + r0 * 32, cnt * ST::kT, &bar[s]);
        }
      };
      fence_async_shared();
      __syncwarp();
      for (int c = 0; c < kStages - 1 && c < nc; ++c) issue(c);
      if (n > 0) Vg[elem_of(rb, 0, lane)] = x0;
      R vprev = x0;
      int depth = 0;  // fork-stack depth of this lane
      for (int c = 0; c < nc; ++c) {
        if (c + kStages - 1 < nc) {
          fence_async_shared();
          __syncwarp();
          issue(c + kStages - 1);
        }
        const int s = c % kStages;
        if (mbar_wait(&bar[s], (phase >> s) & 1u, wait_limit)) {
          phase ^= 1u << s;
          pending &= ~(1u << s);
        } else {
          failed = true;
        }
        if (__any_sync(0xffffffffu, failed)) {
          failed = true;
          break;
        }
        const char* st = wbuf + s * ST::kBytes;
        const int lo = kRowsFwd * c, hi = lo + kRowsFwd < rows ? lo + kRowsFwd : rows;
        if (ST::kStacks && c == 0 && n > 0 &&
            (((const uint8_t*)(st + ST::fTF))[lane] & kForkPop)) {
          stack1[lane] = x0;  // the root is a fork with one other child
          depth = 1;
        }
        for (int i = lo > 1 ? lo : 1; i < hi; ++i) {
          if (i >= n) break;
          const int r = (i - lo) * 32 + lane;
          R vp = vprev;
          uint8_t tf = 0;
          if (TREE) {
            const uint32_t ei = elem_of(rb, i, lane);
            if (ST::kStacks) {
              // the parent row is read from memory only where it is not the
              // previous row and not on the stack
              tf = ((const uint8_t*)(st + ST::fTF))[r];
              if (tf & kForkPush) {
                // the one other child of its parent: the parent's V from the stack
                --depth;
                vp = depth < ST::kStackF ? stack1[depth * 32 + lane]
                                         : Vg[elem_of(rb, A.par[ei], lane)];
              } else if (!(tf & kParPrev)) {
                const uint32_t ep = elem_of(rb, A.par[ei], lane);
                vp = PA_IN(A, ep, A.n_row_elems) ? Vg[ep] : RW::zero();
              }
            } else {
              const int pi = ((const int16_t*)(st + ST::fPAR))[r];
              if (pi != i - 1) {
                vp = PA_IN(A, elem_of(rb, pi, lane), A.n_row_elems) ? Vg[elem_of(rb, pi, lane)]
                                                                     : RW::zero();
              }
            }
          }
          const R vi = RW::fnma(((const R*)(st + ST::fF))[r], vp, ((const R*)(st + ST::fXP))[r]);
          if (PA_IN(A, elem_of(rb, i, lane), A.n_row_elems)) Vg[elem_of(rb, i, lane)] = vi;
          if (TREE && (tf & kForkPop)) {
            if (depth < ST::kStackF) stack1[depth * 32 + lane] = vi;
            ++depth;
          }
          vprev = vi;
        }
      }
    }
    if (__any_sync(0xffffffffu, failed)) {
      failed = true;
      break;
    }
    if (A.prp_diff && has_stc)
      prp = prp_field_step<TREE>(A, rb, lane, L, n, qs_field, A.sp[A.stc_stream].rate_p, A.prp_dg,
                                 A.prp_vdt);
    if (A.ca_stream >= 0 && n > 0 && A.has_ca[L]) ca_field_step<TREE>(A, rb, lane, n);
    if (n > 0) {
      for (int32_t q = pq0; q < pq1; ++q) {
        const int64_t smp = probe0 + (k - k_begin);
        if (smp < A.probe_cap) {
          A.probe_buf[smp * A.n_probe + A.probe_id[q]] =
              RW::to_d(Vg[elem_of(rb, A.probe_row[q], lane)]);
        } else {
          atomicOr(A.err_flags, 1);
        }
      }
    }
    // ---- d. soma gates, detection, compaction --------------------------------
    if (hh) soma.update(v0_new, dt);
    const bool spk = n > 0 && v0_old < th && v0_new >= th;
    const unsigned ball = __ballot_sync(0xffffffffu, spk);
    if (ball) {
      int base = 0;
      if (lane == 0) base = atomicAdd(A.spk_count, __popc(ball));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (spk) {
        const int slot = base + __popc(ball & ((1u << lane) - 1u));
        if (slot < A.spk_cap) {
          A.spk_gid[slot] = A.gid[L];
          A.spk_step[slot] = (int32_t)k;
          A.spk_t[slot] = (double)k * dt + dt * ((th - v0_old) / (v0_new - v0_old));
        }
      }
    }
    spiked_prev = A.replay ? (((rbits >> (k - k_begin)) & 1ull) != 0) : spk;
  }
  if (failed) {
    // a stage did not arrive within the poll limit: report it, then let every
    // copy this warp issued land (bounded by the full limit) before the warp
    // leaves, so that no bulk copy still writes into its shared memory.  A
    // stage's expected parity is unchanged until its wait succeeds.
    if (lane == 0) atomicOr(A.err_flags, 4);
    for (int s = 0; s < kStages; ++s)
      if ((pending >> s) & 1u) mbar_wait(&bar[s], (phase >> s) & 1u, kSpinLimit);
    __syncwarp();
    return;
  }
  if (n > 0) {
    A.spiked_prev[L] = spiked_prev ? 1 : 0;
    if (hh) soma.store(A.gate, A.n_lanes, L);
    if (has_stc) A.prp[L] = prp;
  }
}

template <class PR, bool TREE, int kRowsBack, int kRowsFwd, int kThreads, int kMinBlocks,
          int kStackDepth, bool EZ>
__global__ void __launch_bounds__(kThreads, kMinBlocks) epoch_kernel(const EpochArgs A) {
  using ST = Stage<PR, TREE, kRowsBack, kRowsFwd, kStackDepth, EZ>;
  extern __shared__ __align__(128) char smem_raw[];
  const int g = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  epoch_warp<PR, TREE, kRowsBack, kRowsFwd, kStackDepth, EZ>(
      A, g, smem_raw + (threadIdx.x >> 5) * ST::kWarpBytes);
}

// Several models in one launch (a batch of resident jobs that share the
// precision, the tree class and the epoch length): block b runs groups
// [bmap[b].y, bmap[b].y + warps per block) of model bmap[b].x, whose launch
// arguments the block first copies from args[] into shared memory.  Every
// warp then takes exactly the steps it takes in the model's own launch.
constexpr int kArgsSmemBytes = (int)((sizeof(EpochArgs) + 127) / 128 * 128);
static_assert(sizeof(EpochArgs) % 8 == 0, "launch arguments copy as 8-byte words");

template <class PR, bool TREE, int kRowsBack, int kRowsFwd, int kThreads, int kMinBlocks,
          int kStackDepth, bool EZ>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    epoch_kernel_grouped(const EpochArgs* __restrict__ args, const int2* __restrict__ bmap) {
  using ST = Stage<PR, TREE, kRowsBack, kRowsFwd, kStackDepth, EZ>;
  extern __shared__ __align__(128) char smem_raw[];
  __shared__ __align__(128) char args_raw[kArgsSmemBytes];
  const int2 bm = bmap[blockIdx.x];
  const long long* src = (const long long*)(args + bm.x);
  long long* dst = (long long*)args_raw;
  for (int i = threadIdx.x; i < (int)(sizeof(EpochArgs) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  epoch_warp<PR, TREE, kRowsBack, kRowsFwd, kStackDepth, EZ>(
      *(const EpochArgs*)args_raw, bm.y + (int)(threadIdx.x >> 5),
      smem_raw + (threadIdx.x >> 5) * ST::kWarpBytes);
}

template <class PR, bool TREE, int RB, int RF, int WPB, int MB, int SB, bool EZ>
int launch_epoch_t(const EpochArgs& a, void* stream) {
  constexpr int warps_per_block = WPB;
  const int threads = 32 * warps_per_block;
  const int64_t warps = a.n_narrow;
  const int blocks = (int)((warps * 32 + threads - 1) / threads);
  if (blocks == 0) return 0;
  const int smem = warps_per_block * Stage<PR, TREE, RB, RF, SB, EZ>::kWarpBytes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  static bool attr_set[64] = {false};  // per device; setting it twice is harmless
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(epoch_kernel<PR, TREE, RB, RF, 32 * WPB, MB, SB, EZ>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  epoch_kernel<PR, TREE, RB, RF, 32 * WPB, MB, SB, EZ>
      <<<blocks, threads, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

// Kernel shapes: rows per TMA chunk (backward, forward), warps per block and
// minimum resident blocks per SM (which sets the register budget).  Shape 0 is
// the default; the autotuner times all of them on the model and keeps the
// fastest.
// Trees also choose the fork stacks' depth (24-byte entries): with 8-byte sums
// (FP64, mixed) shape 0 takes 3 backward rows (4 where every E = +0) and 11
// forward rows per chunk and 8 entries (many nested forks; mixed with every
// E = +0: 5 and 12 rows, 10 entries of 16 bytes), shapes 3 and 4 take 4 rows and 2 entries; with FP32 sums
// shape 0 takes 4 rows (5 where every E = +0) and 6 entries; shape 5 has no stacks (trees with long
// branches and few forks); 12 warps per SM fit in each case (4-entry stacks
// that would let shape 1 keep 16 warps per SM on trees made it 33 % slower,
// 6-entry stacks with 8 forward rows 19 %: the random trees' forks nest deeper).
template <class PR, bool TREE, bool EZ>
int launch_epoch_shape(const EpochArgs& a, int shape, void* stream) {
  constexpr bool f64tree = TREE && sizeof(typename PR::S) == 8;
  // (with every E = +0 the g E sums are not staged, which leaves room for a
  // fourth backward row beside 11 forward rows and 8 stack entries)
  // (mixed trees stage neither the g E sums nor the leak E-term and keep
  // 16-byte stack entries: 5 backward and 12 forward rows with 10 entries
  // fit; 0.7 % faster than 4 and 11 rows, then 1.4 % from the product-form
  // entries, 10 of them against 7 of 24 bytes)
  // (FP32 sums with every E = +0 leave room for 5 backward rows as well:
  // 1.6 % faster than 4 on the large network)
  constexpr bool mx = PR::kDeriveEM && f64tree && EZ;
  constexpr bool f32ez = TREE && !f64tree && EZ;
  constexpr int RB0 = (mx || f32ez) ? 5 : (f64tree && !EZ) ? 3 : 4,
                SB0 = mx ? 10 : f64tree ? 8 : 6, RF0 = mx ? 12 : f64tree ? 11 : 12;
  constexpr int RB6 = f64tree ? 5 : 6;
  constexpr int SB4 = f64tree ? 2 : 6;
  switch (shape) {
    case 1: return launch_epoch_t<PR, TREE, 3, 9, 4, 4, 8, EZ>(a, stream);    // 16 warps per SM
    case 2: return launch_epoch_t<PR, TREE, RB6, 16, 2, 4, 8, EZ>(a, stream); // 8 warps, long chunks
    case 3: return launch_epoch_t<PR, TREE, 4, 12, 2, 6, SB4, EZ>(a, stream); // 2-warp blocks
    case 4: return launch_epoch_t<PR, TREE, 4, 12, 1, 12, SB4, EZ>(a, stream);// 1-warp blocks
    case 5: return launch_epoch_t<PR, TREE, 4, 12, 4, 3, 0, EZ>(a, stream);   // trees: no stacks
    default: return launch_epoch_t<PR, TREE, RB0, RF0, 4, 3, SB0, EZ>(a, stream);  // 12 warps per SM
  }
}

// Grouped launches: 4 warps per block, 3 blocks per SM; chains take shape 0's
// geometry, trees shape 5's (no fork stacks: the copied arguments take their
// shared memory).  Results equal those of every other shape.
constexpr int kGroupedWarpsPerBlock = 4;

template <class PR, bool TREE, int RB, int RF, int MB, int SB, bool EZ>
int launch_epoch_grouped_t(const EpochArgs* d_args, const int2* d_bmap, int n_blocks,
                           void* stream) {
  constexpr int WPB = kGroupedWarpsPerBlock;
  if (n_blocks == 0) return 0;
  const int smem = WPB * Stage<PR, TREE, RB, RF, SB, EZ>::kWarpBytes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  static bool attr_set[64] = {false};
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(epoch_kernel_grouped<PR, TREE, RB, RF, 32 * WPB, MB, SB, EZ>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  epoch_kernel_grouped<PR, TREE, RB, RF, 32 * WPB, MB, SB, EZ>
      <<<n_blocks, 32 * WPB, smem, (cudaStream_t)stream>>>(d_args, d_bmap);
  return (int)cudaGetLastError();
}

template <class PR>
int launch_epoch_grouped_impl(const EpochArgs* d_args, const int2* d_bmap, int n_blocks,
                              bool tree, bool ez, void* stream) {
  if (ez)
    return tree ? launch_epoch_grouped_t<PR, true, 4, 12, 3, 0, true>(d_args, d_bmap, n_blocks,
                                                                      stream)
                : launch_epoch_grouped_t<PR, false, 4, 12, 3, 6, true>(d_args, d_bmap, n_blocks,
                                                                       stream);
  return tree ? launch_epoch_grouped_t<PR, true, 4, 12, 3, 0, false>(d_args, d_bmap, n_blocks,
                                                                     stream)
              : launch_epoch_grouped_t<PR, false, 4, 12, 3, 6, false>(d_args, d_bmap, n_blocks,
                                                                      stream);
}

template <class PR>
int launch_epoch_impl(const EpochArgs& a, bool tree, int shape, void* stream) {
  if (a.es_zero)
    return tree ? launch_epoch_shape<PR, true, true>(a, shape, stream)
                : launch_epoch_shape<PR, false, true>(a, shape, stream);
  return tree ? launch_epoch_shape<PR, true, false>(a, shape, stream)
              : launch_epoch_shape<PR, false, false>(a, shape, stream);
}

}  // namespace pa
