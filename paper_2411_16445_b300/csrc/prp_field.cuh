// prp_field.cuh -- one step of a diffusing PRP field (Eq. diffusion on the
// cell's tree, solved like the cable equation), for the time-step kernel and
// for the long steps of the fast-forward.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "int_arith.cuh"

namespace pa {

// The field of the lane's cell (narrow element layout, rows n-1..0 then
// 0..n-1, in global memory): every CV takes the explicit reaction step
// P* = P + rate (src - P) (rate = step / tau_p; synthesis qs V_tot / V_0 at the
// soma only, degradation everywhere), then one backward-Euler diffusion solve
// with the constant matrix of the step (diagonal dg = V/step + sum gD,
// coupling -gD, right-hand side vdt P* with vdt = V/step), eliminated like
// the cable equation: children into parents from the highest row down (other
// children first, the row below last), one correctly rounded reciprocal per
// row.  The Hines scratch f, x' must be free (the voltage solve of the step is
// done).  Explicitly rounded operations: the same arithmetic in every build.
// Returns the soma CV's new concentration.
// WIDE: the cell's rows are contiguous (element (rb << 5) + row, the wide bin's
// layout) instead of lane-interleaved.
template <bool TREE, bool WIDE = false>
__device__ __noinline__ double prp_field_step(const EpochArgs& A, int32_t rb, int lane, int64_t L,
                                              int n, double qs, double rate, const double* dg,
                                              const double* vdt) {
  double* __restrict__ P = A.prp_cv;
  double* __restrict__ F = A.f;
  double* __restrict__ XP = A.xp;
  auto el = [&](int row) -> uint32_t {
    return WIDE ? ((uint32_t)rb << 5) + (uint32_t)row : ((uint32_t)(rb + row) << 5) | (uint32_t)lane;
  };
  double cf = 0.0, ca = 0.0, cx = 0.0, x0 = 0.0;
  bool carry = false;
  for (int i = n - 1; i >= 0; --i) {
    const uint32_t e = el(i);
    const double pv = P[e];
    const double src = (i == 0) ? __dmul_rn(qs, A.prp_src[L]) : 0.0;
    const double ps = __dadd_rn(pv, __dmul_rn(rate, __dsub_rn(src, pv)));
    double d = dg[e];
    double b = __dmul_rn(vdt[e], ps);
    if (TREE) {
      for (int ch = A.och_head[e]; ch >= 0;) {
        const uint32_t ec = el(ch);
        const double ac = A.prp_a[ec];
        d = __fma_rn(-F[ec], ac, d);
        b = __fma_rn(-ac, XP[ec], b);
        ch = A.och_next[ec];
      }
    }
    if (carry) {
      d = __fma_rn(-cf, ca, d);
      b = __fma_rn(-ca, cx, b);
    }
    if (i > 0) {
      const double ai = A.prp_a[e];
      const double rr = rcp_rn_pos(d);
      const double fi = __dmul_rn(ai, rr);
      const double xi = __dmul_rn(b, rr);
      F[e] = fi;
      XP[e] = xi;
      carry = !TREE || A.par[e] == i - 1;
      cf = fi; ca = ai; cx = xi;
    } else {
      x0 = __dmul_rn(b, rcp_rn_pos(d));
    }
  }
  if (n > 0) P[el(0)] = x0;
  double prev = x0;
  for (int i = 1; i < n; ++i) {
    const uint32_t e = el(i);
    double pp = prev;
    if (TREE) {
      const int pi = A.par[e];
      if (pi != i - 1) pp = P[el(pi)];
    }
    const double xi = __fma_rn(-F[e], pp, XP[e]);
    P[e] = xi;
    prev = xi;
  }
  return x0;
}

// One step of the heterosynaptic calcium field of the lane's cell (Eq.
// ca_diffusion_dendrite; narrow element layout): every CV takes the explicit
// reaction C* = C + (dt/tau_C) (q - C) with q = tau_C src / V (src: this step's
// inflow summed by the synapse phase; 0 in CVs without HCA synapses, which the
// phase never writes), then one backward-Euler diffusion solve with the
// constant matrix, eliminated like the PRP field above.
template <bool TREE>
__device__ __noinline__ void ca_field_step(const EpochArgs& A, int32_t rb, int lane, int n) {
  double* __restrict__ C = A.ca_cv;
  double* __restrict__ F = A.f;
  double* __restrict__ XP = A.xp;
  const double tau = A.ca_tau, rate = A.ca_rate;
  auto el = [&](int row) -> uint32_t { return ((uint32_t)(rb + row) << 5) | (uint32_t)lane; };
  double cf = 0.0, ca = 0.0, cx = 0.0, x0 = 0.0;
  bool carry = false;
  for (int i = n - 1; i >= 0; --i) {
    const uint32_t e = el(i);
    const double cv = C[e];
    const double q = __ddiv_rn(__dmul_rn(tau, A.ca_src[e]), A.ca_vol[e]);
    const double cs = __dadd_rn(cv, __dmul_rn(rate, __dsub_rn(q, cv)));
    double d = A.ca_dg[e];
    double b = __dmul_rn(A.ca_vdt[e], cs);
    if (TREE) {
      for (int ch = A.och_head[e]; ch >= 0;) {
        const uint32_t ec = el(ch);
        const double ac = A.ca_a[ec];
        d = __fma_rn(-F[ec], ac, d);
        b = __fma_rn(-ac, XP[ec], b);
        ch = A.och_next[ec];
      }
    }
    if (carry) {
      d = __fma_rn(-cf, ca, d);
      b = __fma_rn(-ca, cx, b);
    }
    if (i > 0) {
      const double ai = A.ca_a[e];
      const double rr = rcp_rn_pos(d);
      const double fi = __dmul_rn(ai, rr);
      const double xi = __dmul_rn(b, rr);
      F[e] = fi;
      XP[e] = xi;
      carry = !TREE || A.par[e] == i - 1;
      cf = fi; ca = ai; cx = xi;
    } else {
      x0 = __dmul_rn(b, rcp_rn_pos(d));
    }
  }
  C[el(0)] = x0;
  double prev = x0;
  for (int i = 1; i < n; ++i) {
    const uint32_t e = el(i);
    double pp = prev;
    if (TREE) {
      const int pi = A.par[e];
      if (pi != i - 1) pp = C[el(pi)];
    }
    const double xi = __fma_rn(-F[e], pp, XP[e]);
    C[e] = xi;
    prev = xi;
  }
}

}  // namespace pa
