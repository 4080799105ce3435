// wide_kernel.cuh -- the epoch kernel for the wide cell bin: one warp per cell.
//
// A large cell whose own rows and synapses would keep one thread busy for a
// whole step (thousands of serial rows or synapses) runs on all 32 lanes of a
// warp.  The cell's CVs are contiguous (element (row_base << 5) + i for CV i),
// as are its synapses in each stream.
//
// Per step, in the same order and with the same operations as the narrow
// kernel (epoch_kernel.cuh), so that both equal the plain definition:
//   a. synapse streams: lanes update 32 synapses at a time in parallel
//      (events, POST_EVENT, plasticity; syn_update), the next row's state
//      loading meanwhile; the per-CV sums and the cell's STC sum S are then
//      folded in canonical synapse order, every lane reading the 32 values by
//      shuffle, so the sums are the sequential ones (a row of exact zeros
//      changes a sum only through the sign rule of zeros, taken from ballots);
//   b. backward pass by branches: a branch is a run of rows i whose parent is
//      i - 1 (contiguous in the numbering), cut after every fork; at a fork the
//      first child's values come from memory like the other children's, applied
//      last as in the narrow kernel.  Branches are scheduled
//      by level (a branch's level exceeds that of every branch hanging off
//      it); the branches of one level run on the lanes in parallel, each
//      eliminated row by row from its last row to its first, children applied
//      in descending index order exactly as in the narrow kernel; a warp
//      barrier separates levels.  The root branch (CV 0, the soma) is the only
//      branch of the top level and runs on lane 0;
//   c. forward pass by levels from the root down; a branch starts from its
//      parent's new voltage (written one level earlier);
//   d. a diffusing PRP field (Eq. diffusion): its reaction and backward-Euler
//      diffusion step by the same branch levels and in the same order as the
//      voltage (prp_field.cuh gives the arithmetic);
//   e. soma on lane 0: HH gates, detection, spike record.
#pragma once
#include "epoch_kernel.cuh"

namespace pa {

constexpr int kWideFwdChunk = 4;  // forward-pass rows whose f and x' load together

// The FP64 HH soma's gate update (HH64::rates, then HH64::gate for m, h, n) on
// the lanes of the cell's warp, operation for operation the sequential one:
// lanes 0-5 each form one rate (am, bm, ah, bh, an, bn) by one instruction
// stream, every form's steps taken on every lane and the lane's own chosen
// by selects; lanes 0-2 then update m, h, n.  Called by the whole warp; the
// gates live on lane 0.
template <bool kF32>
__device__ __forceinline__ void hh64_update_warp(SomaHH<kF32>& soma, double v, double dt,
                                                 int lane) {
  static_assert(!kF32, "FP64 gates only");
  const unsigned full = 0xffffffffu;
  const int q = lane < 6 ? lane : 0;
  // rate q: A vtrap(-(v + B), C) (am, an), A exp(-(v + B) / C) (bm, ah, bn),
  // 1 / (exp(-(v + B) / C) + 1) (bh)
  const double B = q == 0 ? 40.0 : q == 3 ? 35.0 : q == 4 ? 55.0 : 65.0;
  const double Cq = q == 0 ? 10.0 : q == 1 ? 18.0 : q == 2 ? 20.0 : q == 3 ? 10.0
                  : q == 4 ? 10.0 : 80.0;
  const double Aq = q == 0 ? 0.1 : q == 1 ? 4.0 : q == 2 ? 0.07 : q == 4 ? 0.01 : 0.125;
  const bool vt = q == 0 || q == 4, sig = q == 3;
  const double x = -(v + B);
  const double u = x / Cq;
  const double e = model_exp(u);
  const double d = (vt ? x : 1.0) / (vt ? e - 1.0 : e + 1.0);
  double r = (vt || sig) ? d : e;
  if (vt && fabs(u) < 1e-6) r = Cq * (1.0 - 0.5 * u);
  const double rate = sig ? r : Aq * r;
  // gate g on lane g: rates 2g and 2g + 1, the gate's value from lane 0
  const int g = lane < 3 ? lane : 0;
  const double a = __shfl_sync(full, rate, 2 * g), b = __shfl_sync(full, rate, 2 * g + 1);
  const double m0 = __shfl_sync(full, soma.m, 0), h0 = __shfl_sync(full, soma.h, 0),
               n0 = __shfl_sync(full, soma.n, 0);
  const double x0 = g == 0 ? m0 : g == 1 ? h0 : n0;
  const double sab = a + b;
  const double xinf = a / sab;
  const double xn = xinf + (x0 - xinf) * model_exp(-dt * sab);
  soma.m = __shfl_sync(full, xn, 0);
  soma.h = __shfl_sync(full, xn, 1);
  soma.n = __shfl_sync(full, xn, 2);
}

template <class PR, bool EZ>
__global__ void __launch_bounds__(128, 2) wide_kernel(const EpochArgs A) {
  using TS = typename PR::S;
  using TG = typename PR::G;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (w >= A.n_wide) return;  // whole warps only
  const int g = A.n_narrow + w;
  const int64_t L = (int64_t)g * 32;  // the cell's lane slot
  const int n = A.ncv[L];
  const int64_t e0 = (int64_t)A.row_base[g] << 5;  // element of CV 0
  const WideCell wc = A.wcell[w];
  const double dt = A.dt;

  // the cable rows in the policy's row form (FP64, or float-float pairs in
  // PA_MIXED); the diffusing field uses the scratch as FP64
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
  double* __restrict__ Fd = A.f;
  double* __restrict__ XPd = A.xp;
  const int16_t* __restrict__ PAR = A.par;
  const int16_t* __restrict__ OCH = A.och_head;
  const int16_t* __restrict__ OCN = A.och_next;

  // the leak E-term formed from C/dt instead of read, as in the narrow kernel
  const bool em_der = PR::kDeriveEM && A.em_derived[g] != 0;
  const R emk = em_der ? RW::from_d(A.em_k[L]) : RW::zero();
  // soma state: lane 0 owns it (every lane keeps prp and the POST_EVENT flag)
  const bool hh = n > 0 && A.is_hh[L];
  SomaHH<PR::kMech32> soma;
  if (hh && lane == 0) soma.load(A.gate, A.n_lanes, L);
  const double iinj_val = n > 0 ? A.iinj[L] : 0.0;
  const int64_t kon = n > 0 ? A.k_on[L] : 0, koff = n > 0 ? A.k_off[L] : 0;
  const double th = n > 0 ? A.thresh[L] : 0.0;
  bool spiked_prev = n > 0 && A.spiked_prev[L];
  double prp = (n > 0 && A.stc_stream >= 0) ? A.prp[L] : 0.0;
  const bool has_stc = n > 0 && A.stc_stream >= 0 && A.has_stc[L];
  const uint64_t rbits = (A.replay && n > 0) ? A.replay_bits[L] : 0ull;
  const int32_t pq0 = n > 0 ? A.probe_ptr[L] : 0, pq1 = n > 0 ? A.probe_ptr[L + 1] : 0;

  int64_t k_begin = A.k_begin, k_end = A.k_end, k0 = A.k0, probe0 = A.probe_sample0;
  int32_t slot = A.slot;
  if (A.clock) {
    k0 = A.clock->k0;
    k_begin = k0;
    k_end = k0 + A.epoch_len;
    probe0 = A.clock->probe_sample0;
    slot = (int32_t)((k0 / A.epoch_len) % A.n_slots);
  }
  for (int64_t k = k_begin; k < k_end && n > 0; ++k) {
    const int kk = (int)(k - k0);
    const bool post = spiked_prev;
    // ---- a. synapse streams ---------------------------------------------------
    double S = 0.0, qs_field = 0.0;
    for (int s = 0; s < A.n_streams; ++s) {
      const StreamParams& P = A.sp[s];
      const StreamDev& D = A.sd[s];
      const int32_t sb = D.sbase[g], nrow = D.sbase[g + 1] - sb;
      const bool calc = P.kind == SK_GB || P.kind == SK_STC;
      const bool stc = P.kind == SK_STC;
      const uint64_t* cmg = D.cmask + (int64_t)slot * D.n_elem;
      const uint64_t* camg = calc ? D.camask + (int64_t)slot * D.n_elem : nullptr;
      TG* G = (TG*)D.g;
      const typename PR::Ec E = PR::e_const(P.e);
      const typename PR::Dc dg = PR::d_const(P.decay_g);
      typename PR::Acc carry;  // sums of the run crossing into the next row
      // one row of lookahead: the next row's synapse state loads while this
      // row is updated and folded (rows are disjoint; padding elements exist)
      int32_t n_cvf = -1;
      uint64_t n_cm = 0, n_cam = 0;
      TG n_g = PR::zero();
      double n_c = 0.0, n_w = 0.0, n_z = 0.0;
      auto fetch = [&](int t) {
        const uint32_t e = ((uint32_t)(sb + t) << 5) | (uint32_t)lane;
        n_cvf = D.cvf[e];
        n_cm = cmg[e];
        n_g = G[e];
        if (calc) {
          n_cam = camg[e];
          n_c = D.c[e];
          n_w = D.w[e];
        }
        if (stc) n_z = D.z[e];
      };
      if (nrow > 0) fetch(0);
      for (int t = 0; t < nrow; ++t) {
        const uint32_t e = ((uint32_t)(sb + t) << 5) | (uint32_t)lane;
        const int32_t cvf = n_cvf;
        const uint64_t cm = n_cm, cam = n_cam;
        const TG g_old = n_g;
        const double cc = n_c, wv = n_w, zv = n_z;
        if (t + 1 < nrow) fetch(t + 1);
        const bool valid = cvf >= 0;  // padding only after the cell's last synapse
        TG gv = PR::zero();
        double sadd = 0.0;
        if (valid) {
          const bool pre = (cm >> kk) & 1ull;
          const bool capre = calc && ((cam >> kk) & 1ull);
          // Eq. late_phase_weight with the cell's PRP, or that of the synapse's CV
          const double pz = (stc && A.prp_diff) ? A.prp_cv[e0 + (cvf >> 3)] : prp;
          gv = syn_update<PR>(P, D, e, pre, capre, post, g_old, calc ? cc : 0.0,
                              calc ? wv : 0.0, stc ? zv : 0.0, pz, k, dt, A.seed, sadd);
          G[e] = PR::decay(gv, dg);
        }
        // Per-CV sums in canonical order (the narrow kernel's accumulator
        // arithmetic): each lane sums its run from the run's first synapse in
        // this row up to itself, in order, reading the values by shuffle; a run
        // that crosses rows continues from the last lane's sums of the previous
        // row.
        const unsigned smask = __ballot_sync(full, valid && (cvf & 2));
        const unsigned upto = lane == 31 ? full : ((2u << lane) - 1u);
        const unsigned mm = smask & upto;
        const int seg0 = mm ? 31 - __clz(mm) : -1;
        const int src0 = seg0 < 0 ? 0 : seg0;
        const int len = valid ? lane - src0 + 1 : 0;
        const int maxlen = (int)__reduce_max_sync(full, (unsigned)len);
        const int32_t cs = __shfl_sync(full, cvf, src0);
        using Acc = typename PR::Acc;
        const typename Acc::C cv = Acc::template contrib<EZ>(gv, E);  // once, on its own lane
        const typename Acc::C c0 = Acc::shfl_c(cv, src0);
        Acc acc;
        if (seg0 < 0) {
          acc = carry;
          acc.template add_c<EZ>(c0);
        } else {
          // continues the sums of earlier streams unless first on its CV
          acc.template start_c<EZ>(c0, !valid || (cs & 1), GS, ES, (uint32_t)(e0 + (cs >> 3)));
        }
        bool sparse = false;
        if constexpr (Acc::kZeroRuns) {
          // Exact zeros in the in-order sums.  Adding a zero changes a partial
          // sum only when that sum is itself a zero (IEEE: x + 0 = x for
          // x != 0); a sum that has taken a nonzero term is never -0 again
          // (exact cancellation gives +0), and a zero plus a nonzero t is t.
          // So each lane's sum over lanes src0 + 1 .. lane equals the sum of
          // its nonzero terms in order, followed by the sign rule of zeros
          // (add_zeros: +0 if the range holds a +0 and the sum is a zero).
          // Where the row has fewer nonzero terms than the dense fold has
          // steps, only those are added (all-zero rows: none).
          const unsigned nzm = __ballot_sync(full, valid && !Acc::zero_c(cv));
          if (__popc(nzm) + 1 < maxlen) {
            sparse = true;
            const unsigned pg = __ballot_sync(full, valid && Acc::pos_zero_g(cv));
            const unsigned pe = __ballot_sync(full, valid && Acc::pos_zero_e(cv));
            const unsigned rng = len > 1 ? (upto & ~((2u << src0) - 1u)) : 0u;
#pragma unroll 1
            for (unsigned mm = nzm; mm; mm &= mm - 1u) {
              const int qn = __ffs(mm) - 1;
              const typename Acc::C ci = Acc::shfl_c(cv, qn);
              if ((rng >> qn) & 1u) acc.template add_c<EZ>(ci);
            }
            acc.add_zeros((pg & rng) != 0u, (pe & rng) != 0u);
          }
        }
        if (!sparse) {
          for (int it = 1; it < maxlen; ++it) {
            const int src = src0 + it < 31 ? src0 + it : 31;
            const typename Acc::C ci = Acc::shfl_c(cv, src);
            if (it < len) acc.template add_c<EZ>(ci);
          }
        }
        if (valid && (cvf & 4)) acc.template store<EZ>(GS, ES, (uint32_t)(e0 + (cvf >> 3)), E);
        carry = acc.shfl(31);
        if (stc) {
          // the cell's S = sum |h - h0| over its STC synapses, in order.  S
          // starts at +0 and every term is >= +0, so a term of +0 (h = h0
          // exactly) leaves S unchanged: only the nonzero terms are added,
          // still in order
          unsigned nz = __ballot_sync(full, valid && !is_zero_bits(sadd));
#pragma unroll 1
          while (nz) {
            const int q = __ffs(nz) - 1;
            nz &= nz - 1u;
            S = S + __shfl_sync(full, sadd, q);
          }
        }
      }
      __syncwarp();  // this stream's sums are visible to later streams and the solve
      if (s == A.stc_stream && has_stc) {
        const double qs = (S > P.theta_pro) ? P.p_max : 0.0;
        if (A.prp_diff) qs_field = qs;  // the field takes its step after the voltage solve
        else prp = prp + P.rate_p * (qs - prp);
      }
    }

    // ---- b. backward pass by branch levels ---------------------------------------
    double v0_old = 0.0, v0_new = 0.0;
    R x0r = RW::zero();  // the soma's new V in the row form
    const double iinj = (k >= kon && k < koff) ? iinj_val : 0.0;
    for (int lv = 0; lv < wc.n_lvl; ++lv) {
      const int b0 = A.wlvl[wc.lvl0 + lv], b1 = A.wlvl[wc.lvl0 + lv + 1];
      for (int b = b0 + lane; b < b1; b += 32) {
        const int bs = A.wbr_s[wc.br0 + b], be = A.wbr_e[wc.br0 + b];
        // the children of the branch's last row (eliminated at lower levels): the
        // first (be + 1) and the highest other one, loaded with the first row; a
        // row inside a branch has exactly one child, the next row
        const int c1 = A.wbr_c[wc.br0 + b], co = A.wbr_o[wc.br0 + b];
        R f1 = RW::zero(), x1 = RW::zero(), a1 = RW::zero(), fo = RW::zero(), xo = RW::zero(),
          ao = RW::zero();
        int cn = -1;
        if (c1 >= 0) {
          f1 = F[e0 + c1]; x1 = XP[e0 + c1]; a1 = AA[e0 + c1];
        }
        if (co >= 0) {
          fo = F[e0 + co]; xo = XP[e0 + co]; ao = AA[e0 + co]; cn = OCN[e0 + co];
        }
        R cf = RW::zero(), ca = RW::zero(), cx = RW::zero();
        // one row of lookahead: the next row's values load during this row's
        // elimination
        R nv = Vg[e0 + be], ncdt = CDT[e0 + be], ndc = DC[e0 + be],
          nem = em_der ? RW::zero() : EM[e0 + be], na = AA[e0 + be];
        TS ngs = GS[e0 + be], nes = EZ ? PR::s_zero() : ES[e0 + be];
        for (int i = be; i >= bs; --i) {
          const int64_t ei = e0 + i;
          const R v = nv, cdt = ncdt, dcv = ndc, emv = nem, ai = na;
          const R gsv = PR::sum_r(ngs);
          const R esv = PR::sum_r(nes);  // (EZ: unused)
          if (i > bs) {
            const int64_t en = ei - 1;
            nv = Vg[en]; ncdt = CDT[en]; ndc = DC[en]; na = AA[en];
            if (!em_der) nem = EM[en];
            ngs = GS[en];
            if (!EZ) nes = ES[en];
          }
          R d, bb;
          if (i == 0) {
            v0_old = RW::to_d(v);
            if (hh) {
              double gmt, emt;
              soma.currents(A, L, gmt, emt);
              d = RW::add(RW::add(dcv, RW::from_d(gmt)), gsv);
              bb = RW::add(RW::fma(cdt, v, RW::from_d(emt)), RW::from_d(iinj));
            } else {
              d = RW::add(dcv, gsv);
              const R em = em_der ? RW::from_d(A.em_soma[L]) : emv;
              bb = RW::add(RW::fma(cdt, v, em), RW::from_d(iinj));
            }
          } else {
            d = RW::add(dcv, gsv);
            bb = RW::fma(cdt, v, em_der ? RW::mul(cdt, emk) : emv);
          }
          if constexpr (!EZ) {
            bb = RW::add(bb, esv);
          } else if constexpr (std::is_same<R, double>::value) {
            bb = ez_add(bb, (const TS*)ES, (uint32_t)ei);  // (float-float: not added)
          }
          if (i == be) {
            // the other children, highest index first, then the first child
            if (co >= 0) {
              other_child<RW>(ao, fo, xo, d, bb);
              for (int ch = cn; ch >= 0; ch = OCN[e0 + ch]) {  // a third child and more
                const int64_t ec = e0 + ch;
                other_child<RW>(AA[ec], F[ec], XP[ec], d, bb);
              }
            }
            if (c1 >= 0) {
              d = RW::fnma(f1, a1, d);
              bb = RW::fnma(a1, x1, bb);
            }
          } else {
            // row i + 1 of this branch, eliminated just before
            d = RW::fnma(cf, ca, d);
            bb = RW::fnma(ca, cx, bb);
          }
          if (i > 0) {
            const R rr = RW::rcp(d);
            const R fi = RW::mul(ai, rr);
            const R xi = RW::mul(bb, rr);
            F[ei] = fi;
            XP[ei] = xi;
            cf = fi; ca = ai; cx = xi;  // row i - 1 of this branch has i as its first child
          } else {
            x0r = RW::mul(bb, RW::rcp(d));
            v0_new = RW::to_d(x0r);
          }
        }
      }
      __syncwarp();
    }
    // ---- c. forward pass, root level first ------------------------------------------
    for (int lv = wc.n_lvl - 1; lv >= 0; --lv) {
      const int b0 = A.wlvl[wc.lvl0 + lv], b1 = A.wlvl[wc.lvl0 + lv + 1];
      for (int b = b0 + lane; b < b1; b += 32) {
        const int bs = A.wbr_s[wc.br0 + b], be = A.wbr_e[wc.br0 + b];
        R vp;
        int i = bs;
        if (bs == 0) {
          Vg[e0] = x0r;
          vp = x0r;
          i = 1;
        } else {
          vp = Vg[e0 + A.wbr_p[wc.br0 + b]];
        }
        // a chunk of the branch's f and x' is loaded at once (the chain has one
        // FP64 operation per row, far shorter than a load's latency)
        for (; i <= be; i += kWideFwdChunk) {
          R fr[kWideFwdChunk], xr[kWideFwdChunk];
#pragma unroll
          for (int q = 0; q < kWideFwdChunk; ++q) {
            if (i + q <= be) {
              fr[q] = F[e0 + i + q];
              xr[q] = XP[e0 + i + q];
            }
          }
#pragma unroll
          for (int q = 0; q < kWideFwdChunk; ++q) {
            if (i + q <= be) {
              const R vi = RW::fnma(fr[q], vp, xr[q]);
              Vg[e0 + i + q] = vi;
              vp = vi;
            }
          }
        }
      }
      __syncwarp();
    }
    // ---- d. a diffusing PRP field, by the same levels ----------------------------
    if (A.prp_diff && has_stc) {
      const double rate = A.sp[A.stc_stream].rate_p;
      double x0 = 0.0;
      for (int lv = 0; lv < wc.n_lvl; ++lv) {
        const int b0 = A.wlvl[wc.lvl0 + lv], b1 = A.wlvl[wc.lvl0 + lv + 1];
        for (int b = b0 + lane; b < b1; b += 32) {
          const int bs = A.wbr_s[wc.br0 + b], be = A.wbr_e[wc.br0 + b];
          double cf = 0.0, ca = 0.0, cx = 0.0;
          bool carry = false;
          for (int i = be; i >= bs; --i) {
            const int64_t ei = e0 + i;
            const double pv = A.prp_cv[ei];
            const double src = (i == 0) ? __dmul_rn(qs_field, A.prp_src[L]) : 0.0;
            const double ps = __dadd_rn(pv, __dmul_rn(rate, __dsub_rn(src, pv)));
            double d = A.prp_dg[ei];
            double bb = __dmul_rn(A.prp_vdt[ei], ps);
            if (PAR) {
              for (int ch = OCH[ei]; ch >= 0; ch = OCN[e0 + ch]) {
                const int64_t ec = e0 + ch;
                const double ac = A.prp_a[ec];
                d = __fma_rn(-Fd[ec], ac, d);
                bb = __fma_rn(-ac, XPd[ec], bb);
              }
            }
            if (carry) {
              d = __fma_rn(-cf, ca, d);
              bb = __fma_rn(-ca, cx, bb);
            } else if (i == be && PAR && i + 1 < n && PAR[ei + 1] == i) {
              const double ac = A.prp_a[ei + 1];
              d = __fma_rn(-Fd[ei + 1], ac, d);
              bb = __fma_rn(-ac, XPd[ei + 1], bb);
            }
            if (i > 0) {
              const double ai = A.prp_a[ei];
              const double rr = rcp_rn_pos(d);
              const double fi = __dmul_rn(ai, rr);
              const double xi = __dmul_rn(bb, rr);
              Fd[ei] = fi;
              XPd[ei] = xi;
              carry = true;
              cf = fi; ca = ai; cx = xi;
            } else {
              x0 = __dmul_rn(bb, rcp_rn_pos(d));
            }
          }
        }
        __syncwarp();
      }
      for (int lv = wc.n_lvl - 1; lv >= 0; --lv) {
        const int b0 = A.wlvl[wc.lvl0 + lv], b1 = A.wlvl[wc.lvl0 + lv + 1];
        for (int b = b0 + lane; b < b1; b += 32) {
          const int bs = A.wbr_s[wc.br0 + b], be = A.wbr_e[wc.br0 + b];
          double pp;
          int i = bs;
          if (bs == 0) {
            A.prp_cv[e0] = x0;
            pp = x0;
            i = 1;
          } else {
            pp = A.prp_cv[e0 + PAR[e0 + bs]];
          }
          for (; i <= be; ++i) {
            const int64_t ei = e0 + i;
            const double xi = __fma_rn(-Fd[ei], pp, XPd[ei]);
            A.prp_cv[ei] = xi;
            pp = xi;
          }
        }
        __syncwarp();
      }
      prp = __shfl_sync(full, x0, 0);  // the root branch runs on lane 0
    }
    for (int32_t q = pq0 + lane; q < pq1; q += 32) {
      const int64_t smp = probe0 + (k - k_begin);
      if (smp < A.probe_cap) {
        A.probe_buf[smp * A.n_probe + A.probe_id[q]] = RW::to_d(Vg[e0 + A.probe_row[q]]);
      } else {
        atomicOr(A.err_flags, 1);
      }
    }
    // ---- e. soma gates, detection (lane 0) -------------------------------------------
    bool spk = false;
    // (FP64 policy: its unit is compiled without contraction, so the spread
    // update is the sequential one bit for bit; the other policies keep the
    // narrow kernel's code on lane 0)
    constexpr bool kSpreadHH = PR::kId == PrecF64::kId;
    if constexpr (kSpreadHH) {
      if (hh) hh64_update_warp(soma, __shfl_sync(full, v0_new, 0), dt, lane);
    }
    if (lane == 0) {
      if constexpr (!kSpreadHH) {
        if (hh) soma.update(v0_new, dt);
      }
      spk = v0_old < th && v0_new >= th;
      if (spk) {
        const int slot_ = atomicAdd(A.spk_count, 1);
        if (slot_ < A.spk_cap) {
          A.spk_gid[slot_] = A.gid[L];
          A.spk_step[slot_] = (int32_t)k;
          A.spk_t[slot_] = (double)k * dt + dt * ((th - v0_old) / (v0_new - v0_old));
        }
      }
    }
    spk = __shfl_sync(full, spk, 0);
    spiked_prev = A.replay ? (((rbits >> (k - k_begin)) & 1ull) != 0) : spk;
  }
  if (n > 0 && lane == 0) {
    A.spiked_prev[L] = spiked_prev ? 1 : 0;
    if (hh) {
      soma.store(A.gate, A.n_lanes, L);
    }
    if (has_stc) A.prp[L] = prp;
  }
}

template <class PR>
int launch_wide_impl(const EpochArgs& a, void* stream) {
  if (a.n_wide <= 0) return 0;
  const int threads = 128;
  const int blocks = (int)(((int64_t)a.n_wide * 32 + threads - 1) / threads);
  if (a.es_zero)
    wide_kernel<PR, true><<<blocks, threads, 0, (cudaStream_t)stream>>>(a);
  else
    wide_kernel<PR, false><<<blocks, threads, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

// Both cell bins of one epoch (see SideLaunch).
template <class PR>
int launch_bins(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  if (side && a.n_narrow > 0 && a.n_wide > 0) {
    cudaStream_t s0 = (cudaStream_t)stream, s1 = (cudaStream_t)side->stream;
    cudaError_t e = cudaEventRecord((cudaEvent_t)side->fork, s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s1, (cudaEvent_t)side->fork, 0);
    if (e != cudaSuccess) return (int)e;
    int rc = launch_epoch_impl<PR>(a, tree, shape, stream);
    if (rc == 0) rc = launch_wide_impl<PR>(a, side->stream);
    e = cudaEventRecord((cudaEvent_t)side->join, s1);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, (cudaEvent_t)side->join, 0);
    return rc ? rc : (int)e;
  }
  const int rc = launch_epoch_impl<PR>(a, tree, shape, stream);
  return rc ? rc : launch_wide_impl<PR>(a, stream);
}

}  // namespace pa
