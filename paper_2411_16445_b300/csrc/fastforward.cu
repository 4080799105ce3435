// fastforward.cu -- pa_fast_forward: long biological times without spiking
// and calcium dynamics (the '8h-recall' paradigm of the recurrent network with
// tagging and capture).  The membrane state is kept; every conductance and
// calcium decays by its exact factor exp(-T / tau); the slow plasticity
// variables take n_long forward-Euler steps of T / n_long with the calcium
// terms (and so the noise) off, in the order of a full step: per cell, S from
// h before the update, then per synapse z (with the cell's p) and h
// (relaxation to h0), GB w (its cubic drift), then p -- or, for a diffusing
// PRP field, its explicit reaction and backward-Euler diffusion with the long
// step's matrix (z then captures the PRP at its own CV).  Everything stays in
// HBM: no state leaves the device.  Built without contraction like the FP64
// kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "prp_field.cuh"

namespace pa {
namespace {

// prec: 0 = FP64 conductances, 1 = float-float (hi, lo), 2 = FP32
__global__ void ff_decay_kernel(StreamDev D, double decay_g, double decay_c, int prec) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < D.n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (prec == 2) {
      float* g = (float*)D.g;
      g[e] = (float)((double)g[e] * decay_g);
    } else if (prec == 1) {
      float2* g = (float2*)D.g;
      const double v = ((double)g[e].x + (double)g[e].y) * decay_g;
      const float hi = (float)v;
      g[e] = make_float2(hi, (float)(v - (double)hi));
    } else {
      double* g = (double*)D.g;
      g[e] = g[e] * decay_g;
    }
    if (D.c) D.c[e] = D.c[e] * decay_c;
  }
}

// One thread per lane (cell): the long steps of its GB and STC synapses.
template <bool TREE>
__global__ void ff_slow_kernel(const EpochArgs A, const FastForward F) {
  const int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (L >= A.n_lanes) return;
  if (A.ncv[L] == 0) return;
  const int64_t g = L >> 5, l = L & 31;
  const bool wide = g >= A.n_narrow;
  const bool has_stc = A.stc_stream >= 0 && A.has_stc[L];
  const bool field = has_stc && A.prp_diff;
  const int32_t rb = A.row_base[g];
  double p = has_stc ? A.prp[L] : 0.0;
  for (int64_t it = 0; it < F.n_long; ++it) {
    double S = 0.0;
    const double pk = p;
    for (int s = 0; s < A.n_streams; ++s) {
      const StreamParams& P = A.sp[s];
      if (P.kind != SK_GB && P.kind != SK_STC) continue;
      const StreamDev& D = A.sd[s];
      const int64_t sb = D.sbase[g], rows = D.sbase[g + 1] - sb;
      const int64_t cnt = wide ? rows * 32 : rows;
      for (int64_t j = 0; j < cnt; ++j) {
        const int64_t e = wide ? (sb << 5) + j : ((sb + j) << 5) + l;
        if (D.cvf[e] < 0) continue;
        if (P.kind == SK_GB) {
          const double w = D.w[e];
          const double Aw = (w * (1.0 - w)) * (P.w_star - w);
          D.w[e] = w + F.rate_w[s] * (-Aw);
        } else {
          const double h = D.w[e], z = D.z[e], h0 = P.h0;
          S = S + fabs(h - h0);
          const uint32_t cv = (uint32_t)(D.cvf[e] >> 3);
          const double pz =
              field ? A.prp_cv[wide ? ((uint32_t)rb << 5) + cv : ((uint32_t)(rb + cv) << 5) | (uint32_t)l]
                    : pk;
          const double T1 = ((h - h0) > P.theta_tag) ? (pz * P.f_int) * (1.0 - z) : 0.0;
          const double T2 = ((h0 - h) > P.theta_tag) ? (pz * P.f_int) * (z + 0.5) : 0.0;
          D.z[e] = z + F.rate_z[s] * (T1 - T2);
          D.w[e] = h + F.rate_h[s] * (0.1 * (h0 - h));
        }
      }
    }
    if (has_stc) {
      const StreamParams& P = A.sp[A.stc_stream];
      const double qs = (S > P.theta_pro) ? P.p_max : 0.0;
      if (field && wide)
        p = prp_field_step<TREE, true>(A, rb, 0, L, A.ncv[L], qs, F.rate_p, F.prp_dg_long,
                                       F.prp_vdt_long);
      else if (field)
        p = prp_field_step<TREE>(A, rb, (int)l, L, A.ncv[L], qs, F.rate_p, F.prp_dg_long,
                                 F.prp_vdt_long);
      else
        p = pk + F.rate_p * (qs - pk);
    }
  }
  if (has_stc) A.prp[L] = p;
}

}  // namespace

int launch_fast_forward(const EpochArgs& a, const FastForward& f, int prec, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  for (int s = 0; s < a.n_streams; ++s) {
    const int64_t ne = a.sd[s].n_elem;
    if (ne == 0) continue;
    int blocks = (int)((ne + 255) / 256);
    if (blocks > 148 * 16) blocks = 148 * 16;
    ff_decay_kernel<<<blocks, 256, 0, st>>>(a.sd[s], f.decay_g[s], f.decay_c[s], prec);
  }
  if (a.n_lanes > 0) {
    const int blocks = (int)((a.n_lanes + 127) / 128);
    if (f.tree) ff_slow_kernel<true><<<blocks, 128, 0, st>>>(a, f);
    else ff_slow_kernel<false><<<blocks, 128, 0, st>>>(a, f);
  }
  return (int)cudaGetLastError();
}

}  // namespace pa
