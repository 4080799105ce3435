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

// The long-step update of one GB or STC synapse (element e of stream s);
// returns |h - h0| for an STC synapse (0 for GB).
__device__ __forceinline__ double ff_synapse(const EpochArgs& A, const FastForward& F, int s,
                                             int64_t e, double pz) {
  const StreamParams& P = A.sp[s];
  const StreamDev& D = A.sd[s];
  if (P.kind == SK_GB) {
    const double w = D.w[e];
    const double Aw = (w * (1.0 - w)) * (P.w_star - w);
    D.w[e] = w + F.rate_w[s] * (-Aw);
    return 0.0;
  }
  const double h = D.w[e], z = D.z[e], h0 = P.h0;
  const double T1 = ((h - h0) > P.theta_tag) ? (pz * P.f_int) * (1.0 - z) : 0.0;
  const double T2 = ((h0 - h) > P.theta_tag) ? (pz * P.f_int) * (z + 0.5) : 0.0;
  D.z[e] = z + F.rate_z[s] * (T1 - T2);
  D.w[e] = h + F.rate_h[s] * (0.1 * (h0 - h));
  return fabs(h - h0);
}

// A wide-bin cell: the whole warp, its synapses 32 at a time (contiguous, so
// the loads coalesce); the cell's S = sum |h - h0| folded in canonical order
// through shuffles, as the narrow lane sums it; lane 0 then steps p or the
// diffusing PRP field.
template <bool TREE>
__device__ void ff_slow_wide(const EpochArgs& A, const FastForward& F, int64_t g, int lane) {
  const unsigned full = 0xffffffffu;
  const int64_t L = g << 5;
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
      for (int64_t t = 0; t < rows; ++t) {
        const int64_t e = (sb << 5) + t * 32 + lane;
        const int32_t cvf = D.cvf[e];
        double sadd = 0.0;
        if (cvf >= 0) {
          const double pz = field ? A.prp_cv[((uint32_t)rb << 5) + (uint32_t)(cvf >> 3)] : pk;
          sadd = ff_synapse(A, F, s, e, pz);
        }
        if (P.kind == SK_STC) {
#pragma unroll 1
          for (int q = 0; q < 32; ++q) {
            const double sq = __shfl_sync(full, sadd, q);
            if (__shfl_sync(full, cvf, q) >= 0) S = S + sq;
          }
        }
      }
    }
    if (has_stc) {
      const StreamParams& P = A.sp[A.stc_stream];
      const double qs = (S > P.theta_pro) ? P.p_max : 0.0;
      if (field) {
        if (lane == 0)
          p = prp_field_step<TREE, true>(A, rb, 0, L, A.ncv[L], qs, F.rate_p, F.prp_dg_long,
                                         F.prp_vdt_long);
        __syncwarp();
        p = __shfl_sync(full, p, 0);
      } else {
        p = pk + F.rate_p * (qs - pk);
      }
    }
  }
  if (has_stc && lane == 0) A.prp[L] = p;
}

// One thread per lane (cell) of the narrow bin, one warp per cell of the wide
// bin: the long steps of its GB and STC synapses.
template <bool TREE>
__global__ void ff_slow_kernel(const EpochArgs A, const FastForward F) {
  const int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (L >= A.n_lanes) return;
  const int64_t g = L >> 5, l = L & 31;
  const bool wide = g >= A.n_narrow;
  if (wide) {
    if (A.ncv[g << 5] > 0) ff_slow_wide<TREE>(A, F, g, (int)l);
    return;
  }
  if (A.ncv[L] == 0) return;
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
      for (int64_t j = 0; j < rows; ++j) {
        const int64_t e = ((sb + j) << 5) + l;
        if (D.cvf[e] < 0) continue;
        const uint32_t cv = (uint32_t)(D.cvf[e] >> 3);
        const double pz = field ? A.prp_cv[((uint32_t)(rb + cv) << 5) | (uint32_t)l] : pk;
        const double sadd = ff_synapse(A, F, s, e, pz);
        if (P.kind == SK_STC) S = S + sadd;
      }
    }
    if (has_stc) {
      const StreamParams& P = A.sp[A.stc_stream];
      const double qs = (S > P.theta_pro) ? P.p_max : 0.0;
      if (field)
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
