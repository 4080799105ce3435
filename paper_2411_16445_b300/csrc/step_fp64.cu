// step_fp64.cu -- FP64 instantiation of the epoch kernels (both cell bins).
// Built with --fmad=false: no multiply-add contraction beyond the explicit
// fma() calls, so the arithmetic is the plain definition, operation for
// operation.
#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {
int launch_epoch_fp64(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  return launch_bins<PrecF64>(a, tree, shape, stream, side);
}
int launch_epoch_grouped_fp64(const EpochArgs* d_args, const int2* d_bmap, int n_blocks, bool tree,
                            bool ez, void* stream) {
  return launch_epoch_grouped_impl<PrecF64>(d_args, d_bmap, n_blocks, tree, ez, stream);
}
// Steady-state HH gates x_inf = alpha / (alpha + beta) at each soma's v_init.
__global__ void init_gates_kernel(const double* v, double* gate, int64_t n_lanes,
                                  const uint8_t* is_hh) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= n_lanes || !is_hh[L]) return;
  double am, bm, ah, bh, an, bn;
  HH64::rates(v[L], am, bm, ah, bh, an, bn);
  gate[L] = am / (am + bm);
  gate[n_lanes + L] = ah / (ah + bh);
  gate[2 * n_lanes + L] = an / (an + bn);
}

int launch_init_gates(const double* v, void* gate, int64_t n_lanes, const uint8_t* is_hh,
                      void* stream) {
  if (n_lanes == 0) return 0;
  const int threads = 128;
  const int blocks = (int)((n_lanes + threads - 1) / threads);
  init_gates_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(v, (double*)gate, n_lanes,
                                                                  is_hh);
  return (int)cudaGetLastError();
}

}  // namespace pa
