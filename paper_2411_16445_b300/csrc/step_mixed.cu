// step_mixed.cu -- mixed-precision instantiation of the epoch kernels
// (PA_MIXED): synaptic conductances in float-float on the FP32 pipes, event
// weights and STDP traces in FP32, per-CV synaptic sums and everything else
// (voltage, cable coefficients, assembly, Hines solve, HH, calcium, the slow
// plasticity state) in FP64.  Multiply-add contraction stays on: the
// float-float operations are written with explicitly rounded intrinsics.
#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {
int launch_epoch_mixed(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  return launch_bins<PrecMix>(a, tree, shape, stream, side);
}
int launch_epoch_grouped_mixed(const EpochArgs* d_args, const int2* d_bmap, int n_blocks, bool tree,
                            bool ez, void* stream) {
  return launch_epoch_grouped_impl<PrecMix>(d_args, d_bmap, n_blocks, tree, ez, stream);
}
}  // namespace pa
