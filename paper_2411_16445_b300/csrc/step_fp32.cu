// step_fp32.cu -- the FP32-synapse instantiation of the epoch kernels
// (PA_FP32): synaptic conductances, event weights, STDP traces and the per-CV
// synaptic sums in plain FP32; everything else as in PA_MIXED.
#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {
int launch_epoch_fp32(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  return launch_bins<PrecF32>(a, tree, shape, stream, side);
}
int launch_epoch_grouped_fp32(const EpochArgs* d_args, const int2* d_bmap, int n_blocks, bool tree,
                            bool ez, void* stream) {
  return launch_epoch_grouped_impl<PrecF32>(d_args, d_bmap, n_blocks, tree, ez, stream);
}
}  // namespace pa
