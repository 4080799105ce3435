// step_fp64.cu -- FP64 instantiation of the epoch kernel.  Built with
// --fmad=false: no multiply-add contraction beyond the explicit fma() calls,
// so the arithmetic is the plain definition, operation for operation.
#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {
int launch_epoch_fp64(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  return launch_bins<double>(a, tree, shape, stream, side);
}
int launch_init_gates_fp64(const double* v, void* gate, int64_t n_lanes,
                           const uint8_t* is_hh, void* stream) {
  return launch_init_gates_impl<double>(v, gate, n_lanes, is_hh, stream);
}
}  // namespace pa
