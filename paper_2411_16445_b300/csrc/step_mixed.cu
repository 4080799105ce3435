// step_mixed.cu -- mixed-precision instantiation of the epoch kernel:
// synaptic conductances, STDP traces and the per-CV synaptic sums in FP32;
// voltage, cable coefficients, assembly, Hines solve, HH, calcium (a threshold
// variable) and the slow plasticity state in FP64.
#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {
int launch_epoch_mixed(const EpochArgs& a, bool tree, int shape, void* stream, const SideLaunch* side) {
  return launch_bins<float>(a, tree, shape, stream, side);
}
int launch_init_gates_mixed(const double* v, void* gate, int64_t n_lanes,
                           const uint8_t* is_hh, void* stream) {
  return launch_init_gates_impl<float>(v, gate, n_lanes, is_hh, stream);
}
}  // namespace pa
