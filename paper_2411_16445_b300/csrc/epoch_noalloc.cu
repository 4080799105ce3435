// epoch_noalloc.cu -- the epoch kernel with its Hines elimination scratch (the
// per-CV f and x' values of one step) taken from a fixed array in device
// global memory that this library defines, instead of from the model's own
// allocation.  Used by pa_advance_noalloc.
//
// The array is reserved once per GPU when the library is loaded and stays
// reserved until the process exits.  Its contents are not cleared between
// calls: every step writes f and x' of a row before reading them back, so no
// value has to start at zero.  All calls share this one array, so two
// pa_advance_noalloc calls whose work overlaps on the GPU (for instance on two
// streams) race on it and must not be issued that way.
//
// Built with --fmad=false like the FP64 kernel it mirrors, so the FP64 results
// equal those of pa_advance bit for bit.
#include <cuda_runtime.h>

#include "epoch_kernel.cuh"
#include "wide_kernel.cuh"

namespace pa {

// f and x' for up to kNoallocMaxPaddedCV padded CVs (32 MiB of doubles).
constexpr int64_t kNoallocMaxPaddedCV = 2 * 1024 * 1024;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxPaddedCV];

namespace {
constexpr int kMaxDevices = 64;
double* g_scratch_dev_ptr[kMaxDevices] = {nullptr};
}  // namespace

int64_t noalloc_max_padded_cv() { return kNoallocMaxPaddedCV; }

// Returns 0 or a cudaError_t value; -1 if the model is larger than the array.
int launch_epoch_noalloc(const EpochArgs& a, int64_t n_padded_cv, bool tree, bool mixed,
                         int shape, void* stream) {
  if (n_padded_cv > kNoallocMaxPaddedCV) return -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  if (!g_scratch_dev_ptr[dev]) {
    // The name of a __device__ array is only a host-side handle: its device
    // address is looked up once per device, with that device current.
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    g_scratch_dev_ptr[dev] = p;
  }
  EpochArgs b = a;
  b.f = g_scratch_dev_ptr[dev];
  b.xp = g_scratch_dev_ptr[dev] + n_padded_cv;
  int rc = mixed ? launch_epoch_impl<float>(b, tree, shape, stream)
                 : launch_epoch_impl<double>(b, tree, shape, stream);
  if (rc == 0) rc = mixed ? launch_wide_impl<float>(b, stream) : launch_wide_impl<double>(b, stream);
  return rc;
}

}  // namespace pa
