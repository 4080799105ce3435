// epoch_noalloc.cu -- the epoch kernels with their Hines elimination scratch
// (the per-CV f and x' values of one step) taken from a fixed array in device
// global memory that this library defines, instead of from the model's own
// allocation.  Used by pa_advance_noalloc.
//
// The array is reserved on every GPU that loads the library and stays reserved
// until the process exits.  Its contents are not cleared between calls: every
// step writes f and x' of a row before reading them back, so no value has to
// start at zero.  All calls share this one array, so two pa_advance_noalloc
// calls whose work overlaps on the GPU (for instance on two streams) race on it
// and must not be issued that way.
//
// This unit instantiates no kernel: it launches the kernels of the precision
// units (step_fp64.cu, step_mixed.cu, step_fp32.cu), built with their own
// contraction flags, on a copy of the arguments whose scratch pointers name the
// array.  The results therefore equal those of pa_advance bit for bit in every
// precision.
#include <cuda_runtime.h>

#include <atomic>

#include "engine.h"

namespace pa {

// f and x' for up to kNoallocMaxPaddedCV padded CVs (32 MiB of doubles).
constexpr int64_t kNoallocMaxPaddedCV = 2 * 1024 * 1024;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxPaddedCV];

namespace {
constexpr int kMaxDevices = 64;
// The array's device address per device, looked up on the first call there.
// Atomic: first calls from several host threads may race; each stores the
// same address.
std::atomic<double*> g_scratch_dev_ptr[kMaxDevices];
}  // namespace

int64_t noalloc_max_padded_cv() { return kNoallocMaxPaddedCV; }

// Returns 0 or a cudaError_t value; -1 if the model is larger than the array.
int launch_epoch_noalloc(const EpochArgs& a, int64_t n_padded_cv, bool tree, int prec,
                         int shape, void* stream) {
  if (n_padded_cv > kNoallocMaxPaddedCV) return -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  double* base = g_scratch_dev_ptr[dev].load(std::memory_order_acquire);
  if (!base) {
    // The name of a __device__ array is only a host-side handle: its device
    // address is looked up once per device, with that device current.
    e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    g_scratch_dev_ptr[dev].store(base, std::memory_order_release);
  }
  EpochArgs b = a;
  b.f = base;
  b.xp = base + n_padded_cv;
  return launch_epoch(prec, b, tree, shape, stream);
}

}  // namespace pa
