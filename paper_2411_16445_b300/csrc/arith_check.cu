// arith_check.cu -- device self-check of the integer FP64 routines of
// int_arith.cuh against the GPU's own IEEE operations (division by the
// correctly rounded FP64 divide; float->double by the hardware conversion).
// Compiled without contraction like the FP64 kernels that use the routines.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "int_arith.cuh"

namespace pa {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void check_rcp(uint64_t bits, unsigned long long* out) {
  const double d = __longlong_as_double((long long)bits);
  const double got = rcp_rn_pos(d);
  const double want = 1.0 / d;
  const bool same = __double_as_longlong(got) == __double_as_longlong(want) ||
                    (got != got && want != want);
  if (!same) {
    atomicAdd(&out[0], 1ull);
    atomicCAS(&out[3], 0ull, (unsigned long long)bits);
  }
}

// Every single-precision seed: all 2^23 top-fraction patterns of M, each with
// eight low-bit patterns and a pseudo-random exponent.
__global__ void rcp_seed_sweep(uint64_t seed, unsigned long long* out) {
  const uint64_t total = (1ull << 23) * 8;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t top = i >> 3, v = i & 7;
    const uint64_t h = mix64(seed ^ (i * 0x9e3779b97f4a7c15ULL));
    uint64_t low;
    switch (v) {
      case 0: low = 0; break;
      case 1: low = 1; break;
      case 2: low = (1ull << 29) - 1; break;
      case 3: low = 1ull << 28; break;
      default: low = h & ((1ull << 29) - 1); break;
    }
    const uint64_t ex = 1 + (h >> 40) % 2044;
    check_rcp((ex << 52) | (top << 29) | low, out);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&out[2], (unsigned long long)total);
}

// n random inputs: 15/16 positive normals with any exponent that has a normal
// reciprocal, 1/16 arbitrary bit patterns (zeros, subnormals, negatives, huge,
// inf, nan take the fallback).
__global__ void rcp_random(uint64_t seed, int64_t n, unsigned long long* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed + 0x632be59bd9b4e019ULL * (uint64_t)(i + 1));
    uint64_t bits;
    if ((h & 15) == 0) {
      bits = mix64(h);
    } else {
      const uint64_t ex = 1 + (mix64(h) % 2044);
      bits = (ex << 52) | (h >> 12);
    }
    check_rcp(bits, out);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&out[2], (unsigned long long)n);
}

// Every float bit pattern.
__global__ void widen_all(unsigned long long* out) {
  const uint64_t total = 1ull << 32;
  unsigned long long bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float v = __uint_as_float((uint32_t)i);
    const double got = widen_f32(v), want = (double)v;
    if (!(__double_as_longlong(got) == __double_as_longlong(want) ||
          (got != got && want != want)))
      ++bad;
  }
  if (bad) atomicAdd(&out[1], bad);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&out[2], (unsigned long long)total);
}

// FP64 FMA throughput: eight independent FMA chains per thread (enough to
// cover the dependent latency at full occupancy), values kept bounded
// (x <- x a + b with 0 < a < 1); the result is stored only if it hits an
// impossible value, so the chains cannot be removed.
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, double a, double b,
                                                       double* sink) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (threadIdx.x + 1) + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == -1.0) sink[0] = s;
}

}  // namespace

int launch_fma_rate(int blocks, int iters, double* sink, void* stream) {
  fma_rate_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 0.9999999, 1e-7, sink);
  return (int)cudaGetLastError();
}

int launch_arith_check(uint64_t seed, int64_t n_random, unsigned long long* d_out, int n_sm,
                       void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = 8 * (n_sm > 0 ? n_sm : 1);
  rcp_seed_sweep<<<grid, 256, 0, s>>>(seed, d_out);
  if (n_random > 0) rcp_random<<<grid, 256, 0, s>>>(seed, n_random, d_out);
  widen_all<<<grid, 256, 0, s>>>(d_out);
  return (int)cudaGetLastError();
}

}  // namespace pa
