// events.cu -- Poisson drive, CSR spike routing and the spike record.
//
// Events are kept as per-synapse bitmasks, one 64-bit word per synapse and
// epoch slot: bit (k mod E) of slot (k / E) mod n_slots says "a conductance
// event reaches this synapse in step k" (cmask) or "a delayed presynaptic
// calcium jump does" (camask, the second target of Sec. "Multiple
// postsynaptic variables ..." at t_c,delay).  Each connection owns its synapse
// and a cell spikes at most once per step, so an event carries no payload and
// OR-ing bits is order independent: routing is deterministic without a sort.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "rng.cuh"

namespace pa {

// One thread per Poisson-driven synapse: draws its spikes for steps
// [k_from, k_to) (one Threefry call per 8 steps: key = seed, counter =
// {train id, step / 8, 1, 0}; the word of step k is 32-bit half (k mod 2)
// of output word (k mod 8) / 2) and sets the event bits, plus the calcium
// jump t_c,delay later for calcium-plastic synapses.
__global__ void poisson_kernel(const PoissonArgs A, int64_t k_from, int64_t k_to) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int s = A.stream[i];
  const int64_t el = A.elem[i];
  const uint32_t thr = A.thr[i];
  const int32_t dc = A.dc_steps[i];
  const uint64_t sid = (uint64_t)A.conn[i];
  uint64_t* cm = A.cmask[s];
  uint64_t* cam = A.camask[s];
  const int64_t ne = A.n_elem[s];
  uint64_t word[4];
  int64_t have = -1;
  uint64_t bits = 0;
  const int64_t k0 = A.clock ? A.clock->k0 : A.k0;
  if (A.clock) {
    k_from = k0;
    k_to = k0 + A.E;
  }
  const int64_t slot = (k0 / A.E) % A.n_slots;
  for (int64_t k = k_from; k < k_to; ++k) {
    const int64_t blk = k >> 3;
    if (blk != have) {
      threefry4x64_12(sid, (uint64_t)blk, 1, 0, A.seed, 0, 0, 0, word);
      have = blk;
    }
    const int j = (int)(k & 7);
    const uint32_t u = (j & 1) ? (uint32_t)(word[j >> 1] >> 32) : (uint32_t)word[j >> 1];
    if (u < thr) {
      bits |= 1ull << (k - k0);
      if (dc >= 0) {
        const int64_t kc = k + dc;
        const int64_t sc = (kc / A.E) % A.n_slots;
        atomicOr((unsigned long long*)&cam[sc * ne + el], 1ull << (kc % A.E));
      }
    }
  }
  if (bits) atomicOr((unsigned long long*)&cm[slot * ne + el], bits);
}

// One warp per spike of the launch; its lanes walk the source's CSR row.
__global__ void route_kernel(const RouteArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = min(*A.spk_count, A.spk_cap);
  for (int64_t q = warp; q < n; q += nwarps) {
    const int gid = A.spk_gid[q];
    const int64_t ks = A.spk_step[q];
    for (int64_t e = A.out_ptr[gid] + lane; e < A.out_ptr[gid + 1]; e += 32) {
      const int s = A.out_stream[e];
      const int64_t el = A.out_elem[e];
      const int64_t kd = ks + A.out_delay[e];
      const int64_t ne = A.n_elem[s];
      atomicOr((unsigned long long*)&A.cmask[s][((kd / A.E) % A.n_slots) * ne + el],
               1ull << (kd % A.E));
      const int dc = A.dc_steps[s];
      if (dc >= 0) {
        const int64_t kc = kd + dc;
        atomicOr((unsigned long long*)&A.camask[s][((kc / A.E) % A.n_slots) * ne + el],
                 1ull << (kc % A.E));
      }
    }
  }
}

// Appends the launch's spikes to the record (log_count is advanced later by
// finalize_kernel, so every block sees the same base).
__global__ void log_append_kernel(const int32_t* spk_count, int32_t spk_cap, const int32_t* gid,
                                  const int32_t* step, const double* t, int32_t* log_count,
                                  int32_t* log_gid, int64_t* log_step, double* log_t,
                                  int64_t log_cap, int32_t* err_flags) {
  const int n = min(*spk_count, spk_cap);
  const int64_t base = *log_count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = base + i;
    if (o < log_cap) {
      log_gid[o] = gid[i];
      log_step[o] = step[i];
      log_t[o] = t[i];
    } else {
      atomicOr(err_flags, 2);
    }
  }
}

__global__ void finalize_kernel(int32_t* spk_count, int32_t spk_cap, int32_t* log_count,
                                int64_t log_cap) {
  int64_t c = (int64_t)*log_count + min(*spk_count, spk_cap);
  *log_count = (int32_t)(c < log_cap ? c : log_cap);
  *spk_count = 0;
}

// Graph launches: zero the finished epoch's mask slot (the slot is reused for
// epoch + n_slots; no event of the ring's horizon targets it meanwhile).
__global__ void clear_slot_kernel(const SlotClear C, const EpochClock* clock) {
  const int64_t slot = (clock->k0 / C.E) % C.n_slots;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int a = 0; a < C.n; ++a) {
    uint64_t* p = C.base[a] + slot * C.elems[a];
    for (int64_t i = tid; i < C.elems[a]; i += nth) p[i] = 0;
  }
}

__global__ void tick_kernel(EpochClock* clock, int32_t E, int32_t probes) {
  clock->k0 += E;
  if (probes) clock->probe_sample0 += E;
}

__global__ void set_clock_kernel(EpochClock* clock, int64_t k0, int64_t probe_sample0) {
  clock->k0 = k0;
  clock->probe_sample0 = probe_sample0;
}

int launch_clear_and_tick(const SlotClear& c, EpochClock* clock, void* stream) {
  int64_t most = 1;
  for (int a = 0; a < c.n; ++a) most = c.elems[a] > most ? c.elems[a] : most;
  int blocks = (int)((most + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (c.n > 0) clear_slot_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(c, clock);
  tick_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(clock, c.E, c.probes);
  return (int)cudaGetLastError();
}

int launch_set_clock(EpochClock* clock, int64_t k0, int64_t probe_sample0, void* stream) {
  set_clock_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(clock, k0, probe_sample0);
  return (int)cudaGetLastError();
}

int launch_poisson(const PoissonArgs& a, int64_t k_from, int64_t k_to, void* stream) {
  if (a.n == 0 || k_to <= k_from) return 0;
  const int threads = 256;
  const int blocks = (int)((a.n + threads - 1) / threads);
  poisson_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(a, k_from, k_to);
  return (int)cudaGetLastError();
}

int launch_route(const RouteArgs& a, int32_t max_spikes, void* stream) {
  const int threads = 256;
  int blocks = (max_spikes * 32 + threads - 1) / threads;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  route_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int launch_log_append(const int32_t* spk_count, const int32_t* gid, const int32_t* step,
                      const double* t, int32_t max_spikes, int32_t* log_count,
                      int32_t* log_gid, int64_t* log_step, double* log_t, int64_t log_cap,
                      int32_t* err_flags, void* stream) {
  const int threads = 256;
  int blocks = (max_spikes + threads - 1) / threads;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  log_append_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(
      spk_count, max_spikes, gid, step, t, log_count, log_gid, log_step, log_t, log_cap,
      err_flags);
  finalize_kernel<<<1, 1, 0, (cudaStream_t)stream>>>((int32_t*)spk_count, max_spikes, log_count,
                                                     log_cap);
  return (int)cudaGetLastError();
}

}  // namespace pa
