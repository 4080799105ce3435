// model.cu -- host side of the C-ABI: descriptor validation, discretisation,
// device layout, the epoch loop of pa_advance and the read-back calls.
//
// Host arithmetic that feeds the device (CV geometry, per-dt constants) is
// compiled without floating-point contraction, so the FP64 path starts from
// exactly the coefficients the plain definition gives.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include <sched.h>

#include "../../include/plastic_arbor.h"
#include "engine.h"

namespace {

thread_local std::string g_last_error;

int set_err(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_err(PA_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));       \
  } while (0)

constexpr double kPi = 3.14159265358979323846;

int n_params_of(int kind) {
  switch (kind) {
    case PA_MECH_PAS: return 2;
    case PA_MECH_HH: return 6;
    case PA_MECH_EXPSYN: return 2;
    case PA_MECH_GB: return 13;
    case PA_MECH_STC: return 18;
    case PA_MECH_STDP: return 8;
    case PA_MECH_HCA: return 10;
  }
  return -1;
}
// Plasticity noise of a GB/STC stream (Eqs. plasticity_noise_1-2): sigma_pl,
// the optional parameter at index np, and the Euler-Maruyama amplitudes
// sigma_pl sqrt(n dt / tau) for n = 0, 1, 2 thresholds crossed.
void set_noise(pa::StreamParams& P, const pa_mechanism& m, int np, double tau, double dt) {
  P.sigma = m.n_params > np ? m.params[np] : 0.0;
  for (int n = 0; n < 3; ++n)
    P.amp[n] = m.n_params > np ? P.sigma * std::sqrt(((double)n * dt) / tau) : 0.0;
}
bool is_point(int kind) {
  return kind == PA_MECH_EXPSYN || kind == PA_MECH_GB || kind == PA_MECH_STC ||
         kind == PA_MECH_STDP || kind == PA_MECH_HCA;
}

// A bump allocator over one cudaMalloc: every array of a model lives in it.
struct Arena {
  char* base = nullptr;
  size_t used = 0, cap = 0;
  std::vector<std::pair<size_t, size_t>> plan;  // offset, bytes
  size_t reserve(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return off;
  }
};

// The cable rows of a model built by cell kind: per-kind tables (CV i of kind
// q at off[q] + i) expanded into the lane-interleaved layout.  Element e is
// row e / 32, lane e % 32 of its thread-per-cell group, or CV e - 32 row_base
// of a wide group's cell (lane slot 0).  Rows past a cell's last CV and lanes
// without a cell take the padding values (V, C/dt, leak E-term, coupling 0;
// diagonal 1; no parent or children; no tree flags).  Mixed models keep V and
// the coefficients as float-float pairs (the nearest float, then the float
// nearest the remainder).
struct RowKinds {
  const double *cdt, *dc, *em, *a;
  const int16_t *par, *och, *ocn;
  const uint8_t* tf;
  const int32_t* off;        // per kind, n_kind + 1
  const int32_t* lane_kind;  // per lane, -1: no cell
  const double* lane_v0;     // per lane: the cell's initial V
  const int32_t* row_base;   // per group, n_groups + 1
  int64_t n_groups, n_narrow, n_elem;
  int mixed, tree;
  double *V, *CDT, *DC, *EM, *A;
  int16_t *PAR, *OCH, *OCN;
  uint8_t* TF;
};

__device__ __forceinline__ void put_row(double* dst, int64_t e, double x, bool mixed) {
  if (mixed) {
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    reinterpret_cast<float2*>(dst)[e] = make_float2(hi, lo);
  } else {
    dst[e] = x;
  }
}

__global__ void expand_rows_kernel(RowKinds k) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k.n_elem; e += stride) {
    const int32_t row = (int32_t)(e >> 5);
    // the group: the last g with row_base[g] <= row
    int64_t lo = 0, hi = k.n_groups;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (k.row_base[mid] <= row) lo = mid;
      else hi = mid;
    }
    int64_t L, i;
    if (lo < k.n_narrow) {
      L = lo * 32 + (e & 31);
      i = row - k.row_base[lo];
    } else {
      L = lo * 32;
      i = e - ((int64_t)k.row_base[lo] << 5);
    }
    const int32_t q = k.lane_kind[L];
    const int64_t o = q >= 0 ? (int64_t)k.off[q] + i : 0;
    const bool in = q >= 0 && o < (int64_t)k.off[q + 1];
    const bool mixed = k.mixed != 0;
    put_row(k.V, e, in ? k.lane_v0[L] : 0.0, mixed);
    put_row(k.CDT, e, in ? k.cdt[o] : 0.0, mixed);
    put_row(k.DC, e, in ? k.dc[o] : 1.0, mixed);
    put_row(k.EM, e, in ? k.em[o] : 0.0, mixed);
    put_row(k.A, e, in ? k.a[o] : 0.0, mixed);
    if (k.tree) {
      k.PAR[e] = in ? k.par[o] : (int16_t)-1;
      k.OCH[e] = in ? k.och[o] : (int16_t)-1;
      k.OCN[e] = in ? k.ocn[o] : (int16_t)-1;
      k.TF[e] = in ? k.tf[o] : (uint8_t)0;
    }
  }
}

}  // namespace

// An allocator whose value-less construct leaves elements default-initialised
// (uninitialised for arithmetic types): large host arrays are then first
// touched, and filled, by the builder threads that own their ranges.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new ((void*)p) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new ((void*)p) U(std::forward<Args>(args)...);
  }
};
template <class T>
using HostVec = std::vector<T, NoInitAlloc<T>>;

struct pa_model {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = PA_FP64;
  bool tree = false;
  double dt = 0;
  uint64_t seed = 0;
  int64_t n_cells = 0, n_cv = 0, n_conn = 0, n_groups = 0, n_lanes = 0, total_rows = 0;
  int64_t n_narrow = 0, n_wide = 0;       // groups of the thread- and warp-per-cell bins
  int64_t step = 0;
  int32_t E = 1, n_slots = 1;
  int64_t poisson_epoch_done = -1;
  int32_t max_spikes = 0;
  int64_t log_cap = 0;
  int32_t n_probe = 0;
  int64_t probe_cap = 0, probe_samples = 0;
  bool replay = false;
  std::vector<int32_t> rep_gid;
  std::vector<int64_t> rep_step;
  size_t rep_pos = 0;
  // host-side maps
  std::vector<int32_t> lane_of_gid;       // gid -> lane
  std::vector<int32_t> row_base;          // per group
  std::vector<int32_t> cell_ncv;          // per gid
  std::vector<int64_t> cell_cv_off;       // per gid, cell-major CV offsets
  HostVec<int32_t> conn_stream;           // per connection
  HostVec<int64_t> conn_elem;
  HostVec<int32_t> conn_kind;             // PA_MECH_* of the connection
  HostVec<double> conn_weight;
  HostVec<double> conn_h0;
  bool prp_diff = false;                  // the STC mechanism's PRP diffuses (D_p > 0)
  std::vector<uint8_t> cell_ca;           // per gid: the cell has HCA synapses
  std::vector<uint8_t> cell_diff;         // per gid: the cell's PRP is a field over its CVs
  std::vector<double> prp_vol, prp_gsum;  // per element: CV volume, summed gD (fast-forward)
  std::vector<double> ff_dg, ff_vdt;      // the long step's matrix, staged for upload
  double* d_ff_dg = nullptr;              // device copies of the long step's matrix
  double* d_ff_vdt = nullptr;
  size_t w_bytes = 8;    // event weight element (4 in PA_FP32)
  size_t tr_bytes = 8;   // STDP trace element (4 in PA_MIXED, PA_FP32)
  size_t g_bytes = 8;    // conductance element (float2 hi + lo in PA_MIXED, float in PA_FP32)
  size_t sum_bytes = 8;  // per-CV synaptic sum element (4 in PA_FP32)
  int n_streams = 0;
  pa::StreamParams sp[pa::kMaxStreams];
  std::vector<double> mech_params[pa::kMaxStreams];  // each stream's mechanism parameters
  int64_t s_nelem[pa::kMaxStreams];
  // device
  char* dmem = nullptr;
  size_t dbytes = 0;
  pa::EpochArgs ea;
  pa::PoissonArgs pa_args;
  pa::RouteArgs ra;
  uint64_t* replay_bits = nullptr;
  int32_t* rep_spk_count = nullptr;
  int32_t* rep_spk_gid = nullptr;
  int32_t* rep_spk_step = nullptr;
  int32_t* log_count = nullptr;
  int32_t* log_gid = nullptr;
  int64_t* log_step = nullptr;
  double* log_t = nullptr;
  int32_t* err_flags = nullptr;
  std::vector<uint64_t*> mask_bases;  // cmask/camask bases to clear per epoch
  std::vector<int64_t> mask_elems;
  // CUDA-graph launches of whole epochs (PA_FLAG_NO_GRAPHS turns them off)
  bool graphs = true;
  pa::EpochClock* clock = nullptr;          // device
  pa::SlotClear slot_clear;
  cudaStream_t cap_stream = nullptr;        // capture only
  cudaStream_t side_stream = nullptr;       // the wide bin, concurrent with the narrow one
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  pa::SideLaunch side{nullptr, nullptr, nullptr};
  cudaGraphExec_t graph1 = nullptr, graph8 = nullptr;  // 1 and 8 epochs
  int64_t n_graph_launches = 0;
  // kernel statistics
  bool time_kernels = false;
  int64_t n_static_cv = 0;
  int shape = 0;
  float tune_ms[pa::kNumShapes] = {0};
  int64_t n_epoch_launches = 0, n_kernel_launches = 0;
  double epoch_ms = 0, event_ms = 0;
  std::vector<cudaEvent_t> ev_pool;                       // recycled events
  struct Timed { cudaEvent_t a, b, c, d; };               // [a,b): Poisson, [b,c): epoch, [c,d): routing
  std::vector<Timed> pending;
};

namespace {
// the side stream of the wide bin, once both bins are in use
const pa::SideLaunch* side_of(const pa_model* M) { return M->side.stream ? &M->side : nullptr; }
}  // namespace

namespace {

struct SynRec {
  int64_t conn;
  int32_t cv;
};

// Runs fn(begin, end) over contiguous pieces of [0, n) on the host cores this
// process may use (at most 64 threads), shared among the builds that run at
// the same time (a server builds several models at once).  The model builder's
// per-group loops write disjoint elements, so the result does not depend on the
// thread count.  A thread that cannot be started has its piece run on the
// calling thread.  An exception in any piece (an allocation failure) is
// rethrown on the calling thread once every thread has joined.
std::atomic<int> g_parallel_regions{0};
thread_local int64_t tl_build_threads = 0;  // the calling build's cap (0: none)

template <class F>
void parallel_ranges(int64_t n, F&& fn) {
  cpu_set_t cs;
  const int64_t hw = sched_getaffinity(0, sizeof cs, &cs) == 0 ? CPU_COUNT(&cs) : 1;
  const int64_t active = g_parallel_regions.fetch_add(1) + 1;
  struct Leave {
    ~Leave() { g_parallel_regions.fetch_sub(1); }
  } leave;
  const int64_t cap = tl_build_threads > 0 ? tl_build_threads : 64;
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({hw / active, cap, n}));
  if (nt <= 1) {
    fn((int64_t)0, n);
    return;
  }
  std::exception_ptr err;
  std::mutex mu;
  auto run = [&](int64_t b, int64_t e) {
    try {
      fn(b, e);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!err) err = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int64_t t = 1; t < nt; ++t) {
    const int64_t b = n * t / nt, e = n * (t + 1) / nt;
    try {
      th.emplace_back([&run, b, e] { run(b, e); });
    } catch (...) {
      run(b, e);
    }
  }
  run((int64_t)0, n / nt);
  for (auto& x : th) x.join();
  if (err) std::rethrow_exception(err);
}

// Stable counting sort of items 0 .. n-1 into n_buckets buckets: bucket(i)
// gives an item's bucket, or a negative value to leave it out.  ptr receives
// the n_buckets + 1 bucket starts, ready(total) is called with the number of
// kept items, and place(i, slot) is then called once per kept item, the slots
// of a bucket following the item order.  Fixed pieces of the
// items are counted and placed in parallel, so the result does not depend on
// the thread count.
template <class B, class R, class P>
void bucket_scatter(int64_t n, int64_t n_buckets, B&& bucket, std::vector<int64_t>& ptr,
                    R&& ready, P&& place) {
  int64_t np = n < (1 << 16) ? 1 : 16;
  while (np > 1 && (double)np * (double)n_buckets * 8.0 > 512.0 * 1024 * 1024) np /= 2;
  std::vector<int64_t> start((size_t)np * (size_t)n_buckets, 0);
  parallel_ranges(np, [&](int64_t p0, int64_t p1) {
    for (int64_t p = p0; p < p1; ++p)
      for (int64_t i = n * p / np; i < n * (p + 1) / np; ++i) {
        const int64_t q = bucket(i);
        if (q >= 0) start[(size_t)p * n_buckets + q]++;
      }
  });
  ptr.assign((size_t)n_buckets + 1, 0);
  int64_t run = 0;
  for (int64_t q = 0; q < n_buckets; ++q) {
    ptr[q] = run;
    for (int64_t p = 0; p < np; ++p) {
      const int64_t k = start[(size_t)p * n_buckets + q];
      start[(size_t)p * n_buckets + q] = run;
      run += k;
    }
  }
  ptr[n_buckets] = run;
  ready(run);
  parallel_ranges(np, [&](int64_t p0, int64_t p1) {
    for (int64_t p = p0; p < p1; ++p)
      for (int64_t i = n * p / np; i < n * (p + 1) / np; ++i) {
        const int64_t q = bucket(i);
        if (q >= 0) place(i, start[(size_t)p * n_buckets + q]++);
      }
  });
}


template <class V>
std::vector<float> to_f32(const V& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}

// Times every epoch-kernel shape on the model's first epoch and keeps the fastest.
// The whole device arena is copied aside first and restored after each trial,
// so the trials leave no trace in the model's state.
int autotune(pa_model* M) {
  using namespace pa;
  char* snap = nullptr;
  if (cudaMalloc((void**)&snap, M->dbytes) != cudaSuccess) {
    cudaGetLastError();
    return PA_OK;  // no room for a snapshot: keep the default shape
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PA_OK;
  float best = 1e30f;
  int best_shape = M->shape;
  auto fail = [&](cudaError_t e) {
    rc = set_err(PA_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // the first epoch's Poisson drive, so the trials see realistic events
  if (e == cudaSuccess) {
    M->pa_args.k0 = 0;
    e = (cudaError_t)launch_poisson(M->pa_args, 0, M->E, M->stream);
    M->poisson_epoch_done = 0;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(snap, M->dmem, M->dbytes, cudaMemcpyDeviceToDevice, M->stream);
  EpochArgs A = M->ea;
  A.k_begin = 0;
  A.k_end = M->E;
  A.k0 = 0;
  A.slot = 0;
  A.probe_sample0 = 0;
  A.replay = 0;
  for (int s = 0; s < kNumShapes && e == cudaSuccess; ++s) {
    float best_s = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, M->stream);
      if (e == cudaSuccess)
        e = (cudaError_t)launch_epoch(M->precision, A, M->tree, s, M->stream, side_of(M));
      if (e == cudaSuccess) e = cudaEventRecord(e1, M->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best_s) best_s = ms;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(M->dmem, snap, M->dbytes, cudaMemcpyDeviceToDevice, M->stream);
    }
    M->tune_ms[s] = best_s;
    if (best_s < best) {
      best = best_s;
      best_shape = s;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  if (e != cudaSuccess) fail(e);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(snap);
  if (rc == PA_OK) M->shape = best_shape;
  return rc;
}

int build_impl(const pa_cell* cells, int64_t n_cells, const pa_morphology* morphs,
               int64_t n_morph, const pa_mechanism* mechs, int64_t n_mech,
               const pa_connection* conns, int64_t n_conn, const pa_options* opt,
               pa_model** out) {
  using namespace pa;
  if (!out) return set_err(PA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!opt) return set_err(PA_ERR_ARG, "options are NULL");
  if (n_cells < 0 || n_morph < 0 || n_mech < 0 || n_conn < 0)
    return set_err(PA_ERR_ARG, "negative count");
  if (n_cells > (1LL << 30) || n_conn > (1LL << 31) - 1)
    return set_err(PA_ERR_ARG, "too many cells or connections");
  if ((n_cells && !cells) || (n_morph && !morphs) || (n_mech && !mechs) || (n_conn && !conns))
    return set_err(PA_ERR_ARG, "NULL descriptor array with a nonzero count");
  const double dt = opt->dt;
  if (!(dt > 0) || !std::isfinite(dt)) return set_err(PA_ERR_ARG, "dt must be positive");
  if (opt->precision != PA_FP64 && opt->precision != PA_MIXED && opt->precision != PA_FP32)
    return set_err(PA_ERR_ARG, "precision must be PA_FP64, PA_MIXED or PA_FP32");
  const bool w32 = opt->precision == PA_FP32;  // FP32 event weights
  tl_build_threads = (opt->flags >> 12) & 0x3F;
  int max_e = opt->max_epoch_steps > 0 ? opt->max_epoch_steps : 64;
  if (max_e > 64) return set_err(PA_ERR_ARG, "max_epoch_steps must be <= 64");

  // ---- mechanisms -------------------------------------------------------------
  for (int64_t j = 0; j < n_mech; ++j) {
    int np = n_params_of(mechs[j].kind);
    if (np < 0) return set_err(PA_ERR_ARG, "mechanism %lld: unknown kind %d", (long long)j, mechs[j].kind);
    // GB and STC take an optional trailing sigma_pl (plasticity noise; 0 if
    // absent), STC then an optional PRP diffusivity D_p
    const bool noisy_kind = mechs[j].kind == PA_MECH_GB || mechs[j].kind == PA_MECH_STC;
    const bool stc_kind = mechs[j].kind == PA_MECH_STC;
    if (!(mechs[j].n_params == np || (noisy_kind && mechs[j].n_params == np + 1) ||
          (stc_kind && mechs[j].n_params == np + 2)) ||
        !mechs[j].params)
      return set_err(PA_ERR_ARG, "mechanism %lld: expected %d parameters", (long long)j, np);
    if (mechs[j].n_params > np && !(mechs[j].params[np] >= 0.0))
      return set_err(PA_ERR_ARG, "mechanism %lld: sigma_pl must be >= 0", (long long)j);
    if (mechs[j].n_params > np + 1 && !(mechs[j].params[np + 1] >= 0.0))
      return set_err(PA_ERR_ARG, "mechanism %lld: D_p must be >= 0", (long long)j);
    for (int i = 0; i < mechs[j].n_params; ++i)
      if (!std::isfinite(mechs[j].params[i]))
        return set_err(PA_ERR_ARG, "mechanism %lld: non-finite parameter %d", (long long)j, i);
  }
  // streams: one per point mechanism used by a connection, in table order
  std::vector<int> mech_stream(n_mech, -1);
  {
    // over fixed pieces of the connection list; the lowest bad one is reported
    constexpr int64_t kPieces = 64;
    std::vector<std::vector<char>> used_p(kPieces, std::vector<char>(n_mech, 0));
    std::vector<int64_t> bad_p(kPieces, -1);
    parallel_ranges(kPieces, [&](int64_t p0, int64_t p1) {
      for (int64_t p = p0; p < p1; ++p)
        for (int64_t c = n_conn * p / kPieces; c < n_conn * (p + 1) / kPieces; ++c) {
          const int m = conns[c].mech;
          if (m < 0 || m >= n_mech || !is_point(mechs[m].kind)) {
            bad_p[p] = c;
            break;
          }
          used_p[p][m] = 1;
        }
    });
    for (int64_t p = 0; p < kPieces; ++p)
      if (bad_p[p] >= 0)
        return set_err(PA_ERR_ARG, "connection %lld: mechanism must be a synapse",
                       (long long)bad_p[p]);
    std::vector<char> used(n_mech, 0);
    for (int64_t p = 0; p < kPieces; ++p)
      for (int64_t m = 0; m < n_mech; ++m) used[m] |= used_p[p][m];
    int ns = 0, n_stc = 0;
    for (int64_t m = 0; m < n_mech; ++m)
      if (used[m]) {
        if (ns == kMaxStreams) return set_err(PA_ERR_ARG, "more than %d synapse mechanisms in use", kMaxStreams);
        if (mechs[m].kind == PA_MECH_STC) ++n_stc;
        mech_stream[m] = ns++;
      }
    if (n_stc > 1) return set_err(PA_ERR_ARG, "at most one STC mechanism per model");
  }

  pa_model* M = new (std::nothrow) pa_model();
  if (!M) return set_err(PA_ERR_OOM, "host allocation failed");
  struct Guard {
    pa_model*& m;
    bool ok = false;
    ~Guard() { if (!ok && m) pa_free_model(m); }
  } guard{M};
  M->device = opt->device;
  M->stream = (cudaStream_t)opt->stream;
  M->precision = opt->precision;
  M->dt = dt;
  M->seed = opt->seed;
  M->n_cells = n_cells;
  M->n_conn = n_conn;
  M->w_bytes = w32 ? 4 : 8;
  M->tr_bytes = opt->precision == PA_FP64 ? 8 : 4;
  M->g_bytes = opt->precision == PA_FP32 ? 4 : 8;
  M->sum_bytes = opt->precision == PA_FP32 ? 4 : 8;
  M->time_kernels = (opt->flags & PA_FLAG_TIME_KERNELS) != 0;
  M->graphs = (opt->flags & PA_FLAG_NO_GRAPHS) == 0;
  {
    const int forced = ((opt->flags >> 8) & 0xF) - 1;
    if (forced >= pa::kNumShapes) return set_err(PA_ERR_ARG, "shape %d out of range", forced);
    if (forced >= 0) M->shape = forced;
  }
  CUDA_TRY(cudaSetDevice(M->device));

  int n_streams = 0, stc_stream = -1, ca_stream = -1;
  double ca_tau = 0.0, ca_d = 0.0;  // the HCA mechanism's tau_C and D
  double diff_d = 0.0;  // PRP diffusivity [um2/ms]
  int stream_mech[kMaxStreams];
  for (int64_t m = 0; m < n_mech; ++m) {
    int s = mech_stream[m];
    if (s < 0) continue;
    n_streams = std::max(n_streams, s + 1);
    stream_mech[s] = (int)m;
    M->mech_params[s].assign(mechs[m].params, mechs[m].params + mechs[m].n_params);
    const double* p = mechs[m].params;
    StreamParams& P = M->sp[s];
    std::memset(&P, 0, sizeof P);
    P.dc_steps = -1;
    P.e = p[1];
    P.decay_g = std::exp(-dt / p[0]);
    switch (mechs[m].kind) {
      case PA_MECH_EXPSYN: P.kind = SK_EXPSYN; break;
      case PA_MECH_GB:
        P.kind = SK_GB;
        P.decay_c = std::exp(-dt / p[2]);
        P.c_pre = p[3]; P.c_post = p[4]; P.theta_p = p[5]; P.theta_d = p[6];
        P.gamma_p = p[7]; P.gamma_d = p[8]; P.rate_w = dt / p[9]; P.w_star = p[10];
        P.dc_steps = (int32_t)std::llround(p[11] / dt);
        set_noise(P, mechs[m], 13, p[9], dt);
        break;
      case PA_MECH_STC:
        P.kind = SK_STC;
        stc_stream = s;
        P.decay_c = std::exp(-dt / p[2]);
        P.c_pre = p[3]; P.c_post = p[4]; P.theta_p = p[5]; P.theta_d = p[6];
        P.gamma_p = p[7]; P.gamma_d = p[8];
        P.rate_h = dt / p[9]; P.rate_z = dt / p[10]; P.rate_p = dt / p[11];
        P.h0 = p[12]; P.theta_tag = p[13]; P.theta_pro = p[14]; P.p_max = p[15];
        P.f_int = p[16];
        P.dc_steps = (int32_t)std::llround(p[17] / dt);
        set_noise(P, mechs[m], 18, p[9], dt);
        if (mechs[m].n_params > 19 && p[19] > 0.0) {
          M->prp_diff = true;
          diff_d = p[19];
        }
        break;
      case PA_MECH_STDP:
        P.kind = SK_STDP;
        P.tau_pre = p[2];
        P.tau_post = p[3];
        P.a_pre = p[4]; P.a_post = p[5]; P.w_max = p[7];
        break;
      case PA_MECH_HCA:
        // no conductance: g stays 0 (e = 0, decay 1); the injection current in c
        if (!(p[1] > 0) || !(p[8] > 0) || !(p[9] >= 0))
          return set_err(PA_ERR_ARG, "mechanism %lld: tau_I, tau_C > 0 and D >= 0 required",
                         (long long)m);
        if (ca_stream >= 0) return set_err(PA_ERR_ARG, "at most one HCA mechanism per model");
        P.kind = SK_HCA;
        ca_stream = s;
        P.e = 0.0;
        P.decay_g = 1.0;
        P.decay_c = std::exp(-dt / p[1]);
        P.c_pre = p[0];
        P.theta_p = p[5]; P.theta_d = p[6];
        P.hca_kq = (p[2] * 1e6) / (2.0 * 96485.33212);
        P.hca_gpr = (dt * p[3]) * 1e-3;
        P.hca_gdr = (dt * p[4]) * 1e-3;
        ca_tau = p[8];
        ca_d = p[9];
        break;
    }
    if ((P.kind == SK_GB || P.kind == SK_STC) && P.dc_steps < 0)
      return set_err(PA_ERR_ARG, "mechanism %lld: negative t_c_delay", (long long)m);
    P.f = {(float)P.decay_c, (float)P.c_pre, (float)P.c_post, (float)P.theta_p,
           (float)P.theta_d, (float)P.gamma_p, (float)P.gamma_d, (float)P.rate_w,
           (float)P.w_star, (float)P.rate_h, (float)P.rate_z, (float)P.h0,
           (float)P.theta_tag, (float)P.f_int, (float)P.a_pre, (float)P.a_post,
           (float)P.tau_pre, (float)P.tau_post, (float)P.w_max, 0.0f};
  }
  M->n_streams = n_streams;

  // ---- morphologies and cells -------------------------------------------------
  // validated over fixed pieces in parallel; the lowest bad index is reported
  {
    constexpr int64_t kPieces = 64;
    struct PieceErr {
      int64_t bad = -1;
      char msg[192];
    };
    std::vector<PieceErr> pe(kPieces);
    std::vector<char> branched(kPieces, 0);
    parallel_ranges(kPieces, [&](int64_t p0, int64_t p1) {
      for (int64_t pc = p0; pc < p1; ++pc) {
        PieceErr& o = pe[pc];
        for (int64_t mo = n_morph * pc / kPieces; mo < n_morph * (pc + 1) / kPieces && o.bad < 0;
             ++mo) {
          const pa_morphology& g = morphs[mo];
          if (g.n_cv < 1 || g.n_cv > 32767) {
            o.bad = mo;
            snprintf(o.msg, sizeof o.msg, "morphology %lld: n_cv must be in [1, 32767]",
                     (long long)mo);
            break;
          }
          if (!g.parent || !g.length_um || !g.diam_um || !g.region) {
            o.bad = mo;
            snprintf(o.msg, sizeof o.msg, "morphology %lld: NULL array", (long long)mo);
            break;
          }
          for (int i = 0; i < g.n_cv; ++i) {
            int p = g.parent[i];
            if ((i == 0 && p != -1) || (i > 0 && (p < 0 || p >= i))) {
              o.bad = mo;
              snprintf(o.msg, sizeof o.msg, "morphology %lld: parent[%d] = %d invalid",
                       (long long)mo, i, p);
              break;
            }
            if (!(g.length_um[i] > 0) || !(g.diam_um[i] > 0) || !std::isfinite(g.length_um[i]) ||
                !std::isfinite(g.diam_um[i])) {
              o.bad = mo;
              snprintf(o.msg, sizeof o.msg,
                       "morphology %lld: CV %d has non-positive length/diameter", (long long)mo, i);
              break;
            }
            if (i > 0 && p != i - 1) branched[pc] = 1;
          }
        }
      }
    });
    for (const PieceErr& o : pe)
      if (o.bad >= 0) return set_err(PA_ERR_ARG, "%s", o.msg);
    for (char b : branched)
      if (b) M->tree = true;
    M->cell_ncv.resize(n_cells);
    M->cell_cv_off.resize(n_cells + 1, 0);
    parallel_ranges(kPieces, [&](int64_t p0, int64_t p1) {
      for (int64_t pc = p0; pc < p1; ++pc) {
        PieceErr& o = pe[pc];
        for (int64_t c = n_cells * pc / kPieces; c < n_cells * (pc + 1) / kPieces && o.bad < 0;
             ++c) {
          const pa_cell& cl = cells[c];
          const char* why = nullptr;
          if (cl.morph < 0 || cl.morph >= n_morph) why = "bad morphology index";
          for (int which = 0; which < 2 && !why; ++which) {
            int m = which == 0 ? cl.soma_mech : cl.dend_mech;
            if (m < 0 || m >= n_mech ||
                (mechs[m].kind != PA_MECH_PAS && mechs[m].kind != PA_MECH_HH))
              why = "soma/dendrite mechanism must be pas or hh";
          }
          if (!why) {
            const pa_morphology& g = morphs[cl.morph];
            for (int i = 0; i < g.n_cv && !why; ++i) {
              int m = g.region[i] == 0 ? cl.soma_mech : cl.dend_mech;
              if (mechs[m].kind == PA_MECH_HH && i != 0)
                why = "HH is supported on the soma CV (CV 0) only";
            }
          }
          if (!why && (!(cl.cm > 0) || !(cl.ra > 0))) why = "cm and ra must be positive";
          if (why) {
            o.bad = c;
            snprintf(o.msg, sizeof o.msg, "cell %lld: %s", (long long)c, why);
            break;
          }
          M->cell_ncv[c] = morphs[cl.morph].n_cv;
        }
      }
    });
    for (const PieceErr& o : pe)
      if (o.bad >= 0) return set_err(PA_ERR_ARG, "%s", o.msg);
    for (int64_t c = 0; c < n_cells; ++c)
      M->cell_cv_off[c + 1] = M->cell_cv_off[c] + M->cell_ncv[c];
  }
  M->n_cv = M->cell_cv_off[n_cells];

  // ---- cell bins: thread per cell (narrow) or warp per cell (wide) ----------------
  if ((opt->flags & PA_FLAG_NARROW_ONLY) && (opt->flags & PA_FLAG_WIDE_ALL))
    return set_err(PA_ERR_ARG, "PA_FLAG_NARROW_ONLY and PA_FLAG_WIDE_ALL exclude each other");
  std::vector<char> wide(n_cells, 0);
  M->cell_diff.assign(n_cells, 0);
  std::vector<uint8_t> cell_ca(n_cells, 0);  // cells with HCA synapses (narrow bin)
  {
    // synapses per cell: per-piece counts in parallel, then summed per cell
    std::vector<int64_t> cell_syn(n_cells, 0);
    {
      constexpr int64_t kPieces = 16;
      std::vector<std::vector<int32_t>> part(kPieces);
      parallel_ranges(kPieces, [&](int64_t p0, int64_t p1) {
        for (int64_t p = p0; p < p1; ++p) {
          part[p].assign(n_cells, 0);
          for (int64_t c = n_conn * p / kPieces; c < n_conn * (p + 1) / kPieces; ++c)
            if (conns[c].dst_gid >= 0 && conns[c].dst_gid < n_cells) ++part[p][conns[c].dst_gid];
        }
      });
      parallel_ranges(n_cells, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c)
          for (int64_t p = 0; p < kPieces; ++p) cell_syn[c] += part[p][c];
      });
    }
    // cells with a diffusing PRP or heterosynaptic calcium (only where such a
    // mechanism exists)
    bool any_stc = false, any_hca = false;
    for (int64_t m = 0; m < n_mech; ++m) {
      any_stc = any_stc || mechs[m].kind == PA_MECH_STC;
      any_hca = any_hca || mechs[m].kind == PA_MECH_HCA;
    }
    if ((M->prp_diff && any_stc) || any_hca)
      for (int64_t c = 0; c < n_conn; ++c)
        if (conns[c].dst_gid >= 0 && conns[c].dst_gid < n_cells) {
          if (M->prp_diff && mechs[conns[c].mech].kind == PA_MECH_STC)
            M->cell_diff[conns[c].dst_gid] = 1;
          if (mechs[conns[c].mech].kind == PA_MECH_HCA) cell_ca[conns[c].dst_gid] = 1;
        }
    std::vector<int32_t> morph_branches(n_morph, 0);
    for (int64_t j = 0; j < n_morph; ++j)
      for (int i = 0; i < morphs[j].n_cv; ++i)
        morph_branches[j] += (i == 0 || morphs[j].parent[i] != i - 1) ? 1 : 0;
    int n_sm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, M->device));
    const int64_t warps = (n_cells + kLanes - 1) / kLanes;
    const bool few = warps < (int64_t)kWideMaxWarpsPerSM * n_sm, idle = warps < n_sm;
    for (int64_t c = 0; c < n_cells; ++c) {
      const bool branched = M->cell_ncv[c] >= kWideMinCV &&
                            morph_branches[cells[c].morph] >= kWideMinBranches &&
                            cell_syn[c] <= (int64_t)kWideMaxSynPerCV * M->cell_ncv[c];
      const bool heavy = M->cell_ncv[c] + cell_syn[c] >= kWideMinWork;
      // the heterosynaptic calcium field is solved by the thread-per-cell bin only
      wide[c] = !cell_ca[c] &&
                ((opt->flags & PA_FLAG_WIDE_ALL) ||
                 (!(opt->flags & PA_FLAG_NARROW_ONLY) && ((few && branched) || (idle && heavy))));
    }
  }
  // narrow cells sorted by CV count (descending) and dealt into groups of 32
  // lanes; then one group per wide cell (its cell in lane 0, CVs contiguous)
  std::vector<int32_t> order, order_w;
  for (int64_t c = 0; c < n_cells; ++c) (wide[c] ? order_w : order).push_back((int32_t)c);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return M->cell_ncv[x] > M->cell_ncv[y]; });
  std::stable_sort(order_w.begin(), order_w.end(),
                   [&](int32_t x, int32_t y) { return M->cell_ncv[x] > M->cell_ncv[y]; });
  const int64_t n_narrow = ((int64_t)order.size() + kLanes - 1) / kLanes;
  const int64_t n_wide = (int64_t)order_w.size();
  const int64_t n_groups = n_narrow + n_wide;
  const int64_t n_lanes = n_groups * kLanes;
  if (n_groups > (1LL << 30)) return set_err(PA_ERR_ARG, "too many cells");
  M->n_groups = n_groups;
  M->n_narrow = n_narrow;
  M->n_wide = n_wide;
  M->n_lanes = n_lanes;
  M->lane_of_gid.assign(n_cells, -1);
  std::vector<int32_t> lane_gid(n_lanes, -1), lane_ncv(n_lanes, 0);
  for (size_t i = 0; i < order.size(); ++i) {
    lane_gid[i] = order[i];
    lane_ncv[i] = M->cell_ncv[order[i]];
    M->lane_of_gid[order[i]] = (int32_t)i;
  }
  for (int64_t j = 0; j < n_wide; ++j) {
    const int64_t L = (n_narrow + j) * kLanes;
    lane_gid[L] = order_w[j];
    lane_ncv[L] = M->cell_ncv[order_w[j]];
    M->lane_of_gid[order_w[j]] = (int32_t)L;
  }
  M->row_base.assign(n_groups + 1, 0);
  for (int64_t g = 0; g < n_groups; ++g) {
    const int64_t nc = lane_ncv[g * kLanes];
    const int64_t rows = g < n_narrow ? nc : (nc + kLanes - 1) / kLanes;
    if ((int64_t)M->row_base[g] + rows > (1LL << 26))
      return set_err(PA_ERR_ARG, "model too large: more than 2^31 padded CVs");
    M->row_base[g + 1] = M->row_base[g] + (int32_t)rows;
  }
  M->total_rows = M->row_base[n_groups];
  const int64_t n_elem = M->total_rows * kLanes;
  auto elem = [&](int64_t L, int row) -> int64_t {
    const int64_t g = L / kLanes;
    if (g >= n_narrow) return ((int64_t)M->row_base[g] << 5) + row;
    return ((int64_t)M->row_base[g] + row) * kLanes + (L % kLanes);
  };

  // ---- CV discretisation (a CV is a cylinder; Eq. cable) -----------------------
  // Without a diffusing PRP or heterosynaptic calcium (whose tables are built
  // lane by lane below), cells that share their morphology, cm, ra and
  // mechanisms have the same cable rows: each such kind is discretised once
  // into per-kind tables and expand_rows_kernel writes the lane-interleaved
  // rows on the device.  Otherwise the rows are filled here, group by group.
  const bool by_kind = !M->prp_diff && ca_stream < 0;
  const int64_t n_host_rows = by_kind ? 0 : n_elem;
  HostVec<double> h_cdt(n_host_rows), h_dc(n_host_rows), h_em(n_host_rows), h_a(n_host_rows),
      h_V(n_host_rows);
  HostVec<int16_t> h_par, h_och, h_ocn;
  HostVec<uint8_t> h_tf;
  if (M->tree) {
    h_par.resize(n_host_rows);
    h_och.resize(n_host_rows);
    h_ocn.resize(n_host_rows);
    h_tf.resize(n_host_rows);
  }
  // the kinds: a representative cell each, the kind of every lane (-1: no
  // cell) and every lane's initial V
  std::vector<int32_t> kind_rep, lane_kind, kind_off(1, 0);
  std::vector<double> lane_v0;
  if (by_kind) {
    struct KindKey {
      int32_t morph, soma_mech, dend_mech;
      uint64_t cm, ra;
      bool operator==(const KindKey& o) const {
        return morph == o.morph && soma_mech == o.soma_mech && dend_mech == o.dend_mech &&
               cm == o.cm && ra == o.ra;
      }
    };
    struct KindHash {
      size_t operator()(const KindKey& k) const {
        uint64_t h = (uint64_t)(uint32_t)k.morph * 0x9E3779B97F4A7C15ull;
        h ^= ((uint64_t)(uint32_t)k.soma_mech << 32 | (uint32_t)k.dend_mech) + (h << 6) + (h >> 2);
        h ^= k.cm + (h << 6) + (h >> 2);
        h ^= k.ra + (h << 6) + (h >> 2);
        return (size_t)h;
      }
    };
    auto bits = [](double x) {
      uint64_t u;
      std::memcpy(&u, &x, 8);
      return u;
    };
    std::unordered_map<KindKey, int32_t, KindHash> kinds;
    lane_kind.assign(n_lanes, -1);
    lane_v0.assign(n_lanes, 0.0);
    for (int64_t L = 0; L < n_lanes; ++L) {
      if (lane_gid[L] < 0) continue;
      const pa_cell& cl = cells[lane_gid[L]];
      const KindKey key{cl.morph, cl.soma_mech, cl.dend_mech, bits(cl.cm), bits(cl.ra)};
      const auto it = kinds.emplace(key, (int32_t)kind_rep.size());
      if (it.second) {
        kind_rep.push_back(lane_gid[L]);
        kind_off.push_back(kind_off.back() + morphs[cl.morph].n_cv);
      }
      lane_kind[L] = it.first->second;
      lane_v0[L] = cl.v_init;
    }
  }
  const int64_t n_kind = (int64_t)kind_rep.size(), n_kind_cv = kind_off.back();
  std::vector<double> k_cdt(n_kind_cv, 0.0), k_dc(n_kind_cv, 1.0), k_em(n_kind_cv, 0.0),
      k_a(n_kind_cv, 0.0), k_v(n_kind_cv, 0.0);
  std::vector<int16_t> k_par, k_och, k_ocn;
  std::vector<uint8_t> k_tf;
  if (M->tree) {
    k_par.assign(n_kind_cv, (int16_t)-1);
    k_och.assign(n_kind_cv, (int16_t)-1);
    k_ocn.assign(n_kind_cv, (int16_t)-1);
    k_tf.assign(n_kind_cv, (uint8_t)0);
  }
  std::vector<uint8_t> h_is_hh(n_lanes, 0);
  std::vector<double> h_hhg(3 * n_lanes, 0.0), h_hhe(3 * n_lanes, 0.0);
  std::vector<double> h_iinj(n_lanes, 0.0), h_thresh(n_lanes, 0.0);
  // PA_MIXED forms a passive dendrite's leak E-term g E as (C/dt) k, with k
  // one constant per cell, where every cell of a thread-per-cell group has its
  // soma on row 0 only and one passive mechanism on every other row; the soma
  // row's E-term is kept per lane (em_soma)
  std::vector<double> h_emk(n_lanes, 0.0), h_em0(n_lanes, 0.0);
  std::vector<uint8_t> h_emok(n_lanes, 1), h_emder(std::max<int64_t>(n_groups, 1), 0);
  std::vector<int64_t> h_kon(n_lanes, 0), h_koff(n_lanes, 0);
  std::vector<double> h_pcv, h_pdg, h_pa, h_pvdt, h_psrc;
  std::vector<double> h_cadg, h_caa, h_cavdt, h_cavol;
  if (ca_stream >= 0) {
    h_cadg.assign(n_elem, 1.0);
    h_caa.assign(n_elem, 0.0);
    h_cavdt.assign(n_elem, 0.0);
    h_cavol.assign(n_elem, 1.0);
  }
  if (M->prp_diff) {
    h_pdg.assign(n_elem, 1.0);
    h_pa.assign(n_elem, 0.0);
    h_pvdt.assign(n_elem, 0.0);
    h_psrc.assign(n_lanes, 0.0);
    M->prp_vol.assign(n_elem, 0.0);
    M->prp_gsum.assign(n_elem, 0.0);
  }
  // One cell's discretisation (CV geometry, cable coefficients, tree tables,
  // fork flags, the soma's HH conductances, the mixed form's leak E-term
  // ratio) into arrays indexed by at(i) for CV i
  struct HHOut {
    uint8_t is_hh = 0;
    double g[3] = {0.0, 0.0, 0.0}, e[3] = {0.0, 0.0, 0.0};
  };
  struct EmOut {
    uint8_t ok = 0;
    double k = 0.0, em0 = 0.0;
  };
  auto discretise = [&](const pa_cell& cl, auto at, double* cdt_, double* dc_, double* em_,
                        double* a_, double* v_, int16_t* par_, int16_t* och_, int16_t* ocn_,
                        uint8_t* tf_, HHOut& hh, EmOut& eo, std::vector<double>& rhalf,
                        std::vector<double>& gax) {
    const pa_morphology& g = morphs[cl.morph];
    const int n = g.n_cv;
    rhalf.assign(n, 0.0);
    gax.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      const double Lc = g.length_um[i], dia = g.diam_um[i];
      const double r = 0.5 * dia;
      const double A = (kPi * dia) * Lc;               // um2
      const double cap = (cl.cm * A) * 1e-5;            // nF
      const int64_t e = at(i);
      cdt_[e] = cap / dt;                              // uS
      rhalf[i] = ((cl.ra * (0.5 * Lc)) / (kPi * (r * r))) * 1e-2;  // Mohm
      const int m = g.region[i] == 0 ? cl.soma_mech : cl.dend_mech;
      const double* p = mechs[m].params;
      if (mechs[m].kind == PA_MECH_PAS) {
        const double gp = (p[0] * A) * 1e-2;            // S/cm2 * um2 -> uS
        em_[e] = gp * p[1];
        dc_[e] = gp;                                   // leak, folded in below
      } else {
        hh.is_hh = 1;
        hh.g[0] = (p[0] * A) * 1e-2;
        hh.g[1] = (p[1] * A) * 1e-2;
        hh.g[2] = (p[2] * A) * 1e-2;
        hh.e[0] = p[3];
        hh.e[1] = p[4];
        hh.e[2] = p[5];
        dc_[e] = 0.0;                                  // gates enter per step
        em_[e] = 0.0;
      }
      v_[e] = cl.v_init;
    }
    // axial conductance of two half-cylinders in series, summed in CV order
    for (int i = 1; i < n; ++i) {
      const int p = g.parent[i];
      const double gi = 1.0 / (rhalf[i] + rhalf[p]);
      a_[at(i)] = -gi;
      gax[i] += gi;
      gax[p] += gi;
    }
    for (int i = 0; i < n; ++i) {
      const int64_t e = at(i);
      const int m = g.region[i] == 0 ? cl.soma_mech : cl.dend_mech;
      const double base = cdt_[e] + gax[i];
      dc_[e] = mechs[m].kind == PA_MECH_PAS ? base + dc_[e] : base;
    }
    if (M->tree) {
      // other (non-first) children of each node, linked from the highest index down
      for (int i = 1; i < n; ++i) par_[at(i)] = (int16_t)g.parent[i];
      for (int i = 1; i < n; ++i) {
        const int p = g.parent[i];
        if (i == p + 1) continue;  // the first child is eliminated through registers
        // children are visited in increasing i: push to the front -> descending list
        ocn_[at(i)] = och_[at(p)];
        och_[at(p)] = (int16_t)i;
      }
      // fork flags: a row with exactly one other child takes that child's values
      // from the warp's fork stack (LIFO in both passes), the child pushes them
      std::vector<int32_t> n_other(n, 0);
      for (int i = 1; i < n; ++i)
        if (i != g.parent[i] + 1) ++n_other[g.parent[i]];
      for (int i = 0; i < n; ++i) {
        const int64_t e = at(i);
        if (n_other[i] == 1) tf_[e] |= kForkPop;
        if (i > 0 && i != g.parent[i] + 1 && n_other[g.parent[i]] == 1) tf_[e] |= kForkPush;
      }
      // The stacks need the pushes and pops to nest (LIFO) in both sweeps, as in
      // depth-first numberings; a numbering that interleaves subtrees (side
      // branches numbered after the trunk, in trunk order) keeps the linked lists.
      bool nested = true;
      std::vector<int> stk;
      for (int i = n - 1; i >= 0 && nested; --i) {
        const uint8_t f = tf_[at(i)];
        if (f & kForkPop) {
          if (stk.empty() || stk.back() != och_[at(i)]) nested = false;
          else stk.pop_back();
        }
        if (f & kForkPush) stk.push_back(i);
      }
      stk.clear();
      for (int i = 0; i < n && nested; ++i) {
        const uint8_t f = tf_[at(i)];
        if (f & kForkPush) {
          if (stk.empty() || stk.back() != g.parent[i]) nested = false;
          else stk.pop_back();
        }
        if (f & kForkPop) stk.push_back(i);
      }
      if (!nested)
        for (int i = 0; i < n; ++i) tf_[at(i)] = 0;
      // what the kernels with fork stacks read instead of the parent and
      // child-list rows: whether the parent is the previous row (the carried
      // first child), and whether the other children go through the list
      for (int i = 0; i < n; ++i) {
        const int64_t e = at(i);
        if (i > 0 && g.parent[i] == i - 1) tf_[e] |= kParPrev;
        if (n_other[i] > 0 && !(tf_[e] & kForkPop)) tf_[e] |= kOtherList;
      }
    }
    {
      bool ok = g.region[0] == 0;
      for (int i = 1; i < n && ok; ++i)
        ok = g.region[i] != 0 && mechs[cl.dend_mech].kind == PA_MECH_PAS;
      eo.ok = ok ? 1 : 0;
      eo.em0 = em_[at(0)];
      if (ok && n > 1) {
        const double* p = mechs[cl.dend_mech].params;
        // (p0 A 1e-2) e / ((cm A 1e-5) / dt): the CV's area cancels
        eo.k = ((p[0] * 1e-2) * p[1]) * dt / (cl.cm * 1e-5);
      }
    }
  };
  // the kinds' tables (kinds are independent), then each lane's per-cell values
  std::vector<HHOut> kind_hh(n_kind);
  std::vector<EmOut> kind_eo(n_kind);
  parallel_ranges(n_kind, [&](int64_t q0, int64_t q1) {
    std::vector<double> rhalf, gax;
    for (int64_t q = q0; q < q1; ++q) {
      const int64_t o = kind_off[q];
      discretise(cells[kind_rep[q]], [o](int i) { return o + i; }, k_cdt.data(), k_dc.data(),
                 k_em.data(), k_a.data(), k_v.data(), k_par.data(), k_och.data(), k_ocn.data(),
                 k_tf.data(), kind_hh[q], kind_eo[q], rhalf, gax);
    }
  });
  if (by_kind) {
    parallel_ranges(n_lanes, [&](int64_t L0, int64_t L1) {
      for (int64_t L = L0; L < L1; ++L) {
        if (lane_gid[L] < 0) continue;
        const pa_cell& cl = cells[lane_gid[L]];
        const HHOut& hh = kind_hh[lane_kind[L]];
        const EmOut& eo = kind_eo[lane_kind[L]];
        if (hh.is_hh) {
          h_is_hh[L] = 1;
          for (int j = 0; j < 3; ++j) {
            h_hhg[j * n_lanes + L] = hh.g[j];
            h_hhe[j * n_lanes + L] = hh.e[j];
          }
        }
        h_emok[L] = eo.ok;
        h_em0[L] = eo.em0;
        h_emk[L] = eo.k;
        h_iinj[L] = cl.i_step;
        h_kon[L] = std::llround(cl.t_on / dt);
        h_koff[L] = cl.t_off > 1e15 ? INT64_MAX : std::llround(cl.t_off / dt);
        h_thresh[L] = cl.threshold;
      }
    });
  }
  // cells are independent: groups of lanes in parallel
  if (!by_kind) parallel_ranges(n_groups, [&](int64_t g0, int64_t g1) {
  std::vector<double> rhalf, gax, vol, hx, gdx;
  for (int64_t gi = g0; gi < g1; ++gi) {
  {
    // the group's elements (one contiguous range) take their initial values
    const int64_t e0 = (int64_t)M->row_base[gi] * kLanes;
    const int64_t e1 = (int64_t)M->row_base[gi + 1] * kLanes;
    std::fill(h_cdt.begin() + e0, h_cdt.begin() + e1, 0.0);
    std::fill(h_dc.begin() + e0, h_dc.begin() + e1, 1.0);
    std::fill(h_em.begin() + e0, h_em.begin() + e1, 0.0);
    std::fill(h_a.begin() + e0, h_a.begin() + e1, 0.0);
    std::fill(h_V.begin() + e0, h_V.begin() + e1, 0.0);
    if (M->tree) {
      std::fill(h_par.begin() + e0, h_par.begin() + e1, (int16_t)-1);
      std::fill(h_och.begin() + e0, h_och.begin() + e1, (int16_t)-1);
      std::fill(h_ocn.begin() + e0, h_ocn.begin() + e1, (int16_t)-1);
      std::fill(h_tf.begin() + e0, h_tf.begin() + e1, (uint8_t)0);
    }
  }
  for (int64_t L = gi * kLanes; L < (gi + 1) * kLanes; ++L) {
    if (lane_gid[L] < 0) continue;
    const pa_cell& cl = cells[lane_gid[L]];
    const pa_morphology& g = morphs[cl.morph];
    const int n = g.n_cv;
    HHOut hh;
    EmOut eo;
    discretise(cl, [&](int i) { return elem(L, i); }, h_cdt.data(), h_dc.data(), h_em.data(),
               h_a.data(), h_V.data(), h_par.data(), h_och.data(), h_ocn.data(), h_tf.data(), hh,
               eo, rhalf, gax);
    if (hh.is_hh) {
      h_is_hh[L] = 1;
      for (int j = 0; j < 3; ++j) {
        h_hhg[j * n_lanes + L] = hh.g[j];
        h_hhe[j * n_lanes + L] = hh.e[j];
      }
    }
    h_emok[L] = eo.ok;
    h_em0[L] = eo.em0;
    h_emk[L] = eo.k;
    if (M->cell_diff[lane_gid[L]]) {
      // PRP diffusion (Eq. diffusion on the cable's tree): CV volume, the
      // diffusive conductance of two half-cylinders in series
      // D / ((L_i/2)/(pi r_i^2) + (L_p/2)/(pi r_p^2)), summed in CV order
      vol.assign(n, 0.0);
      hx.assign(n, 0.0);
      gdx.assign(n, 0.0);
      for (int i = 0; i < n; ++i) {
        const double Lc = g.length_um[i], r = 0.5 * g.diam_um[i];
        vol[i] = (kPi * (r * r)) * Lc;
        hx[i] = (0.5 * Lc) / (kPi * (r * r));
      }
      for (int i = 1; i < n; ++i) {
        const int p = g.parent[i];
        const double gd = diff_d / (hx[i] + hx[p]);
        h_pa[elem(L, i)] = -gd;
        gdx[i] += gd;
        gdx[p] += gd;
      }
      double vt = 0.0;
      for (int i = 0; i < n; ++i) {
        const int64_t e = elem(L, i);
        h_pvdt[e] = vol[i] / dt;
        h_pdg[e] = (vol[i] / dt) + gdx[i];
        M->prp_vol[e] = vol[i];
        M->prp_gsum[e] = gdx[i];
        vt = vt + vol[i];
      }
      h_psrc[L] = vt / vol[0];  // synthesis at the soma: p_max V_tot / (V_0 tau_p)
    }
    if (cell_ca[lane_gid[L]]) {
      // heterosynaptic calcium (Eq. ca_diffusion_dendrite): the same tree
      // discretisation as the PRP field, with the HCA mechanism's D
      std::vector<double> cvol(n), chx(n), cg(n, 0.0);
      for (int i = 0; i < n; ++i) {
        const double Lc = g.length_um[i], r = 0.5 * g.diam_um[i];
        cvol[i] = (kPi * (r * r)) * Lc;
        chx[i] = (0.5 * Lc) / (kPi * (r * r));
      }
      for (int i = 1; i < n; ++i) {
        const int p = g.parent[i];
        const double gd = ca_d / (chx[i] + chx[p]);
        h_caa[elem(L, i)] = -gd;
        cg[i] += gd;
        cg[p] += gd;
      }
      for (int i = 0; i < n; ++i) {
        const int64_t e = elem(L, i);
        h_cavdt[e] = cvol[i] / dt;
        h_cadg[e] = (cvol[i] / dt) + cg[i];
        h_cavol[e] = cvol[i];
      }
    }
    h_iinj[L] = cl.i_step;
    h_kon[L] = std::llround(cl.t_on / dt);
    h_koff[L] = cl.t_off > 1e15 ? INT64_MAX : std::llround(cl.t_off / dt);
    h_thresh[L] = cl.threshold;
  }
  }
  });

  for (int64_t gi = 0; gi < n_groups; ++gi) {
    uint8_t ok = M->precision == PA_MIXED ? 1 : 0;
    if (gi < n_narrow) {
      for (int64_t L = gi * kLanes; L < (gi + 1) * kLanes; ++L) ok &= h_emok[L];
    } else {
      ok &= h_emok[gi * kLanes];  // a wide cell: its lane slot
    }
    h_emder[gi] = ok;
  }

  // ---- branch tables of the wide cells ------------------------------------------
  // A branch is a run of rows i whose parent is i - 1 (rows are contiguous),
  // cut after every fork.  A branch's level exceeds that of every branch
  // starting at a child of one of its rows, so a level only needs lower levels
  // eliminated; the root branch (row 0) is then the only branch of the top
  // level.
  std::vector<WideCell> h_wcell(n_wide);
  std::vector<int32_t> h_wbr_s, h_wbr_e, h_wlvl;
  // per branch: the parent row of its first row, and the first and the highest
  // other child of its last row (-1: none), so that the kernel loads the
  // children's values when it starts the branch
  std::vector<int32_t> h_wbr_p, h_wbr_c, h_wbr_o;
  for (int64_t j = 0; j < n_wide; ++j) {
    const pa_morphology& gm = morphs[cells[order_w[j]].morph];
    const int n = gm.n_cv;
    std::vector<int32_t> nchild(n, 0);
    for (int i = 1; i < n; ++i) ++nchild[gm.parent[i]];
    // a new branch starts at row 0, at a row whose parent is not the row
    // before, and after every fork (a row with two or more children)
    std::vector<char> is_start(n, 0);
    std::vector<int32_t> bstart, bidx(n);
    for (int i = 0; i < n; ++i) {
      is_start[i] = i == 0 || gm.parent[i] != i - 1 || nchild[i - 1] >= 2;
      if (is_start[i]) bstart.push_back(i);
      bidx[i] = (int32_t)bstart.size() - 1;
    }
    const int nb = (int)bstart.size();
    std::vector<int32_t> lvl(nb, 0);
    for (int i = n - 1; i >= 1; --i) {
      if (!is_start[i]) continue;
      int32_t& up = lvl[bidx[gm.parent[i]]];
      up = std::max(up, lvl[bidx[i]] + 1);
    }
    std::vector<int32_t> ordb(nb);
    for (int b = 0; b < nb; ++b) ordb[b] = b;
    std::stable_sort(ordb.begin(), ordb.end(), [&](int32_t x, int32_t y) { return lvl[x] < lvl[y]; });
    const int n_lvl = lvl[0] + 1;
    if (ordb[nb - 1] != 0 || (nb > 1 && lvl[ordb[nb - 2]] == lvl[0]))
      return set_err(PA_ERR_ARG, "internal: root branch is not alone on the top level");
    WideCell& w = h_wcell[j];
    w.br0 = (int32_t)h_wbr_s.size();
    w.lvl0 = (int32_t)h_wlvl.size();
    w.n_lvl = n_lvl;
    w.pad = 0;
    int b = 0;
    for (int lv = 0; lv <= n_lvl; ++lv) {
      while (b < nb && lvl[ordb[b]] < lv) ++b;
      h_wlvl.push_back(b);
    }
    std::vector<int32_t> och(n, -1);  // highest non-first child
    for (int i = 1; i < n; ++i)
      if (i != gm.parent[i] + 1) och[gm.parent[i]] = std::max(och[gm.parent[i]], i);
    for (int q = 0; q < nb; ++q) {
      const int bb = ordb[q];
      const int bs = bstart[bb], be = bb + 1 < nb ? bstart[bb + 1] - 1 : n - 1;
      h_wbr_s.push_back(bs);
      h_wbr_e.push_back(be);
      h_wbr_p.push_back(bs == 0 ? -1 : gm.parent[bs]);
      h_wbr_c.push_back(be + 1 < n && gm.parent[be + 1] == be ? be + 1 : -1);
      h_wbr_o.push_back(och[be]);
    }
  }

  // ---- synapses: one per connection, streams by mechanism -------------------------
  // (every entry is written by the parallel loops below: the tables by the
  // validation, stream and element by the synapse layout)
  M->conn_stream.resize(n_conn);
  M->conn_elem.resize(n_conn);
  M->conn_kind.resize(n_conn);
  M->conn_weight.resize(n_conn);
  M->conn_h0.resize(n_conn);
  // the synapses of each (stream, lane) pair, by a counting sort: sl_ptr[q] ..
  // sl_ptr[q + 1] in syn_rec, q = stream * n_lanes + lane
  const size_t n_sl = (size_t)n_lanes * (size_t)std::max(n_streams, 1);
  std::vector<int64_t> sl_ptr(n_sl + 1, 0);
  int64_t max_delay = 1, min_delay = INT64_MAX;
  int32_t max_dc = 0;
  std::vector<int64_t> n_out(n_cells + 1, 0);
  HostVec<int32_t> conn_D(n_conn);  // (recurrent connections only)
  // validation and the per-connection tables over fixed pieces of the
  // connection list, in parallel; the lowest bad connection is reported
  {
    constexpr int64_t kPieces = 64;
    static const char* const kWhy[] = {"", "bad dst_gid", "bad dst_cv", "bad weight",
                                       "rate_hz * dt out of range", "bad src_gid",
                                       "delay must be at least one step"};
    struct PieceOut {
      int64_t bad = -1, max_d = 1, min_d = INT64_MAX;
      int why = 0;
      int32_t max_dc = 0;
    };
    std::vector<PieceOut> po(kPieces);
    parallel_ranges(kPieces, [&](int64_t p0, int64_t p1) {
      for (int64_t p = p0; p < p1; ++p) {
        PieceOut& o = po[p];
        for (int64_t c = n_conn * p / kPieces; c < n_conn * (p + 1) / kPieces; ++c) {
          const pa_connection& k = conns[c];
          int why = 0;
          if (k.dst_gid < 0 || k.dst_gid >= n_cells) why = 1;
          else if (k.dst_cv < 0 || k.dst_cv >= M->cell_ncv[k.dst_gid]) why = 2;
          else if (!std::isfinite(k.weight)) why = 3;
          else if (k.src_gid == PA_SRC_POISSON) {
            const double x = ((k.rate_hz * dt) * 1e-3) * 4294967296.0;
            if (!(x >= 0) || x >= 4294967296.0) why = 4;
          } else if (k.src_gid < 0 || k.src_gid >= n_cells) {
            why = 5;
          } else {
            const int64_t D = std::llround(k.delay_ms / dt);
            if (!(D >= 1) || D > (1 << 30)) {
              why = 6;
            } else {
              conn_D[c] = (int32_t)D;
              o.max_d = std::max(o.max_d, D);
              o.min_d = std::min(o.min_d, D);
            }
          }
          if (why) {
            o.bad = c;
            o.why = why;
            break;
          }
          const int s = mech_stream[k.mech];
          if (M->sp[s].dc_steps > o.max_dc) o.max_dc = M->sp[s].dc_steps;
          M->conn_kind[c] = mechs[k.mech].kind;
          M->conn_weight[c] = k.weight;
          M->conn_h0[c] = mechs[k.mech].kind == PA_MECH_STC ? mechs[k.mech].params[12] : 0.0;
        }
      }
    });
    for (const PieceOut& o : po)
      if (o.bad >= 0) return set_err(PA_ERR_ARG, "connection %lld: %s", (long long)o.bad, kWhy[o.why]);
    for (const PieceOut& o : po) {
      max_delay = std::max(max_delay, o.max_d);
      min_delay = std::min(min_delay, o.min_d);
      max_dc = std::max(max_dc, o.max_dc);
    }
  }
  // counting sort of the connections by (stream, lane): per piece of the
  // connection list a count per bucket, then each piece fills its own slots
  // (within a bucket, connections stay in list order)
  HostVec<SynRec> syn_rec(n_conn);
  {
    int64_t np = 16;
    while (np > 1 && (double)np * (double)n_sl * 8.0 > 512.0 * 1024 * 1024) np /= 2;
    std::vector<int64_t> start((size_t)np * n_sl, 0);
    auto bucket = [&](int64_t c) {
      return (size_t)mech_stream[conns[c].mech] * n_lanes + M->lane_of_gid[conns[c].dst_gid];
    };
    parallel_ranges(np, [&](int64_t p0, int64_t p1) {
      for (int64_t p = p0; p < p1; ++p)
        for (int64_t c = n_conn * p / np; c < n_conn * (p + 1) / np; ++c)
          start[(size_t)p * n_sl + bucket(c)]++;
    });
    int64_t run = 0;
    for (size_t q = 0; q < n_sl; ++q) {
      sl_ptr[q] = run;
      for (int64_t p = 0; p < np; ++p) {
        const int64_t k = start[(size_t)p * n_sl + q];
        start[(size_t)p * n_sl + q] = run;
        run += k;
      }
    }
    sl_ptr[n_sl] = run;
    parallel_ranges(np, [&](int64_t p0, int64_t p1) {
      for (int64_t p = p0; p < p1; ++p)
        for (int64_t c = n_conn * p / np; c < n_conn * (p + 1) / np; ++c)
          syn_rec[start[(size_t)p * n_sl + bucket(c)]++] = {c, conns[c].dst_cv};
    });
  }
  // canonical order per lane: (CV, connection); groups in parallel
  parallel_ranges(n_groups, [&](int64_t g0, int64_t g1) {
    for (int s = 0; s < n_streams; ++s)
      for (int64_t L = g0 * kLanes; L < g1 * kLanes; ++L) {
        const size_t q = (size_t)s * n_lanes + L;
        std::sort(syn_rec.begin() + sl_ptr[q], syn_rec.begin() + sl_ptr[q + 1],
                  [](const SynRec& x, const SynRec& y) {
                    return x.cv != y.cv ? x.cv < y.cv : x.conn < y.conn;
                  });
      }
  });
  int E = (int)std::min<int64_t>(min_delay == INT64_MAX ? max_e : min_delay, max_e);
  if (E < 1) E = 1;
  M->E = E;
  M->n_slots = (int32_t)((max_delay + max_dc + E - 1) / E + 2);

  // per stream: canonical order (CV, connection) per lane, padded rows per group
  std::vector<std::vector<int32_t>> s_sbase(n_streams);
  // (filled group by group in the parallel loop below)
  std::vector<HostVec<int32_t>> s_cvf(n_streams);
  std::vector<HostVec<double>> s_weight(n_streams), s_w(n_streams);
  std::vector<HostVec<int32_t>> s_nid(n_streams);   // noise source ids (noisy streams)
  std::vector<uint8_t> h_has_stc(n_lanes, 0), h_has_ca(n_lanes, 0);
  for (int s = 0; s < n_streams; ++s) {
    s_sbase[s].assign(n_groups + 1, 0);
    for (int64_t g = 0; g < n_groups; ++g) {
      size_t mx = 0;
      for (int l = 0; l < kLanes; ++l) {
        const size_t q = (size_t)s * n_lanes + g * kLanes + l;
        mx = std::max(mx, (size_t)(sl_ptr[q + 1] - sl_ptr[q]));
      }
      const int64_t rows = g < n_narrow ? (int64_t)mx : ((int64_t)mx + kLanes - 1) / kLanes;
      if ((int64_t)s_sbase[s][g] + rows > (1LL << 26))
        return set_err(PA_ERR_ARG, "too many synapses in one stream");
      s_sbase[s][g + 1] = s_sbase[s][g] + (int32_t)rows;
    }
    const int64_t ne = (int64_t)s_sbase[s][n_groups] * kLanes;
    M->s_nelem[s] = ne;
    s_cvf[s].resize(ne);
    s_weight[s].resize(ne);
    s_w[s].resize(ne);
    if (M->sp[s].sigma > 0.0) s_nid[s].resize(ne);
  }
  // Per-CV synaptic sums are accumulated in registers over each run of same-CV
  // synapses of a stream (canonical order: mechanism, CV, connection).  Flags:
  // bit 0 "first on this CV over all streams" (the run starts from 0), bit 1 "run
  // starts", bit 2 "run ends" (store the sums).  cvf = (cv << 3) | flags.
  // lanes write disjoint elements and connections: groups in parallel
  std::vector<int64_t> n_static(n_groups, 0);
  parallel_ranges(n_groups, [&](int64_t g0, int64_t g1) {
  for (int64_t gi = g0; gi < g1; ++gi) {
  for (int s = 0; s < n_streams; ++s) {
    // the group's synapse slots (one contiguous range) take their initial values
    const int64_t e0 = (int64_t)s_sbase[s][gi] * kLanes, e1 = (int64_t)s_sbase[s][gi + 1] * kLanes;
    std::fill(s_cvf[s].begin() + e0, s_cvf[s].begin() + e1, -1);
    std::fill(s_weight[s].begin() + e0, s_weight[s].begin() + e1, 0.0);
    std::fill(s_w[s].begin() + e0, s_w[s].begin() + e1, 0.0);
    if (!s_nid[s].empty()) std::fill(s_nid[s].begin() + e0, s_nid[s].begin() + e1, 0);
  }
  for (int64_t L = gi * kLanes; L < (gi + 1) * kLanes; ++L) {
    if (lane_gid[L] < 0) continue;
    const int ncell = M->cell_ncv[lane_gid[L]];
    std::vector<char> touched(ncell, 0);
    const int64_t g = L / kLanes, l = L % kLanes;
    for (int s = 0; s < n_streams; ++s) {
      const int m = stream_mech[s];
      const double* p = mechs[m].params;
      const size_t q = (size_t)s * n_lanes + L;
      const SynRec* v = syn_rec.data() + sl_ptr[q];
      const size_t nv = (size_t)(sl_ptr[q + 1] - sl_ptr[q]);
      for (size_t j = 0; j < nv; ++j) {
        const int64_t e = g < n_narrow ? ((int64_t)s_sbase[s][g] + (int64_t)j) * kLanes + l
                                       : ((int64_t)s_sbase[s][g] << 5) + (int64_t)j;
        const int cv = v[j].cv;
        const bool start = j == 0 || v[j - 1].cv != cv;
        const bool end = j + 1 == nv || v[j + 1].cv != cv;
        const bool first = !touched[cv];
        s_cvf[s][e] = (cv << 3) | (first ? 1 : 0) | (start ? 2 : 0) | (end ? 4 : 0);
        touched[cv] = 1;
        s_weight[s][e] = conns[v[j].conn].weight;
        if (M->sp[s].kind == SK_GB) s_w[s][e] = p[12];
        if (M->sp[s].kind == SK_STDP) s_w[s][e] = p[6];
        if (M->sp[s].kind == SK_HCA) {
          s_w[s][e] = p[7];
          h_has_ca[L] = 1;
        }
        if (M->sp[s].kind == SK_STC) {
          s_w[s][e] = p[12];
          h_has_stc[L] = 1;
        }
        if (!s_nid[s].empty()) s_nid[s][e] = (int32_t)v[j].conn;
        M->conn_stream[v[j].conn] = s;
        M->conn_elem[v[j].conn] = e;
      }
    }
    // Rows whose subtree carries no synapse (statistic only: their eliminated
    // diagonal is constant, but a shortcut for them would split each warp's
    // rows into two paths, since lanes are different cells).
    const pa_morphology& gm = morphs[cells[lane_gid[L]].morph];
    std::vector<char> dyn(ncell, 0);
    for (int i = 0; i < ncell; ++i) dyn[i] = touched[i] || i == 0;
    for (int i = ncell - 1; i >= 1; --i)
      if (dyn[i]) dyn[gm.parent[i]] = 1;
    for (int i = 1; i < ncell; ++i) n_static[g] += dyn[i] ? 0 : 1;
  }
  }
  });
  for (int64_t g = 0; g < n_groups; ++g) M->n_static_cv += n_static[g];
  syn_rec.clear();
  syn_rec.shrink_to_fit();

  // Poisson drives, in connection order
  std::vector<int32_t> ps_stream, ps_dc;
  std::vector<int64_t> ps_conn;
  std::vector<int64_t> ps_elem;
  std::vector<uint32_t> ps_thr;
  {
    std::vector<int64_t> ps_ptr;
    bucket_scatter(
        n_conn, 1, [&](int64_t c) -> int64_t { return conns[c].src_gid == PA_SRC_POISSON ? 0 : -1; },
        ps_ptr,
        [&](int64_t total) {
          ps_stream.resize(total);
          ps_dc.resize(total);
          ps_conn.resize(total);
          ps_elem.resize(total);
          ps_thr.resize(total);
        },
        [&](int64_t c, int64_t q) {
          const int s = M->conn_stream[c];
          const double x = ((conns[c].rate_hz * dt) * 1e-3) * 4294967296.0;
          ps_stream[q] = s;
          ps_elem[q] = M->conn_elem[c];
          ps_conn[q] = conns[c].poisson_id >= 0 ? conns[c].poisson_id : c;
          ps_thr[q] = (uint32_t)std::floor(x);
          ps_dc[q] = M->sp[s].dc_steps;
        });
  }
  // CSR of recurrent connections by source gid (connection order within a row)
  std::vector<uint8_t> out_stream;
  std::vector<int64_t> out_elem;
  std::vector<int32_t> out_delay;
  bucket_scatter(
      n_conn, n_cells,
      [&](int64_t c) -> int64_t {
        return conns[c].src_gid == PA_SRC_POISSON ? -1 : (int64_t)conns[c].src_gid;
      },
      n_out,
      [&](int64_t total) {
        out_stream.resize(total);
        out_elem.resize(total);
        out_delay.resize(total);
      },
      [&](int64_t c, int64_t q) {
        out_stream[q] = (uint8_t)M->conn_stream[c];
        out_elem[q] = M->conn_elem[c];
        out_delay[q] = conn_D[c];
      });
  const int64_t n_edges = n_out[n_cells];
  // probes
  M->n_probe = opt->n_probe;
  if (opt->n_probe < 0 || (opt->n_probe > 0 && (!opt->probe_gid || !opt->probe_cv)))
    return set_err(PA_ERR_ARG, "bad probe list");
  std::vector<int32_t> probe_ptr(n_lanes + 1, 0), probe_row, probe_id;
  {
    std::vector<std::vector<std::pair<int, int>>> pl(n_lanes);
    for (int i = 0; i < opt->n_probe; ++i) {
      const int gid = opt->probe_gid[i], cv = opt->probe_cv[i];
      if (gid < 0 || gid >= n_cells || cv < 0 || cv >= M->cell_ncv[gid])
        return set_err(PA_ERR_ARG, "probe %d: bad location", i);
      pl[M->lane_of_gid[gid]].push_back({cv, i});
    }
    for (int64_t L = 0; L < n_lanes; ++L) {
      probe_ptr[L + 1] = probe_ptr[L] + (int32_t)pl[L].size();
      for (auto& q : pl[L]) {
        probe_row.push_back(q.first);
        probe_id.push_back(q.second);
      }
    }
  }
  M->probe_cap = opt->n_probe > 0 ? (opt->probe_capacity > 0 ? opt->probe_capacity : 65536) : 0;
  M->max_spikes = (int32_t)std::min<int64_t>(n_cells * ((E + 1) / 2) + 32, (1LL << 31) - 1);
  M->log_cap = opt->spike_capacity > 0 ? opt->spike_capacity
                                       : std::max<int64_t>(1 << 20, (int64_t)n_cells * 64);
  if (M->log_cap > (1LL << 31) - 1) M->log_cap = (1LL << 31) - 1;

  // ---- device layout ------------------------------------------------------------
  const size_t tw = M->w_bytes, tg = M->g_bytes, tsum = M->sum_bytes, ttr = M->tr_bytes;
  Arena ar;
  auto R = [&](size_t bytes) { return ar.reserve(bytes); };
  const size_t o_rowbase = R(sizeof(int32_t) * (n_groups + 1));
  const size_t o_ncv = R(sizeof(int32_t) * n_lanes);
  const size_t o_gid = R(sizeof(int32_t) * n_lanes);
  const size_t o_V = R(8 * n_elem);
  const size_t o_cdt = R(8 * n_elem), o_dc = R(8 * n_elem), o_em = R(8 * n_elem),
               o_a = R(8 * n_elem), o_gs = R(tsum * n_elem), o_es = R(tsum * n_elem);
  const size_t o_f = R(8 * n_elem), o_xp = R(8 * n_elem);
  size_t o_par = 0, o_och = 0, o_ocn = 0, o_tf = 0;
  if (M->tree) {
    o_par = R(2 * n_elem);
    o_och = R(2 * n_elem);
    o_ocn = R(2 * n_elem);
    o_tf = R(n_elem);
  }
  const size_t o_ishh = R(n_lanes), o_hhg = R(8 * 3 * n_lanes), o_hhe = R(8 * 3 * n_lanes),
               o_gate = R(8 * 3 * n_lanes), o_iinj = R(8 * n_lanes), o_kon = R(8 * n_lanes),
               o_koff = R(8 * n_lanes), o_th = R(8 * n_lanes), o_sp = R(n_lanes),
               o_prp = R(8 * n_lanes), o_hasstc = R(n_lanes), o_rbits = R(8 * n_lanes);
  const size_t o_emk = R(8 * n_lanes), o_em0 = R(8 * n_lanes), o_emder = R(h_emder.size());
  // per-kind row tables (models built by cell kind), read once by the expansion
  size_t o_kcdt = 0, o_kdc = 0, o_kem = 0, o_ka = 0, o_kpar = 0, o_koch = 0, o_kocn = 0,
         o_ktf = 0, o_kptr = 0, o_lkind = 0, o_lv0 = 0;
  if (by_kind) {
    o_kcdt = R(8 * n_kind_cv); o_kdc = R(8 * n_kind_cv); o_kem = R(8 * n_kind_cv);
    o_ka = R(8 * n_kind_cv); o_kptr = R(4 * (n_kind + 1)); o_lkind = R(4 * n_lanes);
    o_lv0 = R(8 * n_lanes);
    if (M->tree) {
      o_kpar = R(2 * n_kind_cv); o_koch = R(2 * n_kind_cv); o_kocn = R(2 * n_kind_cv);
      o_ktf = R(n_kind_cv);
    }
  }
  size_t o_s[kMaxStreams][12];
  for (int s = 0; s < n_streams; ++s) {
    const int64_t ne = M->s_nelem[s];
    const int kind = M->sp[s].kind;
    o_s[s][0] = R(sizeof(int32_t) * (n_groups + 1));
    o_s[s][1] = R(4 * ne);                    // cvf
    o_s[s][2] = R(tw * ne);                   // weight
    o_s[s][3] = R(tg * ne);                   // g
    o_s[s][4] = (kind == SK_GB || kind == SK_STC || kind == SK_HCA) ? R(8 * ne) : 0;  // c / I
    o_s[s][5] = (kind != SK_EXPSYN) ? R(8 * ne) : 0;                            // w / h
    o_s[s][6] = (kind == SK_STC) ? R(8 * ne) : 0;                               // z
    o_s[s][7] = (kind == SK_STDP) ? R(ttr * ne) : 0;                            // apre
    o_s[s][8] = (kind == SK_STDP) ? R(ttr * ne) : 0;                            // apost
    o_s[s][10] = (kind == SK_STDP) ? R(8 * ne) : 0;                             // kpre, kpost
    o_s[s][9] = R(8 * ne * (size_t)M->n_slots * ((kind == SK_GB || kind == SK_STC) ? 2 : 1));
    o_s[s][11] = M->sp[s].sigma > 0.0 ? R(4 * ne) : 0;                          // noise ids
  }
  const size_t np = ps_conn.size();
  const size_t o_ps_stream = R(4 * np), o_ps_elem = R(8 * np), o_ps_conn = R(8 * np),
               o_ps_thr = R(4 * np), o_ps_dc = R(4 * np);
  const size_t o_out_ptr = R(8 * (n_cells + 1)), o_out_stream = R(n_edges),
               o_out_elem = R(8 * n_edges), o_out_delay = R(4 * n_edges);
  const size_t o_pptr = R(4 * (n_lanes + 1)), o_prow = R(4 * probe_row.size()),
               o_pid = R(4 * probe_id.size()),
               o_pbuf = R(8 * (size_t)M->probe_cap * (size_t)std::max(M->n_probe, 0));
  const size_t o_spk_count = R(4), o_spk_gid = R(4 * (size_t)M->max_spikes),
               o_spk_step = R(4 * (size_t)M->max_spikes), o_spk_t = R(8 * (size_t)M->max_spikes);
  const size_t o_rep_count = R(4), o_rep_gid = R(4 * (size_t)M->max_spikes),
               o_rep_step = R(4 * (size_t)M->max_spikes);
  const size_t o_log_count = R(4), o_log_gid = R(4 * (size_t)M->log_cap),
               o_log_step = R(8 * (size_t)M->log_cap), o_log_t = R(8 * (size_t)M->log_cap);
  const size_t o_err = R(4);
  const size_t o_wcell = R(sizeof(WideCell) * std::max<int64_t>(n_wide, 1));
  const size_t o_wbr_s = R(sizeof(int32_t) * std::max<size_t>(h_wbr_s.size(), 1));
  const size_t o_wbr_e = R(sizeof(int32_t) * std::max<size_t>(h_wbr_e.size(), 1));
  const size_t o_wbr_p = R(sizeof(int32_t) * std::max<size_t>(h_wbr_p.size(), 1));
  const size_t o_wbr_c = R(sizeof(int32_t) * std::max<size_t>(h_wbr_c.size(), 1));
  const size_t o_wbr_o = R(sizeof(int32_t) * std::max<size_t>(h_wbr_o.size(), 1));
  const size_t o_wlvl = R(sizeof(int32_t) * std::max<size_t>(h_wlvl.size(), 1));
  const size_t o_clock = R(sizeof(EpochClock));
  size_t o_cacv = 0, o_casrc = 0, o_cadg = 0, o_caa = 0, o_cavdt = 0, o_cavol = 0, o_hasca = 0;
  if (ca_stream >= 0) {
    o_cacv = R(8 * n_elem); o_casrc = R(8 * n_elem); o_cadg = R(8 * n_elem);
    o_caa = R(8 * n_elem); o_cavdt = R(8 * n_elem); o_cavol = R(8 * n_elem);
    o_hasca = R(n_lanes);
  }
  size_t o_pcv = 0, o_pdg = 0, o_pa = 0, o_pvdt = 0, o_psrc = 0, o_ffdg = 0, o_ffvdt = 0;
  if (M->prp_diff) {
    o_pcv = R(8 * n_elem); o_pdg = R(8 * n_elem); o_pa = R(8 * n_elem);
    o_pvdt = R(8 * n_elem); o_psrc = R(8 * n_lanes);
    o_ffdg = R(8 * n_elem); o_ffvdt = R(8 * n_elem);
  }

  const size_t total = ar.used;
  cudaError_t ce = cudaMalloc((void**)&M->dmem, total);
  if (ce != cudaSuccess) {
    M->dmem = nullptr;
    return set_err(ce == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA,
                   "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(ce));
  }
  M->dbytes = total;
  CUDA_TRY(cudaMemsetAsync(M->dmem, 0, total, M->stream));

  // upload every non-zero array (pageable copies: the source may go out of scope
  // as soon as the call returns)
  int up_rc = 0;
  auto putv = [&](size_t off, const auto& v) {
    if (up_rc || v.empty()) return;
    cudaError_t e3 = cudaMemcpyAsync(M->dmem + off, v.data(), v.size() * sizeof(v[0]),
                                     cudaMemcpyHostToDevice, M->stream);
    if (e3 != cudaSuccess) up_rc = set_err(PA_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e3));
  };
  putv(o_rowbase, M->row_base);
  putv(o_ncv, lane_ncv);
  putv(o_gid, lane_gid);
  // PA_MIXED keeps the cable rows (V, coefficients; the scratch and per-CV sums
  // are written by the kernels) as float-float pairs: each double becomes the
  // nearest float and the float nearest the remainder, in its own 8 bytes
  if (M->precision == PA_MIXED && !by_kind) {
    auto to_ff = [&](HostVec<double>& v) {
      parallel_ranges((int64_t)v.size(), [&](int64_t a, int64_t b) {
        for (int64_t i = a; i < b; ++i) {
          const double x = v[i];
          const float hl[2] = {(float)x, (float)(x - (double)(float)x)};
          std::memcpy(&v[i], hl, sizeof hl);
        }
      });
    };
    to_ff(h_V); to_ff(h_cdt); to_ff(h_dc); to_ff(h_em); to_ff(h_a);
  }
  if (!by_kind) {
    putv(o_V, h_V);
    putv(o_cdt, h_cdt); putv(o_dc, h_dc); putv(o_em, h_em); putv(o_a, h_a);
    if (M->tree) {
      putv(o_par, h_par); putv(o_och, h_och); putv(o_ocn, h_ocn);
      putv(o_tf, h_tf);
    }
  } else {
    putv(o_kcdt, k_cdt); putv(o_kdc, k_dc); putv(o_kem, k_em); putv(o_ka, k_a);
    putv(o_kptr, kind_off); putv(o_lkind, lane_kind); putv(o_lv0, lane_v0);
    if (M->tree) {
      putv(o_kpar, k_par); putv(o_koch, k_och); putv(o_kocn, k_ocn); putv(o_ktf, k_tf);
    }
  }
  putv(o_hhg, h_hhg); putv(o_hhe, h_hhe);
  putv(o_ishh, h_is_hh);
  putv(o_wcell, h_wcell); putv(o_wbr_s, h_wbr_s); putv(o_wbr_e, h_wbr_e); putv(o_wlvl, h_wlvl);
  putv(o_wbr_p, h_wbr_p); putv(o_wbr_c, h_wbr_c); putv(o_wbr_o, h_wbr_o);
  putv(o_iinj, h_iinj); putv(o_kon, h_kon); putv(o_koff, h_koff); putv(o_th, h_thresh);
  putv(o_emk, h_emk); putv(o_em0, h_em0); putv(o_emder, h_emder);
  putv(o_hasstc, h_has_stc);
  if (ca_stream >= 0) {
    putv(o_cadg, h_cadg); putv(o_caa, h_caa); putv(o_cavdt, h_cavdt); putv(o_cavol, h_cavol);
    putv(o_hasca, h_has_ca);
  }
  if (M->prp_diff) {
    putv(o_pdg, h_pdg); putv(o_pa, h_pa); putv(o_pvdt, h_pvdt); putv(o_psrc, h_psrc);
  }
  for (int s = 0; s < n_streams; ++s) {
    putv(o_s[s][0], s_sbase[s]);
    putv(o_s[s][1], s_cvf[s]);
    if (w32) putv(o_s[s][2], to_f32(s_weight[s])); else putv(o_s[s][2], s_weight[s]);
    if (o_s[s][5]) putv(o_s[s][5], s_w[s]);
    if (o_s[s][11]) putv(o_s[s][11], s_nid[s]);
  }
  putv(o_ps_stream, ps_stream); putv(o_ps_elem, ps_elem); putv(o_ps_conn, ps_conn);
  putv(o_ps_thr, ps_thr); putv(o_ps_dc, ps_dc);
  putv(o_out_ptr, n_out); putv(o_out_stream, out_stream); putv(o_out_elem, out_elem);
  putv(o_out_delay, out_delay);
  putv(o_pptr, probe_ptr); putv(o_prow, probe_row); putv(o_pid, probe_id);
  if (up_rc) return up_rc;
  if (by_kind && n_elem > 0) {
    char* D0 = M->dmem;
    RowKinds rk;
    rk.cdt = (const double*)(D0 + o_kcdt); rk.dc = (const double*)(D0 + o_kdc);
    rk.em = (const double*)(D0 + o_kem); rk.a = (const double*)(D0 + o_ka);
    rk.par = (const int16_t*)(D0 + o_kpar); rk.och = (const int16_t*)(D0 + o_koch);
    rk.ocn = (const int16_t*)(D0 + o_kocn); rk.tf = (const uint8_t*)(D0 + o_ktf);
    rk.off = (const int32_t*)(D0 + o_kptr); rk.lane_kind = (const int32_t*)(D0 + o_lkind);
    rk.lane_v0 = (const double*)(D0 + o_lv0); rk.row_base = (const int32_t*)(D0 + o_rowbase);
    rk.n_groups = n_groups; rk.n_narrow = n_narrow; rk.n_elem = n_elem;
    rk.mixed = M->precision == PA_MIXED; rk.tree = M->tree;
    rk.V = (double*)(D0 + o_V); rk.CDT = (double*)(D0 + o_cdt); rk.DC = (double*)(D0 + o_dc);
    rk.EM = (double*)(D0 + o_em); rk.A = (double*)(D0 + o_a);
    rk.PAR = (int16_t*)(D0 + o_par); rk.OCH = (int16_t*)(D0 + o_och);
    rk.OCN = (int16_t*)(D0 + o_ocn); rk.TF = (uint8_t*)(D0 + o_tf);
    const int64_t blocks = std::min<int64_t>((n_elem + 255) / 256, 148 * 16);
    expand_rows_kernel<<<(unsigned)blocks, 256, 0, M->stream>>>(rk);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaStreamSynchronize(M->stream));

  char* D = M->dmem;
  auto P8 = [&](size_t o) { return (void*)(D + o); };
  EpochArgs& A = M->ea;
  std::memset(&A, 0, sizeof A);
  A.seed = M->seed;
  A.n_groups = (int32_t)n_groups;
  A.n_narrow = (int32_t)n_narrow;
  A.n_wide = (int32_t)n_wide;
  A.wcell = (const WideCell*)P8(o_wcell);
  A.wbr_s = (const int32_t*)P8(o_wbr_s);
  A.wbr_e = (const int32_t*)P8(o_wbr_e);
  A.wbr_p = (const int32_t*)P8(o_wbr_p);
  A.wbr_c = (const int32_t*)P8(o_wbr_c);
  A.wbr_o = (const int32_t*)P8(o_wbr_o);
  A.wlvl = (const int32_t*)P8(o_wlvl);
  if (n_narrow > 0 && n_wide > 0) {
    CUDA_TRY(cudaStreamCreateWithFlags(&M->side_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming));
    M->side = {M->side_stream, M->ev_fork, M->ev_join};
  }
  A.dt = dt;
  A.row_base = (const int32_t*)P8(o_rowbase);
  A.ncv = (const int32_t*)P8(o_ncv);
  A.gid = (const int32_t*)P8(o_gid);
  A.V = (double*)P8(o_V);
  A.cdt = (const double*)P8(o_cdt); A.dc = (const double*)P8(o_dc);
  A.em = (const double*)P8(o_em); A.a = (const double*)P8(o_a);
  A.gs = P8(o_gs); A.es = P8(o_es);
  A.f = (double*)P8(o_f); A.xp = (double*)P8(o_xp);
  if (M->tree) {
    A.par = (const int16_t*)P8(o_par);
    A.och_head = (const int16_t*)P8(o_och);
    A.och_next = (const int16_t*)P8(o_ocn);
    A.tflag = (const uint8_t*)P8(o_tf);
  }
  A.is_hh = (const uint8_t*)P8(o_ishh);
  A.hh_g = (const double*)P8(o_hhg); A.hh_e = (const double*)P8(o_hhe);
  A.gate = (double*)P8(o_gate);
  A.iinj = (const double*)P8(o_iinj);
  A.em_k = (const double*)P8(o_emk);
  A.em_soma = (const double*)P8(o_em0);
  A.em_derived = (const uint8_t*)P8(o_emder);
  A.k_on = (const int64_t*)P8(o_kon); A.k_off = (const int64_t*)P8(o_koff);
  A.thresh = (const double*)P8(o_th);
  A.spiked_prev = (uint8_t*)P8(o_sp);
  A.prp = (double*)P8(o_prp);
  A.has_stc = (const uint8_t*)P8(o_hasstc);
  A.stc_stream = stc_stream;
  A.ca_stream = ca_stream;
  if (ca_stream >= 0) {
    A.ca_tau = ca_tau;
    A.ca_rate = dt / ca_tau;
    A.ca_cv = (double*)P8(o_cacv);
    A.ca_src = (double*)P8(o_casrc);
    A.ca_dg = (const double*)P8(o_cadg);
    A.ca_a = (const double*)P8(o_caa);
    A.ca_vdt = (const double*)P8(o_cavdt);
    A.ca_vol = (const double*)P8(o_cavol);
    A.has_ca = (const uint8_t*)P8(o_hasca);
    M->cell_ca = cell_ca;
  }
  if (M->prp_diff) {
    A.prp_diff = 1;
    A.prp_cv = (double*)P8(o_pcv);
    A.prp_dg = (const double*)P8(o_pdg);
    A.prp_a = (const double*)P8(o_pa);
    A.prp_vdt = (const double*)P8(o_pvdt);
    A.prp_src = (const double*)P8(o_psrc);
    M->d_ff_dg = (double*)P8(o_ffdg);
    M->d_ff_vdt = (double*)P8(o_ffvdt);
  }
  A.n_lanes = n_lanes;
  A.n_row_elems = n_elem;
  A.n_streams = n_streams;
  // every reversal potential exactly +0 (a bit test: -0 does not qualify)
  A.es_zero = 1;
  for (int s = 0; s < n_streams; ++s) {
    uint64_t eb;
    std::memcpy(&eb, &M->sp[s].e, sizeof eb);
    if (eb != 0) A.es_zero = 0;
  }
  M->mask_bases.clear();
  M->mask_elems.clear();
  for (int s = 0; s < n_streams; ++s) {
    A.sp[s] = M->sp[s];
    StreamDev& sd = A.sd[s];
    const int64_t ne = M->s_nelem[s];
    const int kind = M->sp[s].kind;
    sd.sbase = (const int32_t*)P8(o_s[s][0]);
    sd.cvf = (const int32_t*)P8(o_s[s][1]);
    sd.weight = P8(o_s[s][2]);
    sd.g = P8(o_s[s][3]);
    sd.c = o_s[s][4] ? (double*)P8(o_s[s][4]) : nullptr;
    sd.w = o_s[s][5] ? (double*)P8(o_s[s][5]) : nullptr;
    sd.z = o_s[s][6] ? (double*)P8(o_s[s][6]) : nullptr;
    sd.apre = o_s[s][7] ? P8(o_s[s][7]) : nullptr;
    sd.apost = o_s[s][8] ? P8(o_s[s][8]) : nullptr;
    sd.kpre = o_s[s][10] ? (int32_t*)P8(o_s[s][10]) : nullptr;
    sd.kpost = o_s[s][10] ? (int32_t*)P8(o_s[s][10]) + ne : nullptr;
    sd.cmask = (uint64_t*)P8(o_s[s][9]);
    sd.camask = (kind == SK_GB || kind == SK_STC) ? sd.cmask + ne * M->n_slots : nullptr;
    sd.nid = o_s[s][11] ? (const int32_t*)P8(o_s[s][11]) : nullptr;
    sd.n_elem = ne;
    M->mask_bases.push_back(sd.cmask);
    M->mask_elems.push_back(ne);
    if (sd.camask) {
      M->mask_bases.push_back(sd.camask);
      M->mask_elems.push_back(ne);
    }
  }
  A.spk_count = (int32_t*)P8(o_spk_count);
  A.spk_gid = (int32_t*)P8(o_spk_gid);
  A.spk_step = (int32_t*)P8(o_spk_step);
  A.spk_t = (double*)P8(o_spk_t);
  A.spk_cap = M->max_spikes;
  A.replay_bits = (const uint64_t*)P8(o_rbits);
  M->replay_bits = (uint64_t*)P8(o_rbits);
  A.probe_ptr = (const int32_t*)P8(o_pptr);
  A.probe_row = (const int32_t*)P8(o_prow);
  A.probe_id = (const int32_t*)P8(o_pid);
  A.probe_buf = (double*)P8(o_pbuf);
  A.probe_cap = M->probe_cap;
  A.n_probe = M->n_probe;
  A.err_flags = (int32_t*)P8(o_err);
  M->err_flags = A.err_flags;
  A.epoch_len = E;
  A.n_slots = M->n_slots;
  A.clock = nullptr;
  M->clock = (EpochClock*)P8(o_clock);
  std::memset(&M->slot_clear, 0, sizeof M->slot_clear);
  M->slot_clear.n = (int32_t)M->mask_bases.size();
  M->slot_clear.n_slots = M->n_slots;
  M->slot_clear.E = E;
  M->slot_clear.probes = M->n_probe > 0 ? 1 : 0;
  for (size_t i = 0; i < M->mask_bases.size(); ++i) {
    M->slot_clear.base[i] = M->mask_bases[i];
    M->slot_clear.elems[i] = M->mask_elems[i];
  }

  PoissonArgs& PA = M->pa_args;
  std::memset(&PA, 0, sizeof PA);
  PA.E = E;
  PA.n_slots = M->n_slots;
  PA.seed = M->seed;
  PA.n = (int64_t)np;
  PA.stream = (const int32_t*)P8(o_ps_stream);
  PA.elem = (const int64_t*)P8(o_ps_elem);
  PA.conn = (const int64_t*)P8(o_ps_conn);
  PA.thr = (const uint32_t*)P8(o_ps_thr);
  PA.dc_steps = (const int32_t*)P8(o_ps_dc);
  RouteArgs& RA = M->ra;
  std::memset(&RA, 0, sizeof RA);
  RA.E = E;
  RA.n_slots = M->n_slots;
  RA.spk_cap = M->max_spikes;
  RA.spk_count = A.spk_count;
  RA.spk_gid = A.spk_gid;
  RA.spk_step = A.spk_step;
  RA.out_ptr = (const int64_t*)P8(o_out_ptr);
  RA.out_stream = (const uint8_t*)P8(o_out_stream);
  RA.out_elem = (const int64_t*)P8(o_out_elem);
  RA.out_delay = (const int32_t*)P8(o_out_delay);
  for (int s = 0; s < n_streams; ++s) {
    PA.cmask[s] = A.sd[s].cmask;
    PA.camask[s] = A.sd[s].camask;
    PA.n_elem[s] = M->s_nelem[s];
    RA.cmask[s] = A.sd[s].cmask;
    RA.camask[s] = A.sd[s].camask;
    RA.n_elem[s] = M->s_nelem[s];
    RA.dc_steps[s] = M->sp[s].dc_steps;
  }
  M->rep_spk_count = (int32_t*)P8(o_rep_count);
  M->rep_spk_gid = (int32_t*)P8(o_rep_gid);
  M->rep_spk_step = (int32_t*)P8(o_rep_step);
  M->log_count = (int32_t*)P8(o_log_count);
  M->log_gid = (int32_t*)P8(o_log_gid);
  M->log_step = (int64_t*)P8(o_log_step);
  M->log_t = (double*)P8(o_log_t);

  // initial HH gates at their steady state for v_init, from the kernels' own
  // rate functions
  {
    std::vector<double> vin(n_lanes, 0.0);
    for (int64_t L = 0; L < n_lanes; ++L)
      if (lane_gid[L] >= 0) vin[L] = cells[lane_gid[L]].v_init;
    double* dv = nullptr;
    CUDA_TRY(cudaMalloc((void**)&dv, sizeof(double) * n_lanes));
    cudaError_t e2 = cudaMemcpyAsync(dv, vin.data(), sizeof(double) * n_lanes,
                                     cudaMemcpyHostToDevice, M->stream);
    int rc = 0;
    if (e2 == cudaSuccess) {
      rc = launch_init_gates(dv, A.gate, n_lanes, A.is_hh, M->stream);
      e2 = cudaStreamSynchronize(M->stream);
    }
    cudaFree(dv);
    if (e2 != cudaSuccess || rc != 0)
      return set_err(PA_ERR_CUDA, "gate initialisation failed: %s",
                     cudaGetErrorString(e2 != cudaSuccess ? e2 : (cudaError_t)rc));
  }
  if ((opt->flags & PA_FLAG_AUTOTUNE) && ((opt->flags >> 8) & 0xF) == 0) {
    int rc = autotune(M);
    if (rc) return rc;
  }
  guard.ok = true;
  *out = M;
  return PA_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
namespace {

int check_device_errors(pa_model* M) {
  int32_t flags = 0;
  CUDA_TRY(cudaMemcpyAsync(&flags, M->err_flags, 4, cudaMemcpyDeviceToHost, M->stream));
  CUDA_TRY(cudaStreamSynchronize(M->stream));
  if (flags) {
    CUDA_TRY(cudaMemsetAsync(M->err_flags, 0, 4, M->stream));
    if (flags & 8)
      return set_err(PA_ERR_CUDA, "an index outside its array was caught by the bounds-checked "
                                  "build and its access skipped; results invalid");
    if (flags & 4)
      return set_err(PA_ERR_TIMEOUT, "a bounded device wait expired (row staging); results invalid");
    return set_err(PA_ERR_CAPACITY, "%s%s",
                   (flags & 1) ? "probe buffer full (read probes more often or raise probe_capacity); " : "",
                   (flags & 2) ? "spike record full (read spikes more often or raise spike_capacity)" : "");
  }
  return PA_OK;
}

cudaEvent_t take_event(pa_model* M) {
  if (!M->ev_pool.empty()) {
    cudaEvent_t e = M->ev_pool.back();
    M->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int collect_timings(pa_model* M) {
  if (M->pending.empty()) return PA_OK;
  CUDA_TRY(cudaStreamSynchronize(M->stream));
  for (auto& t : M->pending) {
    float x = 0, y = 0, z = 0;
    CUDA_TRY(cudaEventElapsedTime(&x, t.a, t.b));
    CUDA_TRY(cudaEventElapsedTime(&y, t.b, t.c));
    CUDA_TRY(cudaEventElapsedTime(&z, t.c, t.d));
    M->event_ms += x + z;
    M->epoch_ms += y;
    for (cudaEvent_t e : {t.a, t.b, t.c, t.d}) M->ev_pool.push_back(e);
  }
  M->pending.clear();
  return PA_OK;
}

int run_window(pa_model* M, int64_t k_begin, int64_t k_end, bool static_scratch = false) {
  using namespace pa;
  const int64_t e = k_begin / M->E;
  const int64_t k0 = e * M->E;
  pa_model::Timed tm{nullptr, nullptr, nullptr, nullptr};
  const bool timed = M->time_kernels && !static_scratch;
  if (timed) {
    if (M->pending.size() >= 4096) {
      int rc = collect_timings(M);
      if (rc) return rc;
    }
    tm = {take_event(M), take_event(M), take_event(M), take_event(M)};
    if (!tm.a || !tm.b || !tm.c || !tm.d) return set_err(PA_ERR_CUDA, "cudaEventCreate failed");
    CUDA_TRY(cudaEventRecord(tm.a, M->stream));
  }
  if (M->poisson_epoch_done != e) {
    M->pa_args.k0 = k0;
    int rc = launch_poisson(M->pa_args, k0, k0 + M->E, M->stream);
    if (rc) return set_err(PA_ERR_CUDA, "poisson launch: %s", cudaGetErrorString((cudaError_t)rc));
    M->poisson_epoch_done = e;
    if (M->pa_args.n > 0) M->n_kernel_launches++;
  }
  EpochArgs& A = M->ea;
  A.k_begin = k_begin;
  A.k_end = k_end;
  A.k0 = k0;
  A.slot = (int32_t)(e % M->n_slots);
  A.probe_sample0 = M->probe_samples;
  A.replay = M->replay ? 1 : 0;
  std::vector<int32_t> rg, rs;
  if (M->replay) {
    std::vector<uint64_t> bits(M->n_lanes, 0);
    while (M->rep_pos < M->rep_gid.size() && M->rep_step[M->rep_pos] < k_end) {
      const int64_t ks = M->rep_step[M->rep_pos];
      const int gid = M->rep_gid[M->rep_pos++];
      if (ks < k_begin || gid < 0 || gid >= M->n_cells) continue;
      bits[M->lane_of_gid[gid]] |= 1ull << (ks - k_begin);
      rg.push_back(gid);
      rs.push_back((int32_t)ks);
    }
    CUDA_TRY(cudaMemcpyAsync(M->replay_bits, bits.data(), 8 * bits.size(),
                             cudaMemcpyHostToDevice, M->stream));
    if ((int64_t)rg.size() > M->max_spikes)
      return set_err(PA_ERR_ARG, "replay list has more than %d spikes in one epoch", M->max_spikes);
    const int32_t nr = (int32_t)rg.size();
    CUDA_TRY(cudaMemcpyAsync(M->rep_spk_count, &nr, 4, cudaMemcpyHostToDevice, M->stream));
    if (nr) {
      CUDA_TRY(cudaMemcpyAsync(M->rep_spk_gid, rg.data(), 4 * rg.size(), cudaMemcpyHostToDevice, M->stream));
      CUDA_TRY(cudaMemcpyAsync(M->rep_spk_step, rs.data(), 4 * rs.size(), cudaMemcpyHostToDevice, M->stream));
    }
  }
  if (timed) CUDA_TRY(cudaEventRecord(tm.b, M->stream));
  int rc = 0;
  if (static_scratch) {
    rc = launch_epoch_noalloc(A, M->total_rows * kLanes, M->tree, M->precision, M->shape,
                              M->stream);
    if (rc == -1)
      return set_err(PA_ERR_ARG, "model has %lld padded CVs; pa_advance_noalloc holds at most %lld",
                     (long long)(M->total_rows * kLanes), (long long)noalloc_max_padded_cv());
  } else {
    rc = launch_epoch(M->precision, A, M->tree, M->shape, M->stream, side_of(M));
  }
  if (rc) return set_err(PA_ERR_CUDA, "epoch launch: %s", cudaGetErrorString((cudaError_t)rc));
  if (timed) CUDA_TRY(cudaEventRecord(tm.c, M->stream));
  M->n_epoch_launches++;
  M->n_kernel_launches += 4;  // epoch, route, record append, record finalize
  RouteArgs RA = M->ra;
  if (M->replay) {
    RA.spk_count = M->rep_spk_count;
    RA.spk_gid = M->rep_spk_gid;
    RA.spk_step = M->rep_spk_step;
  }
  rc = launch_route(RA, M->max_spikes, M->stream);
  if (rc == 0)
    rc = launch_log_append(A.spk_count, A.spk_gid, A.spk_step, A.spk_t, M->max_spikes,
                           M->log_count, M->log_gid, M->log_step, M->log_t, M->log_cap,
                           M->err_flags, M->stream);
  if (M->replay && rc == 0) {
    // replayed spikes have been routed: reset their count for the next window
    rc = (int)cudaMemsetAsync(M->rep_spk_count, 0, 4, M->stream);
  }
  if (rc) return set_err(PA_ERR_CUDA, "route launch: %s", cudaGetErrorString((cudaError_t)rc));
  if (k_end == k0 + M->E) {
    // the epoch is complete: its mask slot becomes the slot of a future epoch
    for (size_t i = 0; i < M->mask_bases.size(); ++i)
      CUDA_TRY(cudaMemsetAsync(M->mask_bases[i] + (int64_t)A.slot * M->mask_elems[i], 0,
                               8 * M->mask_elems[i], M->stream));
  }
  if (timed) {
    CUDA_TRY(cudaEventRecord(tm.d, M->stream));
    M->pending.push_back(tm);
  }
  if (M->n_probe > 0) M->probe_samples += k_end - k_begin;
  return PA_OK;
}

// The launch sequence of one whole epoch, every kernel taking its epoch from the
// device clock, and the clock's advance: what a captured graph holds.
int enqueue_graph_epoch(pa_model* M, cudaStream_t st) {
  using namespace pa;
  int rc = 0;
  if (M->pa_args.n > 0) {
    PoissonArgs P = M->pa_args;
    P.clock = M->clock;
    rc = launch_poisson(P, 0, M->E, st);
  }
  if (rc == 0) {
    EpochArgs A = M->ea;
    A.clock = M->clock;
    A.replay = 0;
    rc = launch_epoch(M->precision, A, M->tree, M->shape, st, side_of(M));
  }
  if (rc == 0) rc = launch_route(M->ra, M->max_spikes, st);
  if (rc == 0)
    rc = launch_log_append(M->ea.spk_count, M->ea.spk_gid, M->ea.spk_step, M->ea.spk_t,
                           M->max_spikes, M->log_count, M->log_gid, M->log_step, M->log_t,
                           M->log_cap, M->err_flags, st);
  if (rc == 0) rc = launch_clear_and_tick(M->slot_clear, M->clock, st);
  return rc;
}

int capture_epochs(pa_model* M, int count, cudaGraphExec_t* out) {
  if (!M->cap_stream)
    CUDA_TRY(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaStreamBeginCapture(M->cap_stream, cudaStreamCaptureModeRelaxed));
  int rc = 0;
  for (int i = 0; i < count && rc == 0; ++i) rc = enqueue_graph_epoch(M, M->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(M->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return set_err(PA_ERR_CUDA, "graph capture: %s", cudaGetErrorString((cudaError_t)rc));
  }
  if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
  return PA_OK;
}

// n whole epochs from the current step (an epoch start) as graph launches.
int run_graph_epochs(pa_model* M, int64_t n) {
  using namespace pa;
  int rc = launch_set_clock(M->clock, M->step, M->probe_samples, M->stream);
  if (rc) return set_err(PA_ERR_CUDA, "clock: %s", cudaGetErrorString((cudaError_t)rc));
  const int per_epoch = (M->pa_args.n > 0 ? 1 : 0) + 4 + (M->slot_clear.n > 0 ? 1 : 0) + 1;
  while (n > 0) {
    const int take = n >= 8 ? 8 : 1;
    cudaGraphExec_t& g = take == 8 ? M->graph8 : M->graph1;
    if (!g) {
      rc = capture_epochs(M, take, &g);
      if (rc) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(g, M->stream));
    ++M->n_graph_launches;
    for (int i = 0; i < take; ++i) {
      M->poisson_epoch_done = M->step / M->E;
      M->step += M->E;
      if (M->n_probe > 0) M->probe_samples += M->E;
    }
    M->n_epoch_launches += take;
    M->n_kernel_launches += (int64_t)take * per_epoch;
    n -= take;
  }
  return PA_OK;
}

}  // namespace

extern "C" {

int pa_build_model(const pa_cell* cells, int64_t n_cells, const pa_morphology* morphs,
                   int64_t n_morph, const pa_mechanism* mechs, int64_t n_mech,
                   const pa_connection* conns, int64_t n_conn, const pa_options* opt,
                   pa_model** out) {
  try {
    return build_impl(cells, n_cells, morphs, n_morph, mechs, n_mech, conns, n_conn, opt, out);
  } catch (const std::bad_alloc&) {
    return set_err(PA_ERR_OOM, "host allocation failed while building the model");
  } catch (...) {
    return set_err(PA_ERR_ARG, "unexpected failure while building the model");
  }
}

int pa_advance(pa_model* M, double t_end_ms, double dt_ms) {
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  if (dt_ms != M->dt) return set_err(PA_ERR_ARG, "dt %.17g differs from the build-time dt %.17g", dt_ms, M->dt);
  const double ks = t_end_ms / M->dt;
  const int64_t k_end = std::llround(ks);
  if (!std::isfinite(ks) || std::fabs(ks - (double)k_end) > 1e-6 * std::max(1.0, std::fabs(ks)))
    return set_err(PA_ERR_ARG, "t_end %.17g is not on the dt grid", t_end_ms);
  if (k_end < M->step) return set_err(PA_ERR_ARG, "t_end lies before the current time");
  try {
    CUDA_TRY(cudaSetDevice(M->device));
    while (M->step < k_end) {
      const int64_t e = M->step / M->E;
      const int64_t whole = M->step == e * M->E ? (k_end - M->step) / M->E : 0;
      if (M->graphs && !M->replay && !M->time_kernels && whole > 0 && M->poisson_epoch_done != e) {
        int rc = run_graph_epochs(M, whole);
        if (rc) return rc;
        continue;
      }
      const int64_t stop = std::min(k_end, (e + 1) * (int64_t)M->E);
      int rc = run_window(M, M->step, stop);
      if (rc) return rc;
      M->step = stop;
    }
  } catch (...) {
    return set_err(PA_ERR_OOM, "host allocation failed in pa_advance");
  }
  return PA_OK;
}

int pa_advance_noalloc(pa_model* M, double t_end_ms, double dt_ms) {
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  if (dt_ms != M->dt) return set_err(PA_ERR_ARG, "dt %.17g differs from the build-time dt %.17g", dt_ms, M->dt);
  if (M->replay) return set_err(PA_ERR_STATE, "pa_advance_noalloc does not run in open-loop replay");
  if (M->total_rows * pa::kLanes > pa::noalloc_max_padded_cv())
    return set_err(PA_ERR_ARG, "model has %lld padded CVs; pa_advance_noalloc holds at most %lld",
                   (long long)(M->total_rows * pa::kLanes), (long long)pa::noalloc_max_padded_cv());
  const double ks = t_end_ms / M->dt;
  const int64_t k_end = std::llround(ks);
  if (!std::isfinite(ks) || std::fabs(ks - (double)k_end) > 1e-6 * std::max(1.0, std::fabs(ks)))
    return set_err(PA_ERR_ARG, "t_end %.17g is not on the dt grid", t_end_ms);
  if (k_end < M->step) return set_err(PA_ERR_ARG, "t_end lies before the current time");
  CUDA_TRY(cudaSetDevice(M->device));
  while (M->step < k_end) {
    const int64_t e = M->step / M->E;
    const int64_t stop = std::min(k_end, (e + 1) * (int64_t)M->E);
    int rc = run_window(M, M->step, stop, true);
    if (rc) return rc;
    M->step = stop;
  }
  return PA_OK;
}

int pa_set_wait_limit(pa_model* M, uint32_t polls) {
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  CUDA_TRY(cudaSetDevice(M->device));
  // captured graphs hold the old arguments: synchronise, drop them, recapture lazily
  CUDA_TRY(cudaStreamSynchronize(M->stream));
  if (M->graph1) cudaGraphExecDestroy(M->graph1);
  if (M->graph8) cudaGraphExecDestroy(M->graph8);
  M->graph1 = M->graph8 = nullptr;
  M->ea.wait_limit = polls;
  return PA_OK;
}

int pa_sync(pa_model* M) {
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  CUDA_TRY(cudaSetDevice(M->device));
  return check_device_errors(M);
}

int pa_read_probes(pa_model* M, double* out, int64_t cap, int64_t* n_out) {
  if (!M || !n_out) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  int rc = check_device_errors(M);
  const int64_t ns = std::min(M->probe_samples, M->probe_cap);
  const int64_t n = ns * M->n_probe;
  *n_out = n;
  if (cap == 0) return rc;
  if (!out || cap < n) return set_err(PA_ERR_ARG, "output holds %lld values, %lld needed", (long long)cap, (long long)n);
  if (n) {
    CUDA_TRY(cudaMemcpyAsync(out, M->ea.probe_buf, 8 * n, cudaMemcpyDeviceToHost, M->stream));
    CUDA_TRY(cudaStreamSynchronize(M->stream));
  }
  M->probe_samples = 0;
  return rc;
}

int pa_read_spikes(pa_model* M, int32_t* gid, int64_t* step, double* t, int64_t cap,
                   int64_t* n_out) {
  if (!M || !n_out) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  int rc = check_device_errors(M);
  int32_t n = 0;
  CUDA_TRY(cudaMemcpyAsync(&n, M->log_count, 4, cudaMemcpyDeviceToHost, M->stream));
  CUDA_TRY(cudaStreamSynchronize(M->stream));
  *n_out = n;
  if (cap == 0) return rc;
  if (cap < n) return set_err(PA_ERR_ARG, "output holds %lld spikes, %d needed", (long long)cap, n);
  std::vector<int32_t> g(n);
  std::vector<int64_t> s(n);
  std::vector<double> tt(n);
  if (n) {
    CUDA_TRY(cudaMemcpyAsync(g.data(), M->log_gid, 4 * (size_t)n, cudaMemcpyDeviceToHost, M->stream));
    CUDA_TRY(cudaMemcpyAsync(s.data(), M->log_step, 8 * (size_t)n, cudaMemcpyDeviceToHost, M->stream));
    CUDA_TRY(cudaMemcpyAsync(tt.data(), M->log_t, 8 * (size_t)n, cudaMemcpyDeviceToHost, M->stream));
  }
  CUDA_TRY(cudaMemsetAsync(M->log_count, 0, 4, M->stream));
  CUDA_TRY(cudaStreamSynchronize(M->stream));
  std::vector<int32_t> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return s[a] != s[b] ? s[a] < s[b] : g[a] < g[b];
  });
  for (int i = 0; i < n; ++i) {
    if (gid) gid[i] = g[idx[i]];
    if (step) step[i] = s[idx[i]];
    if (t) t[i] = tt[idx[i]];
  }
  return rc;
}

int pa_read_state(pa_model* M, int32_t field, double* out, int64_t cap, int64_t* n_out) {
  using namespace pa;
  if (!M || !n_out) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  // element encodings: 8 = double, 4 = float, kFF = float-float pair (hi, lo)
  constexpr size_t kFF = 16;
  const size_t g_code = M->precision == PA_MIXED ? kFF : M->g_bytes;
  // (host arrays left uninitialised: every entry is written by the copy or
  // the conversion)
  auto fetch = [&](const void* dptr, int64_t n, size_t code, HostVec<double>& dst) -> int {
    dst.clear();
    if (n == 0 || !dptr) return 0;
    dst.resize(n);
    const size_t esz = code == kFF ? 8 : code;
    HostVec<char> raw;
    if (code != 8) raw.resize(n * esz);
    void* land = code == 8 ? (void*)dst.data() : (void*)raw.data();
    cudaError_t e = cudaMemcpyAsync(land, dptr, n * esz, cudaMemcpyDeviceToHost, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "read back: %s", cudaGetErrorString(e));
    if (code == 8) return 0;
    const float* f = (const float*)raw.data();
    parallel_ranges(n, [&](int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i)
        dst[i] = code == 4 ? (double)f[i] : (double)f[2 * i] + (double)f[2 * i + 1];
    });
    return 0;
  };
  HostVec<double> tmp;
  if (field == PA_FIELD_V) {
    *n_out = M->n_cv;
    if (cap == 0) return PA_OK;
    if (!out || cap < M->n_cv) return set_err(PA_ERR_ARG, "output too small");
    int rc = fetch(M->ea.V, M->total_rows * kLanes, M->precision == PA_MIXED ? kFF : 8, tmp);
    if (rc) return rc;
    for (int64_t c = 0; c < M->n_cells; ++c) {
      const int64_t L = M->lane_of_gid[c], g = L / kLanes;
      for (int i = 0; i < M->cell_ncv[c]; ++i)
        out[M->cell_cv_off[c] + i] =
            tmp[g < M->n_narrow ? ((int64_t)M->row_base[g] + i) * kLanes + L % kLanes
                                : ((int64_t)M->row_base[g] << 5) + i];
    }
    return PA_OK;
  }
  if (field == PA_FIELD_CA_CV) {
    *n_out = M->n_cv;
    if (cap == 0) return PA_OK;
    if (!out || cap < M->n_cv) return set_err(PA_ERR_ARG, "output too small");
    const bool has = M->ea.ca_stream >= 0;
    int rc = fetch(M->ea.ca_cv, has ? M->total_rows * kLanes : 0, 8, tmp);
    if (rc) return rc;
    for (int64_t c = 0; c < M->n_cells; ++c) {
      const int64_t L = M->lane_of_gid[c], g = L / kLanes;
      for (int i = 0; i < M->cell_ncv[c]; ++i)
        out[M->cell_cv_off[c] + i] =
            (has && M->cell_ca[c]) ? tmp[((int64_t)M->row_base[g] + i) * kLanes + L % kLanes] : 0.0;
    }
    return PA_OK;
  }
  if (field == PA_FIELD_PRP_CV) {
    *n_out = M->n_cv;
    if (cap == 0) return PA_OK;
    if (!out || cap < M->n_cv) return set_err(PA_ERR_ARG, "output too small");
    int rc = fetch(M->ea.prp_cv, M->prp_diff ? M->total_rows * kLanes : 0, 8, tmp);
    if (rc) return rc;
    for (int64_t c = 0; c < M->n_cells; ++c) {
      const int64_t L = M->lane_of_gid[c], g = L / kLanes;
      for (int i = 0; i < M->cell_ncv[c]; ++i)
        out[M->cell_cv_off[c] + i] =
            M->cell_diff[c] ? tmp[g < M->n_narrow ? ((int64_t)M->row_base[g] + i) * kLanes + L % kLanes
                                                  : ((int64_t)M->row_base[g] << 5) + i]
                            : 0.0;
    }
    return PA_OK;
  }
  if (field == PA_FIELD_PRP || field == PA_FIELD_GATES) {
    const int per = field == PA_FIELD_GATES ? 3 : 1;
    *n_out = M->n_cells * per;
    if (cap == 0) return PA_OK;
    if (!out || cap < *n_out) return set_err(PA_ERR_ARG, "output too small");
    int rc = field == PA_FIELD_PRP ? fetch(M->ea.prp, M->n_lanes, 8, tmp)
                                   : fetch(M->ea.gate, 3 * M->n_lanes, 8, tmp);
    if (rc) return rc;
    for (int64_t c = 0; c < M->n_cells; ++c)
      for (int j = 0; j < per; ++j) out[c * per + j] = tmp[j * M->n_lanes + M->lane_of_gid[c]];
    return PA_OK;
  }
  if (field < PA_FIELD_G || field > PA_FIELD_APOST) return set_err(PA_ERR_ARG, "unknown field %d", field);
  *n_out = M->n_conn;
  if (cap == 0) return PA_OK;
  if (!out || cap < M->n_conn) return set_err(PA_ERR_ARG, "output too small");
  std::vector<HostVec<double>> per_stream(M->n_streams);
  for (int s = 0; s < M->n_streams; ++s) {
    const StreamDev& D = M->ea.sd[s];
    const int kind = M->sp[s].kind;
    const void* src = nullptr;
    size_t esz = M->tr_bytes;
    switch (field) {
      case PA_FIELD_G: src = D.g; esz = g_code; break;
      case PA_FIELD_C: src = D.c; esz = 8; break;
      case PA_FIELD_W:
        src = (kind == SK_GB || kind == SK_STDP || kind == SK_HCA) ? D.w : nullptr;
        esz = 8;
        break;
      case PA_FIELD_H: src = kind == SK_STC ? D.w : nullptr; esz = 8; break;
      case PA_FIELD_Z: src = D.z; esz = 8; break;
      case PA_FIELD_APRE: src = D.apre; break;
      case PA_FIELD_APOST: src = D.apost; break;
    }
    int rc = fetch(src, src ? D.n_elem : 0, esz, per_stream[s]);
    if (rc) return rc;
  }
  // STDP traces are stored as (value after the last jump, step of that jump)
  std::vector<std::vector<double>> kstep(M->n_streams);
  if (field == PA_FIELD_APRE || field == PA_FIELD_APOST) {
    for (int s = 0; s < M->n_streams; ++s) {
      const StreamDev& D = M->ea.sd[s];
      if (M->sp[s].kind != SK_STDP) continue;
      std::vector<int32_t> ks(D.n_elem);
      const int32_t* src = field == PA_FIELD_APRE ? D.kpre : D.kpost;
      CUDA_TRY(cudaMemcpyAsync(ks.data(), src, 4 * D.n_elem, cudaMemcpyDeviceToHost, M->stream));
      CUDA_TRY(cudaStreamSynchronize(M->stream));
      kstep[s].assign(ks.begin(), ks.end());
    }
  }
  parallel_ranges(M->n_conn, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      const int s = M->conn_stream[c];
      const auto& v = per_stream[s];
      out[c] = v.empty() ? 0.0 : v[M->conn_elem[c]];
      if (!kstep[s].empty()) {
        const double tau = field == PA_FIELD_APRE ? M->sp[s].tau_pre : M->sp[s].tau_post;
        out[c] *= std::exp(-((double)(M->step - (int64_t)kstep[s][M->conn_elem[c]]) * M->dt) / tau);
      }
    }
  });
  return PA_OK;
}

int pa_read_weights(pa_model* M, double* out, int64_t cap, int64_t* n_out) {
  using namespace pa;
  if (!M || !n_out) return set_err(PA_ERR_ARG, "NULL argument");
  *n_out = M->n_conn;
  if (cap == 0) return PA_OK;
  if (!out || cap < M->n_conn) return set_err(PA_ERR_ARG, "output too small");
  // only the fields the model's mechanisms have
  bool need_w = false, need_hz = false;
  for (int s = 0; s < M->n_streams; ++s) {
    const int kind = M->sp[s].kind;
    need_w = need_w || kind == SK_GB || kind == SK_STDP || kind == SK_HCA;
    need_hz = need_hz || kind == SK_STC;
  }
  HostVec<double> w, h, z;  // (every entry is written by pa_read_state)
  int64_t n;
  int rc = 0;
  if (need_w) {
    w.resize(M->n_conn);
    rc = pa_read_state(M, PA_FIELD_W, w.data(), M->n_conn, &n);
  }
  if (!rc && need_hz) {
    h.resize(M->n_conn);
    z.resize(M->n_conn);
    rc = pa_read_state(M, PA_FIELD_H, h.data(), M->n_conn, &n);
    if (!rc) rc = pa_read_state(M, PA_FIELD_Z, z.data(), M->n_conn, &n);
  }
  if (rc) return rc;
  parallel_ranges(M->n_conn, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; ++c) {
      switch (M->conn_kind[c]) {
        case PA_MECH_GB:
        case PA_MECH_STDP:
        case PA_MECH_HCA: out[c] = w[c]; break;
        case PA_MECH_STC: out[c] = h[c] + M->conn_h0[c] * z[c]; break;
        default: out[c] = M->conn_weight[c];
      }
    }
  });
  return PA_OK;
}

int pa_set_replay(pa_model* M, int64_t n, const int32_t* gid, const int64_t* step) {
  if (!M || n < 0 || (n > 0 && (!gid || !step))) return set_err(PA_ERR_ARG, "bad replay arguments");
  M->rep_gid.assign(gid, gid + n);
  M->rep_step.assign(step, step + n);
  for (int64_t i = 0; i < n; ++i) {
    if (i > 0 && step[i] < step[i - 1]) return set_err(PA_ERR_ARG, "replay spikes must be sorted by step");
    if (step[i] < M->step) return set_err(PA_ERR_ARG, "replay spike before the current step");
  }
  M->rep_pos = 0;
  M->replay = true;
  return PA_OK;
}

int pa_inject_spikes(pa_model* M, int64_t n, const int32_t* gid, const int64_t* step) {
  using namespace pa;
  if (!M || n < 0 || (n > 0 && (!gid || !step))) return set_err(PA_ERR_ARG, "bad spike arguments");
  if (M->replay) return set_err(PA_ERR_STATE, "pa_inject_spikes does not run in open-loop replay");
  for (int64_t i = 0; i < n; ++i) {
    if (gid[i] < 0 || gid[i] >= M->n_cells)
      return set_err(PA_ERR_ARG, "spike %lld: gid %d out of range", (long long)i, gid[i]);
    if (step[i] >= M->step || step[i] < M->step - M->E)
      return set_err(PA_ERR_ARG, "spike %lld: step %lld outside the last epoch [%lld, %lld)",
                     (long long)i, (long long)step[i], (long long)(M->step - M->E),
                     (long long)M->step);
  }
  if (n == 0) return PA_OK;
  CUDA_TRY(cudaSetDevice(M->device));
  // through the replay spike buffers, max_spikes at a time, routed like the
  // model's own spikes (every connection's delay is at least one epoch, so
  // each event lands at or after the current step)
  RouteArgs RA = M->ra;
  RA.spk_count = M->rep_spk_count;
  RA.spk_gid = M->rep_spk_gid;
  RA.spk_step = M->rep_spk_step;
  std::vector<int32_t> g32, s32;
  for (int64_t off = 0; off < n; off += M->max_spikes) {
    const int32_t cnt = (int32_t)std::min<int64_t>(n - off, M->max_spikes);
    g32.assign(gid + off, gid + off + cnt);
    s32.resize(cnt);
    for (int32_t j = 0; j < cnt; ++j) s32[j] = (int32_t)step[off + j];
    CUDA_TRY(cudaMemcpyAsync(M->rep_spk_gid, g32.data(), 4 * (size_t)cnt, cudaMemcpyHostToDevice, M->stream));
    CUDA_TRY(cudaMemcpyAsync(M->rep_spk_step, s32.data(), 4 * (size_t)cnt, cudaMemcpyHostToDevice, M->stream));
    CUDA_TRY(cudaMemcpyAsync(M->rep_spk_count, &cnt, 4, cudaMemcpyHostToDevice, M->stream));
    int rc = launch_route(RA, cnt, M->stream);
    if (rc) return set_err(PA_ERR_CUDA, "route launch: %s", cudaGetErrorString((cudaError_t)rc));
    M->n_kernel_launches++;
    // the host buffers are reused: wait for the copies (and the routing) to finish
    CUDA_TRY(cudaStreamSynchronize(M->stream));
  }
  CUDA_TRY(cudaMemsetAsync(M->rep_spk_count, 0, 4, M->stream));
  return PA_OK;
}

int pa_model_info(const pa_model* M, pa_info* info) {
  if (!M || !info) return set_err(PA_ERR_ARG, "NULL argument");
  info->n_cells = M->n_cells;
  info->n_cv = M->n_cv;
  info->n_conn = M->n_conn;
  info->n_groups = M->n_groups;
  info->n_padded_cv = M->total_rows * pa::kLanes;
  info->step = M->step;
  info->epoch_steps = M->E;
  info->precision = M->precision;
  info->tree = M->tree ? 1 : 0;
  info->n_wide = (int32_t)M->n_wide;
  info->n_streams = M->n_streams;
  info->shape = M->shape;
  info->device_bytes = (int64_t)M->dbytes;
  info->n_static_cv = M->n_static_cv;
  return PA_OK;
}

int pa_get_tuning(const pa_model* M, int32_t* shape, double* trial_ms, int32_t cap) {
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  if (shape) *shape = M->shape;
  for (int32_t s = 0; trial_ms && s < cap && s < pa::kNumShapes; ++s) trial_ms[s] = M->tune_ms[s];
  return PA_OK;
}

int pa_get_kernel_stats(pa_model* M, pa_kernel_stats* out) {
  if (!M || !out) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  int rc = collect_timings(M);
  if (rc) return rc;
  out->epoch_launches = M->n_epoch_launches;
  out->kernel_launches = M->n_kernel_launches;
  out->epoch_kernel_ms = M->epoch_ms;
  out->event_kernels_ms = M->event_ms;
  out->graph_launches = M->n_graph_launches;
  return PA_OK;
}

int pa_reset_kernel_stats(pa_model* M) {
  if (!M) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  int rc = collect_timings(M);
  M->n_epoch_launches = M->n_kernel_launches = M->n_graph_launches = 0;
  M->epoch_ms = M->event_ms = 0;
  return rc;
}

int pa_fast_forward(pa_model* M, double duration_ms, int64_t n_long) {
  using namespace pa;
  if (!M) return set_err(PA_ERR_ARG, "model is NULL");
  if (M->replay) return set_err(PA_ERR_STATE, "pa_fast_forward does not run in open-loop replay");
  if (M->ea.ca_stream >= 0)
    return set_err(PA_ERR_STATE, "pa_fast_forward: heterosynaptic calcium has no long-step scheme");
  const double ks = duration_ms / M->dt;
  const int64_t K = std::llround(ks);
  if (!std::isfinite(ks) || K < 0 || std::fabs(ks - (double)K) > 1e-6 * std::max(1.0, std::fabs(ks)))
    return set_err(PA_ERR_ARG, "duration %.17g is not a whole number of steps", duration_ms);
  if (n_long < 1) return set_err(PA_ERR_ARG, "n_long must be at least 1");
  CUDA_TRY(cudaSetDevice(M->device));
  const double T = (double)K * M->dt;
  const double dtl = T / (double)n_long;
  FastForward F;
  std::memset(&F, 0, sizeof F);
  F.n_long = n_long;
  for (int s = 0; s < M->n_streams; ++s) {
    const StreamParams& P = M->sp[s];
    const double* p = M->mech_params[s].data();
    F.decay_g[s] = std::exp(-T / p[0]);
    F.decay_c[s] = (P.kind == SK_GB || P.kind == SK_STC) ? std::exp(-T / p[2]) : 1.0;
    if (P.kind == SK_GB) F.rate_w[s] = dtl / p[9];
    if (P.kind == SK_STC) {
      F.rate_h[s] = dtl / p[9];
      F.rate_z[s] = dtl / p[10];
      F.rate_p = dtl / p[11];
    }
  }
  F.tree = M->tree;
  if (M->prp_diff) {
    // the diffusing PRP field's matrix for the long step
    const int64_t ne = M->total_rows * kLanes;
    M->ff_dg.assign(ne, 1.0);
    M->ff_vdt.assign(ne, 0.0);
    for (int64_t e = 0; e < ne; ++e)
      if (M->prp_vol[e] > 0.0) {
        M->ff_vdt[e] = M->prp_vol[e] / dtl;
        M->ff_dg[e] = (M->prp_vol[e] / dtl) + M->prp_gsum[e];
      }
    CUDA_TRY(cudaMemcpyAsync(M->d_ff_dg, M->ff_dg.data(), 8 * ne, cudaMemcpyHostToDevice, M->stream));
    CUDA_TRY(cudaMemcpyAsync(M->d_ff_vdt, M->ff_vdt.data(), 8 * ne, cudaMemcpyHostToDevice, M->stream));
    F.prp_dg_long = M->d_ff_dg;
    F.prp_vdt_long = M->d_ff_vdt;
  }
  int rc = launch_fast_forward(M->ea, F, M->precision, M->stream);
  if (rc) return set_err(PA_ERR_CUDA, "fast forward: %s", cudaGetErrorString((cudaError_t)rc));
  // pending events are dropped; no POST_EVENT is due
  for (size_t i = 0; i < M->mask_bases.size(); ++i)
    CUDA_TRY(cudaMemsetAsync(M->mask_bases[i], 0, 8 * M->mask_elems[i] * (size_t)M->n_slots,
                             M->stream));
  CUDA_TRY(cudaMemsetAsync(M->ea.spiked_prev, 0, M->n_lanes, M->stream));
  M->step += K;
  M->poisson_epoch_done = -1;
  return check_device_errors(M);
}

int pa_write_state(pa_model* M, int32_t field, const double* in, int64_t n) {
  using namespace pa;
  if (!M || (!in && n > 0)) return set_err(PA_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaSetDevice(M->device));
  // read-modify-write of the device array (padding entries keep their values)
  auto rmw = [&](void* dptr, int64_t count, size_t esz, auto&& edit) -> int {
    std::vector<char> raw((size_t)count * esz);
    cudaError_t e = cudaMemcpyAsync(raw.data(), dptr, raw.size(), cudaMemcpyDeviceToHost, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "write state: %s", cudaGetErrorString(e));
    edit(raw.data());
    e = cudaMemcpyAsync(dptr, raw.data(), raw.size(), cudaMemcpyHostToDevice, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "write state: %s", cudaGetErrorString(e));
    return PA_OK;
  };
  if (field == PA_FIELD_V) {
    if (n != M->n_cv) return set_err(PA_ERR_ARG, "expected %lld values", (long long)M->n_cv);
    const bool ff = M->precision == PA_MIXED;  // V as float-float pairs
    return rmw(M->ea.V, M->total_rows * kLanes, 8, [&](char* raw) {
      for (int64_t c = 0; c < M->n_cells; ++c) {
        const int64_t L = M->lane_of_gid[c], g = L / kLanes;
        for (int i = 0; i < M->cell_ncv[c]; ++i) {
          const int64_t e = g < M->n_narrow ? ((int64_t)M->row_base[g] + i) * kLanes + L % kLanes
                                            : ((int64_t)M->row_base[g] << 5) + i;
          const double x = in[M->cell_cv_off[c] + i];
          if (ff) {
            const float hl[2] = {(float)x, (float)(x - (double)(float)x)};
            std::memcpy(raw + 8 * e, hl, sizeof hl);
          } else {
            std::memcpy(raw + 8 * e, &x, sizeof x);
          }
        }
      }
    });
  }
  if (field == PA_FIELD_CA_CV) {
    if (n != M->n_cv) return set_err(PA_ERR_ARG, "expected %lld values", (long long)M->n_cv);
    if (M->ea.ca_stream < 0) return PA_OK;
    return rmw(M->ea.ca_cv, M->total_rows * kLanes, 8, [&](char* raw) {
      double* v = (double*)raw;
      for (int64_t c = 0; c < M->n_cells; ++c) {
        if (!M->cell_ca[c]) continue;
        const int64_t L = M->lane_of_gid[c], g = L / kLanes;
        for (int i = 0; i < M->cell_ncv[c]; ++i)
          v[((int64_t)M->row_base[g] + i) * kLanes + L % kLanes] = in[M->cell_cv_off[c] + i];
      }
    });
  }
  if (field == PA_FIELD_PRP_CV || (field == PA_FIELD_PRP && M->prp_diff)) {
    // the field of each diffusing cell (PA_FIELD_PRP: uniform at the cell's
    // value) and the soma value that PA_FIELD_PRP reads back
    const bool per_cv = field == PA_FIELD_PRP_CV;
    const int64_t want = per_cv ? M->n_cv : M->n_cells;
    if (n != want) return set_err(PA_ERR_ARG, "expected %lld values", (long long)want);
    if (M->prp_diff) {
      int rc = rmw(M->ea.prp_cv, M->total_rows * kLanes, 8, [&](char* raw) {
        double* v = (double*)raw;
        for (int64_t c = 0; c < M->n_cells; ++c) {
          if (!M->cell_diff[c]) continue;
          const int64_t L = M->lane_of_gid[c], g = L / kLanes;
          for (int i = 0; i < M->cell_ncv[c]; ++i)
            v[g < M->n_narrow ? ((int64_t)M->row_base[g] + i) * kLanes + L % kLanes
                              : ((int64_t)M->row_base[g] << 5) + i] =
                per_cv ? in[M->cell_cv_off[c] + i] : in[c];
        }
      });
      if (rc) return rc;
    }
    return rmw(M->ea.prp, M->n_lanes, 8, [&](char* raw) {
      double* v = (double*)raw;
      for (int64_t c = 0; c < M->n_cells; ++c) {
        if (per_cv && !M->cell_diff[c]) continue;
        v[M->lane_of_gid[c]] = per_cv ? in[M->cell_cv_off[c]] : in[c];
      }
    });
  }
  if (field == PA_FIELD_PRP || field == PA_FIELD_GATES) {
    const int per = field == PA_FIELD_GATES ? 3 : 1;
    if (n != M->n_cells * per) return set_err(PA_ERR_ARG, "expected %lld values", (long long)(M->n_cells * per));
    return rmw(field == PA_FIELD_PRP ? (void*)M->ea.prp : (void*)M->ea.gate, per * M->n_lanes, 8,
               [&](char* raw) {
                 double* v = (double*)raw;
                 for (int64_t c = 0; c < M->n_cells; ++c)
                   for (int j = 0; j < per; ++j) v[j * M->n_lanes + M->lane_of_gid[c]] = in[c * per + j];
               });
  }
  if (field < PA_FIELD_G || field > PA_FIELD_APOST) return set_err(PA_ERR_ARG, "unknown field %d", field);
  if (n != M->n_conn) return set_err(PA_ERR_ARG, "expected %lld values", (long long)M->n_conn);
  for (int s = 0; s < M->n_streams; ++s) {
    const StreamDev& D = M->ea.sd[s];
    const int kind = M->sp[s].kind;
    void* dst = nullptr;
    int enc = 8;  // 8 = double, 4 = float, 2 = float-float pair (hi, lo)
    switch (field) {
      case PA_FIELD_G:
        dst = D.g;
        enc = M->precision == PA_MIXED ? 2 : (int)M->g_bytes;
        break;
      case PA_FIELD_C: dst = D.c; break;
      case PA_FIELD_W: dst = (kind == SK_GB || kind == SK_STDP || kind == SK_HCA) ? D.w : nullptr; break;
      case PA_FIELD_H: dst = kind == SK_STC ? D.w : nullptr; break;
      case PA_FIELD_Z: dst = D.z; break;
      case PA_FIELD_APRE: dst = D.apre; enc = (int)M->tr_bytes; break;
      case PA_FIELD_APOST: dst = D.apost; enc = (int)M->tr_bytes; break;
    }
    if (!dst) continue;
    int rc = rmw(dst, D.n_elem, enc == 4 ? 4 : 8, [&](char* raw) {
      for (int64_t c = 0; c < M->n_conn; ++c) {
        if (M->conn_stream[c] != s) continue;
        const int64_t e = M->conn_elem[c];
        if (enc == 4) {
          ((float*)raw)[e] = (float)in[c];
        } else if (enc == 2) {
          const float hi = (float)in[c];
          ((float*)raw)[2 * e] = hi;
          ((float*)raw)[2 * e + 1] = (float)(in[c] - (double)hi);
        } else {
          ((double*)raw)[e] = in[c];
        }
      }
    });
    if (rc) return rc;
    if ((field == PA_FIELD_APRE || field == PA_FIELD_APOST) && kind == SK_STDP) {
      // a trace written now: its last jump is the current step
      rc = rmw(field == PA_FIELD_APRE ? (void*)D.kpre : (void*)D.kpost, D.n_elem, 4, [&](char* raw) {
        for (int64_t c = 0; c < M->n_conn; ++c)
          if (M->conn_stream[c] == s) ((int32_t*)raw)[M->conn_elem[c]] = (int32_t)M->step;
      });
      if (rc) return rc;
    }
  }
  return PA_OK;
}

int pa_measure_fp64(int32_t device, double* out) {
  if (!out) return set_err(PA_ERR_ARG, "pa_measure_fp64: NULL output");
  CUDA_TRY(cudaSetDevice(device));
  int n_sm = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  double* sink = nullptr;
  CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = 8 * n_sm, iters = 1 << 14;
  float best = 1e30f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first run warms up
    e = cudaEventRecord(e0, nullptr);
    if (e == cudaSuccess) e = (cudaError_t)pa::launch_fma_rate(blocks, iters, sink, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "pa_measure_fp64: %s", cudaGetErrorString(e));
  const double fmas = (double)blocks * 256.0 * 8.0 * (double)iters;
  out[0] = fmas / (best * 1e-3);
  out[1] = best;
  return PA_OK;
}

int pa_check_arith(int32_t device, uint64_t seed, int64_t n_random, int64_t* out) {
  if (!out || n_random < 0) return set_err(PA_ERR_ARG, "pa_check_arith: bad arguments");
  CUDA_TRY(cudaSetDevice(device));
  int n_sm = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  unsigned long long* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 4 * sizeof(unsigned long long)));
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof h);
  if (e == cudaSuccess) e = (cudaError_t)pa::launch_arith_check(seed, n_random, d, n_sm, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess)
    return set_err(PA_ERR_CUDA, "pa_check_arith: %s", cudaGetErrorString(e));
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)h[i];
  return PA_OK;
}

void pa_free_model(pa_model* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  if (M->dmem) {
    cudaStreamSynchronize(M->stream);
    cudaFree(M->dmem);
  }
  for (auto& t : M->pending)
    for (cudaEvent_t e : {t.a, t.b, t.c, t.d}) cudaEventDestroy(e);
  for (cudaEvent_t e : M->ev_pool) cudaEventDestroy(e);
  if (M->graph1) cudaGraphExecDestroy(M->graph1);
  if (M->graph8) cudaGraphExecDestroy(M->graph8);
  if (M->cap_stream) cudaStreamDestroy(M->cap_stream);
  if (M->side_stream) cudaStreamDestroy(M->side_stream);
  if (M->ev_fork) cudaEventDestroy(M->ev_fork);
  if (M->ev_join) cudaEventDestroy(M->ev_join);
  delete M;
}

const char* pa_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"


// ---------------------------------------------------------------------------
// Batches: several resident models advanced together, one grouped epoch-kernel
// launch per min-delay epoch for all of them (the serving path).

struct pa_batch {
  int device = 0;
  cudaStream_t stream = nullptr;       // every member runs on it
  cudaStream_t cap_stream = nullptr;   // capture only
  static constexpr int kSide = 8;      // branches for the members' small kernels
  cudaStream_t side[kSide] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kSide] = {};
  std::vector<pa_model*> members;
  int precision = -1;
  bool tree = false;
  pa::EpochArgs* d_args = nullptr;     // members' launch arguments (clock-driven)
  int2* d_bmap = nullptr;              // block -> (member, first group)
  size_t cap_args = 0, cap_bmap = 0;
  int n_blocks = 0;
  bool dirty = true;                   // membership changed since the last upload
  cudaGraphExec_t g1 = nullptr, g8 = nullptr;
  int64_t n_launches = 0;              // graph launches
  int64_t n_captures = 0;              // graphs captured (membership changes)
};

namespace {

void batch_drop_graphs(pa_batch* B) {
  if (B->g1) cudaGraphExecDestroy(B->g1);
  if (B->g8) cudaGraphExecDestroy(B->g8);
  B->g1 = B->g8 = nullptr;
}

// Members' arguments and the block map to the device (on membership change).
int batch_upload(pa_batch* B) {
  using namespace pa;
  std::vector<EpochArgs> args(B->members.size());
  std::vector<int2> bmap;
  for (size_t j = 0; j < B->members.size(); ++j) {
    pa_model* M = B->members[j];
    EpochArgs A = M->ea;
    A.clock = M->clock;
    A.replay = 0;
    args[j] = A;
    for (int32_t g0 = 0; g0 < M->n_narrow; g0 += kGroupedWarps) bmap.push_back(make_int2((int)j, g0));
  }
  if (args.size() > B->cap_args) {
    if (B->d_args) cudaFree(B->d_args);
    B->d_args = nullptr;
    B->cap_args = 0;
    CUDA_TRY(cudaMalloc(&B->d_args, sizeof(EpochArgs) * args.size()));
    B->cap_args = args.size();
  }
  if (bmap.size() > B->cap_bmap) {
    if (B->d_bmap) cudaFree(B->d_bmap);
    B->d_bmap = nullptr;
    B->cap_bmap = 0;
    CUDA_TRY(cudaMalloc(&B->d_bmap, sizeof(int2) * bmap.size()));
    B->cap_bmap = bmap.size();
  }
  if (!args.empty())
    CUDA_TRY(cudaMemcpyAsync(B->d_args, args.data(), sizeof(EpochArgs) * args.size(),
                             cudaMemcpyHostToDevice, B->stream));
  if (!bmap.empty())
    CUDA_TRY(cudaMemcpyAsync(B->d_bmap, bmap.data(), sizeof(int2) * bmap.size(),
                             cudaMemcpyHostToDevice, B->stream));
  CUDA_TRY(cudaStreamSynchronize(B->stream));
  B->n_blocks = (int)bmap.size();
  batch_drop_graphs(B);
  B->dirty = false;
  return PA_OK;
}

// One epoch of every member on capture stream st: the members' Poisson draws
// on parallel branches, the grouped epoch kernel, then each member's routing,
// spike record and clock tick on parallel branches.
int batch_enqueue_epoch(pa_batch* B, cudaStream_t st) {
  using namespace pa;
  const int K = pa_batch::kSide;
  auto fork = [&]() -> int {
    CUDA_TRY(cudaEventRecord(B->ev_fork, st));
    for (int k = 0; k < K; ++k) CUDA_TRY(cudaStreamWaitEvent(B->side[k], B->ev_fork, 0));
    return PA_OK;
  };
  auto join = [&]() -> int {
    for (int k = 0; k < K; ++k) {
      CUDA_TRY(cudaEventRecord(B->ev_join[k], B->side[k]));
      CUDA_TRY(cudaStreamWaitEvent(st, B->ev_join[k], 0));
    }
    return PA_OK;
  };
  int rc = fork();
  for (size_t j = 0; j < B->members.size() && rc == 0; ++j) {
    pa_model* M = B->members[j];
    if (M->pa_args.n > 0) {
      PoissonArgs P = M->pa_args;
      P.clock = M->clock;
      rc = launch_poisson(P, 0, M->E, B->side[j % K]);
    }
  }
  if (rc == 0) rc = join();
  bool ez = true;  // the E = +0 kernels serve the batch only if they serve every member
  for (const pa_model* M : B->members) ez = ez && M->ea.es_zero != 0;
  if (rc == 0)
    rc = launch_epoch_grouped(B->precision, B->d_args, B->d_bmap, B->n_blocks, B->tree, ez, st);
  if (rc == 0) rc = fork();
  for (size_t j = 0; j < B->members.size() && rc == 0; ++j) {
    pa_model* M = B->members[j];
    cudaStream_t sj = B->side[j % K];
    rc = launch_route(M->ra, M->max_spikes, sj);
    if (rc == 0)
      rc = launch_log_append(M->ea.spk_count, M->ea.spk_gid, M->ea.spk_step, M->ea.spk_t,
                             M->max_spikes, M->log_count, M->log_gid, M->log_step, M->log_t,
                             M->log_cap, M->err_flags, sj);
    if (rc == 0) rc = launch_clear_and_tick(M->slot_clear, M->clock, sj);
  }
  if (rc == 0) rc = join();
  return rc;
}

int batch_capture(pa_batch* B, int count, cudaGraphExec_t* out) {
  CUDA_TRY(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeRelaxed));
  int rc = 0;
  for (int i = 0; i < count && rc == 0; ++i) rc = batch_enqueue_epoch(B, B->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc < 0 ? rc : set_err(PA_ERR_CUDA, "batch capture: %s", cudaGetErrorString((cudaError_t)rc));
  }
  if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_err(PA_ERR_CUDA, "batch instantiation: %s", cudaGetErrorString(e));
  return PA_OK;
}

}  // namespace

int pa_batch_create(int32_t device, void* stream, pa_batch** out) {
  if (!out) return set_err(PA_ERR_ARG, "NULL output");
  *out = nullptr;
  pa_batch* B = new (std::nothrow) pa_batch();
  if (!B) return set_err(PA_ERR_OOM, "host allocation failed");
  B->device = device;
  B->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking);
  for (int k = 0; k < pa_batch::kSide && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    pa_batch_free(B);
    return set_err(PA_ERR_CUDA, "pa_batch_create: %s", cudaGetErrorString(e));
  }
  *out = B;
  return PA_OK;
}

int pa_batch_add(pa_batch* B, pa_model* M) {
  if (!B || !M) return set_err(PA_ERR_ARG, "NULL argument");
  if (std::find(B->members.begin(), B->members.end(), M) != B->members.end())
    return set_err(PA_ERR_ARG, "model already in the batch");
  if (M->device != B->device) return set_err(PA_ERR_ARG, "a member must be on the batch's device");
  if (M->n_wide > 0) return set_err(PA_ERR_ARG, "a member must have no wide-bin cells (PA_FLAG_NARROW_ONLY)");
  if (M->replay) return set_err(PA_ERR_STATE, "a member cannot be in open-loop replay");
  if (M->step % M->E != 0) return set_err(PA_ERR_STATE, "a member must be at an epoch boundary");
  if (!B->members.empty() && (M->precision != B->precision || M->tree != B->tree))
    return set_err(PA_ERR_ARG, "members must share precision and tree class");
  if (B->members.empty()) {
    B->precision = M->precision;
    B->tree = M->tree;
  }
  if (M->stream != B->stream) {
    // the member moves to the batch's stream, after its own work
    CUDA_TRY(cudaSetDevice(M->device));
    CUDA_TRY(cudaStreamSynchronize(M->stream));
    M->stream = B->stream;
  }
  B->members.push_back(M);
  B->dirty = true;
  return PA_OK;
}

int pa_batch_remove(pa_batch* B, pa_model* M) {
  if (!B || !M) return set_err(PA_ERR_ARG, "NULL argument");
  auto it = std::find(B->members.begin(), B->members.end(), M);
  if (it == B->members.end()) return set_err(PA_ERR_ARG, "model not in the batch");
  B->members.erase(it);
  B->dirty = true;
  return PA_OK;
}

int pa_batch_advance(pa_batch* B, int64_t n_epochs) {
  using namespace pa;
  if (!B || n_epochs < 0) return set_err(PA_ERR_ARG, "bad arguments");
  if (B->members.empty() || n_epochs == 0) return PA_OK;
  CUDA_TRY(cudaSetDevice(B->device));
  for (pa_model* M : B->members)
    if (M->step % M->E != 0) return set_err(PA_ERR_STATE, "a member left its epoch boundary");
  if (B->dirty) {
    int rc = batch_upload(B);
    if (rc) return rc;
  }
  // the members' device clocks from their host positions (a member may have
  // been advanced alone since the last batch advance)
  for (pa_model* M : B->members) {
    int rc = launch_set_clock(M->clock, M->step, M->probe_samples, B->stream);
    if (rc) return set_err(PA_ERR_CUDA, "clock: %s", cudaGetErrorString((cudaError_t)rc));
  }
  int64_t n = n_epochs;
  while (n > 0) {
    const int take = n >= 8 ? 8 : 1;
    cudaGraphExec_t& g = take == 8 ? B->g8 : B->g1;
    if (!g) {
      int rc = batch_capture(B, take, &g);
      if (rc) return rc;
      ++B->n_captures;
    }
    CUDA_TRY(cudaGraphLaunch(g, B->stream));
    ++B->n_launches;
    for (pa_model* M : B->members) {
      for (int i = 0; i < take; ++i) {
        M->poisson_epoch_done = M->step / M->E;
        M->step += M->E;
        if (M->n_probe > 0) M->probe_samples += M->E;
      }
      M->n_epoch_launches += take;
    }
    n -= take;
  }
  return PA_OK;
}

int pa_batch_info(const pa_batch* B, int64_t* out) {
  if (!B || !out) return set_err(PA_ERR_ARG, "NULL argument");
  out[0] = (int64_t)B->members.size();
  out[1] = B->n_blocks;
  out[2] = B->n_launches;
  out[3] = B->n_captures;
  return PA_OK;
}

void pa_batch_free(pa_batch* B) {
  if (!B) return;
  cudaSetDevice(B->device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  batch_drop_graphs(B);
  if (B->d_args) cudaFree(B->d_args);
  if (B->d_bmap) cudaFree(B->d_bmap);
  for (int k = 0; k < pa_batch::kSide; ++k) {
    if (B->side[k]) cudaStreamDestroy(B->side[k]);
    if (B->ev_join[k]) cudaEventDestroy(B->ev_join[k]);
  }
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  delete B;
}
