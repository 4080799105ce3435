// engine.h -- internal data layout shared by the host builder and the kernels.
//
// Layout ("lane-interleaved groups"): cells are sorted by CV count (descending)
// and dealt into groups of 32; one warp advances one group, one thread one
// cell.  Row i of a group holds CV i of its 32 cells in 32 consecutive slots,
// so element (group g, row i, lane l) lives at ((row_base[g] + i) << 5) | l and
// every per-row access of a warp is one coalesced 256-byte (FP64) transaction.
// A group has as many rows as its largest cell; shorter cells leave padding
// rows that are never touched.  Synapses are laid out the same way, one
// "stream" per point mechanism of the model: row j of a stream holds the j-th
// synapse (in the canonical order CV, connection) of each lane's cell.
#pragma once
#include <cstdint>

#include <vector_types.h>

namespace pa {

// Fork flags of a tree row (EpochArgs::tflag).
constexpr uint8_t kForkPop = 1;   // exactly one non-first child: its values are popped here
constexpr uint8_t kForkPush = 2;  // the one non-first child of its parent: pushed here
constexpr uint8_t kParPrev = 4;   // the parent is the previous row (row i - 1)
constexpr uint8_t kOtherList = 8; // non-first children taken through the linked list

constexpr int kLanes = 32;
constexpr int kMaxStreams = 8;
constexpr int kMaxProbeRowsPerLane = 1 << 15;

enum StreamKind : int32_t { SK_EXPSYN = 0, SK_GB = 1, SK_STC = 2, SK_STDP = 3, SK_HCA = 4 };

// Constants of one synapse stream (one point mechanism), derived for the dt.
struct StreamParams {
  int32_t kind;
  int32_t dc_steps;      // presynaptic calcium delay in steps (GB, STC)
  double e;              // reversal potential [mV]
  double decay_g;        // exp(-dt/tau)
  double decay_c;        // exp(-dt/tau_c)
  double c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d;
  double rate_w, w_star; // GB: dt/tau_w, w*
  double rate_h, rate_z, rate_p, h0, theta_tag, theta_pro, p_max, f_int;  // STC
  double a_pre, a_post, tau_pre, tau_post, w_max;                         // STDP
  double sigma;          // GB, STC: plasticity noise sigma_pl (0: none)
  double amp[3];         // sigma_pl sqrt(n dt / tau) with n thresholds crossed
  // HCA (c_pre = I0 [pA], decay_c = exp(-dt/tau_I), theta_p/theta_d [umol/l]):
  // calcium inflow per pA gamma 1e6 / (2 F), dt gamma_p, dt gamma_d per step
  double hca_kq, hca_gpr, hca_gdr;
  // the same constants rounded to FP32, for the FP32-mechanism policy
  struct F32 {
    float decay_c, c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d;
    float rate_w, w_star, rate_h, rate_z, h0, theta_tag, f_int;
    float a_pre, a_post, tau_pre, tau_post, w_max;
    float pad;
  } f;
};

// Device pointers of one synapse stream.  Element index e = ((sbase+j)<<5)|lane.
struct StreamDev {
  const int32_t* cvf;    // (cv << 1) | first-on-CV flag; -1 for padding
  const int32_t* sbase;  // [n_groups + 1] row offsets of each group
  const void* weight;    // uS: double (PA_FP64) or float (PA_MIXED, PA_FP32)
  void* g;               // conductance [uS]: double, float2 hi + lo (PA_MIXED) or float
  double* c;             // calcium (GB, STC)
  double* w;             // GB w, STDP w, STC h
  double* z;             // STC z
  void* apre;            // STDP: trace value right after its last jump, as the weight
  void* apost;           // STDP, as the weight
  int32_t* kpre;         // step of the last jump of apre (STDP)
  int32_t* kpost;        // step of the last jump of apost (STDP)
  uint64_t* cmask;       // [n_slots][n_elem]: bit (k mod E) = conductance event in step k
  uint64_t* camask;      // [n_slots][n_elem]: delayed calcium event (GB, STC)
  const int32_t* nid;    // noise source of each synapse (its connection index; noisy streams)
  int64_t n_elem;
};

// Device-side position of a graph-launched model: the epoch a captured launch
// sequence advances (every launch reads it; the sequence's last kernel moves it
// on by one epoch), so that one captured CUDA graph serves every epoch.
struct EpochClock {
  int64_t k0;              // first step of the epoch
  int64_t probe_sample0;   // probe sample index of step k0
};

// A cell of the wide bin (one warp per cell): its branch list (rows
// [wbr_s, wbr_e] of each branch, sorted by level) and the level offsets into it.
struct WideCell {
  int32_t br0;    // first entry in wbr_s / wbr_e
  int32_t lvl0;   // first entry in wlvl (n_lvl + 1 offsets, relative to br0)
  int32_t n_lvl;
  int32_t pad;
};

// Cell bins.  When the narrow bin alone would give fewer than
// kWideMaxWarpsPerSM warps per SM, the wide bin takes the cells with at least
// kWideMinCV CVs in at least kWideMinBranches branches and at most
// kWideMaxSynPerCV synapses per CV (the per-CV sums are serial runs, so a
// cell whose synapses crowd onto few CVs gains less from a warp).  Below one
// warp per SM the GPU is mostly idle in the narrow bin, and every cell with at
// least kWideMinWork CVs plus synapses is wide.  PA_FLAG_WIDE_ALL: every cell.
constexpr int kWideMinCV = 128;
constexpr int kWideMinBranches = 8;
constexpr int kWideMaxSynPerCV = 2;
constexpr int kWideMaxWarpsPerSM = 4;
constexpr int kWideMinWork = 128;

struct EpochArgs {
  // launch window: steps [k_begin, k_end) all inside epoch [k0, k0 + E); with
  // `clock` set the window is the whole epoch the clock names instead
  int64_t k_begin, k_end, k0;
  int32_t slot;          // mask slot of this epoch
  int32_t epoch_len;     // E
  int32_t n_slots;
  const EpochClock* clock;
  uint64_t seed;         // key of the counter-based generator (plasticity noise)
  int32_t n_groups;      // all groups: narrow [0, n_narrow), then one per wide cell
  int32_t n_narrow;      // groups of 32 cells, one thread per cell
  int32_t n_wide;        // wide cells, one warp per cell
  const WideCell* wcell; // [n_wide]
  const int32_t* wbr_s;  // branch first row
  const int32_t* wbr_e;  // branch last row
  const int32_t* wbr_p;  // parent row of the branch's first row (-1: the root branch)
  const int32_t* wbr_c;  // first child of the branch's last row (-1: none)
  const int32_t* wbr_o;  // highest other child of the branch's last row (-1: none)
  const int32_t* wlvl;   // level offsets
  double dt;
  // groups / lanes
  const int32_t* row_base;   // [n_groups + 1]
  const int32_t* ncv;        // [n_lanes] CV count of the lane's cell (0: empty lane)
  const int32_t* gid;        // [n_lanes] cell gid (-1: empty lane)
  // CV arrays (element index)
  double* V;
  const double* cdt;         // C/dt [uS]
  const double* dc;          // cdt + axial sum (+ leak for passive CVs)
  const double* em;          // leak g E for passive CVs
  const double* a;           // -g_axial to the parent
  void* gs;                  // synaptic conductance per CV: double (float in PA_FP32)
  void* es;                  // synaptic g E per CV: double (float in PA_FP32)
  double* f;                 // elimination scratch
  double* xp;                // elimination scratch
  const int16_t* par;        // tree: parent row (row 0: -1)
  const int16_t* och_head;   // tree: highest-index non-first child (-1: none)
  const int16_t* och_next;   // tree: next lower non-first sibling (-1: none)
  // tree: per row, kForkPop if the row has exactly one non-first child (and its
  // cell's forks nest), kForkPush if the row is the one non-first child of such
  // a row, kParPrev if its parent is row i - 1, kOtherList if its non-first
  // children go through the linked list
  const uint8_t* tflag;
  // soma / cell state (lane index)
  const uint8_t* is_hh;
  const double* hh_g;        // [3][n_lanes] gna, gk, gl [uS]
  const double* hh_e;        // [3][n_lanes] ena, ek, el [mV]
  double* gate;              // [3][n_lanes] m, h, n
  const double* iinj;
  // PA_MIXED, groups (either bin) with em_derived[g]: the leak E-term of a
  // dendrite row is (C/dt) em_k[lane], the soma row's em_soma[lane]
  const double* em_k;
  const double* em_soma;
  const uint8_t* em_derived;
  const int64_t* k_on;
  const int64_t* k_off;
  const double* thresh;
  uint8_t* spiked_prev;
  double* prp;               // STC PRP per lane
  const uint8_t* has_stc;
  int32_t stc_stream;        // index of the STC stream or -1
  // PRP diffusion (Eq. diffusion; an STC mechanism with D_p > 0, every cell with
  // STC synapses in the narrow bin): the PRP concentration, the constant
  // backward-Euler matrix (diagonal V/dt + sum gD, coupling -gD to the parent)
  // and V/dt per CV in the narrow element layout; per lane the soma's synthesis
  // scale V_tot / V_0.  prp[] then holds the soma CV's concentration.
  int32_t prp_diff;
  double* prp_cv;
  const double* prp_dg;
  const double* prp_a;
  const double* prp_vdt;
  const double* prp_src;
  // heterosynaptic calcium (an HCA stream; its cells in the narrow bin): the
  // calcium per CV [umol/l], its backward-Euler matrix (diagonal, coupling),
  // V/dt and V per CV, the step's inflow per CV (summed by the synapse phase)
  int32_t ca_stream;         // index of the HCA stream or -1
  // every stream's reversal potential is exactly +0: g E is the zero of g's
  // sign, so the per-CV g E sums are signed zeros (kernels specialise on this)
  int32_t es_zero;
  double ca_tau, ca_rate;    // tau_C, dt / tau_C
  double* ca_cv;
  double* ca_src;
  const double* ca_dg;
  const double* ca_a;
  const double* ca_vdt;
  const double* ca_vol;
  const uint8_t* has_ca;     // per lane
  int64_t n_lanes;
  // synapse streams
  int32_t n_streams;
  StreamParams sp[kMaxStreams];
  StreamDev sd[kMaxStreams];
  // spike output of this launch
  int32_t* spk_count;
  int32_t* spk_gid;
  int32_t* spk_step;
  double* spk_t;
  int32_t spk_cap;
  // open-loop replay (POST_EVENT source); replay_bits[lane] bit j = spike at k_begin + j
  int32_t replay;
  const uint64_t* replay_bits;
  // probes
  const int32_t* probe_ptr;  // [n_lanes + 1]
  const int32_t* probe_row;
  const int32_t* probe_id;
  double* probe_buf;
  int64_t probe_sample0;     // sample index of step k_begin
  int64_t probe_cap;         // samples
  int32_t n_probe;
  int32_t* err_flags;        // bit 0: probe overflow, bit 1: spike record full,
                             // bit 2: a bounded wait expired
  uint32_t wait_limit;       // polls of a bounded staging wait (0: the default)
  int64_t n_row_elems;       // elements of the CV-row arrays (bounds of the checked build)
};

struct PoissonArgs {
  int64_t k0;                // epoch start (ignored with `clock` set)
  const EpochClock* clock;   // graph launches: the epoch comes from here
  int32_t E;
  int32_t n_slots;
  uint64_t seed;
  int64_t n;                 // Poisson synapses
  const int32_t* stream;     // stream index
  const int64_t* elem;       // element index in the stream
  const int64_t* conn;       // Poisson train id (the connection index by default)
  const uint32_t* thr;       // spike iff u32 < thr
  const int32_t* dc_steps;   // calcium delay (-1: none)
  uint64_t* cmask[kMaxStreams];
  uint64_t* camask[kMaxStreams];
  int64_t n_elem[kMaxStreams];
};

struct RouteArgs {
  int32_t E;
  int32_t n_slots;
  int32_t spk_cap;           // entries in the spike buffer
  const int32_t* spk_count;
  const int32_t* spk_gid;
  const int32_t* spk_step;
  const int64_t* out_ptr;    // [n_cells + 1] CSR by source gid
  const uint8_t* out_stream;
  const int64_t* out_elem;
  const int32_t* out_delay;  // steps
  int32_t dc_steps[kMaxStreams];  // -1: no calcium target
  uint64_t* cmask[kMaxStreams];
  uint64_t* camask[kMaxStreams];
  int64_t n_elem[kMaxStreams];
};

// kernel launchers (defined in the .cu files)
constexpr int kNumShapes = 6;  // kernel shapes (see launch_epoch_shape)
// The narrow kernel over groups [0, n_narrow) and the wide kernel.  With
// `side` (a second stream and two events) and both bins in use, the wide
// kernel runs on the side stream concurrently with the narrow one (fork and
// join through the events, so a stream capture records two parallel
// branches); otherwise one after the other on `stream`.
struct SideLaunch {
  void* stream;  // cudaStream_t
  void* fork;    // cudaEvent_t
  void* join;    // cudaEvent_t
};
int launch_epoch_fp64(const EpochArgs& a, bool tree, int shape, void* stream,
                      const SideLaunch* side = nullptr);
int launch_epoch_mixed(const EpochArgs& a, bool tree, int shape, void* stream,
                       const SideLaunch* side = nullptr);
int launch_epoch_fp32(const EpochArgs& a, bool tree, int shape, void* stream,
                      const SideLaunch* side = nullptr);
// the launcher of precision `prec` (PA_FP64, PA_MIXED, PA_FP32)
inline int launch_epoch(int prec, const EpochArgs& a, bool tree, int shape, void* stream,
                        const SideLaunch* side = nullptr) {
  return prec == 1   ? launch_epoch_mixed(a, tree, shape, stream, side)
         : prec == 2 ? launch_epoch_fp32(a, tree, shape, stream, side)
                     : launch_epoch_fp64(a, tree, shape, stream, side);
}
int launch_init_gates(const double* v, void* gate, int64_t n_lanes, const uint8_t* is_hh,
                      void* stream);
// One launch over several models (narrow bin only): block b runs 4 groups from
// group d_bmap[b].y of model d_bmap[b].x, whose arguments are d_args[d_bmap[b].x].
constexpr int kGroupedWarps = 4;
// (ez: every member model has es_zero set)
int launch_epoch_grouped_fp64(const EpochArgs* d_args, const int2* d_bmap, int n_blocks, bool tree,
                              bool ez, void* stream);
int launch_epoch_grouped_mixed(const EpochArgs* d_args, const int2* d_bmap, int n_blocks,
                               bool tree, bool ez, void* stream);
int launch_epoch_grouped_fp32(const EpochArgs* d_args, const int2* d_bmap, int n_blocks, bool tree,
                              bool ez, void* stream);
inline int launch_epoch_grouped(int prec, const EpochArgs* d_args, const int2* d_bmap,
                                int n_blocks, bool tree, bool ez, void* stream) {
  return prec == 1   ? launch_epoch_grouped_mixed(d_args, d_bmap, n_blocks, tree, ez, stream)
         : prec == 2 ? launch_epoch_grouped_fp32(d_args, d_bmap, n_blocks, tree, ez, stream)
                     : launch_epoch_grouped_fp64(d_args, d_bmap, n_blocks, tree, ez, stream);
}
// Graph launches: zero the mask slot of the clock's epoch in every mask array,
// then advance the clock by one epoch (events.cu).
struct SlotClear {
  int32_t n;                       // mask arrays
  int32_t n_slots, E;
  int32_t probes;                  // advance probe_sample0 too
  uint64_t* base[2 * kMaxStreams];
  int64_t elems[2 * kMaxStreams];  // elements per slot
};
int launch_clear_and_tick(const SlotClear& c, EpochClock* clock, void* stream);
int launch_set_clock(EpochClock* clock, int64_t k0, int64_t probe_sample0, void* stream);

// pa_fast_forward (fastforward.cu): per-stream exact decay factors over the
// fast-forwarded time and long-step rates dt_long / tau.
struct FastForward {
  int64_t n_long;
  double decay_g[kMaxStreams], decay_c[kMaxStreams];
  double rate_w[kMaxStreams], rate_h[kMaxStreams], rate_z[kMaxStreams];
  double rate_p;  // dt_long / tau_p of the STC stream
  // a diffusing PRP field: the long step's matrix diagonal V/dt_long + sum gD
  // and V/dt_long per CV (narrow element layout); tree rows present
  const double* prp_dg_long;
  const double* prp_vdt_long;
  bool tree;
};
int launch_fast_forward(const EpochArgs& a, const FastForward& f, int prec, void* stream);

int launch_epoch_noalloc(const EpochArgs& a, int64_t n_padded_cv, bool tree, int prec,
                         int shape, void* stream);
int64_t noalloc_max_padded_cv();

// Device self-check of int_arith.cuh (arith_check.cu): counts into d_out[0]
// reciprocal mismatches, [1] float-widening mismatches, [2] cases checked,
// [3] the first mismatching reciprocal input (bits).
int launch_arith_check(uint64_t seed, int64_t n_random, unsigned long long* d_out, int n_sm,
                       void* stream);
// FP64 FMA throughput microbenchmark (arith_check.cu): blocks x 256 threads,
// each running 8 independent chains of `iters` FMAs.
int launch_fma_rate(int blocks, int iters, double* sink, void* stream);
int launch_poisson(const PoissonArgs& a, int64_t k_from, int64_t k_to, void* stream);
int launch_route(const RouteArgs& a, int32_t max_spikes, void* stream);
int launch_log_append(const int32_t* spk_count, const int32_t* gid, const int32_t* step,
                      const double* t, int32_t max_spikes, int32_t* log_count,
                      int32_t* log_gid, int64_t* log_step, double* log_t, int64_t log_cap,
                      int32_t* err_flags, void* stream);

}  // namespace pa
