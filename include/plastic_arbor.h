/*
 * plastic_arbor.h -- C-ABI of the B300 engine for the fixed-dt time-step loop of
 * networks of multi-compartment neurons with spike-driven plastic synapses
 * ("Plastic Arbor", arXiv 2411.16445).
 *
 * One call of pa_advance runs, for every cell and every step, the four stages of
 * the loop on the GPU:
 *   1. mechanism currents and state updates: Hodgkin-Huxley soma (the paper's
 *      simple-branchy cells, Sec. "Runtime and memory benchmarking with
 *      large-scale networks"), passive leak, conductance-based exponential
 *      synapses, pair STDP (Eqs. stdp_ode_1-3), Graupner-Brunel calcium
 *      plasticity (Eqs. weight_graupner_brunel, ca_model_graupner_brunel) and
 *      synaptic tagging and capture (Eqs. total_syn_weight .. prp_single_comp),
 *      with the POST_EVENT hook (Sec. "Spike-time detection to simplify
 *      computation") and the delayed second calcium target of the
 *      round_robin_halt policy (Sec. "Multiple postsynaptic variables ...");
 *   2. backward-Euler assembly of the cable equation (Eq. cable) and a Hines
 *      solve of each cell's tree;
 *   3. threshold-crossing spike detection at the soma;
 *   4. event delivery through a CSR connectivity table once per min-delay epoch.
 *
 * Units: mV, ms, um, uS (weights and point conductances), nA, S/cm2 (densities),
 * uF/cm2, ohm cm.
 *
 * Conventions for every entry point:
 *   - All pointers passed in are host pointers owned by the caller; they are
 *     read during the call and may be freed afterwards.  The model owns every
 *     device allocation it makes and releases it in pa_free_model.
 *   - Return value 0 means success.  Negative values are errors (PA_ERR_*); a
 *     human-readable message is then available from pa_last_error() (thread-
 *     local, valid until the next call on the same thread).  No C++ exception
 *     crosses this boundary.
 *   - A model is used by one host thread at a time.
 */
#ifndef PLASTIC_ARBOR_H
#define PLASTIC_ARBOR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PA_OK 0
#define PA_ERR_ARG (-1)      /* invalid descriptor, size or argument */
#define PA_ERR_OOM (-2)      /* device or host allocation failed */
#define PA_ERR_CUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error) */
#define PA_ERR_TIMEOUT (-4)  /* a bounded device wait expired */
#define PA_ERR_CAPACITY (-5) /* a probe or spike record buffer filled up; data were dropped */
#define PA_ERR_STATE (-6)    /* call not valid in the model's current state */

/* mechanism kinds */
#define PA_MECH_PAS 1     /* density, params: g [S/cm2], e [mV] */
#define PA_MECH_HH 2      /* density (soma CV only), params: gnabar, gkbar, gl [S/cm2],
                             ena, ek, el [mV] */
#define PA_MECH_EXPSYN 10 /* point, params: tau [ms], e [mV] */
#define PA_MECH_GB 11     /* point, expsyn + Graupner-Brunel calcium rule; params: tau, e,
                             tau_c, c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d,
                             tau_w [ms], w_star, t_c_delay [ms], w0 [, sigma_pl] */
#define PA_MECH_STC 12    /* point, expsyn + tagging and capture; params: tau, e, tau_c,
                             c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d, tau_h,
                             tau_z, tau_p [ms], h0 [mV], theta_tag [mV], theta_pro [mV],
                             p_max, f_int, t_c_delay [ms] [, sigma_pl [mV] [, D_p]] */
/* PRP diffusion (Eq. diffusion on the cable's tree): with the optional
 * diffusivity D_p > 0 [um2/ms] (1e-11 m2/s = 1e-2 um2/ms) the PRP of every cell
 * with STC synapses is a concentration per CV.  Each step, after the synapse
 * updates (which capture the PRP at their own CV, Eq. late_phase_weight), every
 * CV takes the explicit reaction step P + dt/tau_p (src - P), src = p_max
 * V_tot / V_0 at the soma CV while S > theta_pro and 0 elsewhere (so the total
 * amount follows Eq. prp_single_comp for the mean concentration), then the
 * field takes one backward-Euler diffusion step, V_i (P_i' - P_i)/dt =
 * sum_j gD_ij (P_j' - P_i'), gD = D_p / ((L_i/2)/(pi r_i^2) + (L_j/2)/(pi r_j^2))
 * for adjacent CVs, solved by the same tree elimination as the cable equation.
 * PA_FIELD_PRP then reads the soma CV's concentration.  Both cell bins solve
 * the field (the wide bin by the same branch levels as the voltage).
 * pa_fast_forward takes the same two steps with the long step (its own
 * backward-Euler matrix). */
/* Plasticity noise (Eqs. plasticity_noise_1-2): with the optional trailing
 * sigma_pl > 0, each step adds sigma_pl sqrt(n dt / tau) N(0,1) to w (GB,
 * tau = tau_w) or h (STC, tau = tau_h), n = number of the thresholds theta_p,
 * theta_d the calcium exceeds (Euler-Maruyama).  N(0,1) of synapse (connection)
 * c at step k: Box-Muller from Threefry-4x64-12 with key (seed, 0, 0, 0) and
 * counter (c, k / 4, 2, 0); k mod 4 = 2p + j uses output words 2p, 2p+1 as
 * 53-bit uniforms u1, u2: sqrt(-2 log(1 - u1)) cos (j = 0) or sin (j = 1) of
 * 2 pi u2, with the engine's own log, cos and sin (documented in rng.cuh). */
#define PA_MECH_STDP 13   /* point, expsyn + pair STDP; params: tau, e, tau_pre, tau_post
                             [ms], A_pre, A_post, w0, w_max (w dimensionless, conductance
                             jump = weight * clip(w, 0, w_max)) */
#define PA_MECH_HCA 14    /* point, heterosynaptic calcium (Eqs. ca_injection_current_spine,
                             ca_diffusion_dendrite, heterosyn_weight); params: I0 [pA],
                             tau_I [ms], gamma, gamma_p, gamma_d [1/s], theta_p, theta_d
                             [umol/l], w0, tau_C [ms], D [um2/ms].  No conductance: an
                             event adds I0 to the synapse's injection current I (decay
                             tau_I), whose calcium w gamma I / (2 F) enters the synapse's
                             CV each step; the cell's calcium per CV decays with tau_C and
                             diffuses with D (the explicit reaction, then one backward-
                             Euler diffusion step on the tree, as for the PRP); w follows
                             Eq. heterosyn_weight by forward Euler with its CV's calcium.
                             At most one HCA mechanism per model; its cells run in the
                             narrow bin; pa_fast_forward refuses the model. */

/* arithmetic of the loop */
#define PA_FP64 0   /* everything in FP64: the plain definition, operation for operation */
#define PA_MIXED 1  /* synaptic conductances (exponential decay, event jumps, the per-CV
                       sums of each run of same-CV synapses) and the cable solve (voltage,
                       cable coefficients, per-CV sums, assembly, elimination, back
                       substitution) on the FP32 pipes in float-float form (hi + lo, about
                       48 significand bits); STDP traces in FP32; event weights, HH,
                       calcium and the slow plasticity state (GB w, STC h/z/p, STDP w) in
                       FP64.  Meets the oracle within 1e-5 V and 1e-3 ms. */
#define PA_FP32 2   /* conductances, event weights, STDP traces and the per-CV synaptic
                       sums in plain FP32, and the mechanisms in FP32 (HH rates and gates,
                       calcium, the GB / STC / STDP increments, accumulated into the FP64
                       slow state); the cable solve in FP64.  Each step re-rounds every
                       conductance (2^-24): spike counts match the oracle on the test
                       networks, spike times and voltages do not meet the PA_MIXED bounds
                       (its measured error against the oracle is documented with the
                       engine). */

/* connection source meaning "an independent Poisson train of rate rate_hz" */
#define PA_SRC_POISSON (-1)

/* synapse / cell state fields for pa_read_state */
#define PA_FIELD_G 0       /* synaptic conductance [uS], per connection */
#define PA_FIELD_C 1       /* calcium, per connection (GB, STC) */
#define PA_FIELD_W 2       /* plastic weight w (GB, STDP), per connection */
#define PA_FIELD_H 3       /* early-phase weight h [mV] (STC), per connection */
#define PA_FIELD_Z 4       /* late-phase weight z (STC), per connection */
#define PA_FIELD_APRE 5    /* STDP presynaptic trace, per connection */
#define PA_FIELD_APOST 6   /* STDP postsynaptic trace, per connection */
#define PA_FIELD_V 16      /* membrane potential [mV], per CV in cell-major order */
#define PA_FIELD_PRP 17    /* PRP concentration p (STC), per cell */
#define PA_FIELD_GATES 18  /* HH gates m, h, n of each cell's soma CV: 3 values per cell */
#define PA_FIELD_PRP_CV 19 /* PRP concentration per CV (cell-major) of cells whose PRP
                              diffuses (STC with D_p > 0); 0 on every other CV */
#define PA_FIELD_CA_CV 20  /* heterosynaptic calcium per CV (cell-major) of cells with HCA
                              synapses [umol/l]; 0 on every other CV.  PA_FIELD_C reads an
                              HCA synapse's injection current I [pA], PA_FIELD_W its w */

typedef struct pa_model pa_model;

/* A CV-level morphology: CV i is a cylinder of length length_um[i] and diameter
 * diam_um[i] whose parent is parent[i] (parent[0] = -1, 0 <= parent[i] < i,
 * n_cv <= 32767).  region[i] = 0 selects the cell's soma mechanism, 1 its
 * dendrite mechanism.  CV 0 is the soma: spikes are detected there. */
typedef struct {
  int32_t n_cv;
  const int32_t* parent;
  const double* length_um;
  const double* diam_um;
  const int32_t* region;
} pa_morphology;

/* One cell.  soma_mech / dend_mech index the mechanism table (PAS or HH; HH
 * only on CV 0).  i_step [nA] is injected into CV 0 during steps k with
 * round(t_on/dt) <= k < round(t_off/dt) (t_off > 1e15 means never off). */
typedef struct {
  int32_t morph;
  int32_t soma_mech;
  int32_t dend_mech;
  int32_t reserved;
  double cm;        /* uF/cm2 */
  double ra;        /* ohm cm */
  double i_step;    /* nA */
  double t_on;      /* ms */
  double t_off;     /* ms */
  double v_init;    /* mV */
  double threshold; /* mV: spike iff V_soma^k < threshold <= V_soma^{k+1} */
} pa_cell;

typedef struct {
  int32_t kind;     /* PA_MECH_* */
  int32_t n_params; /* must equal the kind's parameter count */
  const double* params;
} pa_mechanism;

/* One connection = one synapse of mechanism `mech` on CV dst_cv of cell
 * dst_gid.  A spike of src_gid in step k is delivered at the start of step
 * k + round(delay_ms/dt) (>= 1 step); a GB/STC synapse also receives its
 * presynaptic calcium jump round(t_c_delay/dt) steps later.  src_gid =
 * PA_SRC_POISSON drives the synapse with its own Poisson train of rate_hz
 * (delivered in the step it is drawn; delay_ms ignored).  Such a train is
 * identified by poisson_id (a negative value means the connection's index):
 * connections with the same poisson_id and rate receive the same train. */
typedef struct {
  int32_t src_gid;
  int32_t dst_gid;
  int32_t dst_cv;
  int32_t mech;
  double weight;   /* uS */
  double delay_ms;
  double rate_hz;
  int64_t poisson_id;
} pa_connection;

typedef struct {
  double dt;                /* ms, fixed for the model's lifetime */
  uint64_t seed;            /* keys the Poisson trains (Threefry-4x64-12) */
  int32_t precision;        /* PA_FP64, PA_MIXED or PA_FP32 */
  int32_t device;           /* CUDA device ordinal */
  void* stream;             /* cudaStream_t to run on; NULL = the legacy default stream */
  int32_t n_probe;          /* membrane-potential probes recorded after every step */
  const int32_t* probe_gid;
  const int32_t* probe_cv;
  int64_t probe_capacity;   /* samples held between pa_read_probes calls (0: 65536) */
  int64_t spike_capacity;   /* spikes held between pa_read_spikes calls (0: automatic) */
  int32_t max_epoch_steps;  /* upper bound of the epoch length (0: 64); <= 64 */
  int32_t flags;            /* PA_FLAG_* */
} pa_options;

/* pa_options.flags: record CUDA events around every kernel launch on the model's
 * stream so that pa_get_kernel_stats can report device time per kernel kind. */
#define PA_FLAG_TIME_KERNELS 1
/* pa_options.flags: at build time, time every compiled shape of the epoch kernel
 * (rows per TMA chunk, warps per block, register budget) on the model's first
 * epoch and keep the fastest.  The model's state is snapshot and restored
 * around the trials (needs a second copy of the model's device memory for the
 * duration of the build; without room for it the default shape is kept). */
#define PA_FLAG_AUTOTUNE 2
/* pa_options.flags: force epoch-kernel shape s (0 <= s < PA_N_SHAPES) */
#define PA_FLAG_SHAPE(s) ((((s) + 1) & 0xF) << 8)
#define PA_N_SHAPES 6
/* pa_options.flags: launch every kernel directly.  By default pa_advance runs
 * each run of whole min-delay epochs as CUDA-graph launches (the epoch's Poisson,
 * time-step, routing and record kernels captured once, replayed per epoch; 8
 * epochs per launch where they fit).  Partial epochs, open-loop replay and
 * PA_FLAG_TIME_KERNELS always launch directly.  Results are identical. */
#define PA_FLAG_NO_GRAPHS 8
/* pa_options.flags: cell bins.  A cell runs on one thread of a warp that holds
 * 32 cells (the narrow bin), or on a whole warp (the wide bin: its synapses
 * updated 32 at a time, its tree eliminated branch-parallel by levels).  By
 * default, when the narrow bin alone would leave fewer than 4 warps per SM,
 * cells with at least 128 CVs in at least 8 branches and at most 2 synapses
 * per CV are wide; below 1 warp per SM, every cell with at least 128 CVs plus
 * synapses is.  Both bins give identical results.  NARROW_ONLY / WIDE_ALL
 * force every cell into one bin. */
#define PA_FLAG_NARROW_ONLY 16
#define PA_FLAG_WIDE_ALL 32
/* pa_options.flags: at most n host threads (1 <= n <= 63) for this model's
 * build; 0 (the default): the cores the process may use, up to 64, shared
 * among builds running at the same time.  A server that builds models while
 * it launches other models' work keeps cores free this way.  The model does
 * not depend on the thread count. */
#define PA_FLAG_BUILD_THREADS(n) (((n) & 0x3F) << 12)

typedef struct {
  int64_t epoch_launches;   /* epoch (time-step) kernel launches since the last reset */
  int64_t kernel_launches;  /* all kernel launches of the engine since the last reset */
  double epoch_kernel_ms;   /* device time of the epoch kernels (PA_FLAG_TIME_KERNELS) */
  double event_kernels_ms;  /* device time of the Poisson, routing and record kernels */
  int64_t graph_launches;   /* CUDA-graph launches (each runs 1 or 8 whole epochs) */
} pa_kernel_stats;

typedef struct {
  int64_t n_cells, n_cv, n_conn, n_groups, n_padded_cv;
  int64_t step;             /* steps completed */
  int32_t epoch_steps;      /* min-delay epoch length E */
  int32_t precision;
  int32_t tree;             /* 1 if any morphology branches */
  int32_t n_streams;        /* synapse streams (one per point mechanism in use) */
  int32_t shape;            /* epoch-kernel shape in use */
  int32_t n_wide;           /* cells in the warp-per-cell bin */
  int64_t device_bytes;     /* device memory held by the model */
  int64_t n_static_cv;      /* CVs whose subtree carries no synapse (a statistic) */
} pa_info;

/* Validates the descriptors, discretises every morphology (CV = cylinder:
 * area pi d L, C = c_m A, axial conductance of two half-cylinders in series,
 * Eq. cable), lays the state out on the device and uploads it.  On success
 * *out receives the model.  Errors: PA_ERR_ARG (message names the offending
 * element; of several bad connections, the lowest-indexed), PA_ERR_OOM,
 * PA_ERR_CUDA.  The host layout runs on the cores the calling process may use
 * (at most 64 threads, shared among builds that run at the same time); the
 * model does not depend on the thread count.  The descriptor arrays are only
 * read, and only during the call. */
int pa_build_model(const pa_cell* cells, int64_t n_cells, const pa_morphology* morphs,
                   int64_t n_morph, const pa_mechanism* mechs, int64_t n_mech,
                   const pa_connection* conns, int64_t n_conn, const pa_options* opt,
                   pa_model** out);

/* Advances the simulation to t_end_ms (on the dt grid, >= the current time).
 * dt_ms must equal the build-time dt.  Runs asynchronously on the model's
 * stream except that it returns only after the work was enqueued; errors
 * raised by the device (record overflow) are reported by the next
 * pa_read_* / pa_sync call. */
int pa_advance(pa_model* m, double t_end_ms, double dt_ms);

/* pa_advance for callers that must not allocate GPU memory while they run --
 * for example code inside a region whose allocations are owned by another
 * memory manager, or a host thread on a real-time path where a device
 * allocation could stall or fail.  The paper has no counterpart; this is an
 * interface convenience.
 *
 * It advances the model exactly like pa_advance (the same kernels, so the same
 * results bit for bit in every precision), but the Hines elimination scratch
 * of the epoch kernels comes from one array of 32 MiB that the library
 * reserves in device memory on every GPU it is used on, held until the process
 * exits.  The call allocates nothing: no cudaMalloc, no cudaFree, no kernel
 * timing events (PA_FLAG_TIME_KERNELS is ignored here), no CUDA graphs.
 *   - Limit: models of at most 2,097,152 padded CVs (pa_info.n_padded_cv);
 *     larger models get PA_ERR_ARG.  Open-loop replay is not supported
 *     (PA_ERR_STATE).
 *   - The first call on a GPU looks the array's device address up (a one-time
 *     set-up, per device; with CUDA's lazy module loading the driver reserves
 *     the array at that moment).  Make that first call before any stream
 *     capture and outside any region that must not allocate.
 *   - All calls share the one array.  Calls whose GPU work overlaps (two models
 *     advanced concurrently on different streams) race on it; serialise them.
 *   - Nothing in the array needs clearing: each step writes the values before
 *     it reads them. */
int pa_advance_noalloc(pa_model* m, double t_end_ms, double dt_ms);

/* Waits for the model's stream and reports device-side errors. */
int pa_sync(pa_model* m);

/* Poll limit of the epoch kernel's bounded waits for its staged rows (the
 * paper has no counterpart; failure detection of this engine).  polls = 0
 * restores the default (4,194,304 polls, milliseconds).  A wait that runs out
 * makes the kernel stop stepping, let every copy it issued land, and return;
 * the next pa_sync / pa_read_* reports PA_ERR_TIMEOUT and the model's state is
 * then invalid (the CUDA context stays usable).  A limit of a few polls makes
 * waits run out on purpose, which is how the failure path is tested.
 * Synchronises the model's stream and drops its captured CUDA graphs (they are
 * captured again at the next whole-epoch advance). */
int pa_set_wait_limit(pa_model* m, uint32_t polls);

/* Copies the probe samples recorded since the last call into out
 * ([sample][probe], double, cap values) and clears the record.  cap = 0 only
 * queries: *n_out receives the number of values available. */
int pa_read_probes(pa_model* m, double* out, int64_t cap, int64_t* n_out);

/* Copies the spikes recorded since the last call, sorted by (step, gid), into
 * gid / step / t (any may be NULL; cap entries each) and clears the record.
 * t is the interpolated crossing time [ms].  cap = 0 only queries. */
int pa_read_spikes(pa_model* m, int32_t* gid, int64_t* step, double* t, int64_t cap,
                   int64_t* n_out);

/* Plastic weight of every connection in build order: GB and STDP w, STC
 * total weight h + h0 z (Eq. total_syn_weight), static synapses their weight. */
int pa_read_weights(pa_model* m, double* out, int64_t cap, int64_t* n_out);

/* Any state field (PA_FIELD_*), per connection, per CV or per cell. */
int pa_read_state(pa_model* m, int32_t field, double* out, int64_t cap, int64_t* n_out);

/* Open-loop replay: from now on the network's own spikes no longer drive
 * synaptic events or POST_EVENT; instead cell gid[i] is taken to have spiked
 * in step step[i] (sorted by step, all >= the current step).  Own spikes are
 * still detected and recorded. */
int pa_set_replay(pa_model* m, int64_t n, const int32_t* gid, const int64_t* step);

/* Spikes of cells simulated elsewhere -- the exchange step of a network
 * sharded over several GPUs (one model per GPU, each holding its own cells
 * plus passive stand-ins for remote presynaptic cells; the paper runs Arbor
 * with one MPI rank per GPU, Sec. "Runtime and memory benchmarking with
 * large-scale networks").  Cell gid[i] of this model is taken to have spiked in
 * step step[i], which must lie in the last epoch, [current step - E, current
 * step) with E = pa_info.epoch_steps: every connection's delay is at least E,
 * so each of its events is still due.  The events are routed through the
 * model's connection table exactly as for a spike detected here (the delayed
 * calcium targets included); POST_EVENT is not triggered.  Not in open-loop
 * replay.  Synchronises the model's stream. */
int pa_inject_spikes(pa_model* m, int64_t n, const int32_t* gid, const int64_t* step);

int pa_model_info(const pa_model* m, pa_info* info);

/* Writes a state field (the inverse of pa_read_state, same layout and count):
 * per connection for the synapse fields (entries of connections whose kind
 * lacks the field are ignored; a written STDP trace counts as jumping now),
 * per CV for PA_FIELD_V and PA_FIELD_PRP_CV (cells whose PRP diffuses; other
 * entries ignored), per cell for PA_FIELD_PRP (a diffusing cell's field is set
 * uniform) and (3 per cell: m, h, n) PA_FIELD_GATES.  Swaps a saved state into a model, e.g. one built from an
 * edited network (the state-saving mechanism of the '8h-recall' paradigm).
 * Synchronises the model's stream. */
int pa_write_state(pa_model* m, int32_t field, const double* values, int64_t n);

/* Fast-forward (the '8h-recall' paradigm: phases of slow network dynamics):
 * advances the model by duration_ms (whole steps) without spiking and calcium
 * dynamics.  The membrane state is kept, pending events are dropped, every
 * conductance and calcium decays by exp(-duration / tau), and the slow
 * plasticity variables take n_long forward-Euler steps of duration / n_long
 * with the calcium terms (and the noise) off: per cell S = sum |h - h0| (STC,
 * canonical order) from h before the step, then per synapse z (Eq.
 * late_phase_weight with the cell's p), h (Eq. early_phase_weight: 0.1 (h0 - h)
 * / tau_h), GB w (Eq. weight_graupner_brunel: its cubic term), then p (Eq.
 * prp_single_comp; a diffusing PRP field: its reaction and diffusion steps with
 * the long step, z with the PRP at the synapse's CV).  STDP traces decay through their closed form.  All state
 * stays on the device.  Not in open-loop replay. */
int pa_fast_forward(pa_model* m, double duration_ms, int64_t n_long);

/* The epoch-kernel shape in use and, if the model was autotuned, the trial time
 * [ms] of each shape (cap entries of trial_ms; 0 for untried shapes). */
int pa_get_tuning(const pa_model* m, int32_t* shape, double* trial_ms, int32_t cap);

/* Launch counts and (with PA_FLAG_TIME_KERNELS) device times since the last
 * reset.  Synchronises the model's stream. */
int pa_get_kernel_stats(pa_model* m, pa_kernel_stats* out);
int pa_reset_kernel_stats(pa_model* m);

void pa_free_model(pa_model* m);

/* Batches of resident models (the paper has no counterpart: the serving path
 * of this engine, many simulation jobs advanced together).  A batch advances
 * every member by whole min-delay epochs (each member by its own epoch
 * length, at its own dt), each batch epoch ONE launch of the
 * time-step kernel over all members' cell groups (each block copies its
 * member's launch arguments and runs that member's groups exactly as the
 * member's own launch would), with each member's Poisson draws, routing,
 * spike record and epoch clock on parallel branches; the epochs are replayed
 * from CUDA graphs captured per membership (8 epochs per launch where they
 * fit).  Members never share state: every result equals the member's result
 * advanced alone, bit for bit.
 * Members must be on the batch's device (a member built on another stream
 * moves to the batch's stream when added, after its pending work, and stays
 * there), share precision and tree class (chains or branched), have no
 * wide-bin cells (build them with PA_FLAG_NARROW_ONLY), not be in open-loop replay, and be
 * at an epoch boundary when added and advanced.  A member may be removed
 * (and advanced alone, read, freed) between batch advances; remove it before
 * pa_free_model.  pa_batch_advance only enqueues work on the stream. */
typedef struct pa_batch pa_batch;
int pa_batch_create(int32_t device, void* stream, pa_batch** out);
int pa_batch_add(pa_batch* b, pa_model* m);
int pa_batch_remove(pa_batch* b, pa_model* m);
int pa_batch_advance(pa_batch* b, int64_t n_epochs);
/* out[0] members, out[1] blocks of the grouped launch, out[2] graph launches,
 * out[3] graphs captured (one per membership and epoch count in use) */
int pa_batch_info(const pa_batch* b, int64_t* out);
void pa_batch_free(pa_batch* b);

/* Self-check of the engine's integer FP64 arithmetic on GPU `device` (no model
 * needed; the paper has no counterpart).  The solver's row reciprocal 1/d is
 * computed from integer operations and a single-precision seed, and the mixed
 * path widens its FP32 synaptic sums to FP64 by moving bit fields; both must
 * equal the GPU's IEEE operations bit for bit.  Checks every single-precision
 * seed pattern (2^23 x 8 inputs), n_random random doubles and every float bit
 * pattern.  out[0] = reciprocal mismatches, out[1] = widening mismatches,
 * out[2] = cases checked, out[3] = bits of the first mismatching reciprocal
 * input (0 if none).  Synchronous; allocates 32 bytes of device memory. */
int pa_check_arith(int32_t device, uint64_t seed, int64_t n_random, int64_t* out);

/* Measures the GPU's FP64 fused multiply-add throughput (no model needed; the
 * paper has no counterpart; the roofline denominator of the FP64 pipe).  Runs
 * 8 x SMs blocks of 256 threads, each thread 8 independent chains of 16,384
 * FMAs, timed with CUDA events on the legacy default stream, best of five
 * after one warm-up.  out[0] = FMA operations per second (one FMA = 2 flop),
 * out[1] = the best run's milliseconds.  Synchronous; allocates 8 bytes of
 * device memory. */
int pa_measure_fp64(int32_t device, double* out);

const char* pa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
