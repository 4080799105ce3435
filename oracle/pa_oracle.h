/*
 * pa_oracle.h -- declarations of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This header, pa_oracle.c and the Python loader in
 * this folder exist so that the test-suite, the smoke check and the timed CPU
 * baseline of bench.py can compare the CUDA engine with a plain, slow,
 * obviously-correct simulator.  Nothing in the product path may include, link
 * or call anything declared here, and this file includes nothing from the
 * product (the two implementations share no code).
 *
 * The simulated method is the fixed-dt time-step loop of "Plastic Arbor"
 * (arXiv 2411.16445): the cable equation (Eq. cable), conductance-based
 * exponential synapses, Hodgkin-Huxley somata, and the spike-driven plasticity
 * rules of Sec. "Spike-timing-dependent plasticity" (Eqs. stdp_ode_1-3),
 * Sec. "Calcium-based synaptic plasticity" (Eqs. weight_graupner_brunel,
 * ca_model_graupner_brunel) and Sec. "Synaptic tagging and capture" (Eqs.
 * total_syn_weight .. prp_single_comp), with the POST_EVENT hook of
 * Sec. "Spike-time detection" and the two-target delivery of the
 * round_robin_halt policy of Sec. "Multiple postsynaptic variables".
 *
 * Units: mV, ms, um, nF, uS, nA.
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* mechanism kinds (numbering of the descriptor format) */
enum {
  ORC_MECH_PAS = 1,    /* params: g [S/cm2], e [mV]                                  */
  ORC_MECH_HH = 2,     /* params: gnabar, gkbar, gl [S/cm2], ena, ek, el [mV]         */
  ORC_MECH_EXPSYN = 10,/* params: tau [ms], e [mV]                                    */
  ORC_MECH_GB = 11,    /* params: tau, e, tau_c, c_pre, c_post, theta_p, theta_d,
                          gamma_p, gamma_d, tau_w [ms], w_star, t_c_delay [ms], w0
                          [, sigma_pl]                                              */
  ORC_MECH_STC = 12,   /* params: tau, e, tau_c, c_pre, c_post, theta_p, theta_d,
                          gamma_p, gamma_d, tau_h, tau_z, tau_p [ms], h0 [mV],
                          theta_tag [mV], theta_pro [mV], p_max, f_int, t_c_delay
                          [, sigma_pl [, D_p [um2/ms]]]; D_p > 0: the cell's PRP is
                          a concentration per CV that diffuses (Eq. diffusion)      */
  ORC_MECH_STDP = 13,  /* params: tau, e, tau_pre, tau_post, A_pre, A_post, w0, w_max */
  ORC_MECH_HCA = 14    /* heterosynaptic calcium (Eqs. ca_injection_current_spine,
                          ca_diffusion_dendrite, heterosyn_weight); params: I0 [pA],
                          tau_I [ms], gamma (Ca2+ fraction of the current), gamma_p,
                          gamma_d [1/s], theta_p, theta_d [umol/l], w0, tau_C [ms],
                          D [um2/ms]; no conductance */
};

/* per-connection synapse state fields readable with orc_get_syn (STDP traces:
   their value at the current step) */
enum {
  ORC_SYN_G = 0, ORC_SYN_C = 1, ORC_SYN_W = 2, ORC_SYN_H = 3, ORC_SYN_Z = 4,
  ORC_SYN_APRE = 5, ORC_SYN_APOST = 6, ORC_SYN_WEIGHT_TOTAL = 7
};

#define ORC_SRC_POISSON (-1)

typedef struct orc_model orc_model;

/* Builds a model from flat descriptor arrays (all caller-owned, copied).
 * Cells:  morph, soma_mech, dend_mech (indices into the mechanism table),
 *         cm [uF/cm2], ra [ohm cm], i_step [nA], t_on, t_off [ms] (t_off > 1e15:
 *         never off), v_init [mV], threshold [mV].
 * Morphologies: CV-level trees; morph_off[m] is the first CV of morphology m in
 *         parent/length/diam/region; parent[0] = -1 and parent[i] < i.
 * Mechanisms: kind and params[mech_off[j] ..].
 * Connections: src gid (ORC_SRC_POISSON for an independent Poisson train of
 *         rate conn_rate [Hz]), dst gid, dst CV, point-mechanism index, weight
 *         [uS], delay [ms].  Each connection creates one synapse.  conn_pid
 *         (may be NULL) names the Poisson train of a Poisson connection; a
 *         negative entry or a NULL array means "the connection's index".
 * Probes: membrane potential of CV probe_cv of cell probe_gid after each step.
 * Returns 0 or a negative error code; *out receives the model. */
int orc_build(int32_t n_cells, const int32_t* cell_morph, const int32_t* cell_soma_mech,
              const int32_t* cell_dend_mech, const double* cell_cm, const double* cell_ra,
              const double* cell_istep, const double* cell_ton, const double* cell_toff,
              const double* cell_vinit, const double* cell_thresh,
              int32_t n_morph, const int32_t* morph_ncv, const int32_t* morph_off,
              const int32_t* parent, const double* length_um, const double* diam_um,
              const int32_t* region,
              int32_t n_mech, const int32_t* mech_kind, const int32_t* mech_off,
              const double* mech_params, int64_t n_mech_params,
              int64_t n_conn, const int32_t* conn_src, const int32_t* conn_dst,
              const int32_t* conn_cv, const int32_t* conn_mech, const double* conn_weight,
              const double* conn_delay, const double* conn_rate, const int64_t* conn_pid,
              double dt, uint64_t seed, int32_t n_probe, const int32_t* probe_gid,
              const int32_t* probe_cv, orc_model** out);

/* Replaces the network's own spikes as the source of synaptic events and
 * POST_EVENT notifications (open-loop replay): gid[i] spiked in step step[i].
 * The cells still detect and record their own spikes. */
int orc_set_replay(orc_model* m, int64_t n, const int32_t* gid, const int64_t* step);
/* spikes of cells simulated elsewhere, in past steps whose events are still due */
int orc_inject_spikes(orc_model* m, int64_t n, const int32_t* gid, const int64_t* step);

int orc_run(orc_model* m, int64_t n_steps);
int64_t orc_step_count(const orc_model* m);
int64_t orc_n_spikes(const orc_model* m);
void orc_get_spikes(const orc_model* m, int32_t* gid, int64_t* step, double* t);
int64_t orc_n_cv(const orc_model* m);
void orc_get_v(const orc_model* m, double* out);           /* cell-major CV order */
int64_t orc_n_probe_samples(const orc_model* m);
void orc_get_probes(const orc_model* m, double* out);      /* [sample][probe] */
void orc_get_syn(const orc_model* m, int32_t field, double* out); /* connection order */
void orc_get_cell_p(const orc_model* m, double* out);      /* PRP per cell */
void orc_get_prp(const orc_model* m, double* out);  /* PRP per CV of diffusing cells, else 0 */
void orc_get_ca(const orc_model* m, double* out);   /* calcium per CV of HCA cells, else 0 */
void orc_set_ca(orc_model* m, const double* in);    /* per CV; other cells untouched */
void orc_set_prp(orc_model* m, const double* in);   /* per CV; cells without diffusion untouched */
int32_t orc_has_diffusion(const orc_model* m, int32_t cell);
void orc_get_gates(const orc_model* m, double* out);       /* m,h,n of each cell's CV 0 */
void orc_get_cv_geometry(const orc_model* m, double* cap_nF, double* gpas_uS,
                         double* a_uS);                    /* per CV, cell-major */
void orc_free(orc_model* m);
const char* orc_last_error(void);

/* unit-level entry points used by the pins */
double orc_exp(double x);
void orc_hh_rates(double v, double* am, double* bm, double* ah, double* bh, double* an,
                  double* bn);
int orc_hines_solve(int32_t n, const int32_t* parent, const double* d, const double* a,
                    const double* b, double* x);
void orc_threefry4x64_12(const uint64_t ctr[4], const uint64_t key[4], uint64_t out[4]);
uint32_t orc_poisson_u32(uint64_t seed, uint64_t stream, int64_t step);
/* Plasticity noise: the model's logarithm, cos/sin(2 pi v) (which = 0/1) and the
 * Box-Muller normal deviate of noise source `id` at step `step`. */
double orc_log(double x);
double orc_cis2pi(double v, int which);
double orc_normal(uint64_t seed, uint64_t id, int64_t step);
/* Fast-forward K steps with n_long long steps of the slow plasticity variables
 * (a diffusing PRP field: its explicit reaction and backward-Euler diffusion
 * with the long step).  -1 on bad arguments or in replay. */
int orc_fast_forward(orc_model* M, int64_t K, int64_t n_long);
void orc_set_syn(orc_model* M, int32_t field, const double* in);
void orc_set_v(orc_model* M, const double* in);
void orc_set_cell_p(orc_model* M, const double* in);
void orc_set_gates(orc_model* M, const double* in);

#ifdef __cplusplus
}
#endif
#endif
