/*
 * pa_oracle.c -- plain FP64 CPU oracle of the Plastic Arbor time-step loop.
 *
 * TEST INFRASTRUCTURE.  Used only by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py.  It shares no code, header, table
 * or constant generator with the CUDA engine; it is written to be read against
 * the paper (arXiv 2411.16445) line by line, not to be fast.
 *
 * What one step k (t_k = k*dt -> t_{k+1}) computes, in this order:
 *   1. events at t_k: synaptic pre events due at step k (spikes delivered after
 *      their integer delay), independent Poisson pre events, the delayed
 *      presynaptic calcium contributions (t_c,delay of Eqs.
 *      ca_model_graupner_brunel / ca_for_stc_model, the second target of the
 *      round_robin_halt policy), then the POST_EVENT hook for cells that spiked
 *      in step k-1 (Sec. "Spike-time detection to simplify computation").
 *   2. membrane currents at V^k, linearised into the matrix: every current here
 *      is linear in V for fixed gates/conductances, so i = g (V - E) enters as
 *      diagonal g and right-hand side g E.
 *   3. backward-Euler step of the cable equation (Eq. cable) on each cell's
 *      tree, solved by Hines elimination -> V^{k+1}.
 *   4. state updates: HH gates by exponential integration at V^{k+1}; synaptic
 *      conductance and calcium decay; forward-Euler steps of the plasticity
 *      ODEs (Eqs. weight_graupner_brunel, early_phase_weight,
 *      late_phase_weight, prp_single_comp) evaluated with the post-event state
 *      of step k.  The STDP traces (Eqs. stdp_ode_1-2) decay exponentially
 *      between spikes; they are kept as (value, step of the last jump) and
 *      evaluated in closed form, a(t_k) = a_last exp(-(k - k_last) dt / tau),
 *      when an event needs them.
 *   5. threshold detection at the soma CV: a spike in step k iff
 *      V^k < theta <= V^{k+1}.
 *
 * Readings where the paper is silent are listed in the repository's design
 * notes; the ones that fix arithmetic are repeated next to the code.
 * Parity: the HH channel kinetics are "parity unpinned" beyond the published
 * resting gate values, the textbook resting potential and the firing-rate
 * checks of the test-suite; every other
 * function here is pinned by a closed form, a brute-force or library solve, or
 * an invariant (tests/test_oracle_pins.py).
 */
#define _GNU_SOURCE
#include "pa_oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static __thread char g_err[512];
static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}
const char* orc_last_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* exp(x) used by the HH kinetics.  Both the oracle and the engine define the
 * model's exponential as this function so that FP64 results can agree to the
 * last bit (a reading: the paper fixes no exp).  Method: Cody-Waite argument
 * reduction x = k ln2 + r, |r| <= ln2/2, with ln2 split into a 32-bit head
 * (the double nearest ln2 with its low 21 mantissa bits cleared) and a tail,
 * then the degree-13 Taylor polynomial sum r^j/j! by Horner's rule with fused
 * multiply-adds, then scaling by 2^k.  Truncation error < r^14/14! < 5e-18. */
static const double kLn2Hi = 6.93147180369123816490e-01;  /* 0x1.62e42feep-1     */
static const double kLn2Lo = 1.9082149292705877e-10;      /* ln2 - kLn2Hi         */
static const double kInvLn2 = 1.4426950408889634;         /* nearest double 1/ln2 */
static const double kInvFact[14] = {
    1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
    0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05,
    2.7557319223985893e-06, 2.755731922398589e-07, 2.505210838544172e-08,
    2.08767569878681e-09, 1.6059043836821613e-10};

double orc_exp(double x) {
  if (x != x) return x;
  if (x > 709.0) return HUGE_VAL;
  if (x < -708.0) return 0.0;
  double kd = nearbyint(x * kInvLn2);
  double r = (x - kd * kLn2Hi) - kd * kLn2Lo;
  double p = kInvFact[13];
  for (int j = 12; j >= 0; --j) p = fma(p, r, kInvFact[j]);
  int64_t k = (int64_t)kd;
  uint64_t bits = (uint64_t)(k + 1023) << 52;
  double scale;
  memcpy(&scale, &bits, sizeof scale);
  return p * scale;
}

/* ------------------------------------------------------------------------ */
/* Hodgkin-Huxley rate functions (HodgkinHuxley1952, used on the soma of the
 * paper's simple-branchy cells): textbook form with resting potential -65 mV,
 * temperature factor 1 (6.3 C).  vtrap removes the 0/0 of alpha_m, alpha_n. */
static double vtrap(double x, double y) {
  double u = x / y;
  if (fabs(u) < 1e-6) return y * (1.0 - 0.5 * u);
  return x / (orc_exp(u) - 1.0);
}

void orc_hh_rates(double v, double* am, double* bm, double* ah, double* bh, double* an,
                  double* bn) {
  *am = 0.1 * vtrap(-(v + 40.0), 10.0);
  *bm = 4.0 * orc_exp(-(v + 65.0) / 18.0);
  *ah = 0.07 * orc_exp(-(v + 65.0) / 20.0);
  *bh = 1.0 / (orc_exp(-(v + 35.0) / 10.0) + 1.0);
  *an = 0.01 * vtrap(-(v + 55.0), 10.0);
  *bn = 0.125 * orc_exp(-(v + 65.0) / 80.0);
}

/* exponential (cnexp) integration of dx/dt = a (1 - x) - b x over dt */
static double cnexp_gate(double x, double a, double b, double dt) {
  double s = a + b;
  double xinf = a / s;
  return xinf + (x - xinf) * orc_exp(-dt * s);
}

/* ------------------------------------------------------------------------ */
/* Hines elimination for a tree with parent[i] < i (textbook; Hines 1984):
 * for i = n-1 .. 1:  r_i = 1/d_i, f_i = a_i r_i, x'_i = b_i r_i,
 *                    d_p -= f_i a_i,  b_p -= a_i x'_i     (p = parent[i])
 * then x_0 = b_0 / d_0 and, for i = 1 .. n-1, x_i = x'_i - f_i x_{p}.
 * a_i is the (symmetric) off-diagonal entry between i and parent[i].
 * d and b are modified in place; f and xp are scratch of length n. */
static void hines(int64_t n, const int32_t* parent, double* d, const double* a, double* b,
                  double* f, double* xp, double* x) {
  for (int64_t i = n - 1; i >= 1; --i) {
    int32_t p = parent[i];
    double r = 1.0 / d[i];
    f[i] = a[i] * r;
    xp[i] = b[i] * r;
    d[p] = fma(-f[i], a[i], d[p]);
    b[p] = fma(-a[i], xp[i], b[p]);
  }
  x[0] = b[0] * (1.0 / d[0]);
  for (int64_t i = 1; i < n; ++i) x[i] = fma(-f[i], x[parent[i]], xp[i]);
}

int orc_hines_solve(int32_t n, const int32_t* parent, const double* d, const double* a,
                    const double* b, double* x) {
  if (n <= 0) return -1;
  double* dd = (double*)malloc(sizeof(double) * 4 * (size_t)n);
  if (!dd) return -2;
  double* bb = dd + n;
  double* f = bb + n;
  double* xp = f + n;
  memcpy(dd, d, sizeof(double) * n);
  memcpy(bb, b, sizeof(double) * n);
  hines(n, parent, dd, a, bb, f, xp, x);
  free(dd);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Threefry-4x64-12 counter-based generator (Salmon et al. 2011, the generator
 * named in Sec. "Computation with stochastic differential equations"):
 * Threefish-256 rotation schedule, key parity constant 0x1BD11BDAA9FC1A22,
 * key injection after every fourth round.  Used here for Poisson drive. */
static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

void orc_threefry4x64_12(const uint64_t ctr[4], const uint64_t key[4], uint64_t out[4]) {
  static const int rot[8][2] = {{14, 16}, {52, 57}, {23, 40}, {5, 37},
                                {25, 33}, {46, 12}, {58, 22}, {32, 32}};
  uint64_t ks[5];
  ks[4] = 0x1BD11BDAA9FC1A22ULL;
  for (int i = 0; i < 4; ++i) {
    ks[i] = key[i];
    ks[4] ^= key[i];
  }
  uint64_t x0 = ctr[0] + ks[0], x1 = ctr[1] + ks[1], x2 = ctr[2] + ks[2], x3 = ctr[3] + ks[3];
  for (int r = 0; r < 12; ++r) {
    const int* rc = rot[r % 8];
    if ((r & 1) == 0) {
      x0 += x1; x1 = rotl64(x1, rc[0]); x1 ^= x0;
      x2 += x3; x3 = rotl64(x3, rc[1]); x3 ^= x2;
    } else {
      x0 += x3; x3 = rotl64(x3, rc[0]); x3 ^= x0;
      x2 += x1; x1 = rotl64(x1, rc[1]); x1 ^= x2;
    }
    if ((r & 3) == 3) {
      int s = (r >> 2) + 1;
      x0 += ks[s % 5];
      x1 += ks[(s + 1) % 5];
      x2 += ks[(s + 2) % 5];
      x3 += ks[(s + 3) % 5] + (uint64_t)s;
    }
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform 32-bit word for Poisson stream `stream` at step `step`: one
 * Threefry call (key = seed, counter = {stream, step/8, 1, 0}) serves eight
 * consecutive steps; word j = step mod 8 is 32-bit half (j mod 2) of output
 * word j/2, low half first. */
uint32_t orc_poisson_u32(uint64_t seed, uint64_t stream, int64_t step) {
  uint64_t key[4] = {seed, 0, 0, 0};
  uint64_t ctr[4] = {stream, (uint64_t)step >> 3, 1, 0};
  uint64_t out[4];
  orc_threefry4x64_12(ctr, key, out);
  int j = (int)(step & 7);
  uint64_t w = out[j >> 1];
  return (j & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
}

/* ------------------------------------------------------------------------ */
/* Plasticity noise (Eqs. plasticity_noise_1, plasticity_noise_2; Sec.
 * "Computation with stochastic differential equations"): Euler-Maruyama with
 * Delta W = sqrt(dt) N(0,1), the normal deviates by the Box-Muller method from
 * Threefry-4x64-12 uniforms.  The model defines its own logarithm and circular
 * functions (below) so that the deviates are reproducible to the last bit. */

/* Natural logarithm of x > 0 (normal): x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(s), s = (m - 1)/(m + 1), by the odd series
 * s + s^3/3 + ... + s^23/23 in Horner form with fused multiply-adds (|s| < 0.172,
 * so the first omitted term is below 2^-60 relative); e ln2 is added with ln2
 * split into the exponential's 32-bit head and tail.  The coefficients are
 * 1/k rounded to double. */
double orc_log(double x) {
  static const double c[12] = {0.043478260869565216, 0.047619047619047616, 0.05263157894736842,
                               0.058823529411764705, 0.06666666666666667, 0.07692307692307693,
                               0.09090909090909091, 0.1111111111111111, 0.14285714285714285,
                               0.2, 0.3333333333333333, 1.0};
  uint64_t b;
  memcpy(&b, &x, 8);
  int e = (int)((b >> 52) & 0x7ff) - 1022;
  b = (b & 0x800fffffffffffffULL) | (1022ULL << 52); /* m in [0.5, 1) */
  double m;
  memcpy(&m, &b, 8);
  if (m < 0.70710678118654752440) {
    m = m * 2.0;
    e = e - 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double s2 = s * s;
  double p = c[0];
  for (int i = 1; i < 12; ++i) p = fma(p, s2, c[i]);
  double t = s * p;
  double lm = t + t;
  double ed = (double)e;
  double hi = ed * 6.93147180369123816490e-01;
  return hi + fma(ed, 1.9082149292705877e-10, lm);
}

/* cos(2 pi v) (which = 0) or sin(2 pi v) (which = 1) for v in [0, 1): the
 * quadrant q = rint(4v) and the remainder r = v - q/4 (|r| <= 1/8) are exact
 * in binary; t = 2 pi r by one rounded product; the Taylor series of sin t
 * (to t^21) and cos t (to t^22) in Horner form with fused multiply-adds
 * (|t| <= pi/4); coefficients (-1)^k / n! rounded to double. */
double orc_cis2pi(double v, int which) {
  static const double sc[10] = {1.9572941063391263e-20, -8.22063524662433e-18,
                                2.8114572543455206e-15, -7.647163731819816e-13,
                                1.6059043836821613e-10, -2.505210838544172e-08,
                                2.7557319223985893e-06, -0.0001984126984126984,
                                0.008333333333333333, -0.16666666666666666};
  static const double cc[11] = {-8.896791392450574e-22, 4.110317623312165e-19,
                                -1.5619206968586225e-16, 4.779477332387385e-14,
                                -1.1470745597729725e-11, 2.08767569878681e-09,
                                -2.755731922398589e-07, 2.48015873015873e-05,
                                -0.001388888888888889, 0.041666666666666664, -0.5};
  double q = rint(4.0 * v);
  double r = v - 0.25 * q;
  double t = r * 6.283185307179586;
  double t2 = t * t;
  int quad = ((int)q) & 3;
  /* sin(t + quad pi/2) and cos(t + quad pi/2) from sin t and cos t */
  int want_sin = which ? (quad == 0 || quad == 2) : (quad == 1 || quad == 3);
  double val;
  if (want_sin) {
    double sp = sc[0];
    for (int i = 1; i < 10; ++i) sp = fma(sp, t2, sc[i]);
    val = fma(sp * t2, t, t);
  } else {
    double cp = cc[0];
    for (int i = 1; i < 11; ++i) cp = fma(cp, t2, cc[i]);
    val = fma(cp, t2, 1.0);
  }
  /* signs: cos: +cos, -sin, -cos, +sin; sin: +sin, +cos, -sin, -cos */
  int neg = which ? (quad >= 2) : (quad == 1 || quad == 2);
  return neg ? -val : val;
}

/* The normal deviate of noise source `id` at step `step`: one Threefry call
 * (key = seed, counter = {id, step/4, 2, 0}) serves four consecutive steps;
 * step mod 4 = 2p + j takes the Box-Muller pair of words 2p and 2p+1 (53-bit
 * uniforms u1, u2 in [0, 1)): sqrt(-2 log(1 - u1)) times cos (j = 0) or
 * sin (j = 1) of 2 pi u2. */
double orc_normal(uint64_t seed, uint64_t id, int64_t step) {
  uint64_t key[4] = {seed, 0, 0, 0};
  uint64_t ctr[4] = {id, (uint64_t)step >> 2, 2, 0};
  uint64_t out[4];
  orc_threefry4x64_12(ctr, key, out);
  int j = (int)(step & 3);
  double u1 = (double)(out[j & 2] >> 11) * 0x1p-53;
  double u2 = (double)(out[(j & 2) + 1] >> 11) * 0x1p-53;
  double rad = sqrt(-2.0 * orc_log(1.0 - u1));
  return rad * orc_cis2pi(u2, j & 1);
}

/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t syn;
  int32_t type; /* 0: pre (conductance) event, 1: delayed calcium event */
} orc_ev;
typedef struct {
  orc_ev* v;
  int64_t n, cap;
} orc_bucket;

typedef struct {
  int32_t kind;
  double p[20];
  /* derived per-dt constants */
  double decay_g, decay_c;
  double rate_w, rate_h, rate_z, rate_p;
  int64_t dc_steps;
  double sigma;   /* sigma_pl (GB, STC) */
  double diff_d;  /* STC: PRP diffusivity D_p [um2/ms] (0: one pool per cell) */
  double amp[3];  /* Euler-Maruyama noise amplitude with n of the two thresholds crossed:
                     sigma_pl sqrt(n dt / tau) for tau = tau_w (GB) or tau_h (STC) */
  /* HCA: calcium inflow per pA of injection current, gamma 1e6 / (2 F)
     [umol/l um3 / (ms pA)]; dt gamma_p, dt gamma_d per step; dt / tau_C */
  double kq, rate_gp, rate_gd, rate_ca;
} orc_mech;

struct orc_model {
  double dt;
  uint64_t seed;
  int64_t step;
  int32_t n_cells;
  int64_t n_cv;
  int64_t* cv_off;
  int32_t* parent; /* cell-local */
  double *cap, *cdt, *gax, *a, *gpas, *em_pas;
  int32_t* cv_mech; /* mechanism index of the CV's density mechanism */
  double *gna_a, *gk_a, *gl_a;
  double *V, *m, *h, *n;
  double *gs, *es, *d, *b, *f, *xp, *xnew;
  /* PRP diffusion (cells whose STC mechanism has D_p > 0): CV volume [um3],
     diffusive half-length (L/2)/(pi r^2) [1/um], PRP concentration, the
     constant backward-Euler matrix (diagonal, coupling to the parent), V/dt */
  double *vol, *hx, *prp_cv, *prp_d, *prp_a, *prp_vdt, *vtot, *prp_src, *prp_gsum;
  int32_t* has_diff;
  /* heterosynaptic calcium (cells with HCA synapses): concentration per CV
     [umol/l], its backward-Euler matrix, V/dt, the step's inflow per CV */
  double *ca_cv, *ca_d, *ca_a, *ca_vdt, *ca_src;
  int32_t *has_ca, *cell_hca_mech;
  double* istep;
  int64_t *k_on, *k_off;
  double *thresh, *p;
  int32_t *spiked_prev, *spk_flag, *cell_stc_mech;
  double* spk_t;
  int32_t n_mech;
  orc_mech* mech;
  int64_t n_syn;
  int32_t *syn_cell, *syn_mech, *syn_src;
  int64_t* syn_cv; /* global CV index */
  double* syn_weight;
  int64_t* syn_D;
  uint64_t* syn_pid; /* Poisson train of the synapse */
  uint32_t* syn_thr;
  double *g, *c, *w, *hs, *z, *apre, *apost;
  int64_t *apre_k, *apost_k; /* step of the traces' last jump */
  int64_t *cell_syn_off, *cell_syn;
  int64_t *out_off, *out_syn;
  int64_t *poisson_syn, n_poisson;
  int64_t R;
  orc_bucket* q;
  int64_t n_spk, cap_spk;
  int32_t* spk_gid;
  int64_t* spk_step;
  double* spk_time;
  int32_t n_probe;
  int64_t* probe_cv;
  double* probes;
  int64_t n_samples, cap_samples;
  int replay;
  int64_t n_rep, rep_pos;
  int32_t* rep_gid;
  int64_t* rep_step;
};

static int is_point(int32_t k) {
  return k == ORC_MECH_EXPSYN || k == ORC_MECH_GB || k == ORC_MECH_STC || k == ORC_MECH_STDP ||
         k == ORC_MECH_HCA;
}
static int n_params_of(int32_t k) {
  switch (k) {
    case ORC_MECH_PAS: return 2;
    case ORC_MECH_HH: return 6;
    case ORC_MECH_EXPSYN: return 2;
    case ORC_MECH_GB: return 13;
    case ORC_MECH_STC: return 18;
    case ORC_MECH_STDP: return 8;
    case ORC_MECH_HCA: return 10;
  }
  return -1;
}
/* GB and STC take an optional trailing sigma_pl (the noise scale; 0 if absent) */
/* GB and STC take an optional trailing sigma_pl; STC then an optional PRP
 * diffusivity D_p [um2/ms] (Eq. diffusion; 0 or absent: one PRP pool per cell) */
static int accepts_params(int32_t k, int32_t n) {
  int np = n_params_of(k);
  return n == np || ((k == ORC_MECH_GB || k == ORC_MECH_STC) && n == np + 1) ||
         (k == ORC_MECH_STC && n == np + 2);
}

static void push_ev(orc_bucket* bk, int32_t syn, int32_t type) {
  if (bk->n == bk->cap) {
    bk->cap = bk->cap ? 2 * bk->cap : 64;
    bk->v = (orc_ev*)realloc(bk->v, sizeof(orc_ev) * (size_t)bk->cap);
  }
  bk->v[bk->n].syn = syn;
  bk->v[bk->n].type = type;
  bk->n++;
}

#define ALLOC(ptr, n) ((ptr) = calloc((size_t)((n) > 0 ? (n) : 1), sizeof(*(ptr))))

static orc_model* g_sort_model;
static int cmp_syn(const void* x, const void* y) {
  int64_t i = *(const int64_t*)x, j = *(const int64_t*)y;
  const orc_model* M = g_sort_model;
  if (M->syn_mech[i] != M->syn_mech[j]) return M->syn_mech[i] < M->syn_mech[j] ? -1 : 1;
  if (M->syn_cv[i] != M->syn_cv[j]) return M->syn_cv[i] < M->syn_cv[j] ? -1 : 1;
  return i < j ? -1 : (i > j);
}

void orc_free(orc_model* M) {
  if (!M) return;
  void* ptrs[] = {M->cv_off, M->parent, M->cap, M->cdt, M->gax, M->a, M->gpas, M->em_pas,
                  M->cv_mech, M->gna_a, M->gk_a, M->gl_a, M->V, M->m, M->h, M->n, M->gs,
                  M->es, M->d, M->b, M->f, M->xp, M->xnew, M->istep, M->k_on, M->k_off,
                  M->thresh, M->p, M->spiked_prev, M->spk_flag, M->cell_stc_mech, M->spk_t,
                  M->mech, M->syn_cell, M->syn_mech, M->syn_src, M->syn_cv, M->syn_weight,
                  M->syn_D, M->syn_pid, M->syn_thr, M->g, M->c, M->w, M->hs, M->z, M->apre, M->apost, M->apre_k, M->apost_k,
                  M->cell_syn_off, M->cell_syn, M->out_off, M->out_syn, M->poisson_syn,
                  M->spk_gid, M->spk_step, M->spk_time, M->probe_cv, M->probes, M->rep_gid,
                  M->rep_step, M->vol, M->hx, M->prp_cv, M->prp_d, M->prp_a, M->prp_vdt,
                  M->vtot, M->prp_src, M->prp_gsum, M->has_diff, M->ca_cv, M->ca_d,
                  M->ca_a, M->ca_vdt, M->ca_src, M->has_ca, M->cell_hca_mech};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
  if (M->q) {
    for (int64_t i = 0; i < M->R; ++i) free(M->q[i].v);
    free(M->q);
  }
  free(M);
}

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
              const int32_t* probe_cv, orc_model** out) {
  *out = NULL;
  if (!(dt > 0)) return fail(-1, "dt must be positive");
  if (n_cells < 0 || n_morph < 0 || n_mech < 0 || n_conn < 0)
    return fail(-1, "negative count");
  orc_model* M = (orc_model*)calloc(1, sizeof *M);
  M->dt = dt;
  M->seed = seed;
  M->n_cells = n_cells;
  M->n_mech = n_mech;
  ALLOC(M->mech, n_mech);
  for (int32_t j = 0; j < n_mech; ++j) {
    int np = n_params_of(mech_kind[j]);
    if (np < 0) { orc_free(M); return fail(-1, "mechanism %d: unknown kind %d", j, mech_kind[j]); }
    int64_t given = (j + 1 < n_mech ? (int64_t)mech_off[j + 1] : n_mech_params) - mech_off[j];
    if (!accepts_params(mech_kind[j], (int32_t)given)) {
      orc_free(M); return fail(-1, "mechanism %d: %lld parameters", j, (long long)given);
    }
    orc_mech* mc = &M->mech[j];
    mc->kind = mech_kind[j];
    for (int i = 0; i < given; ++i) mc->p[i] = mech_params[mech_off[j] + i];
    mc->sigma = (given > np) ? mc->p[np] : 0.0;
    mc->diff_d = (given > np + 1) ? mc->p[np + 1] : 0.0;
    if (!(mc->diff_d >= 0.0)) { orc_free(M); return fail(-1, "mechanism %d: D_p < 0", j); }
    if (!(mc->sigma >= 0.0)) { orc_free(M); return fail(-1, "mechanism %d: sigma_pl < 0", j); }
    for (int n = 0; n < 3; ++n)
      mc->amp[n] = (given > np) ? mc->sigma * sqrt(((double)n * dt) / mc->p[9]) : 0.0;
    /* per-dt constants: exact exponential decay of the linear ODEs
       (g' = -g/tau, c' = -c/tau_c, a' = -a/tau) and forward-Euler rates */
    if (is_point(mc->kind) && mc->kind != ORC_MECH_HCA) mc->decay_g = exp(-dt / mc->p[0]);
    if (mc->kind == ORC_MECH_HCA) {
      /* Eq. ca_injection_current_spine decays with tau_I; the current's
         calcium (valence 2, Faraday constant 96485.33212 C/mol) in
         umol/l um3 per ms and pA; rates of Eq. heterosyn_weight per second */
      mc->decay_g = 1.0;
      mc->decay_c = exp(-dt / mc->p[1]);
      mc->kq = (mc->p[2] * 1e6) / (2.0 * 96485.33212);
      mc->rate_gp = (dt * mc->p[3]) * 1e-3;
      mc->rate_gd = (dt * mc->p[4]) * 1e-3;
      mc->rate_ca = dt / mc->p[8];
      if (!(mc->p[1] > 0) || !(mc->p[8] > 0) || !(mc->p[9] >= 0)) {
        orc_free(M); return fail(-1, "mechanism %d: tau_I, tau_C > 0 and D >= 0 required", j);
      }
    }
    if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC) {
      mc->decay_c = exp(-dt / mc->p[2]);
      double tcd = mc->kind == ORC_MECH_GB ? mc->p[11] : mc->p[17];
      mc->dc_steps = llround(tcd / dt);
      if (mc->dc_steps < 0) { orc_free(M); return fail(-1, "negative t_c_delay"); }
    }
    if (mc->kind == ORC_MECH_GB) mc->rate_w = dt / mc->p[9];
    if (mc->kind == ORC_MECH_STC) {
      mc->rate_h = dt / mc->p[9];
      mc->rate_z = dt / mc->p[10];
      mc->rate_p = dt / mc->p[11];
    }

  }
  /* CV layout: cell-major */
  ALLOC(M->cv_off, n_cells + 1);
  for (int32_t c = 0; c < n_cells; ++c) {
    int32_t mo = cell_morph[c];
    if (mo < 0 || mo >= n_morph) { orc_free(M); return fail(-1, "cell %d: bad morphology", c); }
    if (morph_ncv[mo] < 1) { orc_free(M); return fail(-1, "morphology %d: no CV", mo); }
    M->cv_off[c + 1] = M->cv_off[c] + morph_ncv[mo];
  }
  int64_t N = M->n_cv = M->cv_off[n_cells];
  ALLOC(M->parent, N); ALLOC(M->cap, N); ALLOC(M->cdt, N); ALLOC(M->gax, N);
  ALLOC(M->a, N); ALLOC(M->gpas, N); ALLOC(M->em_pas, N); ALLOC(M->cv_mech, N);
  ALLOC(M->gna_a, N); ALLOC(M->gk_a, N); ALLOC(M->gl_a, N);
  ALLOC(M->V, N); ALLOC(M->m, N); ALLOC(M->h, N); ALLOC(M->n, N);
  ALLOC(M->gs, N); ALLOC(M->es, N); ALLOC(M->d, N); ALLOC(M->b, N);
  ALLOC(M->f, N); ALLOC(M->xp, N); ALLOC(M->xnew, N);
  ALLOC(M->vol, N); ALLOC(M->hx, N); ALLOC(M->prp_cv, N); ALLOC(M->prp_d, N);
  ALLOC(M->prp_a, N); ALLOC(M->prp_vdt, N); ALLOC(M->vtot, n_cells); ALLOC(M->has_diff, n_cells);
  ALLOC(M->prp_src, n_cells); ALLOC(M->prp_gsum, N);
  ALLOC(M->ca_cv, N); ALLOC(M->ca_d, N); ALLOC(M->ca_a, N); ALLOC(M->ca_vdt, N);
  ALLOC(M->ca_src, N); ALLOC(M->has_ca, n_cells); ALLOC(M->cell_hca_mech, n_cells);
  ALLOC(M->istep, n_cells); ALLOC(M->k_on, n_cells); ALLOC(M->k_off, n_cells);
  ALLOC(M->thresh, n_cells); ALLOC(M->p, n_cells); ALLOC(M->spiked_prev, n_cells);
  ALLOC(M->spk_flag, n_cells); ALLOC(M->spk_t, n_cells); ALLOC(M->cell_stc_mech, n_cells);
  double* rhalf = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  for (int32_t c = 0; c < n_cells; ++c) {
    int32_t mo = cell_morph[c];
    int64_t n = morph_ncv[mo], base = M->cv_off[c], mb = morph_off[mo];
    int32_t ms = cell_soma_mech[c], md = cell_dend_mech[c];
    if (ms < 0 || ms >= n_mech || md < 0 || md >= n_mech ||
        (M->mech[ms].kind != ORC_MECH_PAS && M->mech[ms].kind != ORC_MECH_HH) ||
        (M->mech[md].kind != ORC_MECH_PAS && M->mech[md].kind != ORC_MECH_HH)) {
      free(rhalf); orc_free(M);
      return fail(-1, "cell %d: soma/dendrite mechanism must be pas or hh", c);
    }
    double cm = cell_cm[c], ra = cell_ra[c];
    for (int64_t i = 0; i < n; ++i) {
      int32_t pi = parent[mb + i];
      if ((i == 0 && pi != -1) || (i > 0 && (pi < 0 || pi >= i))) {
        free(rhalf); orc_free(M);
        return fail(-1, "morphology %d: parent[%lld] invalid", mo, (long long)i);
      }
      double L = length_um[mb + i], dia = diam_um[mb + i];
      if (!(L > 0) || !(dia > 0)) {
        free(rhalf); orc_free(M);
        return fail(-1, "morphology %d: non-positive length/diameter", mo);
      }
      /* a CV is a cylinder; area pi d L [um2]; C = cm A 1e-5 [nF];
         half-cylinder axial resistance Ra (L/2) / (pi r^2) 1e-2 [Mohm] */
      double r = 0.5 * dia;
      double A = (M_PI * dia) * L;
      M->parent[base + i] = pi;
      M->cap[base + i] = (cm * A) * 1e-5;
      M->cdt[base + i] = M->cap[base + i] / dt;
      rhalf[base + i] = ((ra * (0.5 * L)) / (M_PI * (r * r))) * 1e-2;
      M->vol[base + i] = (M_PI * (r * r)) * L;
      M->hx[base + i] = (0.5 * L) / (M_PI * (r * r));
      int32_t mj = region[mb + i] == 0 ? ms : md;
      M->cv_mech[base + i] = mj;
      const orc_mech* mc = &M->mech[mj];
      if (mc->kind == ORC_MECH_PAS) {
        M->gpas[base + i] = (mc->p[0] * A) * 1e-2; /* S/cm2 * um2 -> uS */
        M->em_pas[base + i] = M->gpas[base + i] * mc->p[1];
      } else {
        M->gna_a[base + i] = (mc->p[0] * A) * 1e-2;
        M->gk_a[base + i] = (mc->p[1] * A) * 1e-2;
        M->gl_a[base + i] = (mc->p[2] * A) * 1e-2;
      }
    }
    /* axial conductances: two half-cylinders in series between i and parent */
    for (int64_t i = 1; i < n; ++i) {
      int64_t p = base + M->parent[base + i];
      double gi = 1.0 / (rhalf[base + i] + rhalf[p]);
      M->a[base + i] = -gi;
      M->gax[base + i] += gi;
      M->gax[p] += gi;
    }
    double v0 = cell_vinit[c];
    for (int64_t i = 0; i < n; ++i) {
      M->V[base + i] = v0;
      if (M->mech[M->cv_mech[base + i]].kind == ORC_MECH_HH) {
        double am, bm, ah, bh, an, bn;
        orc_hh_rates(v0, &am, &bm, &ah, &bh, &an, &bn);
        M->m[base + i] = am / (am + bm);
        M->h[base + i] = ah / (ah + bh);
        M->n[base + i] = an / (an + bn);
      }
    }
    M->istep[c] = cell_istep[c];
    M->k_on[c] = llround(cell_ton[c] / dt);
    M->k_off[c] = cell_toff[c] > 1e15 ? INT64_MAX : llround(cell_toff[c] / dt);
    M->thresh[c] = cell_thresh[c];
    M->cell_stc_mech[c] = -1;
    M->cell_hca_mech[c] = -1;
  }
  free(rhalf);
  /* synapses, one per connection, in connection order */
  M->n_syn = n_conn;
  ALLOC(M->syn_cell, n_conn); ALLOC(M->syn_mech, n_conn); ALLOC(M->syn_src, n_conn);
  ALLOC(M->syn_cv, n_conn); ALLOC(M->syn_weight, n_conn); ALLOC(M->syn_D, n_conn);
  ALLOC(M->syn_thr, n_conn); ALLOC(M->syn_pid, n_conn); ALLOC(M->g, n_conn); ALLOC(M->c, n_conn); ALLOC(M->w, n_conn);
  ALLOC(M->hs, n_conn); ALLOC(M->z, n_conn); ALLOC(M->apre, n_conn); ALLOC(M->apost, n_conn);
  ALLOC(M->apre_k, n_conn); ALLOC(M->apost_k, n_conn);
  ALLOC(M->poisson_syn, n_conn);
  int64_t maxdelay = 1;
  ALLOC(M->out_off, n_cells + 1);
  for (int64_t s = 0; s < n_conn; ++s) {
    int32_t dst = conn_dst[s], mj = conn_mech[s], src = conn_src[s];
    if (dst < 0 || dst >= n_cells) { orc_free(M); return fail(-1, "connection %lld: bad dst", (long long)s); }
    int64_t ncv = M->cv_off[dst + 1] - M->cv_off[dst];
    if (conn_cv[s] < 0 || conn_cv[s] >= ncv) { orc_free(M); return fail(-1, "connection %lld: bad cv", (long long)s); }
    if (mj < 0 || mj >= n_mech || !is_point(M->mech[mj].kind)) {
      orc_free(M); return fail(-1, "connection %lld: mechanism must be a synapse", (long long)s);
    }
    const orc_mech* mc = &M->mech[mj];
    M->syn_cell[s] = dst;
    M->syn_mech[s] = mj;
    M->syn_src[s] = src;
    M->syn_cv[s] = M->cv_off[dst] + conn_cv[s];
    M->syn_weight[s] = conn_weight[s];
    if (src == ORC_SRC_POISSON) {
      double x = ((conn_rate[s] * dt) * 1e-3) * 4294967296.0;
      if (!(x >= 0) || x >= 4294967296.0) { orc_free(M); return fail(-1, "connection %lld: rate*dt out of range", (long long)s); }
      M->syn_thr[s] = (uint32_t)floor(x);
      M->syn_pid[s] = (conn_pid && conn_pid[s] >= 0) ? (uint64_t)conn_pid[s] : (uint64_t)s;
      M->syn_D[s] = 0;
      M->poisson_syn[M->n_poisson++] = s;
    } else {
      if (src < 0 || src >= n_cells) { orc_free(M); return fail(-1, "connection %lld: bad src", (long long)s); }
      M->syn_D[s] = llround(conn_delay[s] / dt);
      if (M->syn_D[s] < 1) { orc_free(M); return fail(-1, "connection %lld: delay below one step", (long long)s); }
      M->out_off[src + 1]++;
    }
    int64_t tot = M->syn_D[s] + ((mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC) ? mc->dc_steps : 0);
    if (tot > maxdelay) maxdelay = tot;
    /* initial synapse state (readings): GB w = w0; STC h = h0, z = 0, p = 0;
       STDP w = w0; all conductances, calcium and traces start at zero */
    if (mc->kind == ORC_MECH_GB) M->w[s] = mc->p[12];
    if (mc->kind == ORC_MECH_STC) {
      M->hs[s] = mc->p[12];
      if (M->cell_stc_mech[dst] >= 0 && M->cell_stc_mech[dst] != mj) {
        orc_free(M); return fail(-1, "cell %d: STC synapses must share one mechanism", dst);
      }
      M->cell_stc_mech[dst] = mj;
    }
    if (mc->kind == ORC_MECH_STDP) M->w[s] = mc->p[6];
    if (mc->kind == ORC_MECH_HCA) {
      M->w[s] = mc->p[7];
      if (M->cell_hca_mech[dst] >= 0 && M->cell_hca_mech[dst] != mj) {
        orc_free(M); return fail(-1, "cell %d: HCA synapses must share one mechanism", dst);
      }
      M->cell_hca_mech[dst] = mj;
    }
  }
  for (int32_t c = 0; c < n_cells; ++c) M->out_off[c + 1] += M->out_off[c];
  ALLOC(M->out_syn, M->out_off[n_cells]);
  {
    int64_t* fill = (int64_t*)calloc((size_t)n_cells + 1, sizeof(int64_t));
    for (int64_t s = 0; s < n_conn; ++s) {
      if (conn_src[s] == ORC_SRC_POISSON) continue;
      int32_t src = conn_src[s];
      M->out_syn[M->out_off[src] + fill[src]++] = s;
    }
    free(fill);
  }
  /* canonical synapse order of each cell: (mechanism, CV, connection) */
  ALLOC(M->cell_syn_off, n_cells + 1);
  for (int64_t s = 0; s < n_conn; ++s) M->cell_syn_off[M->syn_cell[s] + 1]++;
  for (int32_t c = 0; c < n_cells; ++c) M->cell_syn_off[c + 1] += M->cell_syn_off[c];
  ALLOC(M->cell_syn, n_conn);
  {
    int64_t* fill = (int64_t*)calloc((size_t)n_cells + 1, sizeof(int64_t));
    for (int64_t s = 0; s < n_conn; ++s) {
      int32_t c = M->syn_cell[s];
      M->cell_syn[M->cell_syn_off[c] + fill[c]++] = s;
    }
    free(fill);
  }
  g_sort_model = M;
  for (int32_t c = 0; c < n_cells; ++c)
    qsort(M->cell_syn + M->cell_syn_off[c], (size_t)(M->cell_syn_off[c + 1] - M->cell_syn_off[c]),
          sizeof(int64_t), cmp_syn);
  M->R = maxdelay + 2;
  M->q = (orc_bucket*)calloc((size_t)M->R, sizeof(orc_bucket));
  /* PRP diffusion (Eq. diffusion with the cable equation's solver): the
     diffusion part by backward Euler on the cell's tree,
     V_i (P_i^{k+1} - P*_i)/dt = sum_j gD_ij (P_j^{k+1} - P_i^{k+1}), with gD of
     two half-cylinders in series, D / ((L_i/2)/(pi r_i^2) + (L_p/2)/(pi r_p^2))
     [um3/ms]; the matrix is constant: diagonal V_i/dt + sum gD, coupling -gD. */
  for (int32_t c = 0; c < n_cells; ++c) {
    int32_t mj = M->cell_stc_mech[c];
    if (mj < 0 || !(M->mech[mj].diff_d > 0.0)) continue;
    const double D = M->mech[mj].diff_d;
    int64_t base = M->cv_off[c], n = M->cv_off[c + 1] - base;
    for (int64_t i = 0; i < n; ++i) M->xnew[base + i] = 0.0; /* summed couplings */
    for (int64_t i = 1; i < n; ++i) {
      int64_t p = base + M->parent[base + i];
      double gd = D / (M->hx[base + i] + M->hx[p]);
      M->prp_a[base + i] = -gd;
      M->xnew[base + i] += gd;
      M->xnew[p] += gd;
    }
    double vt = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double v = M->vol[base + i];
      M->prp_vdt[base + i] = v / dt;
      M->prp_gsum[base + i] = M->xnew[base + i];
      M->prp_d[base + i] = (v / dt) + M->xnew[base + i];
      vt = vt + v;
    }
    M->vtot[c] = vt;
    /* synthesis enters the soma CV at p_max V_tot / (V_0 tau_p): the cell's
       total amount then follows the single pool's equation for the mean
       concentration (Eq. prp_single_comp) */
    M->prp_src[c] = vt / M->vol[base];
    M->has_diff[c] = 1;
  }
  /* heterosynaptic calcium: the same backward-Euler diffusion on the cell's
     tree (Eq. ca_diffusion_dendrite), with the mechanism's D */
  for (int32_t c = 0; c < n_cells; ++c) {
    int32_t mj = M->cell_hca_mech[c];
    if (mj < 0) continue;
    const double D = M->mech[mj].p[9];
    int64_t base = M->cv_off[c], n = M->cv_off[c + 1] - base;
    for (int64_t i = 0; i < n; ++i) M->xnew[base + i] = 0.0;
    for (int64_t i = 1; i < n; ++i) {
      int64_t p = base + M->parent[base + i];
      double gd = D / (M->hx[base + i] + M->hx[p]);
      M->ca_a[base + i] = -gd;
      M->xnew[base + i] += gd;
      M->xnew[p] += gd;
    }
    for (int64_t i = 0; i < n; ++i) {
      double v = M->vol[base + i];
      M->ca_vdt[base + i] = v / dt;
      M->ca_d[base + i] = (v / dt) + M->xnew[base + i];
    }
    M->has_ca[c] = 1;
  }
  M->n_probe = n_probe;
  ALLOC(M->probe_cv, n_probe);
  for (int32_t i = 0; i < n_probe; ++i) {
    int32_t gid = probe_gid[i];
    if (gid < 0 || gid >= n_cells || probe_cv[i] < 0 ||
        probe_cv[i] >= M->cv_off[gid + 1] - M->cv_off[gid]) {
      orc_free(M); return fail(-1, "probe %d: bad location", i);
    }
    M->probe_cv[i] = M->cv_off[gid] + probe_cv[i];
  }
  *out = M;
  return 0;
}

int orc_set_replay(orc_model* M, int64_t n, const int32_t* gid, const int64_t* step) {
  free(M->rep_gid);
  free(M->rep_step);
  ALLOC(M->rep_gid, n);
  ALLOC(M->rep_step, n);
  for (int64_t i = 0; i < n; ++i) {
    if (i > 0 && step[i] < step[i - 1]) return fail(-1, "replay spikes must be sorted by step");
    M->rep_gid[i] = gid[i];
    M->rep_step[i] = step[i];
  }
  M->n_rep = n;
  M->rep_pos = 0;
  M->replay = 1;
  while (M->rep_pos < n && M->rep_step[M->rep_pos] < M->step) M->rep_pos++;
  return 0;
}

/* Spikes of cells simulated elsewhere (a shard's stubs for remote presynaptic
   cells): cell gid[i] spiked in step step[i], a past step of the last epoch,
   so that every event it sends is still due (step + delay >= the current
   step).  The events are queued exactly as for a spike detected here. */
static void queue_spike_events(orc_model* M, int32_t gid, int64_t k);
int orc_inject_spikes(orc_model* M, int64_t n, const int32_t* gid, const int64_t* step) {
  for (int64_t i = 0; i < n; ++i) {
    if (gid[i] < 0 || gid[i] >= M->n_cells) return fail(-1, "inject: gid %d out of range", gid[i]);
    if (step[i] >= M->step) return fail(-1, "inject: spike step %lld is not in the past", (long long)step[i]);
    for (int64_t e = M->out_off[gid[i]]; e < M->out_off[gid[i] + 1]; ++e)
      if (step[i] + M->syn_D[M->out_syn[e]] < M->step)
        return fail(-1, "inject: an event of the spike in step %lld is already overdue", (long long)step[i]);
  }
  for (int64_t i = 0; i < n; ++i) queue_spike_events(M, gid[i], step[i]);
  return 0;
}

/* STDP trace value at step k: exact decay since its last jump (Eqs. stdp_ode_1-2
   without spikes in between) */
static double trace_at(double a, int64_t k_last, int64_t k, double dt, double tau) {
  return a * orc_exp(-((double)(k - k_last) * dt) / tau);
}

/* pre event on synapse s in step k (conductance jump; STDP pre update, Eqs.
   stdp_ode_1 and stdp_ode_3 with the conductance contribution clipped at w_max) */
static void pre_event(orc_model* M, int64_t s, int64_t k) {
  const orc_mech* mc = &M->mech[M->syn_mech[s]];
  switch (mc->kind) {
    case ORC_MECH_EXPSYN:
    case ORC_MECH_GB:
      M->g[s] += M->syn_weight[s];
      break;
    case ORC_MECH_STC: {
      /* Eq. total_syn_weight: w = h + h0 z, as a multiple of its baseline h0 */
      double h0 = mc->p[12];
      M->g[s] += M->syn_weight[s] * ((M->hs[s] + h0 * M->z[s]) / h0);
      break;
    }
    case ORC_MECH_HCA:
      /* Eq. ca_injection_current_spine: the current jumps by I0 */
      M->c[s] += mc->p[0];
      break;
    case ORC_MECH_STDP: {
      double wc = M->w[s];
      if (wc < 0.0) wc = 0.0;
      if (wc > mc->p[7]) wc = mc->p[7];
      M->g[s] += M->syn_weight[s] * wc;
      M->apre[s] = trace_at(M->apre[s], M->apre_k[s], k, M->dt, mc->p[2]) + mc->p[4];
      M->apre_k[s] = k;
      M->w[s] += trace_at(M->apost[s], M->apost_k[s], k, M->dt, mc->p[3]);
      break;
    }
  }
}

/* delayed presynaptic calcium jump c_pre (Eq. ca_model_graupner_brunel) */
static void ca_event(orc_model* M, int64_t s) {
  const orc_mech* mc = &M->mech[M->syn_mech[s]];
  if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC) M->c[s] += mc->p[3];
}

/* POST_EVENT in step k -- postsynaptic calcium jump c_post; STDP post update
   (Eqs. stdp_ode_2 and stdp_ode_3) */
static void post_event(orc_model* M, int64_t s, int64_t k) {
  const orc_mech* mc = &M->mech[M->syn_mech[s]];
  if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC) M->c[s] += mc->p[4];
  if (mc->kind == ORC_MECH_STDP) {
    M->apost[s] = trace_at(M->apost[s], M->apost_k[s], k, M->dt, mc->p[3]) + mc->p[5];
    M->apost_k[s] = k;
    M->w[s] += trace_at(M->apre[s], M->apre_k[s], k, M->dt, mc->p[2]);
  }
}

static void queue_spike_events(orc_model* M, int32_t gid, int64_t k) {
  for (int64_t e = M->out_off[gid]; e < M->out_off[gid + 1]; ++e) {
    int64_t s = M->out_syn[e];
    const orc_mech* mc = &M->mech[M->syn_mech[s]];
    push_ev(&M->q[(k + M->syn_D[s]) % M->R], (int32_t)s, 0);
    if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC)
      push_ev(&M->q[(k + M->syn_D[s] + mc->dc_steps) % M->R], (int32_t)s, 1);
  }
}

/* One step of the diffusing PRP field of cell c: the reaction as the
   mechanism's explicit update, P* = P + rate (src - P) in every CV (rate =
   step / tau_p; synthesis only at the soma, degradation everywhere), then the
   diffusion by one backward-Euler solve with diagonal diag[] and right-hand
   side vdt[] P* (vdt = V / step).  Uses the cell's solver scratch. */
static void prp_field_step(orc_model* M, int32_t c, double qs, double rate, const double* diag,
                           const double* vdt) {
  int64_t base = M->cv_off[c], n = M->cv_off[c + 1] - base;
  double *P = M->prp_cv + base, *d = M->d + base, *b = M->b + base, *x = M->xnew + base;
  for (int64_t i = 0; i < n; ++i) {
    double src = (i == 0) ? qs * M->prp_src[c] : 0.0;
    double ps = P[i] + rate * (src - P[i]);
    d[i] = diag[base + i];
    b[i] = vdt[base + i] * ps;
  }
  hines(n, M->parent + base, d, M->prp_a + base, b, M->f + base, M->xp + base, x);
  for (int64_t i = 0; i < n; ++i) P[i] = x[i];
  M->p[c] = P[0];
}

/* One step of the heterosynaptic calcium field of cell c (Eq.
   ca_diffusion_dendrite): the reaction explicitly, C* = C + dt/tau_C (q - C)
   with q = tau_C src / V the inflow's steady concentration in each CV (src
   from this step's injection currents, 0 in CVs without synapses); then the
   diffusion by one backward-Euler solve on the cell's tree. */
static void ca_field_step(orc_model* M, int32_t c) {
  int64_t base = M->cv_off[c], n = M->cv_off[c + 1] - base;
  const orc_mech* mc = &M->mech[M->cell_hca_mech[c]];
  const double tau_c = mc->p[8], r = mc->rate_ca;
  double *C = M->ca_cv + base, *d = M->d + base, *b = M->b + base, *x = M->xnew + base;
  for (int64_t i = 0; i < n; ++i) {
    double q = (tau_c * M->ca_src[base + i]) / M->vol[base + i];
    double cs = C[i] + r * (q - C[i]);
    d[i] = M->ca_d[base + i];
    b[i] = M->ca_vdt[base + i] * cs;
  }
  hines(n, M->parent + base, d, M->ca_a + base, b, M->f + base, M->xp + base, x);
  for (int64_t i = 0; i < n; ++i) C[i] = x[i];
}

/* steps 2-5 for one cell */
static void cell_step(orc_model* M, int32_t c, int64_t k) {
  const double dt = M->dt;
  int64_t base = M->cv_off[c], n = M->cv_off[c + 1] - base;
  const int32_t* par = M->parent + base;
  double *V = M->V + base, *gs = M->gs + base, *es = M->es + base;
  double *d = M->d + base, *b = M->b + base;
  for (int64_t i = 0; i < n; ++i) { gs[i] = 0.0; es[i] = 0.0; }
  if (M->has_ca[c])
    for (int64_t i = 0; i < n; ++i) M->ca_src[base + i] = 0.0;
  /* synaptic conductances summed per CV in the cell's canonical order */
  for (int64_t j = M->cell_syn_off[c]; j < M->cell_syn_off[c + 1]; ++j) {
    int64_t s = M->cell_syn[j];
    int64_t i = M->syn_cv[s] - base;
    double E = M->mech[M->syn_mech[s]].p[1];
    gs[i] = gs[i] + M->g[s];
    es[i] = es[i] + M->g[s] * E;
  }
  double iinj = (k >= M->k_on[c] && k < M->k_off[c]) ? M->istep[c] : 0.0;
  /* backward-Euler matrix: (C/dt + sum g_axial + g_m) V^{k+1} - sum g_axial V_nb^{k+1}
     = C/dt V^k + sum g E + I_inj */
  for (int64_t i = 0; i < n; ++i) {
    int64_t gi = base + i;
    const orc_mech* mc = &M->mech[M->cv_mech[gi]];
    double gm, em;
    if (mc->kind == ORC_MECH_PAS) {
      gm = M->gpas[gi];
      em = M->em_pas[gi];
    } else {
      double mv = M->m[gi], hv = M->h[gi], nv = M->n[gi];
      double gna = M->gna_a[gi] * (((mv * mv) * mv) * hv);
      double gk = M->gk_a[gi] * (((nv * nv) * nv) * nv);
      gm = (gna + gk) + M->gl_a[gi];
      em = ((gna * mc->p[3]) + (gk * mc->p[4])) + (M->gl_a[gi] * mc->p[5]);
    }
    d[i] = ((M->cdt[gi] + M->gax[gi]) + gm) + gs[i];
    b[i] = (fma(M->cdt[gi], V[i], em) + (i == 0 ? iinj : 0.0)) + es[i];
  }
  double v0_old = V[0];
  double* xnew = M->xnew + base;
  hines(n, par, d, M->a + base, b, M->f + base, M->xp + base, xnew);
  for (int64_t i = 0; i < n; ++i) V[i] = xnew[i];
  /* HH gates at V^{k+1} */
  for (int64_t i = 0; i < n; ++i) {
    int64_t gi = base + i;
    if (M->mech[M->cv_mech[gi]].kind != ORC_MECH_HH) continue;
    double am, bm, ah, bh, an, bn;
    orc_hh_rates(V[i], &am, &bm, &ah, &bh, &an, &bn);
    M->m[gi] = cnexp_gate(M->m[gi], am, bm, dt);
    M->h[gi] = cnexp_gate(M->h[gi], ah, bh, dt);
    M->n[gi] = cnexp_gate(M->n[gi], an, bn, dt);
  }
  /* synapse state updates with the post-event values of step k */
  double S = 0.0, pk = M->p[c];
  for (int64_t j = M->cell_syn_off[c]; j < M->cell_syn_off[c + 1]; ++j) {
    int64_t s = M->cell_syn[j];
    const orc_mech* mc = &M->mech[M->syn_mech[s]];
    const double* q = mc->p;
    M->g[s] = M->g[s] * mc->decay_g;
    if (mc->kind == ORC_MECH_GB) {
      /* Eq. weight_graupner_brunel, forward Euler */
      double w = M->w[s], cc = M->c[s];
      double A = (w * (1.0 - w)) * (q[10] - w);
      double P = (cc > q[5]) ? q[7] * (1.0 - w) : 0.0;
      double D = (cc > q[6]) ? q[8] * w : 0.0;
      double wn = w + mc->rate_w * ((P - A) - D);
      /* Eq. plasticity_noise_1, Euler-Maruyama: sigma_pl sqrt(n dt / tau_w) N(0,1)
         with n the number of thresholds the calcium exceeds */
      int nth = (cc > q[5]) + (cc > q[6]);
      if (mc->sigma > 0.0 && nth > 0) wn = wn + mc->amp[nth] * orc_normal(M->seed, (uint64_t)s, k);
      M->w[s] = wn;
      M->c[s] = cc * mc->decay_c;
    } else if (mc->kind == ORC_MECH_STC) {
      double h = M->hs[s], z = M->z[s], cc = M->c[s], h0 = q[12];
      S = S + fabs(h - h0);
      /* Eq. late_phase_weight with the PRP p^k of the cell, or at the synapse's
         CV when PRP diffuses */
      double pz = M->has_diff[c] ? M->prp_cv[M->syn_cv[s]] : pk;
      double T1 = ((h - h0) > q[13]) ? (pz * q[16]) * (1.0 - z) : 0.0;
      double T2 = ((h0 - h) > q[13]) ? (pz * q[16]) * (z + 0.5) : 0.0;
      M->z[s] = z + mc->rate_z * (T1 - T2);
      /* Eq. early_phase_weight, 10 mV potentiation ceiling */
      double P = (cc > q[5]) ? q[7] * (10.0 - h) : 0.0;
      double D = (cc > q[6]) ? q[8] * h : 0.0;
      double hn = h + mc->rate_h * ((0.1 * (h0 - h) + P) - D);
      /* Eq. plasticity_noise_2 with tau_h */
      int nth = (cc > q[5]) + (cc > q[6]);
      if (mc->sigma > 0.0 && nth > 0) hn = hn + mc->amp[nth] * orc_normal(M->seed, (uint64_t)s, k);
      M->hs[s] = hn;
      M->c[s] = cc * mc->decay_c;
    } else if (mc->kind == ORC_MECH_HCA) {
      /* the injection current after this step's events (Eq.
         ca_injection_current_spine) brings w gamma I / (2 F) of calcium into the
         synapse's CV (the source of Eq. ca_diffusion_dendrite), summed per CV in
         canonical order; Eq. heterosyn_weight by forward Euler with the CV's
         calcium before this step's update; then the current decays */
      int64_t ci = M->syn_cv[s] - base;
      double I = M->c[s], w = M->w[s], cl = M->ca_cv[M->syn_cv[s]];
      M->ca_src[base + ci] = M->ca_src[base + ci] + w * (mc->kq * I);
      double P = (cl > q[5]) ? mc->rate_gp * (1.0 - w) : 0.0;
      double D = (cl > q[6]) ? mc->rate_gd * w : 0.0;
      M->w[s] = w + (P - D);
      M->c[s] = I * mc->decay_c;
    }
  }
  if (M->cell_stc_mech[c] >= 0) {
    /* Eq. prp_single_comp: synthesis while the summed early-phase change
       exceeds theta_pro */
    const orc_mech* mc = &M->mech[M->cell_stc_mech[c]];
    double qs = (S > mc->p[14]) ? mc->p[15] : 0.0;
    if (M->has_diff[c]) {
      prp_field_step(M, c, qs, mc->rate_p, M->prp_d, M->prp_vdt);
    } else {
      M->p[c] = pk + mc->rate_p * (qs - pk);
    }
  }
  if (M->has_ca[c]) ca_field_step(M, c);
  /* threshold detection at the soma CV with linear interpolation of the time */
  double th = M->thresh[c];
  M->spk_flag[c] = 0;
  if (v0_old < th && V[0] >= th) {
    M->spk_flag[c] = 1;
    M->spk_t[c] = (double)k * dt + dt * ((th - v0_old) / (V[0] - v0_old));
  }
}

int orc_run(orc_model* M, int64_t n_steps) {
  for (int64_t it = 0; it < n_steps; ++it) {
    int64_t k = M->step;
    orc_bucket* bk = &M->q[k % M->R];
    for (int64_t e = 0; e < bk->n; ++e)
      if (bk->v[e].type == 0) pre_event(M, bk->v[e].syn, k);
    for (int64_t i = 0; i < M->n_poisson; ++i) {
      int64_t s = M->poisson_syn[i];
      if (orc_poisson_u32(M->seed, M->syn_pid[s], k) < M->syn_thr[s]) {
        const orc_mech* mc = &M->mech[M->syn_mech[s]];
        pre_event(M, s, k);
        if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC)
          push_ev(&M->q[(k + mc->dc_steps) % M->R], (int32_t)s, 1);
      }
    }
    for (int64_t e = 0; e < bk->n; ++e)
      if (bk->v[e].type == 1) ca_event(M, bk->v[e].syn);
    bk->n = 0;
    for (int32_t c = 0; c < M->n_cells; ++c) {
      if (!M->spiked_prev[c]) continue;
      for (int64_t j = M->cell_syn_off[c]; j < M->cell_syn_off[c + 1]; ++j)
        post_event(M, M->cell_syn[j], k);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t c = 0; c < M->n_cells; ++c) cell_step(M, c, k);
    for (int32_t c = 0; c < M->n_cells; ++c) {
      if (M->spk_flag[c]) {
        if (M->n_spk == M->cap_spk) {
          M->cap_spk = M->cap_spk ? 2 * M->cap_spk : 1024;
          M->spk_gid = (int32_t*)realloc(M->spk_gid, sizeof(int32_t) * (size_t)M->cap_spk);
          M->spk_step = (int64_t*)realloc(M->spk_step, sizeof(int64_t) * (size_t)M->cap_spk);
          M->spk_time = (double*)realloc(M->spk_time, sizeof(double) * (size_t)M->cap_spk);
        }
        M->spk_gid[M->n_spk] = c;
        M->spk_step[M->n_spk] = k;
        M->spk_time[M->n_spk] = M->spk_t[c];
        M->n_spk++;
      }
    }
    if (!M->replay) {
      for (int32_t c = 0; c < M->n_cells; ++c) {
        M->spiked_prev[c] = M->spk_flag[c];
        if (M->spk_flag[c]) queue_spike_events(M, c, k);
      }
    } else {
      for (int32_t c = 0; c < M->n_cells; ++c) M->spiked_prev[c] = 0;
      while (M->rep_pos < M->n_rep && M->rep_step[M->rep_pos] == k) {
        int32_t gid = M->rep_gid[M->rep_pos++];
        if (gid < 0 || gid >= M->n_cells) continue;
        M->spiked_prev[gid] = 1;
        queue_spike_events(M, gid, k);
      }
    }
    if (M->n_probe > 0) {
      if (M->n_samples == M->cap_samples) {
        M->cap_samples = M->cap_samples ? 2 * M->cap_samples : 1024;
        M->probes = (double*)realloc(M->probes, sizeof(double) * (size_t)M->cap_samples * (size_t)M->n_probe);
      }
      for (int32_t i = 0; i < M->n_probe; ++i)
        M->probes[M->n_samples * M->n_probe + i] = M->V[M->probe_cv[i]];
      M->n_samples++;
    }
    M->step++;
  }
  return 0;
}

/* Fast-forward (the '8h-recall' paradigm, Sec. on the recurrent network with
 * plastic synapses): K steps of simulated time without spiking and calcium
 * dynamics.  The membrane state is kept; pending events are dropped; every
 * conductance and calcium decays by its exact factor exp(-K dt / tau); the slow
 * plasticity variables take n_long forward-Euler steps of K dt / n_long with
 * the calcium terms (and so the noise) off, in the order of a full step: per
 * cell, S from h before the update, then per synapse z (with the cell's p) and
 * h (relaxation to h0), GB w (its cubic drift), then p.  STDP traces decay
 * through their closed form as the clock advances by K. */
int orc_fast_forward(orc_model* M, int64_t K, int64_t n_long) {
  if (K < 0 || n_long < 1 || M->replay) return -1;
  for (int32_t c = 0; c < M->n_cells; ++c)
    if (M->has_ca[c]) return -1; /* calcium dynamics have no long-step scheme */
  const double T = (double)K * M->dt;
  const double dtl = T / (double)n_long;
  /* a diffusing PRP field takes its long steps with the long step's matrix:
     diagonal V/dtl + sum gD, right-hand side V/dtl P* */
  double *dl = calloc((size_t)M->n_cv + 1, sizeof(double)), *vl = calloc((size_t)M->n_cv + 1, sizeof(double));
  if (!dl || !vl) { free(dl); free(vl); return -1; }
  for (int32_t c = 0; c < M->n_cells; ++c)
    if (M->has_diff[c])
      for (int64_t i = M->cv_off[c]; i < M->cv_off[c + 1]; ++i) {
        vl[i] = M->vol[i] / dtl;
        dl[i] = (M->vol[i] / dtl) + M->prp_gsum[i];
      }
  for (int64_t s = 0; s < M->n_syn; ++s) {
    const orc_mech* mc = &M->mech[M->syn_mech[s]];
    M->g[s] = M->g[s] * exp(-T / mc->p[0]);
    if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STC) M->c[s] = M->c[s] * exp(-T / mc->p[2]);
  }
  for (int64_t r = 0; r < M->R; ++r) M->q[r].n = 0;
  for (int32_t c = 0; c < M->n_cells; ++c) M->spiked_prev[c] = 0;
  for (int64_t it = 0; it < n_long; ++it) {
    for (int32_t c = 0; c < M->n_cells; ++c) {
      double S = 0.0, pk = M->p[c];
      for (int64_t j = M->cell_syn_off[c]; j < M->cell_syn_off[c + 1]; ++j) {
        int64_t s = M->cell_syn[j];
        const orc_mech* mc = &M->mech[M->syn_mech[s]];
        const double* q = mc->p;
        if (mc->kind == ORC_MECH_GB) {
          double w = M->w[s];
          double A = (w * (1.0 - w)) * (q[10] - w);
          M->w[s] = w + (dtl / q[9]) * (-A);
        } else if (mc->kind == ORC_MECH_STC) {
          double h = M->hs[s], z = M->z[s], h0 = q[12];
          S = S + fabs(h - h0);
          double pz = M->has_diff[c] ? M->prp_cv[M->syn_cv[s]] : pk;
          double T1 = ((h - h0) > q[13]) ? (pz * q[16]) * (1.0 - z) : 0.0;
          double T2 = ((h0 - h) > q[13]) ? (pz * q[16]) * (z + 0.5) : 0.0;
          M->z[s] = z + (dtl / q[10]) * (T1 - T2);
          M->hs[s] = h + (dtl / q[9]) * (0.1 * (h0 - h));
        }
      }
      if (M->cell_stc_mech[c] >= 0) {
        const orc_mech* mc = &M->mech[M->cell_stc_mech[c]];
        double qs = (S > mc->p[14]) ? mc->p[15] : 0.0;
        if (M->has_diff[c]) prp_field_step(M, c, qs, dtl / mc->p[11], dl, vl);
        else M->p[c] = pk + (dtl / mc->p[11]) * (qs - pk);
      }
    }
  }
  free(dl);
  free(vl);
  M->step += K;
  return 0;
}

/* State setters (the inverse of the getters; a model's state swapped in). */
void orc_set_syn(orc_model* M, int32_t field, const double* in) {
  for (int64_t s = 0; s < M->n_syn; ++s) {
    switch (field) {
      case ORC_SYN_G: M->g[s] = in[s]; break;
      case ORC_SYN_C: M->c[s] = in[s]; break;
      case ORC_SYN_W: M->w[s] = in[s]; break;
      case ORC_SYN_H: M->hs[s] = in[s]; break;
      case ORC_SYN_Z: M->z[s] = in[s]; break;
      case ORC_SYN_APRE: M->apre[s] = in[s]; M->apre_k[s] = M->step; break;
      case ORC_SYN_APOST: M->apost[s] = in[s]; M->apost_k[s] = M->step; break;
    }
  }
}
void orc_set_v(orc_model* M, const double* in) { memcpy(M->V, in, sizeof(double) * (size_t)M->n_cv); }
/* PRP concentration per CV of cells whose PRP diffuses (other CVs: 0) */
void orc_get_prp(const orc_model* M, double* out) {
  memcpy(out, M->prp_cv, sizeof(double) * (size_t)M->n_cv);
}
void orc_set_prp(orc_model* M, const double* in) {
  for (int32_t c = 0; c < M->n_cells; ++c) {
    if (!M->has_diff[c]) continue;
    for (int64_t i = M->cv_off[c]; i < M->cv_off[c + 1]; ++i) M->prp_cv[i] = in[i];
    M->p[c] = M->prp_cv[M->cv_off[c]];
  }
}
int32_t orc_has_diffusion(const orc_model* M, int32_t c) { return M->has_diff[c]; }
/* heterosynaptic calcium per CV of cells with HCA synapses (other CVs: 0) */
void orc_get_ca(const orc_model* M, double* out) {
  memcpy(out, M->ca_cv, sizeof(double) * (size_t)M->n_cv);
}
void orc_set_ca(orc_model* M, const double* in) {
  for (int32_t c = 0; c < M->n_cells; ++c) {
    if (!M->has_ca[c]) continue;
    for (int64_t i = M->cv_off[c]; i < M->cv_off[c + 1]; ++i) M->ca_cv[i] = in[i];
  }
}
/* per cell; the field of a cell whose PRP diffuses is set uniform */
void orc_set_cell_p(orc_model* M, const double* in) {
  memcpy(M->p, in, sizeof(double) * (size_t)M->n_cells);
  for (int32_t c = 0; c < M->n_cells; ++c)
    if (M->has_diff[c])
      for (int64_t i = M->cv_off[c]; i < M->cv_off[c + 1]; ++i) M->prp_cv[i] = in[c];
}
void orc_set_gates(orc_model* M, const double* in) {
  for (int32_t c = 0; c < M->n_cells; ++c) {
    int64_t gi = M->cv_off[c];
    M->m[gi] = in[3 * c];
    M->h[gi] = in[3 * c + 1];
    M->n[gi] = in[3 * c + 2];
  }
}

int64_t orc_step_count(const orc_model* M) { return M->step; }
int64_t orc_n_spikes(const orc_model* M) { return M->n_spk; }
void orc_get_spikes(const orc_model* M, int32_t* gid, int64_t* step, double* t) {
  for (int64_t i = 0; i < M->n_spk; ++i) {
    if (gid) gid[i] = M->spk_gid[i];
    if (step) step[i] = M->spk_step[i];
    if (t) t[i] = M->spk_time[i];
  }
}
int64_t orc_n_cv(const orc_model* M) { return M->n_cv; }
void orc_get_v(const orc_model* M, double* out) { memcpy(out, M->V, sizeof(double) * (size_t)M->n_cv); }
int64_t orc_n_probe_samples(const orc_model* M) { return M->n_samples; }
void orc_get_probes(const orc_model* M, double* out) {
  if (M->n_samples * M->n_probe > 0)
    memcpy(out, M->probes, sizeof(double) * (size_t)(M->n_samples * M->n_probe));
}
void orc_get_syn(const orc_model* M, int32_t field, double* out) {
  for (int64_t s = 0; s < M->n_syn; ++s) {
    const orc_mech* mc = &M->mech[M->syn_mech[s]];
    double v = 0.0;
    switch (field) {
      case ORC_SYN_G: v = M->g[s]; break;
      case ORC_SYN_C: v = M->c[s]; break;
      case ORC_SYN_W: v = M->w[s]; break;
      case ORC_SYN_H: v = M->hs[s]; break;
      case ORC_SYN_Z: v = M->z[s]; break;
      case ORC_SYN_APRE:
        v = mc->kind == ORC_MECH_STDP ? trace_at(M->apre[s], M->apre_k[s], M->step, M->dt, mc->p[2]) : 0.0;
        break;
      case ORC_SYN_APOST:
        v = mc->kind == ORC_MECH_STDP ? trace_at(M->apost[s], M->apost_k[s], M->step, M->dt, mc->p[3]) : 0.0;
        break;
      case ORC_SYN_WEIGHT_TOTAL:
        if (mc->kind == ORC_MECH_STC) v = M->hs[s] + mc->p[12] * M->z[s];
        else if (mc->kind == ORC_MECH_GB || mc->kind == ORC_MECH_STDP || mc->kind == ORC_MECH_HCA)
          v = M->w[s];
        else v = M->syn_weight[s];
        break;
    }
    out[s] = v;
  }
}
void orc_get_cell_p(const orc_model* M, double* out) {
  memcpy(out, M->p, sizeof(double) * (size_t)M->n_cells);
}
void orc_get_gates(const orc_model* M, double* out) {
  for (int32_t c = 0; c < M->n_cells; ++c) {
    int64_t gi = M->cv_off[c];
    out[3 * c] = M->m[gi];
    out[3 * c + 1] = M->h[gi];
    out[3 * c + 2] = M->n[gi];
  }
}
void orc_get_cv_geometry(const orc_model* M, double* cap_nF, double* gpas_uS, double* a_uS) {
  for (int64_t i = 0; i < M->n_cv; ++i) {
    if (cap_nF) cap_nF[i] = M->cap[i];
    if (gpas_uS) gpas_uS[i] = M->gpas[i];
    if (a_uS) a_uS[i] = M->a[i];
  }
}
