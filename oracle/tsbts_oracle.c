/*
 * FP64 CPU oracle of the era-based time-symmetric block time-step (TSBTS)
 * integrator (Kaplan & Saygin, Sec. 2 Eq. 1-4, Alg. 1-2; Sec. 4 Alg. 3).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA library
 * is compared against. It shares no code with the CUDA library. Compile with
 * -ffp-contract=off so that every product and sum is rounded on its own and
 * the results do not depend on the host CPU.
 *
 * Each step follows the paper's order and is written without blocking or
 * reordering. Sums over j run in ascending j. OpenMP, where enabled, only
 * splits independent bodies i (or j in the prediction loop); every
 * per-body result is computed by one thread in a fixed order.
 *
 * Readings taken where the paper is silent or garbled:
 *  R1  Eq. 3 collision term uses the softened distance s; the free-fall
 *      term sqrt(|r_ij| / |a_ij|) with the softened pairwise acceleration
 *      |a_ij| = m_j |d_ij| / s^3 equals sqrt(s^3 / m_j). Hence
 *      delta_t_i = eta / sqrt(q_i), q_i = max_j max(|v_ij|^2/s^2, m_j/s^3).
 *  R2  v_ij uses the predicted velocities of both bodies.
 *  R3  the self term j = i is skipped; phi has no self term.
 *  R4  Plummer softening: a = sum m_j d/(d^2+eps^2)^(3/2),
 *      phi = -sum m_j/(d^2+eps^2)^(1/2).
 *  R5  Eq. 4: delta_t^m is the estimate at the step's start in this pass,
 *      delta_t^(m+1) the estimate at the step's end from the previous pass.
 *  R6  Prediction of body j to the block time T: Taylor (Eq. 2) in the
 *      first pass, for active bodies, and whenever the previous pass's
 *      stored records of j do not bracket T; otherwise time-symmetric
 *      cubic Hermite interpolation between the bracketing records.
 *  R7  Alg. 1 follows its prose: try the largest candidate first, test it
 *      with Eq. 4 at that candidate's own end time; halving is untested.
 *  R8  The previous pass's estimate at a time between two stored records
 *      is linearly interpolated; beyond the stored records the start-of-
 *      step estimate is used.
 *  R9  First pass: the largest power of two <= min(estimate, 2 d) that
 *      divides the body's time.
 *  R10 Steps below 2^-k_max are clamped to 2^-k_max and counted.
 *  R11 Dynamic era = last block time - first block time, clamped to
 *      [dt_max 2^-dyn_min_log2, dt_max] and rounded up to a power of two
 *      (the smallest power of two that holds the span; dt_max is one). The
 *      paper does not say how to round; rounding up is the reading under
 *      which dynamic eras reproduce Sec. 4's finding that their energy
 *      errors are in the range of, and modestly below, those of a fixed
 *      era of dt_max. Rounding down shortens most eras to a fraction of
 *      dt_max, cuts off the largest steps at almost every era end, and
 *      gives errors several times larger.
 *
 * Pins: the record lookup, R8's estimate and R6's prediction are pinned
 * through the exported hooks orc_hist_find, orc_hist_dts_at and
 * orc_predict_prev. Parity partially unpinned: whether passes >= 1
 * interpolate at all (the call site in run_pass) has no observable beyond
 * the scheme's own error. Only the separately written multi-pass replay of
 * tsbts_adjoint_era.c, a second restatement of the same reading, catches
 * its omission.
 */
#include "tsbts_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Pairwise force, potential and time-step criterion (Eq. 3, R1-R4).  */
/* ------------------------------------------------------------------ */

static void force_on(int64_t n, const double* m, const double* r,
                     const double* v, double eps2, int64_t i, double* a_out,
                     double* phi_out, double* q_out) {
  double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0, q = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    const double dx = r[3 * j + 0] - r[3 * i + 0];
    const double dy = r[3 * j + 1] - r[3 * i + 1];
    const double dz = r[3 * j + 2] - r[3 * i + 2];
    const double s2 = dx * dx + dy * dy + dz * dz + eps2;
    const double s = sqrt(s2);
    const double f = m[j] / (s2 * s); /* m_j / s^3 */
    ax += f * dx;
    ay += f * dy;
    az += f * dz;
    ph -= m[j] / s;
    const double wx = v[3 * j + 0] - v[3 * i + 0];
    const double wy = v[3 * j + 1] - v[3 * i + 1];
    const double wz = v[3 * j + 2] - v[3 * i + 2];
    const double c = (wx * wx + wy * wy + wz * wz) / s2; /* |v_ij|^2/s^2 */
    if (c > q) q = c;
    if (f > q) q = f; /* s^3 / m_j = |r_ij| / |a_ij| */
  }
  a_out[0] = ax;
  a_out[1] = ay;
  a_out[2] = az;
  *phi_out = ph;
  *q_out = q;
}

void orc_forces(int64_t n, const double* m, const double* r, const double* v,
                double eps, int64_t n_act, const int32_t* idx, double* a,
                double* phi, double* q) {
  const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < n_act; ++k)
    force_on(n, m, r, v, eps2, idx[k], a + 3 * k, phi + k, q + k);
}

void orc_energy_of(int64_t n, const double* m, const double* r,
                   const double* v, double eps, double* ekin, double* epot) {
  const double eps2 = eps * eps;
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    double wi = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = r[3 * j + 0] - r[3 * i + 0];
      const double dy = r[3 * j + 1] - r[3 * i + 1];
      const double dz = r[3 * j + 2] - r[3 * i + 2];
      wi += m[i] * m[j] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
    }
    w[i] = wi;
  }
  double k = 0.0, p = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                      v[3 * i + 2] * v[3 * i + 2];
    k += 0.5 * m[i] * v2;
    p -= 0.5 * w[i];
  }
  free(w);
  *ekin = k;
  *epot = p;
}

/* ------------------------------------------------------------------ */
/* Block levels and step choice (Eq. 4, Alg. 1, R7-R10).               */
/* ------------------------------------------------------------------ */

int64_t orc_level_ticks(double x, int k_min, int k_max, int64_t* underflow) {
  for (int k = k_min; k <= k_max; ++k)
    if (ldexp(1.0, -k) <= x) return (int64_t)1 << (k_max - k);
  if (underflow) ++*underflow;
  return 1;
}

int64_t orc_forward_step(int64_t tau, int64_t d, double dts, int k_min,
                         int k_max, int64_t* underflow) {
  int64_t c = orc_level_ticks(dts, k_min, k_max, underflow);
  if (c > 2 * d) c = 2 * d;
  while (tau % c != 0) c /= 2;
  return c;
}

int64_t orc_symmetric_step(int64_t tau, int64_t d, double dts, double dte_2d,
                           double dte_d, int k_min, int k_max,
                           int64_t* underflow) {
  const int64_t dt_max = (int64_t)1 << (k_max - k_min);
  const int even = (tau % (2 * d)) == 0;
  if (even && 2 * d <= dt_max &&
      2 * d <= orc_level_ticks((dts + dte_2d) / 2.0, k_min, k_max, 0))
    return 2 * d;
  if (d <= orc_level_ticks((dts + dte_d) / 2.0, k_min, k_max, 0)) return d;
  if (d == 1) {
    if (underflow) ++*underflow;
    return 1;
  }
  return d / 2;
}

/* ------------------------------------------------------------------ */
/* Prediction (Eq. 2) and time-symmetric interpolation (R6).          */
/* ------------------------------------------------------------------ */

static void taylor(const double* r, const double* v, const double* a, double h,
                   double* rp, double* vp) {
  for (int c = 0; c < 3; ++c) {
    rp[c] = r[c] + v[c] * h + 0.5 * a[c] * h * h;
    vp[c] = v[c] + a[c] * h;
  }
}

void orc_hermite(int64_t ta, int64_t tb, int64_t t, int k_max,
                 const double* ra, const double* va, const double* aa,
                 const double* rb, const double* vb, const double* ab,
                 double* r_out, double* v_out) {
  const double x = (double)(t - ta) / (double)(tb - ta);
  const double h = ldexp((double)(tb - ta), -k_max);
  const double h00 = (1.0 + 2.0 * x) * (1.0 - x) * (1.0 - x);
  const double h10 = x * (1.0 - x) * (1.0 - x);
  const double h01 = x * x * (3.0 - 2.0 * x);
  const double h11 = x * x * (x - 1.0);
  for (int c = 0; c < 3; ++c) {
    r_out[c] = h00 * ra[c] + h10 * h * va[c] + h01 * rb[c] + h11 * h * vb[c];
    v_out[c] = h00 * va[c] + h10 * h * aa[c] + h01 * vb[c] + h11 * h * ab[c];
  }
}

/* ------------------------------------------------------------------ */
/* Era history (Sec. 2: predicted r, v, a of every body at every step). */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t tau;
  double r[3], v[3], a[3], dts;
} record;

typedef struct {
  record* rec;
  int64_t len, cap;
} history;

static void hist_push(history* h, const record* x) {
  if (h->len == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 16;
    h->rec = (record*)realloc(h->rec, sizeof(record) * (size_t)h->cap);
  }
  h->rec[h->len++] = *x;
}

/* index of the last record with tau <= t, or -1 */
static int64_t hist_find(const history* h, int64_t t) {
  int64_t lo = 0, hi = h->len - 1, ans = -1;
  while (lo <= hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (h->rec[mid].tau <= t) {
      ans = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  return ans;
}

/* previous pass's estimate at tick t (R8), or fallback */
static double hist_dts_at(const history* h, int64_t t, double fallback) {
  const int64_t k = hist_find(h, t);
  if (k < 0) return fallback;
  if (h->rec[k].tau == t) return h->rec[k].dts;
  if (k + 1 >= h->len) return fallback;
  const record* A = &h->rec[k];
  const record* B = &h->rec[k + 1];
  const double w = (double)(t - A->tau) / (double)(B->tau - A->tau);
  return A->dts + (B->dts - A->dts) * w;
}

/* ------------------------------------------------------------------ */
/* The integrator (Alg. 2 with the era choice of Alg. 3).             */
/* ------------------------------------------------------------------ */

struct orc_sim {
  int64_t n;
  orc_cfg cfg;
  int k_min;
  int64_t dt_max_t;
  double *m, *r, *v, *a, *dts;
  int64_t *tau, *dt;
  /* era-start snapshot; rlast: era-end positions of the previous pass */
  double *r0, *v0, *a0, *dts0, *rlast;
  int64_t *tau0, *dt0;
  /* per-pass scratch */
  double *rp, *vp, *an, *phin, *qn;
  int32_t* act;
  char* is_act;
  history *hprev, *hcur;
  int64_t t_sys;
  int64_t stats[7];
  /* schedule log */
  int32_t *lg_era, *lg_pass, *lg_nact, *lg_i;
  int64_t *lg_tau, *lg_dt;
  int64_t lg_steps, lg_steps_cap, lg_ent, lg_ent_cap;
  int64_t *era_s, *era_e, n_era_log, era_cap;
  /* trace of one body (cfg.trace_body) */
  int32_t *tr_era, *tr_pass, *tr_kind;
  int64_t* tr_tau;
  double* tr_rva;
  int64_t tr_n, tr_cap;
};

static void* xmalloc(size_t bytes) {
  void* p = malloc(bytes ? bytes : 1);
  if (!p) abort();
  return p;
}

static void trace_push(orc_sim* s, int era, int pass, int64_t tau, int kind,
                       const double* r, const double* v, const double* a) {
  if (s->tr_n == s->tr_cap) {
    s->tr_cap = s->tr_cap ? 2 * s->tr_cap : 1024;
    s->tr_era = realloc(s->tr_era, sizeof(int32_t) * (size_t)s->tr_cap);
    s->tr_pass = realloc(s->tr_pass, sizeof(int32_t) * (size_t)s->tr_cap);
    s->tr_kind = realloc(s->tr_kind, sizeof(int32_t) * (size_t)s->tr_cap);
    s->tr_tau = realloc(s->tr_tau, sizeof(int64_t) * (size_t)s->tr_cap);
    s->tr_rva = realloc(s->tr_rva, sizeof(double) * 9 * (size_t)s->tr_cap);
    if (!s->tr_era || !s->tr_pass || !s->tr_kind || !s->tr_tau || !s->tr_rva)
      abort();
  }
  const int64_t k = s->tr_n++;
  s->tr_era[k] = era;
  s->tr_pass[k] = pass;
  s->tr_tau[k] = tau;
  s->tr_kind[k] = kind;
  for (int c = 0; c < 3; ++c) {
    s->tr_rva[9 * k + c] = r[c];
    s->tr_rva[9 * k + 3 + c] = v[c];
    s->tr_rva[9 * k + 6 + c] = a ? a[c] : 0.0;
  }
}

int64_t orc_trace_get(orc_sim* s, int32_t* era, int32_t* pass, int64_t* tau,
                      int32_t* kind, double* rva) {
  const size_t k = (size_t)s->tr_n;
  if (era) memcpy(era, s->tr_era, sizeof(int32_t) * k);
  if (pass) memcpy(pass, s->tr_pass, sizeof(int32_t) * k);
  if (tau) memcpy(tau, s->tr_tau, sizeof(int64_t) * k);
  if (kind) memcpy(kind, s->tr_kind, sizeof(int32_t) * k);
  if (rva) memcpy(rva, s->tr_rva, sizeof(double) * 9 * k);
  return s->tr_n;
}

static void log_step(orc_sim* s, int era, int pass, int64_t tau, int nact) {
  if (s->lg_steps == s->lg_steps_cap) {
    s->lg_steps_cap = s->lg_steps_cap ? 2 * s->lg_steps_cap : 1024;
    s->lg_era = realloc(s->lg_era, sizeof(int32_t) * (size_t)s->lg_steps_cap);
    s->lg_pass = realloc(s->lg_pass, sizeof(int32_t) * (size_t)s->lg_steps_cap);
    s->lg_nact = realloc(s->lg_nact, sizeof(int32_t) * (size_t)s->lg_steps_cap);
    s->lg_tau = realloc(s->lg_tau, sizeof(int64_t) * (size_t)s->lg_steps_cap);
  }
  s->lg_era[s->lg_steps] = era;
  s->lg_pass[s->lg_steps] = pass;
  s->lg_tau[s->lg_steps] = tau;
  s->lg_nact[s->lg_steps] = nact;
  ++s->lg_steps;
}

static void log_entry(orc_sim* s, int32_t i, int64_t dt) {
  if (s->lg_ent == s->lg_ent_cap) {
    s->lg_ent_cap = s->lg_ent_cap ? 2 * s->lg_ent_cap : 4096;
    s->lg_i = realloc(s->lg_i, sizeof(int32_t) * (size_t)s->lg_ent_cap);
    s->lg_dt = realloc(s->lg_dt, sizeof(int64_t) * (size_t)s->lg_ent_cap);
  }
  s->lg_i[s->lg_ent] = i;
  s->lg_dt[s->lg_ent] = dt;
  ++s->lg_ent;
}

static double ticks_to_time(int64_t t, int k_max) {
  return ldexp((double)t, -k_max);
}

/* R6 for a body that is not active in a pass >= 1: its previous-pass
 * record at tn on an exact hit, else the cubic Hermite between the records
 * bracketing tn, else (tn before the first or after the last record) Eq. 2
 * from the body's own state (r, v, a at tick tj). */
static void predict_prev(const history* hp, int64_t tj, const double* r,
                         const double* v, const double* a, int64_t tn,
                         int k_max, double* rp, double* vp) {
  const int64_t k = hist_find(hp, tn);
  if (k >= 0 && hp->rec[k].tau == tn) {
    memcpy(rp, hp->rec[k].r, sizeof(double) * 3);
    memcpy(vp, hp->rec[k].v, sizeof(double) * 3);
  } else if (k >= 0 && k + 1 < hp->len) {
    const record* A = &hp->rec[k];
    const record* B = &hp->rec[k + 1];
    orc_hermite(A->tau, B->tau, tn, k_max, A->r, A->v, A->a, B->r, B->v,
                B->a, rp, vp);
  } else {
    taylor(r, v, a, ticks_to_time(tn - tj, k_max), rp, vp);
  }
}

/* one body's previous-pass records from arrays (tau[len] ascending;
 * r, v, a as (len, 3); dts may be NULL) */
static history hist_of(int64_t len, const int64_t* tau, const double* r,
                       const double* v, const double* a, const double* dts) {
  history h = {0, 0, 0};
  for (int64_t k = 0; k < len; ++k) {
    record x;
    memset(&x, 0, sizeof x);
    x.tau = tau[k];
    if (r) memcpy(x.r, r + 3 * k, sizeof x.r);
    if (v) memcpy(x.v, v + 3 * k, sizeof x.v);
    if (a) memcpy(x.a, a + 3 * k, sizeof x.a);
    x.dts = dts ? dts[k] : 0.0;
    hist_push(&h, &x);
  }
  return h;
}

int64_t orc_hist_find(int64_t len, const int64_t* tau, int64_t t) {
  history h = hist_of(len, tau, NULL, NULL, NULL, NULL);
  const int64_t k = hist_find(&h, t);
  free(h.rec);
  return k;
}

double orc_hist_dts_at(int64_t len, const int64_t* tau, const double* dts,
                       int64_t t, double fallback) {
  history h = hist_of(len, tau, NULL, NULL, NULL, dts);
  const double e = hist_dts_at(&h, t, fallback);
  free(h.rec);
  return e;
}

void orc_predict_prev(int64_t len, const int64_t* tau, const double* r,
                      const double* v, const double* a, int64_t tj,
                      const double* rj, const double* vj, const double* aj,
                      int64_t tn, int k_max, double* rp, double* vp) {
  history h = hist_of(len, tau, r, v, a, NULL);
  predict_prev(&h, tj, rj, vj, aj, tn, k_max, rp, vp);
  free(h.rec);
}

orc_sim* orc_create(int64_t n, const double* m, const double* r,
                    const double* v, const orc_cfg* cfg) {
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->n = n;
  s->cfg = *cfg;
  int k_min = 0;
  while (ldexp(1.0, -k_min) > cfg->dt_max && k_min < cfg->k_max) ++k_min;
  s->k_min = k_min;
  s->dt_max_t = (int64_t)1 << (cfg->k_max - k_min);
  const size_t n3 = sizeof(double) * 3 * (size_t)n, n1 = sizeof(double) * (size_t)n;
  const size_t ni = sizeof(int64_t) * (size_t)n;
  s->m = xmalloc(n1);
  s->r = xmalloc(n3);
  s->v = xmalloc(n3);
  s->a = xmalloc(n3);
  s->dts = xmalloc(n1);
  s->tau = xmalloc(ni);
  s->dt = xmalloc(ni);
  s->r0 = xmalloc(n3);
  s->rlast = xmalloc(n3);
  s->v0 = xmalloc(n3);
  s->a0 = xmalloc(n3);
  s->dts0 = xmalloc(n1);
  s->tau0 = xmalloc(ni);
  s->dt0 = xmalloc(ni);
  s->rp = xmalloc(n3);
  s->vp = xmalloc(n3);
  s->an = xmalloc(n3);
  s->phin = xmalloc(n1);
  s->qn = xmalloc(n1);
  s->act = xmalloc(sizeof(int32_t) * (size_t)n);
  s->is_act = xmalloc((size_t)n);
  s->hprev = (history*)calloc((size_t)n, sizeof(history));
  s->hcur = (history*)calloc((size_t)n, sizeof(history));
  memcpy(s->m, m, n1);
  memcpy(s->r, r, n3);
  memcpy(s->v, v, n3);
  /* Alg. 2 step 1: forces, time-steps and next block times of all bodies */
  for (int64_t i = 0; i < n; ++i) s->act[i] = (int32_t)i;
  orc_forces(n, s->m, s->r, s->v, cfg->eps, n, s->act, s->a, s->phin, s->qn);
  for (int64_t i = 0; i < n; ++i) {
    s->tau[i] = 0;
    s->dts[i] = cfg->eta / sqrt(s->qn[i]);
    s->dt[i] = orc_level_ticks(s->dts[i], k_min, cfg->k_max, &s->stats[4]);
  }
  s->stats[6] = n * n;
  return s;
}

static int64_t era_length(orc_sim* s) {
  if (s->cfg.era_mode == 0) return (int64_t)1 << (s->cfg.k_max - s->cfg.era_log2);
  /* Alg. 3: era = last block time - first block time, clamped (R11) */
  int64_t first = INT64_MAX, last = INT64_MIN;
  for (int64_t i = 0; i < s->n; ++i) {
    const int64_t t = s->tau[i] + s->dt[i];
    if (t < first) first = t;
    if (t > last) last = t;
  }
  int64_t lo = s->dt_max_t >> s->cfg.dyn_min_log2;
  if (lo < 1) lo = 1;
  int64_t e = last - first;
  if (e < lo) e = lo;
  if (e > s->dt_max_t) e = s->dt_max_t;
  int64_t p = 1;
  while (p < e) p *= 2;
  return p;
}

static void run_pass(orc_sim* s, int era_idx, int pass, int64_t tau_e) {
  const int64_t n = s->n;
  const int k_max = s->cfg.k_max;
  /* the pass's history starts with each body's era-start record */
  for (int64_t i = 0; i < n; ++i) {
    record x;
    x.tau = s->tau[i];
    memcpy(x.r, s->r + 3 * i, sizeof x.r);
    memcpy(x.v, s->v + 3 * i, sizeof x.v);
    memcpy(x.a, s->a + 3 * i, sizeof x.a);
    x.dts = s->dts[i];
    s->hcur[i].len = 0;
    hist_push(&s->hcur[i], &x);
  }
  for (;;) {
    /* Alg. 2 steps 3 and 8: the block with the smallest next time */
    int64_t tn = INT64_MAX;
    for (int64_t i = 0; i < n; ++i)
      if (s->tau[i] + s->dt[i] < tn) tn = s->tau[i] + s->dt[i];
    if (tn > tau_e) break;
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
      s->is_act[i] = (s->tau[i] + s->dt[i] == tn);
      if (s->is_act[i]) s->act[na++] = (int32_t)i;
    }
    /* Alg. 2 step 4: predict or interpolate every body to tn (R6) */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      if (pass > 0 && !s->is_act[j]) {
        predict_prev(&s->hprev[j], s->tau[j], s->r + 3 * j, s->v + 3 * j,
                     s->a + 3 * j, tn, k_max, s->rp + 3 * j, s->vp + 3 * j);
      } else {
        const double h = ticks_to_time(tn - s->tau[j], k_max);
        taylor(s->r + 3 * j, s->v + 3 * j, s->a + 3 * j, h, s->rp + 3 * j,
               s->vp + 3 * j);
      }
    }
    const int64_t tb = s->cfg.trace_body;
    if (tb >= 0 && tb < n && !s->is_act[tb])
      trace_push(s, era_idx, pass, tn, 0, s->rp + 3 * tb, s->vp + 3 * tb, NULL);
    /* Alg. 2 step 5: forces on the active bodies */
    orc_forces(n, s->m, s->rp, s->vp, s->cfg.eps, na, s->act, s->an, s->phin,
               s->qn);
    /* Alg. 2 steps 6-7: correct (Eq. 1) and choose the next step */
    int64_t uf = 0;
#pragma omp parallel for schedule(static) reduction(+ : uf)
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = s->act[k];
      const int64_t d = s->dt[i];
      const double h = ticks_to_time(d, k_max);
      for (int c = 0; c < 3; ++c) {
        s->v[3 * i + c] =
            s->v[3 * i + c] + 0.5 * (s->a[3 * i + c] + s->an[3 * k + c]) * h;
        s->r[3 * i + c] = s->rp[3 * i + c];
        s->a[3 * i + c] = s->an[3 * k + c];
      }
      s->tau[i] = tn;
      s->dts[i] = s->cfg.eta / sqrt(s->qn[k]);
      record x;
      x.tau = tn;
      memcpy(x.r, s->r + 3 * i, sizeof x.r);
      memcpy(x.v, s->v + 3 * i, sizeof x.v);
      memcpy(x.a, s->a + 3 * i, sizeof x.a);
      x.dts = s->dts[i];
      hist_push(&s->hcur[i], &x);
      int64_t u = 0;
      if (pass == 0) {
        s->dt[i] = orc_forward_step(tn, d, s->dts[i], s->k_min, k_max, &u);
      } else {
        const double e2 = hist_dts_at(&s->hprev[i], tn + 2 * d, s->dts[i]);
        const double e1 = hist_dts_at(&s->hprev[i], tn + d, s->dts[i]);
        s->dt[i] = orc_symmetric_step(tn, d, s->dts[i], e2, e1, s->k_min,
                                      k_max, &u);
      }
      uf += u;
    }
    if (tb >= 0 && tb < n && s->is_act[tb])
      trace_push(s, era_idx, pass, tn, 1, s->r + 3 * tb, s->v + 3 * tb,
                 s->a + 3 * tb);
    s->stats[4] += uf;
    s->stats[0] += 1;
    s->stats[1] += na * n;
    if (s->cfg.log) {
      log_step(s, era_idx, pass, tn, (int)na);
      for (int64_t k = 0; k < na; ++k) log_entry(s, s->act[k], s->dt[s->act[k]]);
    }
  }
}

/* Converged iteration: this pass took the same block steps as the
 * previous one (every body's record times equal) and its era-end
 * positions are within conv_tol of the previous pass's. */
static int converged(const orc_sim* s) {
  for (int64_t i = 0; i < s->n; ++i) {
    const history* a = &s->hcur[i];
    const history* b = &s->hprev[i];
    if (a->len != b->len) return 0;
    for (int64_t k = 0; k < a->len; ++k)
      if (a->rec[k].tau != b->rec[k].tau) return 0;
    for (int c = 0; c < 3; ++c)
      if (!(fabs(s->r[3 * i + c] - s->rlast[3 * i + c]) < s->cfg.conv_tol))
        return 0;
  }
  return 1;
}

int orc_run(orc_sim* s, double t_end) {
  const int k_max = s->cfg.k_max;
  const double te = ldexp(t_end, k_max);
  if (!(te == floor(te)) || te < (double)s->t_sys) return -1;
  const int64_t tau_end = (int64_t)te;
  const int64_t n = s->n;
  const size_t n3 = sizeof(double) * 3 * (size_t)n, n1 = sizeof(double) * (size_t)n;
  const size_t ni = sizeof(int64_t) * (size_t)n;
  while (s->t_sys < tau_end) {
    int64_t tau_e = s->t_sys + era_length(s);
    if (tau_e > tau_end) tau_e = tau_end;
    const int era_idx = (int)s->stats[2];
    if (s->n_era_log == s->era_cap) {
      s->era_cap = s->era_cap ? 2 * s->era_cap : 64;
      s->era_s = realloc(s->era_s, sizeof(int64_t) * (size_t)s->era_cap);
      s->era_e = realloc(s->era_e, sizeof(int64_t) * (size_t)s->era_cap);
    }
    s->era_s[s->n_era_log] = s->t_sys;
    s->era_e[s->n_era_log] = tau_e;
    ++s->n_era_log;
    memcpy(s->r0, s->r, n3);
    memcpy(s->v0, s->v, n3);
    memcpy(s->a0, s->a, n3);
    memcpy(s->dts0, s->dts, n1);
    memcpy(s->tau0, s->tau, ni);
    memcpy(s->dt0, s->dt, ni);
    for (int p = 0; p < s->cfg.n_iter; ++p) {
      if (p > 0) {
        if (s->cfg.conv_tol > 0.0) memcpy(s->rlast, s->r, n3);
        /* Alg. 2 step 9: restart the era from its first block */
        memcpy(s->r, s->r0, n3);
        memcpy(s->v, s->v0, n3);
        memcpy(s->a, s->a0, n3);
        memcpy(s->dts, s->dts0, n1);
        memcpy(s->tau, s->tau0, ni);
        memcpy(s->dt, s->dt0, ni);
        history* t = s->hprev;
        s->hprev = s->hcur;
        s->hcur = t;
      }
      run_pass(s, era_idx, p, tau_e);
      s->stats[3] += 1;
      if (p > 0 && s->cfg.conv_tol > 0.0 && converged(s)) break;
    }
    s->t_sys = tau_e;
    s->stats[2] += 1;
  }
  s->stats[5] = s->t_sys;
  return 0;
}

void orc_energy(orc_sim* s, double* ekin, double* epot) {
  const int64_t n = s->n;
  double* r = xmalloc(sizeof(double) * 3 * (size_t)n);
  double* v = xmalloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const double h = ticks_to_time(s->t_sys - s->tau[i], s->cfg.k_max);
    taylor(s->r + 3 * i, s->v + 3 * i, s->a + 3 * i, h, r + 3 * i, v + 3 * i);
  }
  orc_energy_of(n, s->m, r, v, s->cfg.eps, ekin, epot);
  free(r);
  free(v);
}

void orc_get_state(orc_sim* s, double* r, double* v, double* a, int64_t* tau,
                   int64_t* dt, double* dts) {
  const int64_t n = s->n;
  if (r) memcpy(r, s->r, sizeof(double) * 3 * (size_t)n);
  if (v) memcpy(v, s->v, sizeof(double) * 3 * (size_t)n);
  if (a) memcpy(a, s->a, sizeof(double) * 3 * (size_t)n);
  if (tau) memcpy(tau, s->tau, sizeof(int64_t) * (size_t)n);
  if (dt) memcpy(dt, s->dt, sizeof(int64_t) * (size_t)n);
  if (dts) memcpy(dts, s->dts, sizeof(double) * (size_t)n);
}

/* Resume at an era end. An era starts from (m, r, v, a, dts, tau, dt) and
 * the system time alone: its first pass predicts with Eq. 2 only and every
 * later pass interpolates records of the same era (Alg. 2 steps 2-9), so
 * these fields are the whole state carried from one era to the next. A
 * state is accepted when it could end an era: every step a power of two
 * within [1, dt_max], every body time a multiple of its step, tau <= t <
 * tau + dt, finite masses and vectors, dts > 0 (+inf allowed: a body that
 * feels no force). */
int orc_set_state(orc_sim* s, int64_t t, const double* m, const double* r,
                  const double* v, const double* a, const int64_t* tau,
                  const int64_t* dt, const double* dts) {
  const int64_t n = s->n;
  if (t < 0) return -1;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t d = dt[i];
    if (d < 1 || d > s->dt_max_t || (d & (d - 1)) != 0) return -1;
    if (tau[i] < 0 || tau[i] % d != 0 || tau[i] > t || tau[i] + d <= t)
      return -1;
    if (!isfinite(m[i]) || !(dts[i] > 0.0)) return -1;
    for (int c = 0; c < 3; ++c)
      if (!isfinite(r[3 * i + c]) || !isfinite(v[3 * i + c]) ||
          !isfinite(a[3 * i + c]))
        return -1;
  }
  const size_t n3 = sizeof(double) * 3 * (size_t)n, n1 = sizeof(double) * (size_t)n;
  const size_t ni = sizeof(int64_t) * (size_t)n;
  memcpy(s->m, m, n1);
  memcpy(s->r, r, n3);
  memcpy(s->v, v, n3);
  memcpy(s->a, a, n3);
  memcpy(s->tau, tau, ni);
  memcpy(s->dt, dt, ni);
  memcpy(s->dts, dts, n1);
  s->t_sys = t;
  return 0;
}

void orc_stats(orc_sim* s, int64_t* out) {
  s->stats[5] = s->t_sys;
  memcpy(out, s->stats, sizeof s->stats);
}

int64_t orc_log_steps(orc_sim* s) { return s->lg_steps; }
int64_t orc_log_entries(orc_sim* s) { return s->lg_ent; }

void orc_log_get(orc_sim* s, int32_t* step_era, int32_t* step_pass,
                 int64_t* step_tau, int32_t* step_nact, int32_t* ent_i,
                 int64_t* ent_dt) {
  const size_t ns = (size_t)s->lg_steps, ne = (size_t)s->lg_ent;
  if (ns) {
    memcpy(step_era, s->lg_era, sizeof(int32_t) * ns);
    memcpy(step_pass, s->lg_pass, sizeof(int32_t) * ns);
    memcpy(step_tau, s->lg_tau, sizeof(int64_t) * ns);
    memcpy(step_nact, s->lg_nact, sizeof(int32_t) * ns);
  }
  if (ne) {
    memcpy(ent_i, s->lg_i, sizeof(int32_t) * ne);
    memcpy(ent_dt, s->lg_dt, sizeof(int64_t) * ne);
  }
}

int64_t orc_era_log(orc_sim* s, int64_t* tau_s, int64_t* tau_e) {
  if (tau_s) memcpy(tau_s, s->era_s, sizeof(int64_t) * (size_t)s->n_era_log);
  if (tau_e) memcpy(tau_e, s->era_e, sizeof(int64_t) * (size_t)s->n_era_log);
  return s->n_era_log;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->era_s);
  free(s->era_e);
  for (int64_t i = 0; i < s->n; ++i) {
    free(s->hprev[i].rec);
    free(s->hcur[i].rec);
  }
  free(s->hprev);
  free(s->hcur);
  free(s->m); free(s->r); free(s->v); free(s->a); free(s->dts);
  free(s->tau); free(s->dt);
  free(s->r0); free(s->rlast); free(s->v0); free(s->a0); free(s->dts0);
  free(s->tau0); free(s->dt0);
  free(s->rp); free(s->vp); free(s->an); free(s->phin); free(s->qn);
  free(s->act); free(s->is_act);
  free(s->lg_era); free(s->lg_pass); free(s->lg_nact); free(s->lg_i);
  free(s->lg_tau); free(s->lg_dt);
  free(s->tr_era); free(s->tr_pass); free(s->tr_kind); free(s->tr_tau);
  free(s->tr_rva);
  free(s);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
