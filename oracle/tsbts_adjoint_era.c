/*
 * FP64 CPU oracle of the adjoint through every pass of one era: reading
 * R14 extended to the symmetrised passes.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this folder. It shares no code
 * with the CUDA library.
 *
 * Forward: the era's passes are replayed on their frozen block schedules,
 * each from the era-start state (r0, v0, a0 = force at r0, tick 0), as the
 * integrator runs them (Alg. 2): at every block step every body is
 * predicted to the block time — active bodies and every body in the first
 * pass with Eq. 2 from its own state; in passes >= 1 a body that is not
 * active from the previous pass's records (R6: the record on an exact hit,
 * the cubic Hermite between the bracketing records, else Eq. 2) — then the
 * Eq. 3 forces on the active bodies and the Eq. 1 correction. A pass's
 * records are each body's era-start state and its state after each of its
 * steps.
 *
 * Reverse: the passes are reversed last to first. Within a pass, steps are
 * reversed as in the single-pass adjoint (tape restore, Eq. 1 adjoint,
 * force vector-Jacobian product, Eq. 2 adjoint); a position cotangent of a
 * body predicted from the previous pass's records goes to those records
 * (Hermite weights h00, h10 h on record A's r, v and h01, h11 h on record
 * B's), and a record's cotangent is added to the body's post-step state
 * when the step that wrote the record is reversed (era-start records: to
 * the era-start state). Every pass starts from the same era-start state,
 * so the passes' era-start cotangents add up; the initial force's
 * cotangent then goes through its vector-Jacobian product.
 *
 * Later eras: an era starts from the state the previous era left, each
 * body at its own tick (a body whose step overshot the era end waits
 * behind it, Sec. 3) with the acceleration of its last correction. The
 * _state variants take that state (r0, v0, a0, tau0) as the input instead
 * of (r0, v0) at tick 0 with a0 the force at r0, and return the cotangent
 * of a0 instead of passing it through the initial force; chained era by
 * era they give the adjoint across eras.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tsbts_oracle.h"

static double tick_time(int64_t t, int k_max) {
  return ldexp((double)t, -k_max);
}

static void* zalloc(size_t bytes) {
  void* p = calloc(bytes ? bytes : 1, 1);
  if (!p) abort();
  return p;
}

/* one pass: its schedule and its records */
typedef struct {
  int64_t S, E;
  const int64_t* tau;   /* S */
  const int64_t* off;   /* S + 1, entry offsets within the pass */
  const int32_t* act;   /* E */
  /* body b owns records rec_off[b] .. rec_off[b+1]-1 in time order; the
   * first is its era-start record */
  int64_t* rec_off;     /* n + 1 */
  int64_t* rec_tau;     /* n + E */
  double* rec_r;        /* (n + E) x 3 */
  double* rec_v;
  double* rec_a;
  int64_t* ent_rec;     /* E: record written by each entry */
  double* pre;          /* E x 10: pre-step r, v, a, tau (tape) */
  double* fin;          /* n x 10: the pass's final state */
  double* grec_r;       /* record cotangents */
  double* grec_v;
} pass_t;

static void pass_setup(pass_t* P, int64_t n, int64_t S, const int64_t* tau,
                       const int64_t* off, const int32_t* act,
                       const int64_t* tau0) {
  P->S = S;
  P->E = S ? off[S] - off[0] : 0;
  P->tau = tau;
  P->off = off;
  P->act = act;
  const int64_t E = P->E, R = n + E;
  P->rec_off = (int64_t*)zalloc(sizeof(int64_t) * (size_t)(n + 1));
  P->rec_tau = (int64_t*)zalloc(sizeof(int64_t) * (size_t)R);
  P->rec_r = (double*)zalloc(sizeof(double) * 3 * (size_t)R);
  P->rec_v = (double*)zalloc(sizeof(double) * 3 * (size_t)R);
  P->rec_a = (double*)zalloc(sizeof(double) * 3 * (size_t)R);
  P->ent_rec = (int64_t*)zalloc(sizeof(int64_t) * (size_t)(E ? E : 1));
  P->pre = (double*)zalloc(sizeof(double) * 10 * (size_t)(E ? E : 1));
  P->fin = (double*)zalloc(sizeof(double) * 10 * (size_t)n);
  P->grec_r = (double*)zalloc(sizeof(double) * 3 * (size_t)R);
  P->grec_v = (double*)zalloc(sizeof(double) * 3 * (size_t)R);
  /* record slots: one era-start record per body, then one per entry */
  int64_t* cnt = (int64_t*)zalloc(sizeof(int64_t) * (size_t)n);
  for (int64_t b = 0; b < n; ++b) cnt[b] = 1;
  for (int64_t e = 0; e < E; ++e) cnt[act[off[0] + e]] += 1;
  for (int64_t b = 0; b < n; ++b) P->rec_off[b + 1] = P->rec_off[b] + cnt[b];
  for (int64_t b = 0; b < n; ++b) cnt[b] = P->rec_off[b] + 1;
  for (int64_t s = 0; s < S; ++s)
    for (int64_t e = off[s] - off[0]; e < off[s + 1] - off[0]; ++e) {
      const int32_t b = act[off[0] + e];
      P->ent_rec[e] = cnt[b];
      P->rec_tau[cnt[b]] = tau[s];
      cnt[b] += 1;
    }
  for (int64_t b = 0; b < n; ++b)
    P->rec_tau[P->rec_off[b]] = tau0 ? tau0[b] : 0;
  free(cnt);
}

static void pass_free(pass_t* P) {
  free(P->rec_off); free(P->rec_tau); free(P->rec_r); free(P->rec_v);
  free(P->rec_a); free(P->ent_rec); free(P->pre); free(P->fin);
  free(P->grec_r); free(P->grec_v);
}

/* how a body was predicted to tick T */
typedef struct {
  int kind;         /* 0: Eq. 2 from its own state, 1: record, 2: Hermite */
  int64_t ra, rb;   /* records used */
  double w[4];      /* Hermite position weights h00, h10 h, h01, h11 h */
} pred_t;

static void taylor3(const double* r, const double* v, const double* a,
                    double h, double* rp, double* vp) {
  for (int c = 0; c < 3; ++c) {
    rp[c] = r[c] + v[c] * h + 0.5 * a[c] * h * h;
    vp[c] = v[c] + a[c] * h;
  }
}

/* R6 prediction of body j to tick T; Q: the previous pass (NULL in the
 * first pass or for an active body) */
static pred_t predict(const pass_t* Q, int64_t j, int64_t T, int k_max,
                      const double* r, const double* v, const double* a,
                      int64_t tj, double* rp, double* vp) {
  pred_t out;
  memset(&out, 0, sizeof out);
  if (Q) {
    /* last record at or before T (records in time order) */
    int64_t lo = Q->rec_off[j], hi = Q->rec_off[j + 1] - 1, k = -1;
    while (lo <= hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (Q->rec_tau[mid] <= T) {
        k = mid;
        lo = mid + 1;
      } else {
        hi = mid - 1;
      }
    }
    if (k >= 0 && Q->rec_tau[k] == T) {
      memcpy(rp, Q->rec_r + 3 * k, sizeof(double) * 3);
      memcpy(vp, Q->rec_v + 3 * k, sizeof(double) * 3);
      out.kind = 1;
      out.ra = k;
      return out;
    }
    if (k >= 0 && k + 1 < Q->rec_off[j + 1]) {
      const int64_t ta = Q->rec_tau[k], tb = Q->rec_tau[k + 1];
      orc_hermite(ta, tb, T, k_max, Q->rec_r + 3 * k, Q->rec_v + 3 * k,
                  Q->rec_a + 3 * k, Q->rec_r + 3 * (k + 1),
                  Q->rec_v + 3 * (k + 1), Q->rec_a + 3 * (k + 1), rp, vp);
      const double x = (double)(T - ta) / (double)(tb - ta);
      const double h = ldexp((double)(tb - ta), -k_max);
      out.kind = 2;
      out.ra = k;
      out.rb = k + 1;
      out.w[0] = (1.0 + 2.0 * x) * (1.0 - x) * (1.0 - x);
      out.w[1] = x * (1.0 - x) * (1.0 - x) * h;
      out.w[2] = x * x * (3.0 - 2.0 * x);
      out.w[3] = x * x * (x - 1.0) * h;
      return out;
    }
  }
  taylor3(r, v, a, tick_time(T - tj, k_max), rp, vp);
  return out;
}

typedef struct {
  int64_t n;
  const double* m;
  double eps;
  int k_max;
  double *r, *v, *a;
  int64_t* tau;
  double *rp, *vp, *f, *phi, *q;
  int64_t* stamp;  /* per body: the step it was last active in */
  int64_t clock;   /* steps visited so far (forward and reverse) */
  const int64_t* tau0;  /* era-start tick of each body (NULL: all 0) */
} era_t;

/* forward replay of pass P (previous pass Q or NULL) from the era start */
static void pass_forward(era_t* X, pass_t* P, const pass_t* Q,
                         const double* r0, const double* v0,
                         const double* a0) {
  const int64_t n = X->n;
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  memcpy(X->r, r0, n3);
  memcpy(X->v, v0, n3);
  memcpy(X->a, a0, n3);
  for (int64_t b = 0; b < n; ++b) {
    X->tau[b] = X->tau0 ? X->tau0[b] : 0;
    const int64_t k = P->rec_off[b];
    memcpy(P->rec_r + 3 * k, r0 + 3 * b, sizeof(double) * 3);
    memcpy(P->rec_v + 3 * k, v0 + 3 * b, sizeof(double) * 3);
    memcpy(P->rec_a + 3 * k, a0 + 3 * b, sizeof(double) * 3);
  }
  for (int64_t s = 0; s < P->S; ++s) {
    const int64_t T = P->tau[s];
    const int64_t e0 = P->off[s] - P->off[0];
    const int64_t na = P->off[s + 1] - P->off[s];
    const int32_t* A = P->act + P->off[s];
    const int64_t stamp = ++X->clock;
    for (int64_t k = 0; k < na; ++k) X->stamp[A[k]] = stamp;
    for (int64_t j = 0; j < n; ++j)
      predict(X->stamp[j] == stamp ? NULL : Q, j, T, X->k_max, X->r + 3 * j,
              X->v + 3 * j, X->a + 3 * j, X->tau[j], X->rp + 3 * j,
              X->vp + 3 * j);
    orc_forces(n, X->m, X->rp, X->vp, X->eps, na, A, X->f, X->phi, X->q);
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      double* t = P->pre + 10 * (e0 + k);
      memcpy(t, X->r + 3 * i, sizeof(double) * 3);
      memcpy(t + 3, X->v + 3 * i, sizeof(double) * 3);
      memcpy(t + 6, X->a + 3 * i, sizeof(double) * 3);
      t[9] = (double)X->tau[i];
      const double h = tick_time(T - X->tau[i], X->k_max);
      for (int c = 0; c < 3; ++c) {
        X->v[3 * i + c] =
            X->v[3 * i + c] + 0.5 * (X->a[3 * i + c] + X->f[3 * k + c]) * h;
        X->r[3 * i + c] = X->rp[3 * i + c];
        X->a[3 * i + c] = X->f[3 * k + c];
      }
      X->tau[i] = T;
      const int64_t rec = P->ent_rec[e0 + k];
      memcpy(P->rec_r + 3 * rec, X->r + 3 * i, sizeof(double) * 3);
      memcpy(P->rec_v + 3 * rec, X->v + 3 * i, sizeof(double) * 3);
      memcpy(P->rec_a + 3 * rec, X->a + 3 * i, sizeof(double) * 3);
    }
  }
  for (int64_t b = 0; b < n; ++b) {
    double* t = P->fin + 10 * b;
    memcpy(t, X->r + 3 * b, sizeof(double) * 3);
    memcpy(t + 3, X->v + 3 * b, sizeof(double) * 3);
    memcpy(t + 6, X->a + 3 * b, sizeof(double) * 3);
    t[9] = (double)X->tau[b];
  }
}

/* force vector-Jacobian product (as in the single-pass adjoint): adds
 * to gp (positions) and gm (masses) */
static void force_vjp(int64_t n, const double* m, const double* p,
                      double eps2, int64_t na, const int32_t* A,
                      const double* lam, double* gp, double* gm) {
  double* gi = (double*)zalloc(sizeof(double) * 3 * (size_t)na);
  for (int64_t k = 0; k < na; ++k) {
    const int64_t i = A[k];
    const double lx = lam[3 * k], ly = lam[3 * k + 1], lz = lam[3 * k + 2];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = p[3 * j] - p[3 * i], dy = p[3 * j + 1] - p[3 * i + 1],
                   dz = p[3 * j + 2] - p[3 * i + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + eps2;
      const double s = sqrt(s2), s3 = s2 * s, s5 = s3 * s2;
      const double ld = lx * dx + ly * dy + lz * dz;
      gx += m[j] * (lx / s3 - 3.0 * ld * dx / s5);
      gy += m[j] * (ly / s3 - 3.0 * ld * dy / s5);
      gz += m[j] * (lz / s3 - 3.0 * ld * dz / s5);
    }
    gi[3 * k] = gx;
    gi[3 * k + 1] = gy;
    gi[3 * k + 2] = gz;
  }
  for (int64_t j = 0; j < n; ++j) {
    double gx = 0.0, gy = 0.0, gz = 0.0, mm = 0.0;
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      if (i == j) continue;
      const double lx = lam[3 * k], ly = lam[3 * k + 1], lz = lam[3 * k + 2];
      const double dx = p[3 * j] - p[3 * i], dy = p[3 * j + 1] - p[3 * i + 1],
                   dz = p[3 * j + 2] - p[3 * i + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + eps2;
      const double s = sqrt(s2), s3 = s2 * s, s5 = s3 * s2;
      const double ld = lx * dx + ly * dy + lz * dz;
      gx += m[j] * (lx / s3 - 3.0 * ld * dx / s5);
      gy += m[j] * (ly / s3 - 3.0 * ld * dy / s5);
      gz += m[j] * (lz / s3 - 3.0 * ld * dz / s5);
      mm += ld / s3;
    }
    gp[3 * j] += gx;
    gp[3 * j + 1] += gy;
    gp[3 * j + 2] += gz;
    gm[j] += mm;
  }
  for (int64_t k = 0; k < na; ++k)
    for (int c = 0; c < 3; ++c) gp[3 * (int64_t)A[k] + c] -= gi[3 * k + c];
  free(gi);
}

/* a0_in NULL: a0 is the force at r0 */
static void era_forward(era_t* X, pass_t* passes, int64_t n_pass,
                        const double* r0, const double* v0,
                        const double* a0_in, double* a0) {
  const int64_t n = X->n;
  if (a0_in) {
    memcpy(a0, a0_in, sizeof(double) * 3 * (size_t)n);
  } else {
    int32_t* all = (int32_t*)zalloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
    orc_forces(n, X->m, r0, v0, X->eps, n, all, a0, X->phi, X->q);
    free(all);
  }
  for (int64_t p = 0; p < n_pass; ++p)
    pass_forward(X, &passes[p], p ? &passes[p - 1] : NULL, r0, v0, a0);
}

static void setup(era_t* X, int64_t n, const double* m, double eps, int k_max,
                  pass_t* passes, int64_t n_pass, const int64_t* pass_off,
                  const int64_t* step_tau, const int64_t* step_off,
                  const int32_t* act, const int64_t* tau0) {
  X->n = n;
  X->tau0 = tau0;
  X->m = m;
  X->eps = eps;
  X->k_max = k_max;
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  X->r = (double*)zalloc(n3);
  X->v = (double*)zalloc(n3);
  X->a = (double*)zalloc(n3);
  X->rp = (double*)zalloc(n3);
  X->vp = (double*)zalloc(n3);
  X->f = (double*)zalloc(n3);
  X->phi = (double*)zalloc(sizeof(double) * (size_t)n);
  X->q = (double*)zalloc(sizeof(double) * (size_t)n);
  X->tau = (int64_t*)zalloc(sizeof(int64_t) * (size_t)n);
  X->stamp = (int64_t*)zalloc(sizeof(int64_t) * (size_t)n);
  X->clock = 0;
  for (int64_t p = 0; p < n_pass; ++p) {
    const int64_t s0 = pass_off[p], s1 = pass_off[p + 1];
    pass_setup(&passes[p], n, s1 - s0, step_tau + s0, step_off + s0, act,
               tau0);
  }
}

static void teardown(era_t* X, pass_t* passes, int64_t n_pass) {
  free(X->r); free(X->v); free(X->a); free(X->rp); free(X->vp); free(X->f);
  free(X->phi); free(X->q); free(X->tau); free(X->stamp);
  for (int64_t p = 0; p < n_pass; ++p) pass_free(&passes[p]);
}

void orc_era_replay_state(int64_t n, const double* m, const double* r0,
                          const double* v0, const double* a0_in,
                          const int64_t* tau0, double eps, int k_max,
                          int64_t n_pass, const int64_t* pass_off,
                          const int64_t* step_tau, const int64_t* step_off,
                          const int32_t* act, double* r_out, double* v_out,
                          double* a_out, int64_t* tau_out) {
  era_t X;
  pass_t* passes = (pass_t*)zalloc(sizeof(pass_t) * (size_t)n_pass);
  setup(&X, n, m, eps, k_max, passes, n_pass, pass_off, step_tau, step_off,
        act, tau0);
  double* a0 = (double*)zalloc(sizeof(double) * 3 * (size_t)n);
  era_forward(&X, passes, n_pass, r0, v0, a0_in, a0);
  if (r_out) memcpy(r_out, X.r, sizeof(double) * 3 * (size_t)n);
  if (v_out) memcpy(v_out, X.v, sizeof(double) * 3 * (size_t)n);
  if (a_out) memcpy(a_out, X.a, sizeof(double) * 3 * (size_t)n);
  if (tau_out) memcpy(tau_out, X.tau, sizeof(int64_t) * (size_t)n);
  free(a0);
  teardown(&X, passes, n_pass);
  free(passes);
}

void orc_era_replay(int64_t n, const double* m, const double* r0,
                    const double* v0, double eps, int k_max, int64_t n_pass,
                    const int64_t* pass_off, const int64_t* step_tau,
                    const int64_t* step_off, const int32_t* act,
                    double* r_out, double* v_out) {
  orc_era_replay_state(n, m, r0, v0, NULL, NULL, eps, k_max, n_pass,
                       pass_off, step_tau, step_off, act, r_out, v_out, NULL,
                       NULL);
}

void orc_era_replay_state_vjp(int64_t n, const double* m, const double* r0,
                              const double* v0, const double* a0_in,
                              const int64_t* tau0, double eps, int k_max,
                              int64_t n_pass, const int64_t* pass_off,
                              const int64_t* step_tau,
                              const int64_t* step_off, const int32_t* act,
                              const double* gr_T, const double* gv_T,
                              const double* ga_T, double* g_r0, double* g_v0,
                              double* g_a0, double* g_m) {
  era_t X;
  pass_t* passes = (pass_t*)zalloc(sizeof(pass_t) * (size_t)n_pass);
  setup(&X, n, m, eps, k_max, passes, n_pass, pass_off, step_tau, step_off,
        act, tau0);
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  double* a0 = (double*)zalloc(n3);
  era_forward(&X, passes, n_pass, r0, v0, a0_in, a0);
  const double eps2 = eps * eps;
  double* gR = (double*)zalloc(n3);
  double* gV = (double*)zalloc(n3);
  double* gA = (double*)zalloc(n3);
  double* gp = (double*)zalloc(n3);
  double* lam = (double*)zalloc(n3);
  double* G0r = (double*)zalloc(n3);
  double* G0v = (double*)zalloc(n3);
  double* G0a = (double*)zalloc(n3);
  double* gm = (double*)zalloc(sizeof(double) * (size_t)n);
  for (int64_t p = n_pass - 1; p >= 0; --p) {
    pass_t* P = &passes[p];
    const pass_t* Q = p ? &passes[p - 1] : NULL;
    /* the pass's final state; only the last pass reaches the loss */
    for (int64_t b = 0; b < n; ++b) {
      const double* t = P->fin + 10 * b;
      memcpy(X.r + 3 * b, t, sizeof(double) * 3);
      memcpy(X.v + 3 * b, t + 3, sizeof(double) * 3);
      memcpy(X.a + 3 * b, t + 6, sizeof(double) * 3);
      X.tau[b] = (int64_t)t[9];
    }
    memset(gR, 0, n3);
    memset(gV, 0, n3);
    memset(gA, 0, n3);
    if (p == n_pass - 1) {
      if (gr_T) memcpy(gR, gr_T, n3);
      if (gv_T) memcpy(gV, gv_T, n3);
      if (ga_T) memcpy(gA, ga_T, n3);
    }
    for (int64_t s = P->S - 1; s >= 0; --s) {
      const int64_t T = P->tau[s];
      const int64_t e0 = P->off[s] - P->off[0];
      const int64_t na = P->off[s + 1] - P->off[s];
      const int32_t* A = P->act + P->off[s];
      const int64_t stamp = ++X.clock;
      for (int64_t k = 0; k < na; ++k) {
        const int64_t i = A[k];
        X.stamp[i] = stamp;
        /* the record this step wrote: its cotangent joins the post-step
         * state's */
        const int64_t rec = P->ent_rec[e0 + k];
        for (int c = 0; c < 3; ++c) {
          gR[3 * i + c] += P->grec_r[3 * rec + c];
          gV[3 * i + c] += P->grec_v[3 * rec + c];
        }
        /* back to the pre-step state */
        const double* t = P->pre + 10 * (e0 + k);
        memcpy(X.r + 3 * i, t, sizeof(double) * 3);
        memcpy(X.v + 3 * i, t + 3, sizeof(double) * 3);
        memcpy(X.a + 3 * i, t + 6, sizeof(double) * 3);
        X.tau[i] = (int64_t)t[9];
      }
      pred_t* how = (pred_t*)zalloc(sizeof(pred_t) * (size_t)n);
      for (int64_t j = 0; j < n; ++j)
        how[j] = predict(X.stamp[j] == stamp ? NULL : Q, j, T, k_max,
                         X.r + 3 * j, X.v + 3 * j, X.a + 3 * j, X.tau[j],
                         X.rp + 3 * j, X.vp + 3 * j);
      memset(gp, 0, n3);
      /* Eq. 1: r_i' = p_i, v_i' = v_i + (a_i + f_i) h / 2, a_i' = f_i */
      for (int64_t k = 0; k < na; ++k) {
        const int64_t i = A[k];
        const double h = tick_time(T - X.tau[i], k_max);
        for (int c = 0; c < 3; ++c) {
          lam[3 * k + c] = gA[3 * i + c] + 0.5 * h * gV[3 * i + c];
          gp[3 * i + c] = gR[3 * i + c];
          gA[3 * i + c] = 0.5 * h * gV[3 * i + c];
          gR[3 * i + c] = 0.0;
        }
      }
      force_vjp(n, m, X.rp, eps2, na, A, lam, gp, gm);
      /* the predictions: Eq. 2 on the body's state, or the previous
       * pass's records */
      for (int64_t j = 0; j < n; ++j) {
        const double* g = gp + 3 * j;
        if (how[j].kind == 0) {
          const double h = tick_time(T - X.tau[j], k_max);
          for (int c = 0; c < 3; ++c) {
            gR[3 * j + c] += g[c];
            gV[3 * j + c] += h * g[c];
            gA[3 * j + c] += 0.5 * h * h * g[c];
          }
        } else if (how[j].kind == 1) {
          double* q = Q->grec_r + 3 * how[j].ra;
          for (int c = 0; c < 3; ++c) q[c] += g[c];
        } else {
          double* ra = Q->grec_r + 3 * how[j].ra;
          double* va = Q->grec_v + 3 * how[j].ra;
          double* rb = Q->grec_r + 3 * how[j].rb;
          double* vb = Q->grec_v + 3 * how[j].rb;
          for (int c = 0; c < 3; ++c) {
            ra[c] += how[j].w[0] * g[c];
            va[c] += how[j].w[1] * g[c];
            rb[c] += how[j].w[2] * g[c];
            vb[c] += how[j].w[3] * g[c];
          }
        }
      }
      free(how);
    }
    /* the pass began at the era start; its era-start records too */
    for (int64_t b = 0; b < n; ++b) {
      const int64_t k = P->rec_off[b];
      for (int c = 0; c < 3; ++c) {
        G0r[3 * b + c] += gR[3 * b + c] + P->grec_r[3 * k + c];
        G0v[3 * b + c] += gV[3 * b + c] + P->grec_v[3 * k + c];
        G0a[3 * b + c] += gA[3 * b + c];
      }
    }
  }
  memset(gp, 0, n3);
  if (a0_in) {
    /* a0 is an input: its cotangent is returned */
    if (g_a0) memcpy(g_a0, G0a, n3);
  } else {
    /* the initial force a0 = f(r0) on every body */
    int32_t* all = (int32_t*)zalloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
    force_vjp(n, m, r0, eps2, n, all, G0a, gp, gm);
    free(all);
    if (g_a0) memset(g_a0, 0, n3);
  }
  for (int64_t x = 0; x < 3 * n; ++x) {
    if (g_r0) g_r0[x] = G0r[x] + gp[x];
    if (g_v0) g_v0[x] = G0v[x];
  }
  if (g_m) memcpy(g_m, gm, sizeof(double) * (size_t)n);
  free(a0); free(gR); free(gV); free(gA); free(gp); free(lam);
  free(G0r); free(G0v); free(G0a); free(gm);
  teardown(&X, passes, n_pass);
  free(passes);
}

void orc_era_replay_vjp(int64_t n, const double* m, const double* r0,
                        const double* v0, double eps, int k_max,
                        int64_t n_pass, const int64_t* pass_off,
                        const int64_t* step_tau, const int64_t* step_off,
                        const int32_t* act, const double* gr_T,
                        const double* gv_T, double* g_r0, double* g_v0,
                        double* g_m) {
  orc_era_replay_state_vjp(n, m, r0, v0, NULL, NULL, eps, k_max, n_pass,
                           pass_off, step_tau, step_off, act, gr_T, gv_T,
                           NULL, g_r0, g_v0, NULL, g_m);
}
