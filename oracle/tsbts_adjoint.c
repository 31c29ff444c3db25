/*
 * FP64 CPU oracle of the adjoint of a frozen block schedule (reading R14).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this folder: the plain, slow
 * reference that the CUDA adjoint is compared against. It shares no code
 * with the CUDA library.
 *
 * The replay runs the final pass of an era as plain block steps: Taylor
 * prediction of every body to the block time (Eq. 2), the force sums of
 * Eq. 3 on the active bodies at the predicted positions, and the Eq. 1
 * correction of the active bodies. The schedule (block times and active
 * sets) is an input and is not differentiated.
 *
 * Reverse mode is written out from the chain rule, step by step in reverse
 * order. The pre-step state of every active body is taped in the forward
 * sweep and restored before its step is reversed, so no arithmetic is run
 * backwards. The cotangent of a pair term of the force,
 *   f_i = sum_{j != i} m_j d_ij / s_ij^3,  d_ij = p_j - p_i,
 *   s_ij^2 = |d_ij|^2 + eps^2,
 * given lam_i = dL/df_i, is
 *   g_ij = m_j (lam_i / s^3 - 3 (lam_i . d_ij) d_ij / s^5),
 * added to p_j and subtracted from p_i, and lam_i . d_ij / s^3 added to m_j.
 * Each sum runs in ascending order; OpenMP splits only independent bodies.
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

/* Eq. 2 for every body from its own time tau_j to tick T. */
static void predict_all(int64_t n, const double* r, const double* v,
                        const double* a, const int64_t* tau, int64_t T,
                        int k_max, double* p) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    const double h = tick_time(T - tau[j], k_max);
    for (int c = 0; c < 3; ++c)
      p[3 * j + c] =
          r[3 * j + c] + v[3 * j + c] * h + 0.5 * a[3 * j + c] * h * h;
  }
}

typedef struct {
  double r[3], v[3], a[3];
  int64_t tau;
} snap;

/* Forward sweep. r, v, a, tau receive the final state; if tape is not
 * NULL, tape[e] receives the pre-step state of schedule entry e. */
static void forward(int64_t n, const double* m, const double* r0,
                    const double* v0, double eps, int k_max, int64_t n_steps,
                    const int64_t* step_tau, const int64_t* step_off,
                    const int32_t* act, double* r, double* v, double* a,
                    int64_t* tau, snap* tape) {
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  double* p = (double*)zalloc(n3);
  double* f = (double*)zalloc(n3);
  double* phi = (double*)zalloc(sizeof(double) * (size_t)n);
  double* q = (double*)zalloc(sizeof(double) * (size_t)n);
  int32_t* all = (int32_t*)zalloc(sizeof(int32_t) * (size_t)n);
  memcpy(r, r0, n3);
  memcpy(v, v0, n3);
  for (int64_t i = 0; i < n; ++i) {
    tau[i] = 0;
    all[i] = (int32_t)i;
  }
  orc_forces(n, m, r, v, eps, n, all, a, phi, q);
  for (int64_t s = 0; s < n_steps; ++s) {
    const int64_t T = step_tau[s];
    const int64_t na = step_off[s + 1] - step_off[s];
    const int32_t* A = act + step_off[s];
    predict_all(n, r, v, a, tau, T, k_max, p);
    /* the criterion output q is not used: the schedule is frozen */
    orc_forces(n, m, p, v, eps, na, A, f, phi, q);
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      if (tape) {
        snap* x = &tape[step_off[s] + k];
        memcpy(x->r, r + 3 * i, sizeof x->r);
        memcpy(x->v, v + 3 * i, sizeof x->v);
        memcpy(x->a, a + 3 * i, sizeof x->a);
        x->tau = tau[i];
      }
      const double h = tick_time(T - tau[i], k_max);
      for (int c = 0; c < 3; ++c) {
        v[3 * i + c] = v[3 * i + c] + 0.5 * (a[3 * i + c] + f[3 * k + c]) * h;
        r[3 * i + c] = p[3 * i + c];
        a[3 * i + c] = f[3 * k + c];
      }
      tau[i] = T;
    }
  }
  free(p);
  free(f);
  free(phi);
  free(q);
  free(all);
}

void orc_replay(int64_t n, const double* m, const double* r0, const double* v0,
                double eps, int k_max, int64_t n_steps, const int64_t* step_tau,
                const int64_t* step_off, const int32_t* act, double* r_out,
                double* v_out) {
  double* a = (double*)zalloc(sizeof(double) * 3 * (size_t)n);
  int64_t* tau = (int64_t*)zalloc(sizeof(int64_t) * (size_t)n);
  forward(n, m, r0, v0, eps, k_max, n_steps, step_tau, step_off, act, r_out,
          v_out, a, tau, NULL);
  free(a);
  free(tau);
}

/* Cotangent of the force sums on bodies A[0..na) at positions p, given
 * lam[k] = dL/df_{A[k]}: adds to gp (positions) and gm (masses). The pair
 * sum is split by endpoint so that each body's sum is one loop. */
static void force_vjp(int64_t n, const double* m, const double* p,
                      double eps2, int64_t na, const int32_t* A,
                      const double* lam, double* gp, double* gm) {
  double* gi = (double*)zalloc(sizeof(double) * 3 * (size_t)na);
  /* the i endpoint: -sum_j g_ij */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < na; ++k) {
    const int64_t i = A[k];
    const double lx = lam[3 * k], ly = lam[3 * k + 1], lz = lam[3 * k + 2];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = p[3 * j + 0] - p[3 * i + 0];
      const double dy = p[3 * j + 1] - p[3 * i + 1];
      const double dz = p[3 * j + 2] - p[3 * i + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + eps2;
      const double s = sqrt(s2);
      const double s3 = s2 * s;
      const double s5 = s3 * s2;
      const double ld = lx * dx + ly * dy + lz * dz;
      gx += m[j] * (lx / s3 - 3.0 * ld * dx / s5);
      gy += m[j] * (ly / s3 - 3.0 * ld * dy / s5);
      gz += m[j] * (lz / s3 - 3.0 * ld * dz / s5);
    }
    gi[3 * k] = gx;
    gi[3 * k + 1] = gy;
    gi[3 * k + 2] = gz;
  }
  /* the j endpoint: +sum_i g_ij, and the mass cotangent */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < n; ++j) {
    double gx = 0.0, gy = 0.0, gz = 0.0, mm = 0.0;
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      if (i == j) continue;
      const double lx = lam[3 * k], ly = lam[3 * k + 1], lz = lam[3 * k + 2];
      const double dx = p[3 * j + 0] - p[3 * i + 0];
      const double dy = p[3 * j + 1] - p[3 * i + 1];
      const double dz = p[3 * j + 2] - p[3 * i + 2];
      const double s2 = dx * dx + dy * dy + dz * dz + eps2;
      const double s = sqrt(s2);
      const double s3 = s2 * s;
      const double s5 = s3 * s2;
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

void orc_replay_vjp(int64_t n, const double* m, const double* r0,
                    const double* v0, double eps, int k_max, int64_t n_steps,
                    const int64_t* step_tau, const int64_t* step_off,
                    const int32_t* act, const double* gr_T, const double* gv_T,
                    double* g_r0, double* g_v0, double* g_m) {
  const size_t n3 = sizeof(double) * 3 * (size_t)n;
  const int64_t n_ent = n_steps > 0 ? step_off[n_steps] : 0;
  const double eps2 = eps * eps;
  double* r = (double*)zalloc(n3);
  double* v = (double*)zalloc(n3);
  double* a = (double*)zalloc(n3);
  double* p = (double*)zalloc(n3);
  double* gp = (double*)zalloc(n3);
  double* gR = (double*)zalloc(n3);
  double* gV = (double*)zalloc(n3);
  double* gA = (double*)zalloc(n3);
  double* lam = (double*)zalloc(n3);
  double* gm = (double*)zalloc(sizeof(double) * (size_t)n);
  int64_t* tau = (int64_t*)zalloc(sizeof(int64_t) * (size_t)n);
  int32_t* all = (int32_t*)zalloc(sizeof(int32_t) * (size_t)n);
  snap* tape = (snap*)zalloc(sizeof(snap) * (size_t)n_ent);
  forward(n, m, r0, v0, eps, k_max, n_steps, step_tau, step_off, act, r, v, a,
          tau, tape);
  memcpy(gR, gr_T, n3);
  memcpy(gV, gv_T, n3);
  for (int64_t s = n_steps - 1; s >= 0; --s) {
    const int64_t T = step_tau[s];
    const int64_t na = step_off[s + 1] - step_off[s];
    const int32_t* A = act + step_off[s];
    /* back to the state before step s */
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      const snap* x = &tape[step_off[s] + k];
      memcpy(r + 3 * i, x->r, sizeof x->r);
      memcpy(v + 3 * i, x->v, sizeof x->v);
      memcpy(a + 3 * i, x->a, sizeof x->a);
      tau[i] = x->tau;
    }
    predict_all(n, r, v, a, tau, T, k_max, p);
    memset(gp, 0, n3);
    /* Eq. 1: r_i' = p_i, v_i' = v_i + (a_i + f_i) h / 2, a_i' = f_i */
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = A[k];
      const double h = tick_time(T - tau[i], k_max);
      for (int c = 0; c < 3; ++c) {
        lam[3 * k + c] = gA[3 * i + c] + 0.5 * h * gV[3 * i + c];
        gp[3 * i + c] = gR[3 * i + c];
        gA[3 * i + c] = 0.5 * h * gV[3 * i + c];
        gR[3 * i + c] = 0.0;
      }
    }
    force_vjp(n, m, p, eps2, na, A, lam, gp, gm);
    /* Eq. 2: p_j = r_j + v_j h + a_j h^2 / 2 */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      const double h = tick_time(T - tau[j], k_max);
      for (int c = 0; c < 3; ++c) {
        gR[3 * j + c] += gp[3 * j + c];
        gV[3 * j + c] += h * gp[3 * j + c];
        gA[3 * j + c] += 0.5 * h * h * gp[3 * j + c];
      }
    }
  }
  /* the initial force a0 = f(r0) on every body */
  for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
  memset(gp, 0, n3);
  force_vjp(n, m, r0, eps2, n, all, gA, gp, gm);
  for (int64_t x = 0; x < 3 * n; ++x) {
    g_r0[x] = gR[x] + gp[x];
    g_v0[x] = gV[x];
  }
  memcpy(g_m, gm, sizeof(double) * (size_t)n);
  free(r); free(v); free(a); free(p); free(gp); free(gR); free(gV);
  free(gA); free(lam); free(gm); free(tau); free(all); free(tape);
}

double orc_loss_msr(int64_t n, const double* m, const double* r, double* g_r,
                    double* g_m) {
  double M = 0.0, S = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double r2 = r[3 * i] * r[3 * i] + r[3 * i + 1] * r[3 * i + 1] +
                      r[3 * i + 2] * r[3 * i + 2];
    M += m[i];
    S += m[i] * r2;
  }
  const double L = S / M;
  for (int64_t i = 0; i < n; ++i) {
    const double r2 = r[3 * i] * r[3 * i] + r[3 * i + 1] * r[3 * i + 1] +
                      r[3 * i + 2] * r[3 * i + 2];
    if (g_r)
      for (int c = 0; c < 3; ++c) g_r[3 * i + c] = 2.0 * m[i] * r[3 * i + c] / M;
    if (g_m) g_m[i] = (r2 - L) / M;
  }
  return L;
}
