/*
 * FP64 CPU oracle of the time-symmetric block time-step (TSBTS) integrator
 * with fixed or dynamic era (Kaplan & Saygin, Sec. 2-4).
 *
 * TEST INFRASTRUCTURE ONLY. This header and its implementation are the
 * slow, plain reference that the CUDA library is checked against. Only the
 * test suite, the smoke check and the bench's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Units: G = 1. Time is kept as integer ticks, 2^k_max ticks per time unit.
 * Arrays of vectors are row-major (n, 3) doubles: x, y, z per body.
 */
#ifndef TSBTS_ORACLE_H
#define TSBTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Plummer-softened force, potential and time-step criterion on bodies
 * idx[0..n_act) from all bodies j != i (Sec. 2 Eq. 3, Sec. 3 softening):
 *   a_i   = sum_j m_j d_ij / s^3,  phi_i = -sum_j m_j / s,
 *   q_i   = max_j max(|v_ij|^2 / s^2, m_j / s^3),
 * with d_ij = r_j - r_i and s^2 = |d_ij|^2 + eps^2. The time-step estimate
 * of Eq. 3 is then eta / sqrt(q_i). j runs in ascending order. */
void orc_forces(int64_t n, const double* m, const double* r, const double* v,
                double eps, int64_t n_act, const int32_t* idx,
                double* a, double* phi, double* q);

/* Kinetic and softened potential energy of a state (Sec. 3 energy error). */
void orc_energy_of(int64_t n, const double* m, const double* r,
                   const double* v, double eps, double* ekin, double* epot);

/* Largest power-of-two step 2^-k <= x with k_min <= k <= k_max, in ticks
 * (Eq. 4). Below 2^-k_max it returns 1 tick and increments *underflow. */
int64_t orc_level_ticks(double x, int k_min, int k_max, int64_t* underflow);

/* First-pass (standard block step) choice of the next step. */
int64_t orc_forward_step(int64_t tau, int64_t d, double dts, int k_min,
                         int k_max, int64_t* underflow);

/* Symmetrised choice of the next step (Alg. 1 and its prose), given the
 * start-of-step estimate dts and the previous pass's estimates at the two
 * candidate end times tau + 2d and tau + d. */
int64_t orc_symmetric_step(int64_t tau, int64_t d, double dts, double dte_2d,
                           double dte_d, int k_min, int k_max,
                           int64_t* underflow);

/* Time-symmetric cubic Hermite interpolation between two stored records
 * at ticks ta < tb, evaluated at tick t (ta <= t <= tb). */
void orc_hermite(int64_t ta, int64_t tb, int64_t t, int k_max,
                 const double* ra, const double* va, const double* aa,
                 const double* rb, const double* vb, const double* ab,
                 double* r_out, double* v_out);

/* One body's previous-pass records, given as arrays (tau[len] strictly
 * ascending; r, v, a as (len, 3) rows), for the pins of readings R6 and
 * R8: the index of the last record with tau <= t (-1 if none); the
 * previous pass's step estimate at tick t (the record's on an exact hit,
 * linear in time between two records, `fallback` before the first or
 * after the last); and the prediction of a non-active body to tick tn in a
 * pass >= 1 (the record on an exact hit, cubic Hermite between the
 * bracketing records, else Eq. 2 from its own state rj, vj, aj at tj). */
int64_t orc_hist_find(int64_t len, const int64_t* tau, int64_t t);
double orc_hist_dts_at(int64_t len, const int64_t* tau, const double* dts,
                       int64_t t, double fallback);
void orc_predict_prev(int64_t len, const int64_t* tau, const double* r,
                      const double* v, const double* a, int64_t tj,
                      const double* rj, const double* vj, const double* aj,
                      int64_t tn, int k_max, double* rp, double* vp);

typedef struct {
  int n_iter;        /* passes per era (1 = plain block steps) */
  int era_mode;      /* 0 fixed, 1 dynamic */
  int era_log2;      /* fixed era = 2^-era_log2 time units */
  int k_max;         /* smallest step 2^-k_max; ticks per unit = 2^k_max */
  int dyn_min_log2;  /* dynamic era lower limit = dt_max * 2^-dyn_min_log2 */
  int log;           /* record the block schedule */
  double eps, eta, dt_max;
  double conv_tol;   /* > 0: converged iteration — after pass p >= 1 the
                        era stops when every body's record times equal the
                        previous pass's (same block schedule) and every
                        era-end position differs from the previous pass's
                        by less than conv_tol; n_iter is then the upper
                        bound. 0: always n_iter passes. */
  int64_t trace_body; /* >= 0: record this body's state at every block step
                        of every pass (orc_trace_get); -1: off */
} orc_cfg;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(int64_t n, const double* m, const double* r,
                    const double* v, const orc_cfg* cfg);
/* Integrate whole eras until the system time reaches t_end. Returns 0, or
 * -1 if t_end is not a whole number of ticks or lies in the past. */
int orc_run(orc_sim* s, double t_end);
/* Energy at the system time; bodies behind it are Taylor-predicted (Eq. 2). */
void orc_energy(orc_sim* s, double* ekin, double* epot);
void orc_get_state(orc_sim* s, double* r, double* v, double* a, int64_t* tau,
                   int64_t* dt, double* dts);
/* Replace the state with one that ends an era at system time t (ticks):
 * masses, r, v, a at each body's own time tau, steps dt (ticks) and step
 * estimates dts. Returns 0, or -1 (nothing changed) when the state could not
 * end an era: a step not a power of two in [1, dt_max], tau not a multiple
 * of dt, not tau <= t < tau + dt, a non-finite value, or dts <= 0. */
int orc_set_state(orc_sim* s, int64_t t, const double* m, const double* r,
                  const double* v, const double* a, const int64_t* tau,
                  const int64_t* dt, const double* dts);
/* stats: [0] block steps, [1] interactions (sum n_act * n), [2] eras,
 * [3] passes, [4] step underflows, [5] system time in ticks,
 * [6] initial interactions */
void orc_stats(orc_sim* s, int64_t* out);
int64_t orc_log_steps(orc_sim* s);
int64_t orc_log_entries(orc_sim* s);
/* per block step: era index, pass, tau_next, n_act; per active body, in
 * ascending index within its step: body index and new step in ticks */
void orc_log_get(orc_sim* s, int32_t* step_era, int32_t* step_pass,
                 int64_t* step_tau, int32_t* step_nact, int32_t* ent_i,
                 int64_t* ent_dt);
/* era bounds [tau_s, tau_e] in ticks, in order; returns the era count
 * (pass NULL pointers to query the count) */
int64_t orc_era_log(orc_sim* s, int64_t* tau_s, int64_t* tau_e);
/* The traced body (cfg.trace_body), one entry per block step of every
 * pass: era index, pass, block time (ticks), kind and the state rva = r, v,
 * a (9 doubles). kind 0: the body is not active and (r, v) is the
 * prediction the step's forces used (a unused); kind 1: the body is
 * active and (r, v, a) is its corrected state (Eq. 1). Returns the entry
 * count (pass NULL pointers to query it). */
int64_t orc_trace_get(orc_sim* s, int32_t* era, int32_t* pass, int64_t* tau,
                      int32_t* kind, double* rva);
void orc_destroy(orc_sim* s);
void orc_set_threads(int n);
int orc_get_threads(void);

/* Adjoint of a frozen block schedule (reading R14): the schedule of an
 * era's final pass is replayed with Taylor prediction only, as in a first
 * pass, and differentiated in reverse mode. The schedule is n_steps block
 * steps; step s ends at tick step_tau[s] (strictly increasing) and moves
 * the bodies act[step_off[s] .. step_off[s+1]). Start: (r0, v0) at tick 0
 * with a0 = force on every body at r0. Each step predicts every body with
 * Eq. 2 from its own time, computes the force (Eq. 3 sums) on the active
 * bodies at the predicted positions and corrects them with Eq. 1 over
 * their own step (block time minus their previous time). */

/* Forward replay: final positions and velocities (each body at the time of
 * its last step, or at tick 0 if it never moves). */
void orc_replay(int64_t n, const double* m, const double* r0, const double* v0,
                double eps, int k_max, int64_t n_steps, const int64_t* step_tau,
                const int64_t* step_off, const int32_t* act, double* r_out,
                double* v_out);

/* Reverse mode: given cotangents gr_T, gv_T of the final positions and
 * velocities, the cotangents of r0, v0 and m. Gradients with respect to
 * m are summed over every force evaluation, the initial one included. */
void orc_replay_vjp(int64_t n, const double* m, const double* r0,
                    const double* v0, double eps, int k_max, int64_t n_steps,
                    const int64_t* step_tau, const int64_t* step_off,
                    const int32_t* act, const double* gr_T, const double* gv_T,
                    double* g_r0, double* g_v0, double* g_m);

/* The adjoint through every pass of one era (reading R14 extended to the
 * symmetrised passes): the era's n_pass passes are replayed on their
 * frozen schedules, each from (r0, v0) at tick 0 with a0 = the force at
 * r0, with Eq. 2 prediction in the first pass and for active bodies and
 * the previous pass's records (R6) for the others in passes >= 1, as the
 * integrator runs them. Pass p's steps are pass_off[p] .. pass_off[p+1]-1
 * of step_tau and step_off (entry offsets into act, not restarting per
 * pass). orc_era_replay gives the last pass's final state;
 * orc_era_replay_vjp the cotangents of r0, v0 and m for cotangents gr_T,
 * gv_T of that state, through every pass and its records. */
void orc_era_replay(int64_t n, const double* m, const double* r0,
                    const double* v0, double eps, int k_max, int64_t n_pass,
                    const int64_t* pass_off, const int64_t* step_tau,
                    const int64_t* step_off, const int32_t* act,
                    double* r_out, double* v_out);
void orc_era_replay_vjp(int64_t n, const double* m, const double* r0,
                        const double* v0, double eps, int k_max,
                        int64_t n_pass, const int64_t* pass_off,
                        const int64_t* step_tau, const int64_t* step_off,
                        const int32_t* act, const double* gr_T,
                        const double* gv_T, double* g_r0, double* g_v0,
                        double* g_m);

/* The same era replay from a general era-start state: body j at tick
 * tau0[j] (NULL: all 0) with acceleration a0[j] (NULL: the force at r0),
 * as a later era starts from what the era before it left (Sec. 3: a body
 * whose step overshot the era end waits behind it). The block ticks of
 * every pass exceed every tau0. Outputs (each may be NULL) the last pass's
 * final r, v, a and tick of every body. The _vjp variant takes cotangents
 * of that final r, v, a (each may be NULL for zero) and returns those of
 * r0, v0, m and a0 (g_a0: zero when a0 is NULL, its cotangent then going
 * through the initial force). Chained era by era: the adjoint across eras. */
void orc_era_replay_state(int64_t n, const double* m, const double* r0,
                          const double* v0, const double* a0,
                          const int64_t* tau0, double eps, int k_max,
                          int64_t n_pass, const int64_t* pass_off,
                          const int64_t* step_tau, const int64_t* step_off,
                          const int32_t* act, double* r_out, double* v_out,
                          double* a_out, int64_t* tau_out);
void orc_era_replay_state_vjp(int64_t n, const double* m, const double* r0,
                              const double* v0, const double* a0,
                              const int64_t* tau0, double eps, int k_max,
                              int64_t n_pass, const int64_t* pass_off,
                              const int64_t* step_tau,
                              const int64_t* step_off, const int32_t* act,
                              const double* gr_T, const double* gv_T,
                              const double* ga_T, double* g_r0, double* g_v0,
                              double* g_a0, double* g_m);

/* Mass-weighted mean-square radius about the origin,
 * L = sum_i m_i |r_i|^2 / sum_i m_i, with its partial derivatives with
 * respect to r (g_r) and m (g_m); either may be NULL. */
double orc_loss_msr(int64_t n, const double* m, const double* r, double* g_r,
                    double* g_m);

#ifdef __cplusplus
}
#endif
#endif
