// Launchers of the block-step kernels (k_step.cu) used by the host engine.
#pragma once

#include <climits>

#include "tsbts_internal.cuh"

namespace tsbts {

void launch_pass_begin(Ctl* ctl, long long tau_s, long long tau_e, int pass,
                       int era, int n, cudaStream_t s);
void launch_pass_setup(const Bodies& B, const Params& P, const History& cur,
                       cudaStream_t s);
// pdl: launch with programmatic stream serialization
cudaError_t launch_select_predict(const Bodies& B, const Params& P,
                                  const History& HA, const History& HB, int p,
                                  bool pdl, cudaStream_t s);
cudaError_t launch_correct(const Bodies& B, const Params& P,
                           const History& HA, const History& HB, int p,
                           int grid, bool pdl, cudaStream_t s);
void launch_copy_state(const Bodies& dst, const Bodies& src, cudaStream_t s);
// converged iteration: ctl->notconv |= (this pass differs from the last);
// nrec = records of the running pass, rlast = positions after the last pass
void launch_converged(const Bodies& B, const History& cur,
                      const History& prev, double* const rlast[3], double tol,
                      long long nrec, Ctl* ctl, int sms, cudaStream_t s);
// the running pass's appended records -> previous-pass records in CSR order
void launch_history_to_csr(const Bodies& B, const History& append,
                           const History& csr, const Ctl* ctl, int sms,
                           cudaStream_t s);
void launch_next_time_extrema(const Bodies& B, Ctl* ctl, cudaStream_t s);
void launch_load_aos(const Bodies& B, const double* m, const double* r,
                     const double* v, Ctl* ctl, cudaStream_t s);
void launch_init_jdata(const Bodies& B, const Params& P, cudaStream_t s);
// B.mf from B.m (after the masses change)
void launch_masses_to_float(const Bodies& B, cudaStream_t s);
void launch_init_finalize(const Bodies& B, const Params& P, const int* nsplit,
                          cudaStream_t s);
void launch_energy(const Bodies& B, const Params& P, long long T, double* w,
                   double* out, int sms, cudaStream_t s);
// Eq. 2 prediction of every body to tick T into the FP64 j arrays
void launch_energy_predict(const Bodies& B, const Params& P, long long T,
                           cudaStream_t s);

// ensembles of independent clusters (k_ensemble.cu)
int ens_max_clusters();
ForceLaunch ens_force_launch_shape(int precision, int device);
void launch_ens_pass_begin(const Ens& E, long long tau_s, cudaStream_t s);
// dynamic eras: each cluster's era end from its bodies' next block times
// (Alg. 3), capped at tau_end; *E.undone counts the clusters not yet there
void launch_ens_era(const Bodies& B, const Ens& E, long long dtmax_t,
                    int dyn_min_log2, long long tau_end, cudaStream_t s);
// every cluster's era start becomes its era end
void launch_ens_era_end(const Ens& E, cudaStream_t s);
void launch_ens_pass_setup(const Bodies& B, const Params& P, const Ens& E,
                           const History& cur, cudaStream_t s);
// one global block step (five launches); ev0/ev1 (nullable) bracket the
// force launch
void launch_ens_step(const Bodies& B, const Params& P, const Ens& E,
                     const History& HA, const History& HB,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaEvent_t ev0, cudaEvent_t ev1, unsigned evflags,
                     cudaStream_t s);
void launch_ens_init(const Bodies& B, const Params& P, const Ens& E,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaStream_t s);
void launch_ens_energy(const Bodies& B, const Params& P, const Ens& E,
                       long long T, double* w, double* ek, double* ep,
                       cudaStream_t s);

// ---------------------------------------------------------------------
// Adjoint of a frozen block schedule (k_adjoint.cu).
// ---------------------------------------------------------------------

// replay state of every body, structure of arrays
struct AdjState {
  double* r[3];
  double* v[3];
  double* a[3];
  long long* tau;
};
// cotangents of the replay state and of the masses
struct AdjCot {
  double* gr[3];
  double* gv[3];
  double* ga[3];
  double* gm;
};
// pre-step state of schedule entries base, base + 1, ...: components
// r (0..2), v (3..5), a (6..8); tau == nullptr: no tape
struct AdjTape {
  double* x[9];
  long long* tau;
  long long base;
};
// Eq. 2 prediction of every body to the block time: FP64 positions, and
// for the mixed path the packed j records (p_hi, m) and (p_lo, 0)
struct AdjPred {
  const double* m;
  double* p[3];
  float4* jhi;
  float4* jlo;
};
// the active bodies of the step being reversed, by slot k (their order in
// the schedule): the force cotangent lam, the cotangent gp0 of the new
// position, the predicted position (FP64 ap; mixed ahi/alo) and lam in
// FP32 (alam); slot[j] is body j's slot, -1 if it is not active
struct AdjSlots {
  double* lam[3];
  double* gp0[3];
  double* ap[3];
  float4* ahi;
  float4* alo;
  float4* alam;
  int* slot;
};
// work split of one side of the force vector-Jacobian product: `tpt`
// threads per target (a power of two <= 8), 128 / tpt targets per block,
// S splits of `chunk` sources, `groups` target groups
struct VjpSide {
  int tpt, S, chunk, groups;
};
// i side: targets are the active bodies, sources every body; j side:
// targets every body, sources the active bodies
struct VjpShape {
  VjpSide si, sj;
};
VjpShape vjp_shape(int n, int n_act, int sms);
// results of one force vector-Jacobian product: u[3] per active slot (i
// side) and G[3], Z per body in g[4] (j side); split partials and the
// per-group completion counters (zero between launches)
struct VjpOut {
  double* u[3];
  double* g[4];
  double* f[3];  // replay force sums per active slot
  double* part_i;
  double* part_j;
  int* cnt_i;
  int* cnt_j;
};
// the end of a reverse step (Eq. 2 adjoint of every body, with the force
// cotangents of its VjpOut) and the start of the step before it (tape
// restore, Eq. 1 adjoint, prediction); either may be inactive
struct AdjBackFin {
  int active;
  long long T;
  AdjSlots Sl;
};
struct AdjBackPrep {
  int active;
  int all;  // every body active at T = 0: the initial force
  long long T;
  long long e_lo;
  AdjSlots Sl;
};
// Records of an era's passes (adjoint through every pass, Sec. 2): the
// position and velocity of each schedule entry's body after its step,
// their cotangents, the block tick of every entry and the entry links. A
// body's era-start state (r0, v0 at tick tau0) is its first record in
// every pass.
// kind/ra/rb: how each body that is not active was placed at the step
// being reversed (0: Eq. 2 from its own state; 1: record ra; 2: cubic
// Hermite between records ra and rb; ra = -1 is the era-start record).
struct AdjRecs {
  double* r[3];
  double* v[3];
  double* gr[3];
  double* gv[3];
  const long long* tau;
  const long long* tau0;  // era-start tick of each body
  const long long* next_e;
  const long long* prev_e;
  const double* r0[3];
  const double* v0[3];
  int* kind;
  long long* ra;
  long long* rb;
};
// The pass being replayed or reversed. on: it has a previous pass Q
// (entries [lo, hi); first[j]: body j's first entry in Q, LLONG_MAX if
// none), whose records place the bodies that are not active at a step;
// cur[j]: body j's last record in Q at or before the current block tick
// (-1: the era-start record); g0r/g0v: the cotangents of Q's era-start
// records. write: the pass's entries write their records (a pass follows
// it); inject: in reverse, an entry's record cotangent joins the
// cotangent of the body's state after that step.
struct AdjPass {
  int on, write, inject;
  long long lo, hi;
  const long long* first;
  long long* cur;
  double* g0r[3];
  double* g0v[3];
};

// the era-start state: (m, r, v) at tick 0 (a_in, tau_in nullptr; the
// initial force follows) or a general state with accelerations and ticks
void launch_adj_load(int n, const double* m_in, const double* r_in,
                     const double* v_in, const double* a_in,
                     const long long* tau_in, int mixed, double* m_out,
                     const AdjState& St, const AdjPred& P, int* err,
                     cudaStream_t s);
// initial accelerations from the force partials, then the prediction to
// T_next (< 0: none)
// (fsum[0] != nullptr: the accelerations are fsum, else the force
// kernel's split partials)
void launch_adj_init_accel(int n, const double* part, const int* nsplit,
                           double* const fsum[3], long long T_next,
                           double inv_ticks, int mixed, const AdjState& St,
                           const AdjPred& P, int* err, cudaStream_t s);
// prediction of every body to tick T; in a pass with a previous pass (Q.on)
// the bodies not active at T (fwd_e[j] >= e_hi) are placed from Q's records
void launch_adj_predict(int n, long long T, double inv_ticks, int mixed,
                        const AdjState& St, const AdjPred& P,
                        const long long* fwd_e, long long e_hi,
                        const AdjRecs& R, const AdjPass& Q, cudaStream_t s);
// Eq. 1 for the bodies of schedule entries [e_lo, e_hi) (fwd_e: each
// body's next entry; their records written when Q.write), then the
// prediction of every body to T_next (active there: entries below
// e_hi_next)
void launch_adj_correct_predict(int n, int n_act, long long T, long long e_lo,
                                long long e_hi, long long T_next,
                                long long e_hi_next, double inv_ticks,
                                int mixed, const double* part,
                                const int* nsplit, double* const fsum[3],
                                const AdjState& St, const AdjPred& P,
                                const AdjTape& Tp, long long* fwd_e,
                                const long long* next_e, const AdjRecs& R,
                                const AdjPass& Q, int* err, cudaStream_t s);
// mixed replay force on the active bodies idx[0..n_act) into O.f (the i
// side's work split)
void launch_adj_force(int n, int n_act, const int* idx, double eps2,
                      const AdjPred& P, const VjpSide& si, const VjpOut& O,
                      cudaStream_t s);
void launch_adj_back_step(int n, double inv_ticks, int mixed,
                          const AdjBackFin& F, const AdjBackPrep& R,
                          const AdjState& St, const AdjTape& Tp,
                          long long* cur_e, const long long* prev_e,
                          const AdjCot& C, const AdjPred& P, const VjpOut& O,
                          const AdjRecs& Rc, const AdjPass& Q, int* err,
                          cudaStream_t s);
// end of one pass's reverse sweep: G0 += the cotangents of the state (and
// of the pass's era-start records g0r/g0v, which are then cleared); the
// state's cotangents become G0 when `last` (the first pass) else zero
void launch_adj_pass_end(int n, const AdjCot& C, const AdjCot& G0,
                         double* const g0r[3], double* const g0v[3], int last,
                         cudaStream_t s);
void launch_adj_vjp(int mixed, int n, int n_act, const int* idx, double eps2,
                    const AdjPred& P, const AdjSlots& Sl, const VjpShape& V,
                    const VjpOut& O, cudaStream_t s);
// L = sum m |r|^2 / sum m into out[0] (out[1] = sum m) and the cotangent
// seeds dL/dr, dL/dm (velocity and acceleration cotangents zero)
void launch_adj_loss(int n, const double* m, const AdjState& St, double* out,
                     const AdjCot& C, cudaStream_t s);
// seeds from (n, 3) cotangents of the final r, v and a (nullable: zero)
void launch_adj_seed(int n, const double* gr, const double* gv,
                     const double* ga, const AdjCot& C, cudaStream_t s);
// three structure-of-arrays components -> row-major (n, 3)
void launch_soa_to_aos(int n, double* const src[3], double* dst,
                       cudaStream_t s);

}  // namespace tsbts
