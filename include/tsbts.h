/*
 * tsbts.h - C ABI of the GB300 (sm_103a) library for the era-based
 * time-symmetric block time-step (TSBTS) N-body integrator of Kaplan &
 * Saygin ("A Dynamic Era-Based Time-Symmetric Block Time-Step Algorithm
 * with Parallel Implementations"), Sec. 2-4.
 *
 * Conventions shared by every entry point:
 *  - Units: G = 1. Times are doubles in N-body time units; internally
 *    every time is an integer tick count, 2^k_max ticks per time unit.
 *  - Vectors are row-major (n, 3) float64 arrays: x, y, z per body.
 *  - Inputs are copied; the library never frees caller memory and keeps
 *    no pointer to it after the call returns.
 *  - Every call returns a tsbts_status. No C++ exception and no CUDA error
 *    crosses this boundary. After TSBTS_ERR_CUDA, TSBTS_ERR_NONFINITE or
 *    TSBTS_ERR_TIMEOUT a context is poisoned: further calls on it return
 *    TSBTS_ERR_STATE until tsbts_destroy. tsbts_last_error gives a message.
 *  - A context is used by one host thread at a time.
 *  - The library has no CPU fallback: without a usable CUDA device,
 *    tsbts_create returns TSBTS_ERR_CUDA.
 */
#ifndef TSBTS_H
#define TSBTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSBTS_OK = 0,
  TSBTS_ERR_ARG = -1,        /* invalid argument; nothing was changed */
  TSBTS_ERR_CUDA = -2,       /* CUDA runtime error (context poisoned) */
  TSBTS_ERR_NONFINITE = -3,  /* non-finite input or force (poisoned) */
  TSBTS_ERR_TIMEOUT = -4,    /* a bounded device wait gave up (poisoned) */
  TSBTS_ERR_HISTORY = -6,    /* era history could not grow (no memory) */
  TSBTS_ERR_STATE = -7       /* call out of order, or context poisoned */
} tsbts_status;

typedef enum { TSBTS_FP64 = 0, TSBTS_MIXED = 1 } tsbts_precision;

/* Integrator settings (Sec. 3 "era size", Sec. 4 Alg. 3, Sec. 2 Alg. 2).
 * tsbts_config_default fills the defaults listed beside each field. */
typedef struct {
  int precision;     /* tsbts_precision; default TSBTS_FP64.
                        FP64: all pairwise arithmetic in FP64, rounded op by
                        op in the order of the plain definition.
                        MIXED: FP32 pairwise terms on double-single (hi+lo)
                        relative coordinates, compensated FP32 sums folded
                        per j-tile; FP64 positions, velocities, times and
                        energy. */
  int n_iter;        /* passes per era (Alg. 2 "iteration limit"); 1 = plain
                        block steps; default 3 */
  int era_mode;      /* 0 = fixed era (Sec. 3), 1 = dynamic era (Alg. 3:
                        last minus first next block time, clamped to
                        [dt_max 2^-dyn_min_log2, dt_max], rounded up to a
                        power of two); default 0 */
  int era_log2;      /* fixed era = 2^-era_log2 time units, 0..k_max;
                        default 3 */
  int dyn_min_log2;  /* dynamic era lower limit = dt_max * 2^-dyn_min_log2;
                        default 3 (Sec. 4 uses 2^-3 of the largest step) */
  int k_max;         /* smallest step 2^-k_max, 1..40; default 20 */
  int exact_order;   /* FP64 only: 1 = every force sum runs over j in
                        ascending order in one thread (bit-identical to a
                        sequential FP64 loop, slow for small active sets);
                        0 = j-split across thread blocks with a fixed-order
                        second stage (deterministic, different rounding);
                        -1 = automatic: exact when n <= 8192. Default -1 */
  int device;        /* CUDA device ordinal; default 0 */
  void* stream;      /* cudaStream_t to run on, or NULL for a private
                        stream owned by the context; default NULL */
  int graph_steps;   /* block steps per captured CUDA graph launch; 0 = plain
                        stream launches; default 32 */
  double conv_tol;   /* converged iteration (0 = off, the paper's fixed
                        pass count): after pass p >= 1 an era stops early
                        when pass p took the same block steps as pass p - 1
                        (every body's record times equal) and every body's
                        position at the end of the pass is within conv_tol
                        of pass p - 1's; n_iter still bounds the passes.
                        Single systems only; default 0 */
  int64_t max_pass_steps; /* watchdog: a pass that takes more block steps
                        than this stops with TSBTS_ERR_TIMEOUT (0 = the
                        bound no working step loop can exceed: one step per
                        tick of the era); default 0 */
} tsbts_config;

typedef struct tsbts_ctx tsbts_ctx;

/* Counters of one context since tsbts_init. */
typedef struct {
  int64_t block_steps;    /* block steps over all passes */
  int64_t interactions;   /* sum over block steps of n_act * n (the pairs
                             evaluated, self pairs counted) */
  int64_t eras;
  int64_t passes;
  int64_t dt_underflow;   /* steps clamped up to 2^-k_max */
  int64_t era_restarts;   /* eras re-run after the history buffer grew */
  int64_t history_capacity; /* records per pass buffer */
  int64_t t_sys_ticks;    /* system time in ticks */
  double force_ms;        /* device time in the force kernel, summed over
                             the timed launches (tsbts_set_timing), else 0 */
  int64_t force_launches;   /* force launches timed */
  int64_t kernel_launches;  /* kernels of this library launched by the
                               context since tsbts_init */
  int64_t force_interactions; /* interactions (n_act * n) of the block
                                 steps whose force launch was timed */
} tsbts_stats;

void tsbts_config_default(tsbts_config* cfg);

/* Create a context on cfg->device. Returns TSBTS_ERR_ARG for a bad config,
 * TSBTS_ERR_CUDA if the device cannot be used. *out is NULL on error. */
int tsbts_create(tsbts_ctx** out, const tsbts_config* cfg);

/* Alg. 2 step 1: read the bodies, compute all forces and the first steps.
 * m[n], r[n*3], v[n*3] are HOST pointers and are copied. eps >= 0 is the
 * Plummer softening length (Sec. 3), eta > 0 the accuracy parameter of
 * Eq. 3, dt_max = 2^-k (0 <= k <= k_max) the largest step. Sets the system
 * time to 0. TSBTS_ERR_ARG: n < 1, a bad parameter, or dt_max not a power
 * of two in range; TSBTS_ERR_NONFINITE: a non-finite input. */
int tsbts_init(tsbts_ctx* ctx, int64_t n, const double* m, const double* r,
               const double* v, double eps, double eta, double dt_max);

/* Same as tsbts_init with DEVICE pointers (read on the context's stream
 * before the call returns). */
int tsbts_init_device(tsbts_ctx* ctx, int64_t n, const double* m_dev,
                      const double* r_dev, const double* v_dev, double eps,
                      double eta, double dt_max);

/* Alg. 2 step 1 for an ensemble of independent clusters integrated
 * together (the batched form of the method; each cluster is its own
 * N-body system with its own block times and its own softening). Cluster
 * c owns bodies offsets[c] .. offsets[c+1]-1 of the HOST arrays m[n],
 * r[n*3], v[n*3] (n = offsets[n_clusters], offsets[0] = 0, every cluster
 * non-empty, 1 <= n_clusters <= 4096); eps[n_clusters] its softening
 * lengths. eta and dt_max as in tsbts_init. With a fixed era (era_mode
 * 0) tsbts_step_era advances every cluster over the same eras; with the
 * dynamic era (era_mode 1) every cluster takes its own eras (Alg. 3 on its
 * own bodies, as a lone run of that cluster would), and tsbts_step_era
 * returns once every cluster has reached t_end. tsbts_state returns all
 * bodies; tsbts_energy returns the sums over the clusters; the schedule log
 * is not recorded; converged iteration (conv_tol > 0) is refused. */
int tsbts_init_ensemble(tsbts_ctx* ctx, int64_t n_clusters,
                        const int64_t* offsets, const double* m,
                        const double* r, const double* v, const double* eps,
                        double eta, double dt_max);

/* Per-cluster kinetic and potential energy of an ensemble at the system
 * time (HOST arrays of n_clusters doubles, each may be NULL). */
int tsbts_ensemble_energy(tsbts_ctx* ctx, double* ekin, double* epot);

/* Alg. 2 steps 2-11 (Alg. 3 for the dynamic era): integrate whole eras,
 * each with n_iter passes, until the system time reaches t_end. t_end must
 * be a whole number of ticks and not before the system time
 * (TSBTS_ERR_ARG). The last era ends at t_end. *t_reached (may be NULL)
 * receives the new system time. Bodies whose step overshoots an era end
 * wait for a later era (Sec. 4), so body times may lag the system time.
 * TSBTS_ERR_NONFINITE: a force or step estimate became non-finite;
 * TSBTS_ERR_TIMEOUT: a pass stopped advancing the block time or took more
 * block steps than config.max_pass_steps (both poison the context). */
int tsbts_step_era(tsbts_ctx* ctx, double t_end, double* t_reached);

/* Kinetic, softened potential and total energy at the system time (the
 * relative energy error of Sec. 3 is formed from these). Bodies behind the
 * system time are predicted with Eq. 2. Always FP64; the pair sum for each
 * body runs in ascending j and the body sums in ascending i. */
int tsbts_energy(tsbts_ctx* ctx, double* ekin, double* epot, double* etot);

/* Copy the state to HOST buffers (each may be NULL): *t system time;
 * m[n]; r, v, a [n*3] at each body's own time; tau_ticks[n] body times;
 * dt_ticks[n] current steps. */
int tsbts_state(tsbts_ctx* ctx, double* t, double* m, double* r, double* v,
                double* a, int64_t* tau_ticks, int64_t* dt_ticks);

/* Copy each body's step estimate (Eq. 3 with Plummer softening: eta over
 * the square root of the time-step criterion, at the body's own time) to
 * the HOST array dts[n]. With tsbts_state it forms a checkpoint. */
int tsbts_step_estimates(tsbts_ctx* ctx, double* dts);

/* Resume at an era end (Alg. 2 steps 2 and 10: an era starts from the
 * bodies' m, r, v, a, step estimates, times and steps and the system time
 * alone; its first pass uses Eq. 2 and later passes only records of the
 * same era). HOST arrays as tsbts_state writes them, plus dts[n] from
 * tsbts_step_estimates; t is the system time (a whole number of ticks).
 * The context must hold a single system initialised with the same n;
 * eps, eta and dt_max stay. A state saved at an era end of a run with the
 * same configuration continues bit for bit like the uninterrupted run.
 * TSBTS_ERR_ARG (nothing changed) unless every dt is a power of two in
 * [1, dt_max] ticks, every tau a multiple of its dt with tau <= t <
 * tau + dt, every value finite and every dts > 0 (+inf allowed);
 * TSBTS_ERR_STATE for an ensemble. The arrays are read before the call
 * returns. */
int tsbts_set_state(tsbts_ctx* ctx, double t, const double* m,
                    const double* r, const double* v, const double* a,
                    const int64_t* tau_ticks, const int64_t* dt_ticks,
                    const double* dts);

int tsbts_get_stats(tsbts_ctx* ctx, tsbts_stats* out);

/* Time force launches with CUDA events around them; the sums appear in
 * tsbts_stats (force_ms, force_launches, force_interactions). period = 0:
 * off; 1: every block step; k > 1: the block steps of every k-th chunk of
 * steps (one graph replay or stream batch), a sample that keeps the cost
 * of the events (which also serialise the step's launches) to about 1/k.
 * TSBTS_ERR_ARG for period < 0. */
int tsbts_set_timing(tsbts_ctx* ctx, int period);

/* Record the block schedule of the following calls: per block step the
 * era index, pass, block time and active count, and per active body its
 * index and new step. capacity_entries bounds the body entries (steps are
 * bounded by the same number); 0 disables. Entries beyond capacity are
 * dropped and counted. Active bodies of one step may be stored in any
 * order. */
int tsbts_schedule_log(tsbts_ctx* ctx, int64_t capacity_entries);
/* Sizes of the recorded log; dropped counts entries that did not fit. */
int tsbts_schedule_size(tsbts_ctx* ctx, int64_t* steps, int64_t* entries,
                        int64_t* dropped);
/* Copy the log to HOST arrays sized from tsbts_schedule_size. */
int tsbts_schedule_get(tsbts_ctx* ctx, int32_t* step_era, int32_t* step_pass,
                       int64_t* step_tau, int32_t* step_nact, int32_t* ent_i,
                       int64_t* ent_dt);

const char* tsbts_last_error(const tsbts_ctx* ctx);
void tsbts_destroy(tsbts_ctx* ctx);

/* Alg. 2 step 5 on its own (Sec. 2 Eq. 3, Sec. 3 softening): for each
 * active body i = idx[k], k < n_act,
 *   a[k]   = sum_{j != i} m_j d_ij / s^3,
 *   phi[k] = -sum_{j != i} m_j / s,
 *   q[k]   = max_{j != i} max(|v_ij|^2 / s^2, m_j / s^3),
 * with d_ij = r_j - r_i, v_ij = v_j - v_i, s^2 = |d_ij|^2 + eps^2; the step
 * estimate of Eq. 3 is eta / sqrt(q). All pointers are DEVICE pointers:
 * m[n], r[n*3], v[n*3], idx[n_act] (int32, each in [0, n), repeats
 * allowed), outputs a[n_act*3], phi[n_act], q[n_act] (caller-allocated).
 * precision is a tsbts_precision; exact_order as in tsbts_config (FP64).
 * Runs on `stream` (cudaStream_t, NULL = legacy default stream) and is
 * asynchronous: outputs are ready when the stream reaches this point.
 * Scratch memory (packed j records and j-split partial sums) is allocated
 * by the library on first use per device, grown as needed and kept until
 * tsbts_release_scratch. TSBTS_ERR_ARG: n < 1, n_act < 0, n or n_act above
 * 2^31 - 1, or eps < 0. */
int tsbts_force(int precision, int exact_order, int64_t n, const double* m,
                const double* r, const double* v, double eps, int64_t n_act,
                const int32_t* idx, double* a, double* phi, double* q,
                void* stream);

/* Free the scratch memory of tsbts_force on the current device. */
int tsbts_release_scratch(void);

/* tsbts_force for callers that cannot allocate device memory: code whose
 * device memory is managed entirely by someone else (a framework allocator
 * that has reserved the device, a fixed real-time budget) and code that must
 * not call cudaMalloc or cudaFree because those calls can synchronise the
 * device. The paper has no counterpart; this is a property of the library.
 *
 * Same arguments, results and tolerances as tsbts_force: DEVICE pointers
 * m[n], r[n*3], v[n*3], idx[n_act] (int32, each value in [0, n); the
 * library does not check them), a[n_act*3], phi[n_act], q[n_act] (the FP64
 * path with ascending-j sums gives identical results; other paths may
 * round differently because the work plan is chosen without
 * measurement). It
 * allocates nothing and calls no allocating routine: its scratch (packed j
 * records and j-split partial sums) is a fixed array of about 9 MB inside
 * the library that every GPU loading the library holds until the process
 * exits. Limits: n <= 65536 and n_act <= 65536, else TSBTS_ERR_ARG.
 * The first call on a device looks up the array's device address; make
 * that first call before any stream capture. Every call on a device shares
 * the one array, so calls that overlap on the GPU (different streams or
 * threads without ordering) race and give wrong results; each call writes
 * all the scratch it reads, so nothing needs clearing between calls. */
int tsbts_force_static(int precision, int exact_order, int64_t n,
                       const double* m, const double* r, const double* v,
                       double eps, int64_t n_act, const int32_t* idx,
                       double* a, double* phi, double* q, void* stream);

/* ---------------------------------------------------------------------
 * Adjoint of a frozen block schedule.
 *
 * The paper defines no adjoint; this is the reading taken here. The
 * gradient of a function of the bodies' final state with respect to their
 * initial positions, velocities and masses is taken through one era's
 * final-pass block schedule (tsbts_adjoint_init), or through all its
 * passes (tsbts_adjoint_init_era), replayed as plain block steps: every
 * body is predicted to the block time (with Eq. 2 from its own time; in a
 * later pass of an era from the previous pass's records), the active
 * bodies get the force sums of Eq. 3 at the predicted positions and are
 * corrected with Eq. 1 over their own step. The schedule (block times and
 * active sets) is held fixed and is not differentiated; the step criterion
 * plays no part. Reverse mode runs the chain rule step by step backwards,
 * with the force's vector-Jacobian product computed by dedicated kernels.
 *
 * A context that holds an adjoint may also hold an integrator (tsbts_init)
 * or an ensemble; they share only the device, the stream and the precision.
 * --------------------------------------------------------------------- */

typedef struct {
  int64_t steps;               /* block steps of the schedule */
  int64_t entries;             /* sum of the active counts */
  int64_t checkpoint_every;    /* 0: the whole schedule is taped */
  int64_t checkpoints;         /* full-state checkpoints held */
  int64_t tape_entries;        /* pre-step records the tape holds */
  int64_t tape_bytes;          /* device bytes of the tape */
  int64_t checkpoint_bytes;    /* device bytes of the checkpoints */
  int64_t device_bytes;        /* all device memory of the adjoint */
  int64_t pairs_forward;       /* pair terms of the last forward call */
  int64_t pairs_backward;      /* pair terms of the last reverse sweep
                                  (force VJP both ends, plus recomputed
                                  forward steps) */
  double forward_ms;           /* device time of the last forward call */
  double backward_ms;          /* device time of the last reverse sweep */
  int64_t kernel_launches;     /* kernels launched by the adjoint */
  int64_t passes;              /* passes of the era replayed */
} tsbts_adjoint_stats;

/* Set up the adjoint of a schedule over n bodies with softening eps >= 0.
 * The schedule is n_steps block steps in HOST arrays: step s ends at tick
 * step_tau[s] (2^k_max ticks per time unit, strictly increasing, > 0) and
 * moves the bodies act[step_off[s] .. step_off[s+1]) (step_off[0] = 0,
 * every step non-empty, each body at most once per step, each in [0, n)).
 * Arrays are copied. checkpoint_every = 0 tapes the pre-step state of
 * every entry during the forward replay (80 bytes per entry); K > 0 keeps
 * only a full-state checkpoint every K steps (88 bytes per body each) and
 * recomputes each K-step segment, taped, during the reverse sweep.
 * Precision, k_max, exact_order, device and stream come from the context's
 * config; with graph_steps > 0 the whole forward replay and the whole
 * reverse sweep are each captured once as a CUDA graph (on the first call)
 * and replayed, with graph_steps = 0 every kernel is a stream launch.
 * TSBTS_ERR_ARG: a bad size or schedule. */
int tsbts_adjoint_init(tsbts_ctx* ctx, int64_t n, double eps,
                       int64_t n_steps, const int64_t* step_tau,
                       const int64_t* step_off, const int32_t* act,
                       int64_t checkpoint_every);

/* Adjoint through every pass of one era (Sec. 2, Alg. 2: each pass after
 * the first places a body that is not active at a block time from the
 * previous pass's records: the record itself on an exact hit, else the
 * cubic Hermite between the two records that bracket the block time, else,
 * past the body's last record, Eq. 2 from its own state). A body's records
 * of a pass are its era-start state and its state after each of its steps
 * in that pass.
 *
 * n_pass >= 1 passes; pass p is steps pass_off[p] .. pass_off[p+1] - 1
 * (pass_off[0] = 0; with n_pass > 1 every pass has at least one step).
 * step_tau, step_off and act hold every step of every pass in order, in
 * the layout of tsbts_adjoint_init (step_off runs on across the passes);
 * the ticks increase from > 0 within each pass, since each pass restarts
 * from the era start at tick 0. The forward replay returns the last pass's
 * final state; reverse mode differentiates through every pass, the
 * cotangent of an interpolated position passing to the records it came
 * from with the Hermite weights. Memory beyond tsbts_adjoint_init: 104
 * bytes per entry of every pass but the last (records, their cotangents
 * and ticks), 16 bytes per body per pass for the record bookkeeping, and
 * a final state per pass when nothing is checkpointed; checkpointed
 * segments (checkpoint_every) stay within one pass. n_pass = 1 is
 * tsbts_adjoint_init. TSBTS_ERR_ARG: a bad size or schedule. */
int tsbts_adjoint_init_era(tsbts_ctx* ctx, int64_t n, double eps,
                           int64_t n_pass, const int64_t* pass_off,
                           const int64_t* step_tau, const int64_t* step_off,
                           const int32_t* act, int64_t checkpoint_every);

/* Forward replay from masses m[n], positions r0[n*3] and velocities
 * v0[n*3] at tick 0 (initial accelerations: the force on every body at
 * r0). r_T, v_T [n*3] (each may be NULL) receive each body's final state,
 * at the time of its last step (tick 0 if it never moves). device_ptrs = 1:
 * every pointer is a DEVICE pointer on the context's device, read and
 * written in order on the context's stream; 0: HOST pointers. The call
 * returns when the results are written. The inputs are kept for
 * tsbts_adjoint_vjp. TSBTS_ERR_NONFINITE: non-finite input or force. */
int tsbts_adjoint_forward(tsbts_ctx* ctx, const double* m, const double* r0,
                          const double* v0, double* r_T, double* v_T,
                          int device_ptrs);

/* Reverse mode of the last forward replay: given the cotangents gr_T, gv_T
 * [n*3] of the final positions and velocities (either may be NULL for
 * zero), writes g_r0, g_v0 [n*3] and g_m [n] (each may be NULL), the
 * cotangents of r0, v0 and m; the mass cotangent sums every force
 * evaluation, the initial one included. Pointers as in
 * tsbts_adjoint_forward. TSBTS_ERR_STATE: no forward replay yet. */
int tsbts_adjoint_vjp(tsbts_ctx* ctx, const double* gr_T, const double* gv_T,
                      double* g_r0, double* g_v0, double* g_m,
                      int device_ptrs);

/* Forward replay from a general era-start state, for the adjoint across
 * eras: a later era starts from the state the era before it left, each
 * body at its own tick tau0[j] (a body whose step overshot the era end
 * waits behind it, Sec. 3) with the acceleration a0[n*3] of its last
 * correction. a0 = NULL (and tau0 = NULL) is tsbts_adjoint_forward: tick
 * 0 and a0 the force at r0; tau0 = NULL with a0 given: every body at tick
 * 0. Every tau0 must be >= 0 and below every pass's first block tick
 * (TSBTS_ERR_ARG). Outputs the final r_T, v_T, a_T [n*3] and ticks
 * tau_T[n] (each may be NULL), the input state of the next era. Pointers
 * as in tsbts_adjoint_forward. */
int tsbts_adjoint_forward_state(tsbts_ctx* ctx, const double* m,
                                const double* r0, const double* v0,
                                const double* a0, const int64_t* tau0,
                                double* r_T, double* v_T, double* a_T,
                                int64_t* tau_T, int device_ptrs);

/* Reverse mode of the last forward replay with cotangents of the final
 * r, v and a (each may be NULL for zero): writes the cotangents of r0, v0,
 * a0 and m (each may be NULL). After a replay from a general start state
 * g_a0 is the start accelerations' cotangent (and no initial force is
 * differentiated); after one from tick 0 it is zero, a0 being the force
 * at r0. Chaining this era by era, last to first, each era's (g_r0, g_v0,
 * g_a0) being the previous era's (gr_T, gv_T, ga_T) and the g_m summed,
 * differentiates across eras. TSBTS_ERR_STATE: no forward replay yet. */
int tsbts_adjoint_vjp_state(tsbts_ctx* ctx, const double* gr_T,
                            const double* gv_T, const double* ga_T,
                            double* g_r0, double* g_v0, double* g_a0,
                            double* g_m, int device_ptrs);

/* Forward replay and reverse mode of the loss
 *   L = sum_i m_i |r_i(T)|^2 / sum_i m_i
 * (the mass-weighted mean-square radius about the origin of the final
 * positions): *loss and the gradients g_r0, g_v0 [n*3], g_m [n] (each may
 * be NULL; dL/dm includes the loss's own dependence on m). Pointers as in
 * tsbts_adjoint_forward (with device_ptrs = 1, loss is a device double). */
int tsbts_adjoint_loss_grad(tsbts_ctx* ctx, const double* m, const double* r0,
                            const double* v0, double* loss, double* g_r0,
                            double* g_v0, double* g_m, int device_ptrs);

int tsbts_adjoint_get_stats(tsbts_ctx* ctx, tsbts_adjoint_stats* out);

/* Measured throughput of one execution pipe of the current device, the
 * denominator of the force kernels' rooflines (the pair term of Eq. 3 is
 * bound by the FMA pipe, not by the tensor cores or memory). kind:
 *   0 = FP32 fma (1 FMA-pipe op per lane and instruction),
 *   1 = packed FP32 fma.f32x2 (2 ops per lane and instruction),
 *   2 = FP64 fma, 3 = FP32 rsqrt (special-function unit).
 * Every thread of an 8-blocks-per-SM grid runs 8 independent chains of
 * `iters` operations (1 <= iters <= 2^30); one warm-up launch, then one
 * launch timed with CUDA events on the legacy default stream. Writes lane
 * operations per second to *ops_per_s and the timed launch's duration to
 * *ms (may be NULL). Allocates 4 bytes of device memory for the call.
 * TSBTS_ERR_ARG: bad kind, iters or null output. */
int tsbts_pipe_peak(int kind, int64_t iters, double* ops_per_s, double* ms);

/* Library version string. */
const char* tsbts_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSBTS_H */
