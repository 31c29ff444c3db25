// Host side of the adjoint of a frozen block schedule (include/tsbts.h,
// tsbts_adjoint_*): schedule validation and bookkeeping, device memory,
// the forward replay and the reverse sweep with optional checkpointing.
//
// The schedule is known on the host, so every launch's active count, force
// plan and vector-Jacobian work split is fixed when the adjoint is set up;
// no step reads its size back from the device.
//
// Memory: full-state arrays of n bodies, a tape of the pre-step state of
// schedule entries (all of them, or one checkpointed segment), and
// full-state checkpoints every K steps. With checkpointing the reverse
// sweep recomputes each segment's forward steps from its checkpoint.
//
// Several passes of one era are one schedule whose entries run on across
// the passes (each body's entry links too); every pass restarts from the
// era-start state. Every pass but the last also keeps its records (each
// entry's post-step position and velocity) and their cotangents, which the
// next pass's predictions and their reverse mode use; checkpointed
// segments stay within one pass.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"

namespace tsbts {

struct AdjCtx {
  int n = 0;
  double eps = 0;
  int mixed = 0;
  int exact = 0;
  int k_max = 20;
  double inv_ticks = 0;
  long long S = 0;  // steps
  long long E = 0;  // entries
  long long K = 0;  // checkpoint every K steps (0: tape everything)
  long long n_ckpt = 0;
  long long tape_cap = 0;
  long long n_pass = 1;
  std::vector<long long> tau, off;
  std::vector<long long> pass_off;  // first step of each pass, then S
  // checkpointed segments [seg0, seg1) of pass seg_pass; ckpt_of[s]: the
  // segment that starts at step s, else -1
  std::vector<long long> seg0, seg1, seg_pass, ckpt_of;
  // several passes: records of every pass but the last (E_rec entries),
  // each body's first and last entry in those passes ((n_pass - 1) x n),
  // the forward and reverse record cursors, the era-start cotangents of
  // two consecutive passes (g0[p & 1]: r then v), their sum G0 over the
  // passes, the era-start state and each pass's final state (taped mode)
  long long E_rec = 0;
  AdjRecs Rc{};
  long long* q_first = nullptr;
  long long* q_last = nullptr;
  long long* qf = nullptr;
  long long* qr = nullptr;
  double* g0[2][6] = {};
  double* g0_block = nullptr;
  double* G0_block = nullptr;
  double* grec_block = nullptr;
  AdjCot G0{};
  AdjState St0{};
  std::vector<AdjState> fins;
  std::vector<long long*> ckpt_qf;
  std::vector<Plan> plans;      // forward force plan per step
  std::vector<VjpShape> shapes; // reverse work split per step
  VjpShape shape_init{};
  Plan plan_init{};
  ForceLaunch fl{};
  std::vector<void*> allocs;
  long long bytes = 0, tape_bytes = 0, ckpt_bytes = 0;
  // device
  int* act = nullptr;           // E
  long long* prev_e = nullptr;  // E: the same body's previous entry or -1
  long long* next_e = nullptr;  // E: its next entry, or LLONG_MAX
  long long* last_e = nullptr;  // n: each body's last entry or -1
  long long* first_e = nullptr; // n: each body's first entry or LLONG_MAX
  long long* cur_e = nullptr;   // n: reverse cursor
  long long* fwd_e = nullptr;   // n: forward cursor
  int* iota = nullptr;          // n
  double* m = nullptr;
  double* io = nullptr;         // 10 n doubles: host inputs / outputs
  long long* tau_io = nullptr;  // n ticks: host start / final ticks
  // the last forward replay started from a general state (r, v, a, tick)
  // instead of (r, v) at tick 0 with the initial force
  int state_mode = 0;
  long long first_tick = LLONG_MAX;  // smallest first block tick of a pass
  AdjState St{};
  std::vector<AdjState> ckpt;
  std::vector<long long*> ckpt_fwd;  // forward cursor at each checkpoint
  AdjState fin{};  // final state of the forward replay (taped mode)
  AdjTape Tp{};
  AdjPred P{};
  AdjSlots Sl[2]{};  // slots of even and odd steps (step -1: initial)
  VjpOut O{};
  AdjCot C{};
  float4* jv = nullptr;         // zero velocities for the force kernel
  double* part = nullptr;
  long long part_cap = 0;
  int* nsplit = nullptr;
  int* err = nullptr;
  double* loss = nullptr;       // L, sum m
  bool have_forward = false;
  // statistics
  long long pairs_fwd = 0, pairs_bwd = 0, launches = 0;
  double fwd_ms = 0, bwd_ms = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // captured forward replay [0] and reverse sweep [1], from tick 0 (+0) or
  // from a general start state (+2), and their kernels
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  long long graph_kernels[4] = {0, 0, 0, 0};
};

}  // namespace tsbts

namespace {

template <class T>
T* adj_alloc(AdjCtx& A, size_t count) {
  A.bytes += (long long)(sizeof(T) * (count ? count : 1));
  return dalloc<T>(A.allocs, count);
}

AdjState alloc_state(AdjCtx& A, int n) {
  AdjState s{};
  for (int c = 0; c < 3; ++c) {
    s.r[c] = adj_alloc<double>(A, n);
    s.v[c] = adj_alloc<double>(A, n);
    s.a[c] = adj_alloc<double>(A, n);
  }
  s.tau = adj_alloc<long long>(A, n);
  return s;
}

void copy_state(const AdjState& dst, const AdjState& src, int n,
                cudaStream_t s) {
  const size_t b = sizeof(double) * (size_t)n;
  for (int c = 0; c < 3; ++c) {
    ck(cudaMemcpyAsync(dst.r[c], src.r[c], b, cudaMemcpyDeviceToDevice, s),
       "checkpoint copy");
    ck(cudaMemcpyAsync(dst.v[c], src.v[c], b, cudaMemcpyDeviceToDevice, s),
       "checkpoint copy");
    ck(cudaMemcpyAsync(dst.a[c], src.a[c], b, cudaMemcpyDeviceToDevice, s),
       "checkpoint copy");
  }
  ck(cudaMemcpyAsync(dst.tau, src.tau, sizeof(long long) * (size_t)n,
                     cudaMemcpyDeviceToDevice, s),
     "checkpoint copy");
}

void adj_free(tsbts_ctx* c) {
  if (!c->adj) return;
  if (c->s) cudaStreamSynchronize(c->s);
  for (cudaGraphExec_t g : c->adj->graph)
    if (g) cudaGraphExecDestroy(g);
  free_list(c->adj->allocs);
  for (cudaEvent_t e : c->adj->ev)
    if (e) cudaEventDestroy(e);
  delete c->adj;
  c->adj = nullptr;
}

int adj_ready(tsbts_ctx* c) {
  if (!c) return TSBTS_ERR_ARG;
  if (c->poisoned) return fail(c, TSBTS_ERR_STATE, "context is poisoned");
  if (!c->adj) return fail(c, TSBTS_ERR_STATE, "tsbts_adjoint_init not called");
  return TSBTS_OK;
}

ForceArgs force_args(const AdjCtx& A) {
  ForceArgs fa{};
  fa.n = A.n;
  fa.m = A.m;
  for (int d = 0; d < 3; ++d) {
    fa.x[d] = A.P.p[d];
    fa.w[d] = A.St.v[d];  // the step criterion is not used
  }
  fa.jhi = A.P.jhi;
  fa.jlo = A.P.jlo;
  fa.jv = A.jv;
  fa.nsplit_out = A.nsplit;
  fa.part = A.part;
  fa.part_cap = A.part_cap;
  fa.eps2 = A.eps * A.eps;
  fa.eps2f = (float)(A.eps * A.eps);
  fa.exact = A.exact;
  fa.has_plan = 1;
  return fa;
}

// the force on the active bodies of a step: the lean mixed replay kernel
// (sums into A.O.f), or the integrator's FP64 force kernel (ascending-j
// sums in exact mode; partials summed by the correction kernel)
void launch_step_force(tsbts_ctx* c, AdjCtx& A, const int* idx, int n_act,
                       const Plan& plan, const VjpSide& si) {
  if (A.mixed) {
    launch_adj_force(A.n, n_act, idx, A.eps * A.eps, A.P, si, A.O, c->s);
    return;
  }
  ForceArgs fa = force_args(A);
  fa.idx = idx;
  fa.n_act_fixed = n_act;
  fa.plan = plan;
  ck(launch_force(A.mixed, fa, A.fl, c->s), "replay force");
}

// accelerations of the force launch: A.O.f (mixed) or none (partials)
double* const* fsum_of(AdjCtx& A) {
  static double* const none[3] = {nullptr, nullptr, nullptr};
  return A.mixed ? A.O.f : none;
}

// plans of the FP64 force kernel for every step (the mixed replay uses its
// own kernel and the reverse sweep's work splits)
void choose_plans(tsbts_ctx* c, AdjCtx& A) {
  (void)c;
  A.plan_init = plan_force(A.mixed, A.exact, A.n, A.n, A.fl.grid, A.part_cap);
  for (long long s = 0; s < A.S; ++s)
    A.plans[s] = plan_force(A.mixed, A.exact, (int)(A.off[s + 1] - A.off[s]),
                            A.n, A.fl.grid, A.part_cap);
}

// The pass p seen by the kernels, with record cursor `cur` (forward or
// reverse); all off for a lone pass.
AdjPass pass_desc(const AdjCtx& A, long long p, long long* cur) {
  AdjPass Q{};
  if (A.n_pass == 1) return Q;
  Q.write = Q.inject = p + 1 < A.n_pass;
  Q.cur = cur;
  if (p > 0) {
    Q.on = 1;
    Q.lo = A.off[A.pass_off[p - 1]];
    Q.hi = A.off[A.pass_off[p]];
    Q.first = A.q_first + (p - 1) * (long long)A.n;
    for (int c = 0; c < 3; ++c) {
      Q.g0r[c] = A.g0[(p - 1) & 1][c];
      Q.g0v[c] = A.g0[(p - 1) & 1][3 + c];
    }
  }
  return Q;
}

// Replay steps [s0, s1) of pass p from the current state (bodies already
// predicted to the block time of step s0); with a tape, record the
// pre-step state of their entries. With save_ckpt, the checkpoint of a
// segment (state, entry and record cursors) is saved before its first step.
void replay_steps(tsbts_ctx* c, AdjCtx& A, long long s0, long long s1,
                  const AdjTape& tape, bool save_ckpt, long long p) {
  const AdjPass Q = pass_desc(A, p, A.qf);
  const size_t nb = sizeof(long long) * (size_t)A.n;
  for (long long s = s0; s < s1; ++s) {
    if (save_ckpt && A.K > 0 && A.ckpt_of[s] >= 0) {
      const long long g = A.ckpt_of[s];
      copy_state(A.ckpt[g], A.St, A.n, c->s);
      ck(cudaMemcpyAsync(A.ckpt_fwd[g], A.fwd_e, nb,
                         cudaMemcpyDeviceToDevice, c->s),
         "checkpoint copy");
      if (A.n_pass > 1)
        ck(cudaMemcpyAsync(A.ckpt_qf[g], A.qf, nb, cudaMemcpyDeviceToDevice,
                           c->s),
           "checkpoint copy");
    }
    const long long T = A.tau[s];
    const int na = (int)(A.off[s + 1] - A.off[s]);
    launch_step_force(c, A, A.act + A.off[s], na, A.plans[s], A.shapes[s].si);
    const bool more = s + 1 < s1;
    launch_adj_correct_predict(A.n, na, T, A.off[s], A.off[s + 1],
                               more ? A.tau[s + 1] : -1,
                               more ? A.off[s + 2] : 0, A.inv_ticks, A.mixed,
                               A.part, A.nsplit, fsum_of(A), A.St, A.P, tape,
                               A.fwd_e, A.next_e, A.Rc, Q, A.err, c->s);
    A.launches += 2;
  }
  ck(cudaGetLastError(), "replay launches");
}

// prediction of every body to the block time of step s of pass p
void predict_to(tsbts_ctx* c, AdjCtx& A, long long s, long long p) {
  launch_adj_predict(A.n, A.tau[s], A.inv_ticks, A.mixed, A.St, A.P, A.fwd_e,
                     A.off[s + 1], A.Rc, pass_desc(A, p, A.qf), c->s);
  A.launches += 1;
}

AdjBackPrep start_of(const AdjCtx& A, long long s) {
  AdjBackPrep R{};
  R.active = 1;
  if (s < 0) {  // the initial force
    R.all = 1;
    R.T = 0;
    R.e_lo = 0;
    R.Sl = A.Sl[1];
  } else {
    R.T = A.tau[s];
    R.e_lo = A.off[s];
    R.Sl = A.Sl[s & 1];
  }
  return R;
}

AdjBackFin end_of(const AdjCtx& A, long long s) {
  AdjBackFin F{};
  F.active = 1;
  F.T = s < 0 ? 0 : A.tau[s];
  F.Sl = A.Sl[s < 0 ? 1 : (s & 1)];
  return F;
}

void back_step(tsbts_ctx* c, AdjCtx& A, const AdjBackFin& F,
               const AdjBackPrep& R, const AdjPass& Q) {
  launch_adj_back_step(A.n, A.inv_ticks, A.mixed, F, R, A.St, A.Tp, A.cur_e,
                       A.prev_e, A.C, A.P, A.O, A.Rc, Q, A.err, c->s);
  A.launches += 1;
}

void vjp_of(tsbts_ctx* c, AdjCtx& A, long long s) {
  const double eps2 = A.eps * A.eps;
  if (s < 0)
    launch_adj_vjp(A.mixed, A.n, A.n, A.iota, eps2, A.P, A.Sl[1],
                   A.shape_init, A.O, c->s);
  else
    launch_adj_vjp(A.mixed, A.n, (int)(A.off[s + 1] - A.off[s]),
                   A.act + A.off[s], eps2, A.P, A.Sl[s & 1], A.shapes[s], A.O,
                   c->s);
  A.launches += 1;
}

// Reverse steps s1 - 1 down to s0 of pass p, whose tape is loaded; step
// s0 - 1 is started too when it needs no tape (a lone pass's initial force,
// s0 = 0).
void reverse_steps(tsbts_ctx* c, AdjCtx& A, long long s1, long long s0,
                   long long p) {
  const AdjBackFin none_f{};
  AdjBackPrep none_r{};
  const AdjPass Q = pass_desc(A, p, A.qr);
  back_step(c, A, none_f, start_of(A, s1 - 1), Q);
  for (long long s = s1 - 1; s >= s0; --s) {
    vjp_of(c, A, s);
    // (a lone pass from tick 0: the initial force is started here)
    const bool before =
        s > s0 || (s0 == 0 && A.n_pass == 1 && !A.state_mode);
    back_step(c, A, end_of(A, s), before ? start_of(A, s - 1) : none_r, Q);
  }
  ck(cudaGetLastError(), "reverse launches");
}

void check_err(tsbts_ctx* c, AdjCtx& A, const char* what, int* rc) {
  int e = 0;
  ck(cudaMemcpyAsync(&e, A.err, sizeof e, cudaMemcpyDeviceToHost, c->s),
     "read error flag");
  ck(cudaStreamSynchronize(c->s), "synchronize");
  if (e) *rc = fail(c, TSBTS_ERR_NONFINITE, what);
}

// All work of the forward replay, inputs read from A.io (m, r0, v0, and in
// state mode a0) and A.tau_io (state mode: tau0).
void enqueue_forward(tsbts_ctx* c, AdjCtx& A) {
  const size_t n = (size_t)A.n;
  const bool st = A.state_mode != 0;
  launch_adj_load(A.n, A.io, A.io + n, A.io + 4 * n, st ? A.io + 7 * n : nullptr,
                  st ? A.tau_io : nullptr, A.mixed, A.m, A.St, A.P, A.err,
                  c->s);
  ck(cudaMemcpyAsync(A.fwd_e, A.first_e, sizeof(long long) * n,
                     cudaMemcpyDeviceToDevice, c->s),
     "copy entry cursors");
  A.launches += 1;
  if (!st) {
    // the initial force, then the prediction to the first block time
    launch_step_force(c, A, A.iota, A.n, A.plan_init, A.shape_init.si);
    launch_adj_init_accel(A.n, A.part, A.nsplit, fsum_of(A),
                          A.S > 0 ? A.tau[0] : -1, A.inv_ticks, A.mixed,
                          A.St, A.P, A.err, c->s);
    A.launches += 2;
  } else if (A.S > 0) {
    predict_to(c, A, 0, 0);
  }
  if (A.n_pass > 1) copy_state(A.St0, A.St, A.n, c->s);
  AdjTape none{};
  for (long long p = 0; p < A.n_pass; ++p) {
    const long long s0 = A.pass_off[p], s1 = A.pass_off[p + 1];
    if (p > 0) {
      // every pass starts from the era-start state, its record cursors at
      // the era-start records
      copy_state(A.St, A.St0, A.n, c->s);
      ck(cudaMemsetAsync(A.qf, 0xFF, sizeof(long long) * n, c->s),
         "memset");
      predict_to(c, A, s0, p);
    }
    replay_steps(c, A, s0, s1, A.K == 0 ? A.Tp : none, true, p);
    if (A.K == 0 && p + 1 < A.n_pass) copy_state(A.fins[p], A.St, A.n, c->s);
  }
  // the taped reverse sweep starts from the final state; keep it so that
  // every sweep of this forward replay can start there
  if (A.K == 0) copy_state(A.fin, A.St, A.n, c->s);
}

// All work of the reverse sweep, from the seeds already in A.C.
void enqueue_backward(tsbts_ctx* c, AdjCtx& A) {
  const size_t nb = sizeof(long long) * (size_t)A.n;
  ck(cudaMemcpyAsync(A.cur_e, A.last_e, nb, cudaMemcpyDeviceToDevice, c->s),
     "copy entry cursors");
  const bool multi = A.n_pass > 1;
  if (multi) {
    ck(cudaMemsetAsync(A.G0_block, 0, sizeof(double) * 9 * (size_t)A.n, c->s),
       "memset");
    ck(cudaMemsetAsync(A.g0_block, 0, sizeof(double) * 12 * (size_t)A.n,
                       c->s),
       "memset");
    ck(cudaMemsetAsync(A.grec_block, 0,
                       sizeof(double) * 6 * (size_t)std::max(A.E_rec, 1LL),
                       c->s),
       "memset");
  }
  for (long long p = A.n_pass - 1; p >= 0; --p) {
    const long long s0 = A.pass_off[p], s1 = A.pass_off[p + 1];
    if (p > 0)
      ck(cudaMemcpyAsync(A.qr, A.q_last + (p - 1) * (long long)A.n, nb,
                         cudaMemcpyDeviceToDevice, c->s),
         "copy record cursors");
    if (A.K == 0) {
      copy_state(A.St, p + 1 == A.n_pass ? A.fin : A.fins[p], A.n, c->s);
      reverse_steps(c, A, s1, s0, p);
    } else {
      for (long long g = A.n_ckpt - 1; g >= 0; --g) {
        if (A.seg_pass[g] != p) continue;
        const long long t0 = A.seg0[g], t1 = A.seg1[g];
        copy_state(A.St, A.ckpt[g], A.n, c->s);
        ck(cudaMemcpyAsync(A.fwd_e, A.ckpt_fwd[g], nb,
                           cudaMemcpyDeviceToDevice, c->s),
           "checkpoint copy");
        if (multi)
          ck(cudaMemcpyAsync(A.qf, A.ckpt_qf[g], nb, cudaMemcpyDeviceToDevice,
                             c->s),
             "checkpoint copy");
        predict_to(c, A, t0, p);
        AdjTape tape = A.Tp;
        tape.base = A.off[t0];
        replay_steps(c, A, t0, t1, tape, false, p);
        A.Tp.base = tape.base;
        reverse_steps(c, A, t1, t0, p);
      }
      A.Tp.base = 0;
    }
    if (multi) {
      launch_adj_pass_end(A.n, A.C, A.G0, A.g0[p & 1], A.g0[p & 1] + 3,
                          p == 0, c->s);
      A.launches += 1;
    }
  }
  // the initial force a0 = f(r0) (a lone pass's last reverse step has
  // started it); from a general start state the cotangents of (r0, v0, a0)
  // are those of the state now
  if (!A.state_mode) {
    const AdjPass lone{};
    if (multi) back_step(c, A, AdjBackFin{}, start_of(A, -1), lone);
    vjp_of(c, A, -1);
    back_step(c, A, end_of(A, -1), AdjBackPrep{}, lone);
  }
  ck(cudaGetLastError(), "reverse launches");
}

// Run the work of `enq` on the stream: directly (graph_steps == 0), or by
// replaying its CUDA graph, captured at the first call (the schedule, the
// plans and every buffer address are fixed for the life of the adjoint).
void run_work(tsbts_ctx* c, AdjCtx& A, int which,
              void (*enq)(tsbts_ctx*, AdjCtx&)) {
  if (c->cfg.graph_steps == 0) {
    enq(c, A);
    return;
  }
  which += 2 * A.state_mode;
  cudaGraphExec_t& exec = A.graph[which];
  if (!exec) {
    const long long l0 = A.launches;
    cudaGraph_t g;
    ck(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal),
       "begin capture");
    try {
      enq(c, A);
    } catch (...) {
      cudaStreamEndCapture(c->s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    ck(cudaStreamEndCapture(c->s, &g), "end capture");
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    ck(e, "graph instantiate");
    A.graph_kernels[which] = A.launches - l0;
    A.launches = l0;
  }
  ck(cudaGraphLaunch(exec, c->s), "graph launch");
  A.launches += A.graph_kernels[which];
}

int forward_impl(tsbts_ctx* c, AdjCtx& A) {
  ck(cudaMemsetAsync(A.err, 0, sizeof(int), c->s), "memset");
  ck(cudaEventRecord(A.ev[0], c->s), "event");
  run_work(c, A, 0, enqueue_forward);
  ck(cudaEventRecord(A.ev[1], c->s), "event");
  int rc = TSBTS_OK;
  check_err(c, A, "non-finite input or force in the replay", &rc);
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, A.ev[0], A.ev[1]), "event time");
  A.fwd_ms = ms;
  A.pairs_fwd = (A.E + A.n) * (long long)A.n;
  A.have_forward = rc == TSBTS_OK;
  return rc;
}

int backward_impl(tsbts_ctx* c, AdjCtx& A) {
  ck(cudaMemsetAsync(A.err, 0, sizeof(int), c->s), "memset");
  ck(cudaEventRecord(A.ev[0], c->s), "event");
  run_work(c, A, 1, enqueue_backward);
  ck(cudaEventRecord(A.ev[1], c->s), "event");
  int rc = TSBTS_OK;
  check_err(c, A, "non-finite cotangent in the reverse sweep", &rc);
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, A.ev[0], A.ev[1]), "event time");
  A.bwd_ms = ms;
  // two-sided force VJP of every step and of the initial force, plus the
  // forward steps recomputed from checkpoints
  A.pairs_bwd = 2 * (A.E + A.n) * (long long)A.n +
                (A.K > 0 ? A.E * (long long)A.n : 0);
  return rc;
}

void to_out(tsbts_ctx* c, AdjCtx& A, double* const src[3], double* dst,
            bool dev) {
  if (!dst) return;
  double* d = dev ? dst : A.io;
  launch_soa_to_aos(A.n, src, d, c->s);
  A.launches += 1;
  if (!dev)
    ck(cudaMemcpyAsync(dst, A.io, sizeof(double) * 3 * (size_t)A.n,
                       cudaMemcpyDeviceToHost, c->s),
       "copy out");
  ck(cudaStreamSynchronize(c->s), "synchronize");
}

// inputs into A.io (m, r0, v0, a0) and A.tau_io (tau0), from host or
// device arrays; the replay always reads them there, so a captured graph
// serves every call
void stage_in(tsbts_ctx* c, AdjCtx& A, const double* m, const double* r,
              const double* v, const double* a, const long long* tau,
              bool dev) {
  const size_t n = (size_t)A.n;
  const cudaMemcpyKind kind =
      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ck(cudaMemcpyAsync(A.io, m, sizeof(double) * n, kind, c->s), "copy m");
  ck(cudaMemcpyAsync(A.io + n, r, sizeof(double) * 3 * n, kind, c->s),
     "copy r");
  ck(cudaMemcpyAsync(A.io + 4 * n, v, sizeof(double) * 3 * n, kind, c->s),
     "copy v");
  if (a)
    ck(cudaMemcpyAsync(A.io + 7 * n, a, sizeof(double) * 3 * n, kind, c->s),
       "copy a");
  if (a && tau)
    ck(cudaMemcpyAsync(A.tau_io, tau, sizeof(long long) * n, kind, c->s),
       "copy tau");
  else if (a)
    ck(cudaMemsetAsync(A.tau_io, 0, sizeof(long long) * n, c->s), "memset");
}

// Records of every pass but the last, and the bookkeeping of the passes
// (several passes only).
void setup_records(tsbts_ctx* ctx, AdjCtx& A, const int32_t* act) {
  const int ni = A.n;
  const long long nq = A.n_pass - 1;
  A.E_rec = A.off[A.pass_off[nq]];
  std::vector<long long> first((size_t)(nq * ni), LLONG_MAX),
      last((size_t)(nq * ni), -1), tau((size_t)std::max(A.E_rec, 1LL), 0);
  for (long long p = 0; p < nq; ++p)
    for (long long s = A.pass_off[p]; s < A.pass_off[p + 1]; ++s)
      for (long long e = A.off[s]; e < A.off[s + 1]; ++e) {
        const long long k = p * ni + act[e];
        if (first[k] == LLONG_MAX) first[k] = e;
        last[k] = e;
        tau[e] = A.tau[s];
      }
  const size_t er = (size_t)std::max(A.E_rec, 1LL);
  A.q_first = adj_alloc<long long>(A, first.size());
  A.q_last = adj_alloc<long long>(A, last.size());
  long long* ent_tau = adj_alloc<long long>(A, er);
  ck(cudaMemcpyAsync(A.q_first, first.data(), sizeof(long long) * first.size(),
                     cudaMemcpyHostToDevice, ctx->s),
     "copy schedule");
  ck(cudaMemcpyAsync(A.q_last, last.data(), sizeof(long long) * last.size(),
                     cudaMemcpyHostToDevice, ctx->s),
     "copy schedule");
  ck(cudaMemcpyAsync(ent_tau, tau.data(), sizeof(long long) * er,
                     cudaMemcpyHostToDevice, ctx->s),
     "copy schedule");
  A.qf = adj_alloc<long long>(A, ni);
  A.qr = adj_alloc<long long>(A, ni);
  A.St0 = alloc_state(A, ni);
  AdjRecs& R = A.Rc;
  double* rv = adj_alloc<double>(A, 6 * er);
  A.grec_block = adj_alloc<double>(A, 6 * er);
  for (int c = 0; c < 3; ++c) {
    R.r[c] = rv + c * er;
    R.v[c] = rv + (3 + c) * er;
    R.gr[c] = A.grec_block + c * er;
    R.gv[c] = A.grec_block + (3 + c) * er;
    R.r0[c] = A.St0.r[c];
    R.v0[c] = A.St0.v[c];
  }
  R.tau = ent_tau;
  R.tau0 = A.St0.tau;
  R.next_e = A.next_e;
  R.prev_e = A.prev_e;
  R.kind = adj_alloc<int>(A, ni);
  R.ra = adj_alloc<long long>(A, ni);
  R.rb = adj_alloc<long long>(A, ni);
  A.g0_block = adj_alloc<double>(A, 12 * (size_t)ni);
  for (int k = 0; k < 2; ++k)
    for (int c = 0; c < 6; ++c) A.g0[k][c] = A.g0_block + (6 * k + c) * (size_t)ni;
  A.G0_block = adj_alloc<double>(A, 9 * (size_t)ni);
  for (int c = 0; c < 3; ++c) {
    A.G0.gr[c] = A.G0_block + c * (size_t)ni;
    A.G0.gv[c] = A.G0_block + (3 + c) * (size_t)ni;
    A.G0.ga[c] = A.G0_block + (6 + c) * (size_t)ni;
  }
}

}  // namespace

void adjoint_release(tsbts_ctx* c) { adj_free(c); }

namespace {

// Set-up of the adjoint of n_pass passes (pass p: steps pass_off[p] ..
// pass_off[p + 1]) of one schedule (tsbts_adjoint_init_era).
int adjoint_init(tsbts_ctx* ctx, int64_t n, double eps, int64_t n_pass,
                 const int64_t* pass_off, const int64_t* step_tau,
                 const int64_t* step_off, const int32_t* act,
                 int64_t checkpoint_every) {
  if (!ctx) return TSBTS_ERR_ARG;
  if (ctx->poisoned) return fail(ctx, TSBTS_ERR_STATE, "context is poisoned");
  if (n < 1 || n > (1LL << 24))
    return fail(ctx, TSBTS_ERR_ARG, "n must be in [1, 2^24]");
  if (!(eps >= 0.0) || !std::isfinite(eps))
    return fail(ctx, TSBTS_ERR_ARG, "eps must be finite and >= 0");
  if (n_pass < 1 || !pass_off)
    return fail(ctx, TSBTS_ERR_ARG, "n_pass must be >= 1 with pass offsets");
  if (pass_off[0] != 0)
    return fail(ctx, TSBTS_ERR_ARG, "pass_off[0] must be 0");
  for (int64_t p = 0; p < n_pass; ++p)
    if (pass_off[p + 1] < pass_off[p] + (n_pass > 1 ? 1 : 0))
      return fail(ctx, TSBTS_ERR_ARG,
                  n_pass > 1 ? "every pass needs at least one step"
                             : "negative step count");
  const int64_t n_steps = pass_off[n_pass];
  if (checkpoint_every < 0)
    return fail(ctx, TSBTS_ERR_ARG, "negative checkpoint count");
  if (n_steps > 0 && (!step_tau || !step_off || !act))
    return fail(ctx, TSBTS_ERR_ARG, "null schedule array");
  if (n_steps > 0 && step_off[0] != 0)
    return fail(ctx, TSBTS_ERR_ARG, "step_off[0] must be 0");
  // validate the schedule: increasing ticks, non-empty steps, bodies in
  // range and distinct within a step
  // (within each pass, which restarts at the era start)
  std::vector<long long> stamp((size_t)n, -1);
  for (int64_t p = 0, s = 0; s < n_steps; ++s) {
    while (s >= pass_off[p + 1]) ++p;
    if (step_tau[s] <= (s > pass_off[p] ? step_tau[s - 1] : 0))
      return fail(ctx, TSBTS_ERR_ARG, "block ticks must increase from > 0");
    if (step_tau[s] > (1LL << 62))
      return fail(ctx, TSBTS_ERR_ARG, "block tick out of range");
    const int64_t na = step_off[s + 1] - step_off[s];
    if (na < 1 || na > n)
      return fail(ctx, TSBTS_ERR_ARG,
                  "step " + std::to_string(s) + " has a bad active count");
    for (int64_t e = step_off[s]; e < step_off[s + 1]; ++e) {
      const int32_t i = act[e];
      if (i < 0 || i >= n)
        return fail(ctx, TSBTS_ERR_ARG, "body index out of range");
      if (stamp[i] == s)
        return fail(ctx, TSBTS_ERR_ARG, "body repeated within a step");
      stamp[i] = s;
    }
  }
  const long long E = n_steps ? step_off[n_steps] : 0;
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    adj_free(ctx);
    ctx->adj = new AdjCtx;
    AdjCtx& A = *ctx->adj;
    A.n = (int)n;
    A.eps = eps;
    A.mixed = ctx->cfg.precision == TSBTS_MIXED;
    A.exact = !A.mixed && (ctx->cfg.exact_order == 1 ||
                           (ctx->cfg.exact_order < 0 && n <= 8192));
    A.k_max = ctx->cfg.k_max;
    A.inv_ticks = std::ldexp(1.0, -ctx->cfg.k_max);
    A.S = n_steps;
    A.E = E;
    A.K = checkpoint_every >= n_steps ? 0 : checkpoint_every;
    A.n_pass = n_pass;
    A.pass_off.assign(pass_off, pass_off + n_pass + 1);
    A.tau.assign(step_tau, step_tau + n_steps);
    A.off.assign(step_off, step_off + n_steps + 1);
    if (n_steps == 0) A.off.assign(1, 0);
    A.fl = force_launch_shape(A.mixed, ctx->cfg.device);
    // entry links: the same body's previous and next entries, and each
    // body's first and last entries
    const size_t e1 = (size_t)std::max<long long>(E, 1);
    std::vector<long long> prev(e1, -1), next(e1, LLONG_MAX),
        last((size_t)n, -1), first((size_t)n, LLONG_MAX);
    for (long long e = 0; e < E; ++e) {
      const int i = act[e];
      prev[e] = last[i];
      if (last[i] >= 0) next[last[i]] = e;
      if (first[i] == LLONG_MAX) first[i] = e;
      last[i] = e;
    }
    const int ni = (int)n;
    A.act = adj_alloc<int>(A, E);
    A.prev_e = adj_alloc<long long>(A, E);
    A.next_e = adj_alloc<long long>(A, E);
    A.last_e = adj_alloc<long long>(A, ni);
    A.first_e = adj_alloc<long long>(A, ni);
    A.cur_e = adj_alloc<long long>(A, ni);
    A.fwd_e = adj_alloc<long long>(A, ni);
    A.iota = adj_alloc<int>(A, ni);
    std::vector<int> iota(ni);
    for (int k = 0; k < ni; ++k) iota[k] = k;
    if (E) {
      ck(cudaMemcpyAsync(A.act, act, sizeof(int) * E, cudaMemcpyHostToDevice,
                         ctx->s), "copy schedule");
      ck(cudaMemcpyAsync(A.prev_e, prev.data(), sizeof(long long) * E,
                         cudaMemcpyHostToDevice, ctx->s), "copy schedule");
      ck(cudaMemcpyAsync(A.next_e, next.data(), sizeof(long long) * E,
                         cudaMemcpyHostToDevice, ctx->s), "copy schedule");
    }
    ck(cudaMemcpyAsync(A.last_e, last.data(), sizeof(long long) * ni,
                       cudaMemcpyHostToDevice, ctx->s), "copy schedule");
    ck(cudaMemcpyAsync(A.first_e, first.data(), sizeof(long long) * ni,
                       cudaMemcpyHostToDevice, ctx->s), "copy schedule");
    ck(cudaMemcpyAsync(A.iota, iota.data(), sizeof(int) * ni,
                       cudaMemcpyHostToDevice, ctx->s), "copy iota");
    A.m = adj_alloc<double>(A, ni);
    A.io = adj_alloc<double>(A, 10 * (size_t)ni);
    A.tau_io = adj_alloc<long long>(A, ni);
    for (long long p = 0; p < n_pass; ++p)
      if (A.pass_off[p + 1] > A.pass_off[p])
        A.first_tick = std::min(A.first_tick, A.tau[A.pass_off[p]]);
    A.St = alloc_state(A, ni);
    for (int c = 0; c < 3; ++c) {
      A.P.p[c] = adj_alloc<double>(A, ni);
      A.C.gr[c] = adj_alloc<double>(A, ni);
      A.C.gv[c] = adj_alloc<double>(A, ni);
      A.C.ga[c] = adj_alloc<double>(A, ni);
      A.O.u[c] = adj_alloc<double>(A, ni);
    }
    for (int c = 0; c < 4; ++c) A.O.g[c] = adj_alloc<double>(A, ni);
    for (int c = 0; c < 3; ++c) A.O.f[c] = adj_alloc<double>(A, ni);
    for (AdjSlots& Sl : A.Sl) {
      for (int c = 0; c < 3; ++c) {
        Sl.lam[c] = adj_alloc<double>(A, ni);
        Sl.gp0[c] = adj_alloc<double>(A, ni);
        Sl.ap[c] = adj_alloc<double>(A, ni);
      }
      Sl.ahi = adj_alloc<float4>(A, ni);
      Sl.alo = adj_alloc<float4>(A, ni);
      Sl.alam = adj_alloc<float4>(A, ni);
      Sl.slot = adj_alloc<int>(A, ni);
    }
    A.P.m = A.m;
    A.C.gm = adj_alloc<double>(A, ni);
    A.P.jhi = adj_alloc<float4>(A, ni);
    A.P.jlo = adj_alloc<float4>(A, ni);
    A.jv = adj_alloc<float4>(A, ni);
    ck(cudaMemsetAsync(A.jv, 0, sizeof(float4) * ni, ctx->s), "memset");
    A.part_cap = std::max<long long>(A.fl.part_cap, 5LL * ni);
    A.part = adj_alloc<double>(A, A.part_cap);
    A.nsplit = adj_alloc<int>(A, 1);
    A.err = adj_alloc<int>(A, 1);
    A.loss = adj_alloc<double>(A, 2);
    // tape: every entry, or the largest checkpointed segment (segments of
    // K steps within each pass)
    const long long before_tape = A.bytes;
    if (A.K == 0) {
      A.tape_cap = E;
    } else {
      A.ckpt_of.assign((size_t)A.S, -1);
      for (long long p = 0; p < A.n_pass; ++p)
        for (long long s0 = A.pass_off[p]; s0 < A.pass_off[p + 1];
             s0 += A.K) {
          const long long s1 = std::min(A.pass_off[p + 1], s0 + A.K);
          A.ckpt_of[s0] = (long long)A.seg0.size();
          A.seg0.push_back(s0);
          A.seg1.push_back(s1);
          A.seg_pass.push_back(p);
          A.tape_cap = std::max(A.tape_cap, A.off[s1] - A.off[s0]);
        }
      A.n_ckpt = (long long)A.seg0.size();
    }
    for (int k = 0; k < 9; ++k) A.Tp.x[k] = adj_alloc<double>(A, A.tape_cap);
    A.Tp.tau = adj_alloc<long long>(A, A.tape_cap);
    A.Tp.base = 0;
    A.tape_bytes = A.bytes - before_tape;
    const long long before_ckpt = A.bytes;
    for (long long g = 0; g < A.n_ckpt; ++g) {
      A.ckpt.push_back(alloc_state(A, ni));
      A.ckpt_fwd.push_back(adj_alloc<long long>(A, ni));
      if (A.n_pass > 1) A.ckpt_qf.push_back(adj_alloc<long long>(A, ni));
    }
    if (A.K == 0) {
      A.fin = alloc_state(A, ni);
      for (long long p = 0; p + 1 < A.n_pass; ++p)
        A.fins.push_back(alloc_state(A, ni));
    }
    A.ckpt_bytes = A.bytes - before_ckpt;
    if (A.n_pass > 1) setup_records(ctx, A, act);
    // reverse work splits and their partial-sum buffers
    A.shapes.resize(A.S);
    A.plans.resize(A.S);
    long long cap_i = 0, cap_j = 0, grp_i = 0, grp_j = 0;
    auto need = [&](const VjpShape& v) {
      cap_i = std::max(cap_i, (long long)v.si.groups * v.si.S * 4 * 128 /
                                  v.si.tpt);
      cap_j = std::max(cap_j, (long long)v.sj.groups * v.sj.S * 4 * 128 /
                                  v.sj.tpt);
      grp_i = std::max<long long>(grp_i, v.si.groups);
      grp_j = std::max<long long>(grp_j, v.sj.groups);
    };
    A.shape_init = vjp_shape(ni, ni, ctx->sms);
    need(A.shape_init);
    for (long long s = 0; s < A.S; ++s) {
      const int na = (int)(A.off[s + 1] - A.off[s]);
      A.shapes[s] = vjp_shape(ni, na, ctx->sms);
      need(A.shapes[s]);
    }
    A.O.part_i = adj_alloc<double>(A, cap_i);
    A.O.part_j = adj_alloc<double>(A, cap_j);
    A.O.cnt_i = adj_alloc<int>(A, grp_i);
    A.O.cnt_j = adj_alloc<int>(A, grp_j);
    ck(cudaMemsetAsync(A.O.cnt_i, 0, sizeof(int) * grp_i, ctx->s), "memset");
    ck(cudaMemsetAsync(A.O.cnt_j, 0, sizeof(int) * grp_j, ctx->s), "memset");
    choose_plans(ctx, A);
    ck(cudaEventCreate(&A.ev[0]), "event");
    ck(cudaEventCreate(&A.ev[1]), "event");
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  } catch (const std::bad_alloc&) {
    return fail(ctx, TSBTS_ERR_CUDA, "host out of memory");
  }
}

}  // namespace

extern "C" {

int tsbts_adjoint_init(tsbts_ctx* ctx, int64_t n, double eps, int64_t n_steps,
                       const int64_t* step_tau, const int64_t* step_off,
                       const int32_t* act, int64_t checkpoint_every) {
  if (ctx && n_steps < 0)
    return fail(ctx, TSBTS_ERR_ARG, "negative step or checkpoint count");
  const int64_t pass_off[2] = {0, n_steps};
  return adjoint_init(ctx, n, eps, 1, pass_off, step_tau, step_off, act,
                      checkpoint_every);
}

int tsbts_adjoint_init_era(tsbts_ctx* ctx, int64_t n, double eps,
                           int64_t n_pass, const int64_t* pass_off,
                           const int64_t* step_tau, const int64_t* step_off,
                           const int32_t* act, int64_t checkpoint_every) {
  return adjoint_init(ctx, n, eps, n_pass, pass_off, step_tau, step_off, act,
                      checkpoint_every);
}

int tsbts_adjoint_forward_state(tsbts_ctx* ctx, const double* m,
                                const double* r0, const double* v0,
                                const double* a0, const int64_t* tau0,
                                double* r_T, double* v_T, double* a_T,
                                int64_t* tau_T, int device_ptrs) {
  int rc = adj_ready(ctx);
  if (rc) return rc;
  if (!m || !r0 || !v0) return fail(ctx, TSBTS_ERR_ARG, "null input pointer");
  if (tau0 && !a0)
    return fail(ctx, TSBTS_ERR_ARG, "start ticks need start accelerations");
  AdjCtx& A = *ctx->adj;
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    const bool dev = device_ptrs != 0;
    if (tau0) {
      // every body's start tick must lie before every block tick
      std::vector<long long> t((size_t)A.n);
      if (dev) {
        ck(cudaMemcpyAsync(t.data(), tau0, sizeof(long long) * (size_t)A.n,
                           cudaMemcpyDeviceToHost, ctx->s),
           "copy tau0");
        ck(cudaStreamSynchronize(ctx->s), "synchronize");
      } else {
        std::memcpy(t.data(), tau0, sizeof(long long) * (size_t)A.n);
      }
      for (long long x : t)
        if (x < 0 || x >= A.first_tick)
          return fail(ctx, TSBTS_ERR_ARG,
                      "start ticks must be >= 0 and before every block "
                      "tick");
    }
    A.have_forward = false;
    A.state_mode = a0 ? 1 : 0;
    stage_in(ctx, A, m, r0, v0, a0, (const long long*)tau0, dev);
    rc = forward_impl(ctx, A);
    if (rc) return rc;
    to_out(ctx, A, A.St.r, r_T, dev);
    to_out(ctx, A, A.St.v, v_T, dev);
    to_out(ctx, A, A.St.a, a_T, dev);
    if (tau_T) {
      ck(cudaMemcpyAsync(tau_T, A.St.tau, sizeof(long long) * (size_t)A.n,
                         dev ? cudaMemcpyDeviceToDevice
                             : cudaMemcpyDeviceToHost,
                         ctx->s),
         "copy tau");
      ck(cudaStreamSynchronize(ctx->s), "synchronize");
    }
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_adjoint_forward(tsbts_ctx* ctx, const double* m, const double* r0,
                          const double* v0, double* r_T, double* v_T,
                          int device_ptrs) {
  return tsbts_adjoint_forward_state(ctx, m, r0, v0, nullptr, nullptr, r_T,
                                     v_T, nullptr, nullptr, device_ptrs);
}

namespace {

int vjp_out(tsbts_ctx* ctx, AdjCtx& A, double* g_r0, double* g_v0,
            double* g_a0, double* g_m, bool dev) {
  to_out(ctx, A, A.C.gr, g_r0, dev);
  to_out(ctx, A, A.C.gv, g_v0, dev);
  to_out(ctx, A, A.C.ga, g_a0, dev);
  if (g_m)
    ck(cudaMemcpyAsync(g_m, A.C.gm, sizeof(double) * A.n,
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->s),
       "copy g_m");
  ck(cudaStreamSynchronize(ctx->s), "synchronize");
  return TSBTS_OK;
}

}  // namespace

int tsbts_adjoint_vjp_state(tsbts_ctx* ctx, const double* gr_T,
                            const double* gv_T, const double* ga_T,
                            double* g_r0, double* g_v0, double* g_a0,
                            double* g_m, int device_ptrs) {
  int rc = adj_ready(ctx);
  if (rc) return rc;
  AdjCtx& A = *ctx->adj;
  if (!A.have_forward)
    return fail(ctx, TSBTS_ERR_STATE, "tsbts_adjoint_forward not called");
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    const double *dgr = gr_T, *dgv = gv_T, *dga = ga_T;
    const size_t n3 = 3 * (size_t)A.n;
    if (!device_ptrs) {
      const double* src[3] = {gr_T, gv_T, ga_T};
      const double** dst[3] = {&dgr, &dgv, &dga};
      for (int k = 0; k < 3; ++k) {
        if (!src[k]) continue;
        ck(cudaMemcpyAsync(A.io + k * n3, src[k], sizeof(double) * n3,
                           cudaMemcpyHostToDevice, ctx->s),
           "copy cotangent");
        *dst[k] = A.io + k * n3;
      }
    }
    launch_adj_seed(A.n, dgr, dgv, dga, A.C, ctx->s);
    A.launches += 1;
    rc = backward_impl(ctx, A);
    if (rc) return rc;
    return vjp_out(ctx, A, g_r0, g_v0, g_a0, g_m, device_ptrs != 0);
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_adjoint_vjp(tsbts_ctx* ctx, const double* gr_T, const double* gv_T,
                      double* g_r0, double* g_v0, double* g_m,
                      int device_ptrs) {
  return tsbts_adjoint_vjp_state(ctx, gr_T, gv_T, nullptr, g_r0, g_v0,
                                 nullptr, g_m, device_ptrs);
}

int tsbts_adjoint_loss_grad(tsbts_ctx* ctx, const double* m, const double* r0,
                            const double* v0, double* loss, double* g_r0,
                            double* g_v0, double* g_m, int device_ptrs) {
  int rc = tsbts_adjoint_forward(ctx, m, r0, v0, nullptr, nullptr,
                                 device_ptrs);
  if (rc) return rc;
  AdjCtx& A = *ctx->adj;
  try {
    launch_adj_loss(A.n, A.m, A.St, A.loss, A.C, ctx->s);
    A.launches += 2;
    if (loss)
      ck(cudaMemcpyAsync(loss, A.loss, sizeof(double),
                         device_ptrs ? cudaMemcpyDeviceToDevice
                                     : cudaMemcpyDeviceToHost,
                         ctx->s),
         "copy loss");
    rc = backward_impl(ctx, A);
    if (rc) return rc;
    return vjp_out(ctx, A, g_r0, g_v0, nullptr, g_m, device_ptrs != 0);
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_adjoint_get_stats(tsbts_ctx* ctx, tsbts_adjoint_stats* out) {
  int rc = adj_ready(ctx);
  if (rc) return rc;
  if (!out) return fail(ctx, TSBTS_ERR_ARG, "null stats pointer");
  const AdjCtx& A = *ctx->adj;
  std::memset(out, 0, sizeof *out);
  out->steps = A.S;
  out->entries = A.E;
  out->checkpoint_every = A.K;
  out->checkpoints = A.n_ckpt;
  out->tape_entries = A.tape_cap;
  out->tape_bytes = A.tape_bytes;
  out->checkpoint_bytes = A.ckpt_bytes;
  out->device_bytes = A.bytes;
  out->pairs_forward = A.pairs_fwd;
  out->pairs_backward = A.pairs_bwd;
  out->forward_ms = A.fwd_ms;
  out->backward_ms = A.bwd_ms;
  out->kernel_launches = A.launches;
  out->passes = A.n_pass;
  return TSBTS_OK;
}

}  // extern "C"
