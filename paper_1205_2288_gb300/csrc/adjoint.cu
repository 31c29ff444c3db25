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
#include <algorithm>
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
  std::vector<long long> tau, off;
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
  long long* last_e = nullptr;  // n: each body's last entry or -1
  long long* cur_e = nullptr;   // n
  int* iota = nullptr;          // n
  double* m = nullptr;
  double* io = nullptr;         // 7 n doubles: host inputs / outputs
  AdjState St{};
  std::vector<AdjState> ckpt;
  AdjState fin{};  // final state of the forward replay (taped mode)
  AdjTape Tp{};
  AdjPred P{};
  AdjSlots Sl{};
  AdjCot C{};
  float4* jv = nullptr;         // zero velocities for the force kernel
  double* part = nullptr;
  long long part_cap = 0;
  int* nsplit = nullptr;
  double* part_i = nullptr;
  double* part_j = nullptr;
  int* err = nullptr;
  double* loss = nullptr;       // L, sum m
  bool have_forward = false;
  // statistics
  long long pairs_fwd = 0, pairs_bwd = 0, launches = 0;
  double fwd_ms = 0, bwd_ms = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
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

void launch_step_force(tsbts_ctx* c, AdjCtx& A, const int* idx, int n_act,
                       const Plan& plan) {
  ForceArgs fa = force_args(A);
  fa.idx = idx;
  fa.n_act_fixed = n_act;
  fa.plan = plan;
  ck(launch_force(A.mixed, fa, A.fl, c->s), "replay force");
}

// forward plans for every step, measured for the mixed path when a tuned
// table exists for (device, n)
void choose_plans(tsbts_ctx* c, AdjCtx& A) {
  const std::vector<Plan>* tp =
      A.mixed && A.n <= (1 << 20) ? tuned_plans(c->cfg.device, A.n, A.fl.grid)
                                  : nullptr;
  auto pick = [&](int na) {
    Plan p = plan_force(A.mixed, A.exact, na, A.n, A.fl.grid, A.part_cap);
    if (tp && (long long)(*tp)[na].S * 5 * na <= A.part_cap) p = (*tp)[na];
    return p;
  };
  A.plan_init = pick(A.n);
  for (long long s = 0; s < A.S; ++s)
    A.plans[s] = pick((int)(A.off[s + 1] - A.off[s]));
}

// Replay steps [s0, s1) from the current state; with a tape, record the
// pre-step state of their entries. Checkpoint k is saved before step k K.
void replay_steps(tsbts_ctx* c, AdjCtx& A, long long s0, long long s1,
                  const AdjTape& tape, bool save_ckpt) {
  for (long long s = s0; s < s1; ++s) {
    if (save_ckpt && A.K > 0 && s % A.K == 0) {
      copy_state(A.ckpt[s / A.K], A.St, A.n, c->s);
    }
    const long long T = A.tau[s];
    const int na = (int)(A.off[s + 1] - A.off[s]);
    const int* idx = A.act + A.off[s];
    launch_adj_predict(A.n, T, A.inv_ticks, A.mixed, A.St, A.P, c->s);
    launch_step_force(c, A, idx, na, A.plans[s]);
    launch_adj_correct(na, idx, T, A.inv_ticks, A.part, A.nsplit, A.St, A.P,
                       tape, A.off[s], A.err, c->s);
    A.launches += 3;
  }
  ck(cudaGetLastError(), "replay launches");
}

void reverse_steps(tsbts_ctx* c, AdjCtx& A, long long s1, long long s0) {
  const double eps2 = A.eps * A.eps;
  for (long long s = s1 - 1; s >= s0; --s) {
    const long long T = A.tau[s];
    const int na = (int)(A.off[s + 1] - A.off[s]);
    launch_adj_back_prep(A.n, T, A.inv_ticks, A.off[s], 0, A.mixed, A.St,
                         A.Tp, A.cur_e, A.prev_e, A.C, A.P, A.Sl, c->s);
    launch_adj_vjp(A.mixed, A.n, na, A.act + A.off[s], eps2, A.P, A.Sl,
                   A.shapes[s], A.part_i, A.part_j, c->s);
    launch_adj_back_finalize(A.n, na, T, A.inv_ticks, A.shapes[s], A.part_i,
                             A.part_j, A.P, A.Sl, A.St, A.C, A.err, c->s);
    A.launches += 3;
    A.pairs_bwd += 2LL * na * A.n;
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

// forward replay from inputs on the device (AoS)
int forward_impl(tsbts_ctx* c, AdjCtx& A, const double* dm, const double* dr,
                 const double* dv) {
  ck(cudaMemsetAsync(A.err, 0, sizeof(int), c->s), "memset");
  ck(cudaEventRecord(A.ev[0], c->s), "event");
  launch_adj_load(A.n, dm, dr, dv, A.mixed, A.m, A.St, A.P, A.err, c->s);
  ForceArgs fa = force_args(A);
  fa.idx = A.iota;
  fa.n_act_fixed = A.n;
  fa.plan = A.plan_init;
  ck(launch_force(A.mixed, fa, A.fl, c->s), "initial force");
  launch_adj_init_accel(A.n, A.part, A.nsplit, A.St, A.err, c->s);
  A.launches += 3;
  AdjTape none{};
  replay_steps(c, A, 0, A.S, A.K == 0 ? A.Tp : none, true);
  // the taped reverse sweep starts from the final state; keep it so that
  // every sweep of this forward replay can start there
  if (A.K == 0) copy_state(A.fin, A.St, A.n, c->s);
  ck(cudaEventRecord(A.ev[1], c->s), "event");
  int rc = TSBTS_OK;
  check_err(c, A, "non-finite input or force in the replay", &rc);
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, A.ev[0], A.ev[1]), "event time");
  A.fwd_ms = ms;
  A.pairs_fwd = (long long)A.n * A.n + A.E * (long long)A.n;
  A.have_forward = rc == TSBTS_OK;
  return rc;
}

// reverse sweep from the seeds already in A.C
int backward_impl(tsbts_ctx* c, AdjCtx& A) {
  ck(cudaMemsetAsync(A.err, 0, sizeof(int), c->s), "memset");
  ck(cudaEventRecord(A.ev[0], c->s), "event");
  A.pairs_bwd = 0;
  ck(cudaMemcpyAsync(A.cur_e, A.last_e, sizeof(long long) * (size_t)A.n,
                     cudaMemcpyDeviceToDevice, c->s),
     "copy entry cursors");
  if (A.K == 0) {
    copy_state(A.St, A.fin, A.n, c->s);
    reverse_steps(c, A, A.S, 0);
  } else {
    for (long long g = A.n_ckpt - 1; g >= 0; --g) {
      const long long s0 = g * A.K, s1 = std::min(A.S, s0 + A.K);
      copy_state(A.St, A.ckpt[g], A.n, c->s);
      AdjTape tape = A.Tp;
      tape.base = A.off[s0];
      replay_steps(c, A, s0, s1, tape, false);
      A.pairs_bwd += (A.off[s1] - A.off[s0]) * (long long)A.n;
      A.Tp.base = tape.base;
      reverse_steps(c, A, s1, s0);
    }
    A.Tp.base = 0;
  }
  // the initial force a0 = f(r0): every body active at tick 0
  const double eps2 = A.eps * A.eps;
  launch_adj_back_prep(A.n, 0, A.inv_ticks, 0, 1, A.mixed, A.St, A.Tp,
                       A.cur_e, A.prev_e, A.C, A.P, A.Sl, c->s);
  launch_adj_vjp(A.mixed, A.n, A.n, A.iota, eps2, A.P, A.Sl, A.shape_init,
                 A.part_i, A.part_j, c->s);
  launch_adj_back_finalize(A.n, A.n, 0, A.inv_ticks, A.shape_init, A.part_i,
                           A.part_j, A.P, A.Sl, A.St, A.C, A.err, c->s);
  A.launches += 3;
  A.pairs_bwd += 2LL * A.n * A.n;
  ck(cudaGetLastError(), "reverse launches");
  ck(cudaEventRecord(A.ev[1], c->s), "event");
  int rc = TSBTS_OK;
  check_err(c, A, "non-finite cotangent in the reverse sweep", &rc);
  float ms = 0;
  ck(cudaEventElapsedTime(&ms, A.ev[0], A.ev[1]), "event time");
  A.bwd_ms = ms;
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

// inputs on the device: host arrays are staged through A.io
void stage_in(tsbts_ctx* c, AdjCtx& A, const double* m, const double* r,
              const double* v, bool dev, const double** dm, const double** dr,
              const double** dv) {
  if (dev) {
    *dm = m;
    *dr = r;
    *dv = v;
    return;
  }
  const size_t n = (size_t)A.n;
  ck(cudaMemcpyAsync(A.io, m, sizeof(double) * n, cudaMemcpyHostToDevice,
                     c->s), "copy m");
  ck(cudaMemcpyAsync(A.io + n, r, sizeof(double) * 3 * n,
                     cudaMemcpyHostToDevice, c->s), "copy r");
  ck(cudaMemcpyAsync(A.io + 4 * n, v, sizeof(double) * 3 * n,
                     cudaMemcpyHostToDevice, c->s), "copy v");
  *dm = A.io;
  *dr = A.io + n;
  *dv = A.io + 4 * n;
}

}  // namespace

void adjoint_release(tsbts_ctx* c) { adj_free(c); }

extern "C" {

int tsbts_adjoint_init(tsbts_ctx* ctx, int64_t n, double eps, int64_t n_steps,
                       const int64_t* step_tau, const int64_t* step_off,
                       const int32_t* act, int64_t checkpoint_every) {
  if (!ctx) return TSBTS_ERR_ARG;
  if (ctx->poisoned) return fail(ctx, TSBTS_ERR_STATE, "context is poisoned");
  if (n < 1 || n > (1LL << 24))
    return fail(ctx, TSBTS_ERR_ARG, "n must be in [1, 2^24]");
  if (!(eps >= 0.0) || !std::isfinite(eps))
    return fail(ctx, TSBTS_ERR_ARG, "eps must be finite and >= 0");
  if (n_steps < 0 || checkpoint_every < 0)
    return fail(ctx, TSBTS_ERR_ARG, "negative step or checkpoint count");
  if (n_steps > 0 && (!step_tau || !step_off || !act))
    return fail(ctx, TSBTS_ERR_ARG, "null schedule array");
  if (n_steps > 0 && step_off[0] != 0)
    return fail(ctx, TSBTS_ERR_ARG, "step_off[0] must be 0");
  // validate the schedule: increasing ticks, non-empty steps, bodies in
  // range and distinct within a step
  std::vector<long long> stamp((size_t)n, -1);
  for (int64_t s = 0; s < n_steps; ++s) {
    if (step_tau[s] <= (s ? step_tau[s - 1] : 0))
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
    A.tau.assign(step_tau, step_tau + n_steps);
    A.off.assign(step_off, step_off + n_steps + 1);
    if (n_steps == 0) A.off.assign(1, 0);
    A.fl = force_launch_shape(A.mixed, ctx->cfg.device);
    // entry links: previous entry of the same body, last entry per body
    std::vector<long long> prev((size_t)std::max<long long>(E, 1), -1),
        last((size_t)n, -1);
    for (long long e = 0; e < E; ++e) {
      const int i = act[e];
      prev[e] = last[i];
      last[i] = e;
    }
    const int ni = (int)n;
    A.act = adj_alloc<int>(A, E);
    A.prev_e = adj_alloc<long long>(A, E);
    A.last_e = adj_alloc<long long>(A, ni);
    A.cur_e = adj_alloc<long long>(A, ni);
    A.iota = adj_alloc<int>(A, ni);
    std::vector<int> iota(ni);
    for (int k = 0; k < ni; ++k) iota[k] = k;
    if (E) {
      ck(cudaMemcpyAsync(A.act, act, sizeof(int) * E, cudaMemcpyHostToDevice,
                         ctx->s), "copy schedule");
      ck(cudaMemcpyAsync(A.prev_e, prev.data(), sizeof(long long) * E,
                         cudaMemcpyHostToDevice, ctx->s), "copy schedule");
    }
    ck(cudaMemcpyAsync(A.last_e, last.data(), sizeof(long long) * ni,
                       cudaMemcpyHostToDevice, ctx->s), "copy schedule");
    ck(cudaMemcpyAsync(A.iota, iota.data(), sizeof(int) * ni,
                       cudaMemcpyHostToDevice, ctx->s), "copy iota");
    A.m = adj_alloc<double>(A, ni);
    A.io = adj_alloc<double>(A, 7 * (size_t)ni);
    A.St = alloc_state(A, ni);
    for (int c = 0; c < 3; ++c) {
      A.P.p[c] = adj_alloc<double>(A, ni);
      A.Sl.lam[c] = adj_alloc<double>(A, ni);
      A.Sl.gp0[c] = adj_alloc<double>(A, ni);
      A.Sl.ap[c] = adj_alloc<double>(A, ni);
      A.C.gr[c] = adj_alloc<double>(A, ni);
      A.C.gv[c] = adj_alloc<double>(A, ni);
      A.C.ga[c] = adj_alloc<double>(A, ni);
    }
    A.P.m = A.m;
    A.C.gm = adj_alloc<double>(A, ni);
    A.P.jhi = adj_alloc<float4>(A, ni);
    A.P.jlo = adj_alloc<float4>(A, ni);
    A.jv = adj_alloc<float4>(A, ni);
    ck(cudaMemsetAsync(A.jv, 0, sizeof(float4) * ni, ctx->s), "memset");
    A.Sl.ahi = adj_alloc<float4>(A, ni);
    A.Sl.alo = adj_alloc<float4>(A, ni);
    A.Sl.alam = adj_alloc<float4>(A, ni);
    A.Sl.slot = adj_alloc<int>(A, ni);
    A.part_cap = std::max<long long>(A.fl.part_cap, 5LL * ni);
    A.part = adj_alloc<double>(A, A.part_cap);
    A.nsplit = adj_alloc<int>(A, 1);
    A.err = adj_alloc<int>(A, 1);
    A.loss = adj_alloc<double>(A, 2);
    // tape: every entry, or the largest checkpointed segment
    const long long before_tape = A.bytes;
    if (A.K == 0) {
      A.tape_cap = E;
    } else {
      A.n_ckpt = (A.S + A.K - 1) / A.K;
      for (long long g = 0; g < A.n_ckpt; ++g) {
        const long long s0 = g * A.K, s1 = std::min(A.S, s0 + A.K);
        A.tape_cap = std::max(A.tape_cap, A.off[s1] - A.off[s0]);
      }
    }
    for (int k = 0; k < 9; ++k) A.Tp.x[k] = adj_alloc<double>(A, A.tape_cap);
    A.Tp.tau = adj_alloc<long long>(A, A.tape_cap);
    A.Tp.base = 0;
    A.tape_bytes = A.bytes - before_tape;
    const long long before_ckpt = A.bytes;
    for (long long g = 0; g < A.n_ckpt; ++g) A.ckpt.push_back(alloc_state(A, ni));
    if (A.K == 0) A.fin = alloc_state(A, ni);
    A.ckpt_bytes = A.bytes - before_ckpt;
    // reverse work splits and their partial-sum buffers
    A.shapes.resize(A.S);
    A.plans.resize(A.S);
    long long cap_i = 0, cap_j = 0;
    auto need = [&](const VjpShape& v, long long na) {
      cap_i = std::max(cap_i, (long long)v.si.S * 3 * na);
      cap_j = std::max(cap_j, (long long)v.sj.S * 4 * ni);
    };
    A.shape_init = vjp_shape(ni, ni, ctx->sms);
    need(A.shape_init, ni);
    for (long long s = 0; s < A.S; ++s) {
      const int na = (int)(A.off[s + 1] - A.off[s]);
      A.shapes[s] = vjp_shape(ni, na, ctx->sms);
      need(A.shapes[s], na);
    }
    A.part_i = adj_alloc<double>(A, cap_i);
    A.part_j = adj_alloc<double>(A, cap_j);
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

int tsbts_adjoint_forward(tsbts_ctx* ctx, const double* m, const double* r0,
                          const double* v0, double* r_T, double* v_T,
                          int device_ptrs) {
  int rc = adj_ready(ctx);
  if (rc) return rc;
  if (!m || !r0 || !v0) return fail(ctx, TSBTS_ERR_ARG, "null input pointer");
  AdjCtx& A = *ctx->adj;
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    const double *dm, *dr, *dv;
    stage_in(ctx, A, m, r0, v0, device_ptrs != 0, &dm, &dr, &dv);
    if (A.mixed && A.n <= (1 << 20) &&
        !tuned_plans(ctx->cfg.device, A.n, A.fl.grid)) {
      // measured force plans for this n, timed on the initial positions
      launch_adj_load(A.n, dm, dr, dv, A.mixed, A.m, A.St, A.P, A.err, ctx->s);
      std::vector<Plan> t;
      ForceArgs base = force_args(A);
      base.idx = A.iota;
      base.has_plan = 0;
      ck(autotune_mixed_plans(ctx->cfg.device, base, A.fl, A.nsplit, ctx->s,
                              &t),
         "force plan autotuning");
      choose_plans(ctx, A);
    }
    rc = forward_impl(ctx, A, dm, dr, dv);
    if (rc) return rc;
    to_out(ctx, A, A.St.r, r_T, device_ptrs != 0);
    to_out(ctx, A, A.St.v, v_T, device_ptrs != 0);
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

namespace {

int vjp_out(tsbts_ctx* ctx, AdjCtx& A, double* g_r0, double* g_v0,
            double* g_m, bool dev) {
  to_out(ctx, A, A.C.gr, g_r0, dev);
  to_out(ctx, A, A.C.gv, g_v0, dev);
  if (g_m)
    ck(cudaMemcpyAsync(g_m, A.C.gm, sizeof(double) * A.n,
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->s),
       "copy g_m");
  ck(cudaStreamSynchronize(ctx->s), "synchronize");
  return TSBTS_OK;
}

}  // namespace

int tsbts_adjoint_vjp(tsbts_ctx* ctx, const double* gr_T, const double* gv_T,
                      double* g_r0, double* g_v0, double* g_m,
                      int device_ptrs) {
  int rc = adj_ready(ctx);
  if (rc) return rc;
  AdjCtx& A = *ctx->adj;
  if (!A.have_forward)
    return fail(ctx, TSBTS_ERR_STATE, "tsbts_adjoint_forward not called");
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    const double *dgr = gr_T, *dgv = gv_T;
    const size_t n3 = 3 * (size_t)A.n;
    if (!device_ptrs) {
      if (gr_T)
        ck(cudaMemcpyAsync(A.io, gr_T, sizeof(double) * n3,
                           cudaMemcpyHostToDevice, ctx->s), "copy gr");
      if (gv_T)
        ck(cudaMemcpyAsync(A.io + n3, gv_T, sizeof(double) * n3,
                           cudaMemcpyHostToDevice, ctx->s), "copy gv");
      dgr = gr_T ? A.io : nullptr;
      dgv = gv_T ? A.io + n3 : nullptr;
    }
    launch_adj_seed(A.n, dgr, dgv, A.C, ctx->s);
    A.launches += 1;
    rc = backward_impl(ctx, A);
    if (rc) return rc;
    return vjp_out(ctx, A, g_r0, g_v0, g_m, device_ptrs != 0);
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
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
    return vjp_out(ctx, A, g_r0, g_v0, g_m, device_ptrs != 0);
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
  return TSBTS_OK;
}

}  // extern "C"
