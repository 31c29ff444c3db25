// Host engine and C ABI of the TSBTS library (include/tsbts.h).
//
// One context owns the bodies, the era snapshot and two era-history
// buffers in HBM, and drives Alg. 2 / Alg. 3 (Sec. 2, Sec. 4): eras, each
// with n_iter passes restarted from the era-start snapshot, each pass a
// device-resident loop of block steps. The host launches block steps in
// chunks (stream launches or a captured CUDA graph of `graph_steps`
// steps); kernels read the step state from the control block and return
// once the pass is over, so the host synchronises once per chunk, not
// once per block step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "engine.cuh"
#include "era_rule.h"

using namespace tsbts;

namespace {

const char* kVersion = "tsbts-gb300 0.1 (sm_103a)";

// clusters of tsbts_init_ensemble, host arrays
struct EnsInput {
  int64_t nc;
  const int64_t* offsets;  // nc + 1
  const double* eps;       // nc
};

bool valid_dt_max(double dt_max, int k_max, int* k_min) {
  for (int k = 0; k <= k_max; ++k)
    if (std::ldexp(1.0, -k) == dt_max) {
      *k_min = k;
      return true;
    }
  return false;
}

void alloc_history(tsbts_ctx* c, int b, long long cap) {
  free_list(c->hist_allocs[b]);
  History& h = c->H[b];
  auto& L = c->hist_allocs[b];
  h.tau = dalloc<long long>(L, cap);
  for (int d = 0; d < 3; ++d) {
    h.r[d] = dalloc<double>(L, cap);
    h.v[d] = dalloc<double>(L, cap);
    h.a[d] = dalloc<double>(L, cap);
  }
  h.dts = dalloc<double>(L, cap);
  h.body = dalloc<int>(L, cap);
  h.seq = dalloc<int>(L, cap);
  h.cap = cap;
  c->graph_dirty = true;
}

void release_graph(tsbts_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gexec_t) cudaGraphExecDestroy(c->gexec_t);
  c->gexec = nullptr;
  c->gexec_t = nullptr;
  c->graph_dirty = true;
}

// keep_history: the era-history buffers survive (a re-initialisation with
// the same body count reuses what earlier eras grew them to, so the first
// era of the new run does not overflow and re-run again)
void release_all(tsbts_ctx* c, bool keep_history = false) {
  release_graph(c);
  if (c->s) cudaStreamSynchronize(c->s);
  free_list(c->allocs);
  if (!keep_history) {
    free_list(c->hist_allocs[0]);
    free_list(c->hist_allocs[1]);
    c->H[0] = History{};
    c->H[1] = History{};
  }
  free_list(c->lg_allocs);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  c->h_ctl = nullptr;
  c->inited = false;
}

void read_ctl(tsbts_ctx* c) {
  ck(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                     c->s),
     "read control block");
  ck(cudaStreamSynchronize(c->s), "synchronize");
}

ForceArgs force_args_engine(tsbts_ctx* c, int p) {
  ForceArgs fa{};
  fa.n = c->n;
  fa.m = c->B.m;
  for (int d = 0; d < 3; ++d) {
    fa.x[d] = c->B.pr[d];
    fa.w[d] = c->B.pv[d];
  }
  fa.jhi = c->B.jhi;
  fa.jlo = c->B.jlo;
  fa.jv = c->B.jv;
  fa.idx = c->B.act;
  fa.n_act_fixed = -1;
  fa.n_act_ptr = &c->d_ctl->slot[p].cnt;
  fa.nsplit_out = &c->d_ctl->slot[p].nsplit;
  fa.done = &c->d_ctl->done;
  fa.part = c->B.part;
  fa.part_cap = c->B.part_cap;
  fa.eps2 = c->eps * c->eps;
  fa.eps2f = (float)(c->eps * c->eps);
  fa.exact = c->exact;
  fa.plans = nullptr;
  return fa;
}

// active counts of the plan buckets: 1, 2, 4, ... below n, then n
std::vector<int> plan_buckets(int n) {
  std::vector<int> b;
  for (long long k = 1; k < n; k *= 2) b.push_back((int)k);
  b.push_back(n);
  return b;
}

// work plan of the force kernel per bucket of active counts, chosen on the
// host by the cost model (the mixed path replaces them with measured plans
// after the first force launch); passed to every launch by value
void build_plan_table(tsbts_ctx* c) {
  const std::vector<int> b = plan_buckets(c->n);
  c->pt = PlanTable{};
  c->pt.nb = (int)b.size();
  for (size_t k = 0; k < b.size(); ++k)
    c->pt.b[k] = plan_force(c->cfg.precision, c->exact, b[k], c->n,
                            c->fl.grid, c->B.part_cap);
}

// one block step: A (select + predict), B (force), C (correct). Plain
// stream order between them: launched with programmatic stream
// serialization the next kernel's blocks start early and wait on the GPU,
// which measured slower per block step on GB300. Timing events inside a
// captured graph are external event nodes, so that they are recorded (and
// timed) at every replay.
void enqueue_step(tsbts_ctx* c, int p, int ev_slot, bool capturing) {
  const History& HA = c->H[0];
  const History& HB = c->H[1];
  const unsigned evflags =
      capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (c->ensemble) {
    launch_ens_step(c->B, c->P, c->E, HA, HB, c->efl, c->cfg.precision,
                    c->exact, ev_slot >= 0 ? c->ev[2 * ev_slot] : nullptr,
                    ev_slot >= 0 ? c->ev[2 * ev_slot + 1] : nullptr, evflags,
                    c->s);
    ck(cudaGetLastError(), "ensemble step launch");
    return;
  }
  ck(launch_select_predict(c->B, c->P, HA, HB, p, false, c->s),
     "select/predict launch");
  if (ev_slot >= 0)
    ck(cudaEventRecordWithFlags(c->ev[2 * ev_slot], c->s, evflags), "event");
  ck(launch_force(c->cfg.precision, force_args_engine(c, p), c->fl, c->s,
                  &c->pt, false),
     "force launch");
  if (ev_slot >= 0)
    ck(cudaEventRecordWithFlags(c->ev[2 * ev_slot + 1], c->s, evflags),
       "event");
  ck(launch_correct(c->B, c->P, HA, HB, p, c->correct_grid, false, c->s),
     "correct launch");
}

void ensure_events(tsbts_ctx* c, int steps) {
  while ((int)c->ev.size() < 2 * steps) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "cudaEventCreate");
    c->ev.push_back(e);
  }
}

// the graph of graph_steps block steps, with (timed) or without event
// nodes around each force launch
void build_graph(tsbts_ctx* c, bool timed) {
  cudaGraphExec_t& ex = timed ? c->gexec_t : c->gexec;
  const int G = c->cfg.graph_steps;
  if (timed) ensure_events(c, G);
  cudaGraph_t g;
  ck(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal),
     "begin capture");
  try {
    for (int k = 0; k < G; ++k) enqueue_step(c, k & 1, timed ? k : -1, true);
  } catch (...) {
    cudaStreamEndCapture(c->s, &g);
    throw;
  }
  ck(cudaStreamEndCapture(c->s, &g), "end capture");
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  ck(e, "graph instantiate");
}

// whether the next chunk of block steps carries timing events: every
// timing-th chunk (the sample that tsbts_stats reports)
bool timed_chunk(tsbts_ctx* c) {
  return c->timing > 0 && (c->chunk_no++ % c->timing) == 0;
}

void accumulate_timing(tsbts_ctx* c, int real_steps,
                       unsigned long long inter) {
  for (int k = 0; k < real_steps; ++k) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]),
       "event elapsed");
    c->force_ms += ms;
    c->force_launches += 1;
  }
  c->force_inter += (long long)inter;
}

struct NoProgress {};

// Every block step advances the block time by at least one tick, so a pass
// has at most (tau_e - t_sys) steps; a chunk without any step that did not
// end the pass means the step loop is broken.
void check_progress(tsbts_ctx* c, int real, long long pass_steps,
                    long long tau_e) {
  if (real <= 0 || pass_steps > tau_e - c->t_sys ||
      (c->cfg.max_pass_steps > 0 && pass_steps > c->cfg.max_pass_steps))
    throw NoProgress{};
}

// run one pass; returns the device error bits
int run_pass(tsbts_ctx* c, int pass, long long tau_e, long long est_steps) {
  // H[0] collects this pass's records; H[1] holds the previous pass's
  launch_pass_begin(c->d_ctl, c->t_sys, tau_e, pass, (int)c->eras, c->n, c->s);
  if (c->ensemble) {
    launch_ens_pass_begin(c->E, c->t_sys, c->s);
    launch_ens_pass_setup(c->B, c->P, c->E, c->H[0], c->s);
    c->launches += 3;
  } else {
    launch_pass_setup(c->B, c->P, c->H[0], c->s);
    c->launches += 2;
  }
  ck(cudaGetLastError(), "pass set-up");
  const int per_step = c->ensemble ? 5 : 3;  // kernels per block step
  const int G = c->cfg.graph_steps;
  unsigned long long steps0 = c->h_ctl->steps;
  long long pass_steps = 0;
  unsigned long long inter0 = c->h_ctl->inter;
  if (G > 0) {
    if (c->graph_dirty) {
      release_graph(c);
      c->graph_dirty = false;
    }
    for (;;) {
      const bool timed = timed_chunk(c);
      cudaGraphExec_t& ex = timed ? c->gexec_t : c->gexec;
      if (!ex) build_graph(c, timed);
      ck(cudaGraphLaunch(ex, c->s), "graph launch");
      c->launches += (long long)per_step * G;
      read_ctl(c);
      const int real = (int)(c->h_ctl->steps - steps0);
      steps0 = c->h_ctl->steps;
      if (timed) accumulate_timing(c, real, c->h_ctl->inter - inter0);
      inter0 = c->h_ctl->inter;
      if (c->h_ctl->done || c->h_ctl->err) break;
      check_progress(c, real, pass_steps += real, tau_e);
    }
  } else {
    long long chunk = std::max<long long>(4, std::min<long long>(
                                                  est_steps / 2 + 1, 256));
    int p = 0;
    for (;;) {
      const bool timed = timed_chunk(c);
      if (timed) ensure_events(c, (int)chunk);
      for (long long k = 0; k < chunk; ++k) {
        enqueue_step(c, p, timed ? (int)k : -1, false);
        c->launches += per_step;
        p ^= 1;
      }
      read_ctl(c);
      const int real = (int)(c->h_ctl->steps - steps0);
      steps0 = c->h_ctl->steps;
      if (timed) accumulate_timing(c, real, c->h_ctl->inter - inter0);
      inter0 = c->h_ctl->inter;
      if (c->h_ctl->done || c->h_ctl->err) break;
      check_progress(c, real, pass_steps += real, tau_e);
      chunk = std::min<long long>(chunk * 2, 256);
    }
  }
  c->passes += 1;
  const long long nrec = std::max(c->h_ctl->slot[0].nrec, c->h_ctl->slot[1].nrec);
  c->max_rec = std::max(c->max_rec, nrec);
  return c->h_ctl->err;
}

long long era_ticks(tsbts_ctx* c) {
  if (c->cfg.era_mode == 0) return 1LL << (c->cfg.k_max - c->cfg.era_log2);
  // Alg. 3 from the device's block-time extrema (era_rule.h)
  const long long lo0 = LLONG_MAX, hi0 = LLONG_MIN;
  ck(cudaMemcpyAsync(&c->d_ctl->first, &lo0, sizeof lo0,
                     cudaMemcpyHostToDevice, c->s), "era reset");
  ck(cudaMemcpyAsync(&c->d_ctl->last, &hi0, sizeof hi0,
                     cudaMemcpyHostToDevice, c->s), "era reset");
  launch_next_time_extrema(c->B, c->d_ctl, c->s);
  c->launches += 1;
  read_ctl(c);
  return tsbts_dynamic_era_ticks(c->h_ctl->first, c->h_ctl->last,
                                 c->dtmax_t, c->cfg.dyn_min_log2);
}

// Dynamic eras of an ensemble: every cluster's next era end (Alg. 3 on its
// own bodies, capped at tau_end); false once every cluster has reached
// tau_end.
bool ensemble_eras(tsbts_ctx* c, long long tau_end) {
  ck(cudaMemsetAsync(c->E.undone, 0, sizeof(int), c->s), "memset");
  launch_ens_era(c->B, c->E, c->dtmax_t, c->cfg.dyn_min_log2, tau_end, c->s);
  c->launches += 1;
  int undone = 0;
  ck(cudaMemcpyAsync(&undone, c->E.undone, sizeof undone,
                     cudaMemcpyDeviceToHost, c->s),
     "read era state");
  ck(cudaStreamSynchronize(c->s), "synchronize");
  return undone > 0;
}

int step_era_impl(tsbts_ctx* c, long long tau_end) {
  // an ensemble with dynamic eras runs global eras in which every cluster
  // takes its own era (a cluster already at tau_end takes none); the
  // passes' block steps stop at each cluster's own era end
  const bool own_eras = c->ensemble && c->E.ts;
  while (c->t_sys < tau_end) {
    if (own_eras && !ensemble_eras(c, tau_end)) {
      c->t_sys = tau_end;
      break;
    }
    const long long tau_e =
        own_eras ? tau_end : std::min(c->t_sys + era_ticks(c), tau_end);
    launch_copy_state(c->snap, c->B, c->s);
    c->launches += 1;
    // counters at the era start: an era re-run after the history grew
    // counts (and logs) only the run that is kept
    read_ctl(c);
    const Ctl saved = *c->h_ctl;
    const long long saved_passes = c->passes;
    const double saved_force_ms = c->force_ms;
    const long long saved_force_n = c->force_launches;
    const long long saved_force_inter = c->force_inter;
    for (;;) {
      bool grow = false;
      long long est = 0;
      const bool conv = c->cfg.conv_tol > 0.0;
      for (int p = 0; p < c->cfg.n_iter; ++p) {
        if (p > 0) {
          if (conv)
            for (int d = 0; d < 3; ++d)
              ck(cudaMemcpyAsync(c->rlast[d], c->B.r[d],
                                 sizeof(double) * c->n,
                                 cudaMemcpyDeviceToDevice, c->s),
                 "keep pass end");
          launch_copy_state(c->B, c->snap, c->s);
          c->launches += 1;
        }
        const unsigned long long s0 = c->h_ctl->steps;
        const int e = run_pass(c, p, tau_e, est);
        est = (long long)(c->h_ctl->steps - s0);
        if (!e && conv && p > 0) {
          // R15: stop once a pass repeats the previous one
          const long long nrec =
              std::max(c->h_ctl->slot[0].nrec, c->h_ctl->slot[1].nrec);
          const int zero = 0;
          ck(cudaMemcpyAsync(&c->d_ctl->notconv, &zero, sizeof zero,
                             cudaMemcpyHostToDevice, c->s),
             "reset convergence flag");
          launch_converged(c->B, c->H[0], c->H[1], c->rlast, c->cfg.conv_tol,
                           nrec, c->d_ctl, c->sms, c->s);
          ck(cudaGetLastError(), "convergence check");
          c->launches += 1;
          read_ctl(c);
          if (!c->h_ctl->notconv) break;
        }
        if (!e && p + 1 < c->cfg.n_iter) {
          // the next pass interpolates from these records, body-major
          launch_history_to_csr(c->B, c->H[0], c->H[1], c->d_ctl, c->sms,
                                c->s);
          ck(cudaGetLastError(), "history reorder");
          c->launches += 4;
        }
        if (e & kErrHistory) {
          grow = true;
          break;
        }
        if (e & kErrNonFinite)
          return fail(c, TSBTS_ERR_NONFINITE,
                      "non-finite force or step estimate (era " +
                          std::to_string(c->eras) + ")");
        if (e)
          return fail(c, TSBTS_ERR_CUDA,
                      "internal block-step invariant broken (bits " +
                          std::to_string(e) + ")");
      }
      if (!grow) break;
      // the history did not fit: grow both buffers, re-run the era (record
      // indices are 32-bit)
      const long long cap = std::min<long long>(
          std::max(c->H[0].cap * 4, c->max_rec * 2), 0x7fffffffLL);
      if (c->max_rec >= cap)
        return fail(c, TSBTS_ERR_HISTORY,
                    "era history exceeds 2^31 records; use a shorter era");
      ck(cudaStreamSynchronize(c->s), "synchronize");
      alloc_history(c, 0, cap);
      alloc_history(c, 1, cap);
      int zero = 0;
      ck(cudaMemcpyAsync(&c->d_ctl->err, &zero, sizeof zero,
                         cudaMemcpyHostToDevice, c->s), "clear error");
      // steps, interactions, underflows, then the log counters
      ck(cudaMemcpyAsync(&c->d_ctl->steps, &saved.steps,
                         3 * sizeof(unsigned long long),
                         cudaMemcpyHostToDevice, c->s), "roll back counters");
      ck(cudaMemcpyAsync(&c->d_ctl->log_steps, &saved.log_steps,
                         3 * sizeof(long long), cudaMemcpyHostToDevice, c->s),
         "roll back counters");
      ck(cudaStreamSynchronize(c->s), "synchronize");
      *c->h_ctl = saved;
      c->passes = saved_passes;
      c->force_ms = saved_force_ms;
      c->force_launches = saved_force_n;
      c->force_inter = saved_force_inter;
      launch_copy_state(c->B, c->snap, c->s);
      c->launches += 1;
      c->restarts += 1;
    }
    if (own_eras) {
      launch_ens_era_end(c->E, c->s);
      c->launches += 1;
    } else {
      c->t_sys = tau_e;
    }
    c->eras += 1;
  }
  return TSBTS_OK;
}

void setup_bodies(tsbts_ctx* c, int n) {
  Bodies& B = c->B;
  B = Bodies{};
  B.n = n;
  auto& L = c->allocs;
  B.m = dalloc<double>(L, n);
  B.mf = dalloc<float>(L, n);
  for (int d = 0; d < 3; ++d) {
    B.r[d] = dalloc<double>(L, n);
    B.v[d] = dalloc<double>(L, n);
    B.a[d] = dalloc<double>(L, n);
    B.pr[d] = dalloc<double>(L, n);
    B.pv[d] = dalloc<double>(L, n);
  }
  B.dts = dalloc<double>(L, n);
  B.tau = dalloc<long long>(L, n);
  B.dt = dalloc<long long>(L, n);
  B.jhi = dalloc<float4>(L, n);
  B.jlo = dalloc<float4>(L, n);
  B.jv = dalloc<float4>(L, n);
  B.act = dalloc<int>(L, n);
  B.cursor = dalloc<int>(L, n);
  B.hcnt = dalloc<int>(L, n);
  B.hoff = dalloc<int>(L, (size_t)n + 1);
  B.scan_tmp = dalloc<int>(L, (size_t)(n + 1023) / 1024);
  ck(cudaMemsetAsync(B.hoff, 0, sizeof(int) * ((size_t)n + 1), c->s),
     "memset");
  B.seg_ta = dalloc<long long>(L, n);
  B.seg_tb = dalloc<long long>(L, n);
  B.seg = dalloc<double>(L, 18 * (size_t)n);
  B.part_cap = force_partial_capacity(c->fl, n);
  B.part = dalloc<double>(L, B.part_cap);
  Bodies& S = c->snap;
  S = Bodies{};
  S.n = n;
  for (int d = 0; d < 3; ++d) {
    S.r[d] = dalloc<double>(L, n);
    S.v[d] = dalloc<double>(L, n);
    S.a[d] = dalloc<double>(L, n);
  }
  S.dts = dalloc<double>(L, n);
  S.tau = dalloc<long long>(L, n);
  S.dt = dalloc<long long>(L, n);
  c->d_ctl = dalloc<Ctl>(L, 1);
  for (int d = 0; d < 3; ++d) c->rlast[d] = dalloc<double>(L, n);
  c->d_w = dalloc<double>(L, n);
  c->d_eout = dalloc<double>(L, 2);
  c->d_nsplit = dalloc<int>(L, 1);
  ck(cudaMallocHost(&c->h_ctl, sizeof(Ctl)), "cudaMallocHost");
  std::memset(c->h_ctl, 0, sizeof(Ctl));
  ck(cudaMemsetAsync(c->d_ctl, 0, sizeof(Ctl), c->s), "memset");
  const long long cap = std::max<long long>(8LL * n, 1LL << 16);
  if (c->H[0].cap < cap || c->H[1].cap != c->H[0].cap) {
    alloc_history(c, 0, cap);
    alloc_history(c, 1, cap);
  }
}

// device arrays of an ensemble: body offsets, cluster of each body, per-
// cluster softening, block-step state and work-list prefixes
void setup_ensemble(tsbts_ctx* c, const EnsInput& in) {
  const int nc = (int)in.nc, n = c->n;
  auto& L = c->allocs;
  std::vector<int> off(nc + 1), cl(n);
  std::vector<double> e2(nc);
  std::vector<float> e2f(nc);
  for (int k = 0; k <= nc; ++k) off[k] = (int)in.offsets[k];
  for (int k = 0; k < nc; ++k) {
    for (int i = off[k]; i < off[k + 1]; ++i) cl[i] = k;
    e2[k] = in.eps[k] * in.eps[k];
    e2f[k] = (float)e2[k];
  }
  Ens& E = c->E;
  E = Ens{};
  E.nc = nc;
  int* d_off = dalloc<int>(L, nc + 1);
  int* d_cl = dalloc<int>(L, n);
  double* d_e2 = dalloc<double>(L, nc);
  float* d_e2f = dalloc<float>(L, nc);
  ck(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (nc + 1),
                     cudaMemcpyHostToDevice, c->s), "copy offsets");
  ck(cudaMemcpyAsync(d_cl, cl.data(), sizeof(int) * n,
                     cudaMemcpyHostToDevice, c->s), "copy clusters");
  ck(cudaMemcpyAsync(d_e2, e2.data(), sizeof(double) * nc,
                     cudaMemcpyHostToDevice, c->s), "copy eps");
  ck(cudaMemcpyAsync(d_e2f, e2f.data(), sizeof(float) * nc,
                     cudaMemcpyHostToDevice, c->s), "copy eps");
  E.off = d_off;
  E.cl = d_cl;
  E.eps2 = d_e2;
  E.eps2f = d_e2f;
  E.tau_c = dalloc<long long>(L, nc);
  E.tau_next = dalloc<long long>(L, nc);
  E.cnt = dalloc<int>(L, nc);
  E.hist = dalloc<int>(L, (size_t)nc * kMaxLevels);
  E.act = dalloc<int>(L, n);
  E.plan = dalloc<Plan>(L, nc);
  E.item_off = dalloc<int>(L, nc + 1);
  E.act_base = dalloc<int>(L, nc + 1);
  E.part_off = dalloc<long long>(L, nc + 1);
  E.totals = dalloc<int>(L, 8);
  ck(cudaMemsetAsync(E.totals, 0, sizeof(int) * 8, c->s), "memset");
  c->d_ek = dalloc<double>(L, nc);
  c->d_ep = dalloc<double>(L, nc);
  c->efl = ens_force_launch_shape(c->cfg.precision, c->cfg.device);
  E.part_cap = c->B.part_cap;
  if (c->cfg.era_mode == 1) {
    // each cluster its own dynamic era, from system time 0
    E.ts = dalloc<long long>(L, nc);
    E.te = dalloc<long long>(L, nc);
    E.undone = dalloc<int>(L, 1);
    ck(cudaMemsetAsync(E.ts, 0, sizeof(long long) * nc, c->s), "memset");
  }
  c->nc = nc;
  c->ensemble = true;
}

int init_common(tsbts_ctx* c, int64_t n, const double* m, const double* r,
                const double* v, double eps, double eta, double dt_max,
                bool host, const EnsInput* ens = nullptr) {
  if (!c) return TSBTS_ERR_ARG;
  if (c->poisoned) return fail(c, TSBTS_ERR_STATE, "context is poisoned");
  if (n < 1 || n > (1LL << 24))
    return fail(c, TSBTS_ERR_ARG, "n must be in [1, 2^24]");
  if (!m || !r || !v) return fail(c, TSBTS_ERR_ARG, "null input pointer");
  if (!(eps >= 0.0) || !std::isfinite(eps))
    return fail(c, TSBTS_ERR_ARG, "eps must be finite and >= 0");
  if (ens) {
    if (ens->nc < 1 || ens->nc > ens_max_clusters() || !ens->offsets ||
        !ens->eps)
      return fail(c, TSBTS_ERR_ARG, "bad cluster count or null array");
    if (ens->offsets[0] != 0 || ens->offsets[ens->nc] != n)
      return fail(c, TSBTS_ERR_ARG, "offsets must run from 0 to n");
    for (int64_t k = 0; k < ens->nc; ++k) {
      if (ens->offsets[k + 1] <= ens->offsets[k])
        return fail(c, TSBTS_ERR_ARG, "every cluster needs at least one body");
      if (!(ens->eps[k] >= 0.0) || !std::isfinite(ens->eps[k]))
        return fail(c, TSBTS_ERR_ARG, "eps must be finite and >= 0");
    }
    if (c->cfg.conv_tol > 0.0)
      return fail(c, TSBTS_ERR_ARG,
                  "ensembles run the fixed pass count (conv_tol = 0)");
  }
  if (!(eta > 0.0) || !std::isfinite(eta))
    return fail(c, TSBTS_ERR_ARG, "eta must be finite and > 0");
  int k_min = 0;
  if (!valid_dt_max(dt_max, c->cfg.k_max, &k_min))
    return fail(c, TSBTS_ERR_ARG, "dt_max must be 2^-k with 0 <= k <= k_max");
  if (c->cfg.era_mode == 0 && c->cfg.era_log2 > c->cfg.k_max)
    return fail(c, TSBTS_ERR_ARG, "era_log2 must be <= k_max");
  try {
    ck(cudaSetDevice(c->cfg.device), "cudaSetDevice");
    release_all(c, c->inited && c->n == n);
    c->n = (int)n;
    c->eps = eps;
    c->eta = eta;
    c->k_min = k_min;
    c->dtmax_t = 1LL << (c->cfg.k_max - k_min);
    c->t_sys = 0;
    c->eras = c->passes = c->restarts = c->max_rec = 0;
    c->force_ms = 0;
    c->force_launches = 0;
    c->force_inter = 0;
    c->chunk_no = 0;
    c->launches = 0;
    c->exact = c->cfg.precision == TSBTS_FP64 &&
               (c->cfg.exact_order == 1 ||
                (c->cfg.exact_order < 0 && n <= 8192));
    c->fl = force_launch_shape(c->cfg.precision, c->cfg.device);
    // one warp per block spreads the FP64 correction over the SMs
    c->correct_grid = std::max(1, std::min(c->sms * 32, (c->n + 31) / 32));
    c->ensemble = false;
    c->nc = 0;
    setup_bodies(c, (int)n);
    if (ens) {
      c->pt = PlanTable{};
      setup_ensemble(c, *ens);
    } else {
      build_plan_table(c);
    }
    Params& P = c->P;
    P = Params{};
    P.eps2 = eps * eps;
    P.eta = eta;
    P.inv_ticks = std::ldexp(1.0, -c->cfg.k_max);
    P.dtmax_t = c->dtmax_t;
    P.k_min = k_min;
    P.k_max = c->cfg.k_max;
    P.precision = c->cfg.precision;
    P.exact = c->exact;
    P.ctl = c->d_ctl;
    P.lg_cap = 0;
    // inputs to the device
    const double *dm = m, *dr = r, *dv = v;
    std::vector<void*> tmp;
    if (host) {
      double* t = dalloc<double>(tmp, 7 * (size_t)n);
      ck(cudaMemcpyAsync(t, m, sizeof(double) * n, cudaMemcpyHostToDevice,
                         c->s), "copy m");
      ck(cudaMemcpyAsync(t + n, r, sizeof(double) * 3 * n,
                         cudaMemcpyHostToDevice, c->s), "copy r");
      ck(cudaMemcpyAsync(t + 4 * n, v, sizeof(double) * 3 * n,
                         cudaMemcpyHostToDevice, c->s), "copy v");
      dm = t;
      dr = t + n;
      dv = t + 4 * n;
    }
    launch_load_aos(c->B, dm, dr, dv, c->d_ctl, c->s);
    // Alg. 2 step 1: forces on every body, first steps
    launch_init_jdata(c->B, P, c->s);
    if (c->ensemble) {
      launch_ens_init(c->B, P, c->E, c->efl, c->cfg.precision, c->exact, c->s);
      ck(cudaGetLastError(), "init kernels");
      c->launches = 6;
    } else {
      ForceArgs fa = force_args_engine(c, 0);
      fa.n_act_fixed = c->n;
      fa.n_act_ptr = nullptr;
      fa.nsplit_out = c->d_nsplit;
      fa.done = nullptr;
      fa.plan = plan_force(c->cfg.precision, c->exact, c->n, c->n,
                           c->fl.grid, c->B.part_cap);
      fa.has_plan = 1;
      ck(launch_force(c->cfg.precision, fa, c->fl, c->s), "init force");
      launch_init_finalize(c->B, P, c->d_nsplit, c->s);
      ck(cudaGetLastError(), "init kernels");
      c->launches = 4;
    }
    read_ctl(c);
    free_list(tmp);
    if (c->h_ctl->err & kErrNonFinite)
      return fail(c, TSBTS_ERR_NONFINITE, "non-finite input or initial force");
    if (c->cfg.precision == TSBTS_MIXED && !c->ensemble &&
        c->n <= (1 << 20)) {
      // measured work plans on this device for this n (first context only;
      // later contexts reuse the cached table)
      std::vector<Plan> t;
      ForceArgs base = force_args_engine(c, 0);
      ck(autotune_mixed_plans(c->cfg.device, base, c->fl, c->d_nsplit, c->s,
                              &t),
         "force plan autotuning");
      // (a tuned plan is used only where its partial sums fit this
      // context's buffer)
      const std::vector<int> b = plan_buckets(c->n);
      for (size_t k = 0; k < b.size(); ++k)
        if ((long long)t[b[k]].S * 5 * b[k] <= c->B.part_cap)
          c->pt.b[k] = t[b[k]];
    }
    c->inited = true;
    c->graph_dirty = true;
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(c, f);
  } catch (const std::bad_alloc&) {
    return fail(c, TSBTS_ERR_CUDA, "host out of memory");
  }
}

int check_ready(tsbts_ctx* c) {
  if (!c) return TSBTS_ERR_ARG;
  if (c->poisoned) return fail(c, TSBTS_ERR_STATE, "context is poisoned");
  if (!c->inited) return fail(c, TSBTS_ERR_STATE, "tsbts_init not called");
  return TSBTS_OK;
}

// ---------------------------------------------------------------------
// scratch of the stand-alone force entry point, per device
// ---------------------------------------------------------------------
struct Scratch {
  int n_cap = 0;
  long long part_cap = 0;
  double* soa = nullptr;  // 7 n doubles (x, y, z, vx, vy, vz, m)
  float4* j4 = nullptr;   // 3 n float4
  double* part = nullptr;
  int* nsplit = nullptr;
  int* iota = nullptr;    // 0, 1, ..., n_cap - 1 (active list for tuning)
};
std::mutex g_scratch_mu;
std::vector<Scratch> g_scratch;

}  // namespace

extern "C" {

void tsbts_config_default(tsbts_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->precision = TSBTS_FP64;
  cfg->n_iter = 3;
  cfg->era_mode = 0;
  cfg->era_log2 = 3;
  cfg->dyn_min_log2 = 3;
  cfg->k_max = 20;
  cfg->exact_order = -1;
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->graph_steps = 32;
  cfg->conv_tol = 0.0;
  cfg->max_pass_steps = 0;
}

int tsbts_create(tsbts_ctx** out, const tsbts_config* cfg) {
  if (!out || !cfg) return TSBTS_ERR_ARG;
  *out = nullptr;
  if (cfg->precision != TSBTS_FP64 && cfg->precision != TSBTS_MIXED)
    return TSBTS_ERR_ARG;
  if (cfg->n_iter < 1 || cfg->n_iter > 64) return TSBTS_ERR_ARG;
  if (cfg->era_mode != 0 && cfg->era_mode != 1) return TSBTS_ERR_ARG;
  if (cfg->k_max < 1 || cfg->k_max > 40) return TSBTS_ERR_ARG;
  if (cfg->era_log2 < 0 || cfg->era_log2 > cfg->k_max) return TSBTS_ERR_ARG;
  if (cfg->dyn_min_log2 < 0 || cfg->dyn_min_log2 > 40) return TSBTS_ERR_ARG;
  if (cfg->graph_steps < 0 || cfg->graph_steps > 4096 ||
      (cfg->graph_steps & 1))
    return TSBTS_ERR_ARG;
  if (!(cfg->conv_tol >= 0.0) || !std::isfinite(cfg->conv_tol) ||
      cfg->max_pass_steps < 0)
    return TSBTS_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 ||
      cfg->device >= ndev) {
    cudaGetLastError();
    return TSBTS_ERR_CUDA;
  }
  tsbts_ctx* c = new (std::nothrow) tsbts_ctx;
  if (!c) return TSBTS_ERR_CUDA;
  c->cfg = *cfg;
  try {
    ck(cudaSetDevice(cfg->device), "cudaSetDevice");
    ck(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount,
                              cfg->device), "device attribute");
    if (cfg->stream) {
      c->s = (cudaStream_t)cfg->stream;
    } else {
      ck(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking),
         "cudaStreamCreate");
      c->own_stream = true;
    }
  } catch (const CudaFail&) {
    delete c;
    return TSBTS_ERR_CUDA;
  }
  *out = c;
  return TSBTS_OK;
}

int tsbts_init(tsbts_ctx* ctx, int64_t n, const double* m, const double* r,
               const double* v, double eps, double eta, double dt_max) {
  if (ctx && m && r && v && n > 0 && n <= (1LL << 24)) {
    for (int64_t i = 0; i < n; ++i) {
      bool ok = std::isfinite(m[i]);
      for (int d = 0; d < 3; ++d)
        ok = ok && std::isfinite(r[3 * i + d]) && std::isfinite(v[3 * i + d]);
      if (!ok)
        return fail(ctx, TSBTS_ERR_NONFINITE,
                    "non-finite input at body " + std::to_string(i));
    }
  }
  return init_common(ctx, n, m, r, v, eps, eta, dt_max, true);
}

int tsbts_init_device(tsbts_ctx* ctx, int64_t n, const double* m_dev,
                      const double* r_dev, const double* v_dev, double eps,
                      double eta, double dt_max) {
  return init_common(ctx, n, m_dev, r_dev, v_dev, eps, eta, dt_max, false);
}

int tsbts_step_era(tsbts_ctx* ctx, double t_end, double* t_reached) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  const double te = std::ldexp(t_end, ctx->cfg.k_max);
  if (!std::isfinite(te) || te != std::floor(te) || te > 9.0e18 ||
      (long long)te < ctx->t_sys)
    return fail(ctx, TSBTS_ERR_ARG,
                "t_end must be a whole number of ticks, not in the past");
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    rc = step_era_impl(ctx, (long long)te);
    if (t_reached) *t_reached = std::ldexp((double)ctx->t_sys, -ctx->cfg.k_max);
    return rc;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  } catch (const NoProgress&) {
    return fail(ctx, TSBTS_ERR_TIMEOUT,
                "block-step loop made no progress or passed its step "
                "limit");
  } catch (const std::bad_alloc&) {
    return fail(ctx, TSBTS_ERR_HISTORY, "host out of memory");
  }
}

int tsbts_ensemble_energy(tsbts_ctx* ctx, double* ekin, double* epot) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!ctx->ensemble)
    return fail(ctx, TSBTS_ERR_STATE, "context holds no ensemble");
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    launch_ens_energy(ctx->B, ctx->P, ctx->E, ctx->t_sys, ctx->d_w, ctx->d_ek,
                      ctx->d_ep, ctx->s);
    ck(cudaGetLastError(), "energy kernels");
    ctx->launches += 3;
    if (ekin)
      ck(cudaMemcpyAsync(ekin, ctx->d_ek, sizeof(double) * ctx->nc,
                         cudaMemcpyDeviceToHost, ctx->s), "read energy");
    if (epot)
      ck(cudaMemcpyAsync(epot, ctx->d_ep, sizeof(double) * ctx->nc,
                         cudaMemcpyDeviceToHost, ctx->s), "read energy");
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_init_ensemble(tsbts_ctx* ctx, int64_t n_clusters,
                        const int64_t* offsets, const double* m,
                        const double* r, const double* v, const double* eps,
                        double eta, double dt_max) {
  if (!ctx) return TSBTS_ERR_ARG;
  if (!offsets || n_clusters < 1)
    return fail(ctx, TSBTS_ERR_ARG, "bad cluster count or null offsets");
  const int64_t n = offsets[n_clusters];
  if (m && r && v && n > 0 && n <= (1LL << 24)) {
    for (int64_t i = 0; i < n; ++i) {
      bool ok = std::isfinite(m[i]);
      for (int d = 0; d < 3; ++d)
        ok = ok && std::isfinite(r[3 * i + d]) && std::isfinite(v[3 * i + d]);
      if (!ok)
        return fail(ctx, TSBTS_ERR_NONFINITE,
                    "non-finite input at body " + std::to_string(i));
    }
  }
  const EnsInput in{n_clusters, offsets, eps};
  return init_common(ctx, n, m, r, v, 0.0, eta, dt_max, true, &in);
}

int tsbts_energy(tsbts_ctx* ctx, double* ekin, double* epot, double* etot) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ctx->ensemble) {
    // totals over the clusters, each cluster's sums added in cluster order
    std::vector<double> k(ctx->nc), p(ctx->nc);
    rc = tsbts_ensemble_energy(ctx, k.data(), p.data());
    if (rc) return rc;
    double ks = 0.0, ps = 0.0;
    for (int c = 0; c < ctx->nc; ++c) {
      ks += k[c];
      ps += p[c];
    }
    if (ekin) *ekin = ks;
    if (epot) *epot = ps;
    if (etot) *etot = ks + ps;
    return TSBTS_OK;
  }
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    launch_energy(ctx->B, ctx->P, ctx->t_sys, ctx->d_w, ctx->d_eout, ctx->sms,
                  ctx->s);
    ck(cudaGetLastError(), "energy kernels");
    ctx->launches += 3;
    double e[2];
    ck(cudaMemcpyAsync(e, ctx->d_eout, sizeof e, cudaMemcpyDeviceToHost,
                       ctx->s), "read energy");
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    if (ekin) *ekin = e[0];
    if (epot) *epot = e[1];
    if (etot) *etot = e[0] + e[1];
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_state(tsbts_ctx* ctx, double* t, double* m, double* r, double* v,
                double* a, int64_t* tau_ticks, int64_t* dt_ticks) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    const int n = ctx->n;
    std::vector<double> buf(3 * (size_t)n);
    auto vec = [&](double* dst, double* const src[3]) {
      if (!dst) return;
      for (int d = 0; d < 3; ++d)
        ck(cudaMemcpyAsync(buf.data() + (size_t)d * n, src[d],
                           sizeof(double) * n, cudaMemcpyDeviceToHost,
                           ctx->s), "read state");
      ck(cudaStreamSynchronize(ctx->s), "synchronize");
      for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
          dst[3 * (size_t)i + d] = buf[(size_t)d * n + i];
    };
    if (t) *t = std::ldexp((double)ctx->t_sys, -ctx->cfg.k_max);
    if (m)
      ck(cudaMemcpyAsync(m, ctx->B.m, sizeof(double) * n,
                         cudaMemcpyDeviceToHost, ctx->s), "read m");
    if (tau_ticks)
      ck(cudaMemcpyAsync(tau_ticks, ctx->B.tau, sizeof(int64_t) * n,
                         cudaMemcpyDeviceToHost, ctx->s), "read tau");
    if (dt_ticks)
      ck(cudaMemcpyAsync(dt_ticks, ctx->B.dt, sizeof(int64_t) * n,
                         cudaMemcpyDeviceToHost, ctx->s), "read dt");
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    vec(r, ctx->B.r);
    vec(v, ctx->B.v);
    vec(a, ctx->B.a);
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_step_estimates(tsbts_ctx* ctx, double* dts) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!dts) return fail(ctx, TSBTS_ERR_ARG, "null output pointer");
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    ck(cudaMemcpyAsync(dts, ctx->B.dts, sizeof(double) * ctx->n,
                       cudaMemcpyDeviceToHost, ctx->s), "read dts");
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_set_state(tsbts_ctx* ctx, double t, const double* m,
                    const double* r, const double* v, const double* a,
                    const int64_t* tau_ticks, const int64_t* dt_ticks,
                    const double* dts) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ctx->ensemble)
    return fail(ctx, TSBTS_ERR_STATE, "set_state takes a single system");
  if (!m || !r || !v || !a || !tau_ticks || !dt_ticks || !dts)
    return fail(ctx, TSBTS_ERR_ARG, "null state pointer");
  const double tt = std::ldexp(t, ctx->cfg.k_max);
  if (!std::isfinite(tt) || tt != std::floor(tt) || tt < 0.0 || tt > 9.0e18)
    return fail(ctx, TSBTS_ERR_ARG, "t must be a whole number of ticks >= 0");
  const long long T = (long long)tt;
  const int n = ctx->n;
  // a state that could end an era (era_rule.h), checked before any copy
  const long long bad = tsbts_first_bad_body(T, ctx->dtmax_t, n, m, r, v, a,
                                             tau_ticks, dt_ticks, dts);
  if (bad >= 0)
    return fail(ctx, TSBTS_ERR_ARG,
                "state cannot end an era at body " + std::to_string(bad));
  try {
    ck(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
    // body-major host vectors to the per-component device arrays
    std::vector<double> buf(9 * (size_t)n);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        buf[(size_t)c * n + i] = r[3 * (size_t)i + c];
        buf[(size_t)(3 + c) * n + i] = v[3 * (size_t)i + c];
        buf[(size_t)(6 + c) * n + i] = a[3 * (size_t)i + c];
      }
    auto put = [&](void* dst, const void* src, size_t bytes) {
      ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->s),
         "copy state");
    };
    const size_t nd = sizeof(double) * n;
    put(ctx->B.m, m, nd);
    for (int c = 0; c < 3; ++c) {
      put(ctx->B.r[c], buf.data() + (size_t)c * n, nd);
      put(ctx->B.v[c], buf.data() + (size_t)(3 + c) * n, nd);
      put(ctx->B.a[c], buf.data() + (size_t)(6 + c) * n, nd);
    }
    put(ctx->B.tau, tau_ticks, sizeof(long long) * n);
    put(ctx->B.dt, dt_ticks, sizeof(long long) * n);
    put(ctx->B.dts, dts, nd);
    launch_masses_to_float(ctx->B, ctx->s);
    ctx->launches += 1;
    ck(cudaGetLastError(), "float masses");
    // the host buffers are read before the call returns
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    ctx->t_sys = T;
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_get_stats(tsbts_ctx* ctx, tsbts_stats* out) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!out) return fail(ctx, TSBTS_ERR_ARG, "null stats pointer");
  try {
    read_ctl(ctx);
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
  std::memset(out, 0, sizeof *out);
  out->block_steps = (int64_t)ctx->h_ctl->steps;
  out->interactions = (int64_t)ctx->h_ctl->inter;
  out->eras = ctx->eras;
  out->passes = ctx->passes;
  out->dt_underflow = (int64_t)ctx->h_ctl->underflow;
  out->era_restarts = ctx->restarts;
  out->history_capacity = ctx->H[0].cap;
  out->t_sys_ticks = ctx->t_sys;
  out->force_ms = ctx->force_ms;
  out->force_launches = ctx->force_launches;
  out->force_interactions = ctx->force_inter;
  out->kernel_launches = ctx->launches;
  return TSBTS_OK;
}

int tsbts_set_timing(tsbts_ctx* ctx, int period) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (period < 0)
    return fail(ctx, TSBTS_ERR_ARG, "timing period must be >= 0");
  ctx->timing = period;
  return TSBTS_OK;
}

int tsbts_schedule_log(tsbts_ctx* ctx, int64_t capacity_entries) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (capacity_entries < 0)
    return fail(ctx, TSBTS_ERR_ARG, "capacity must be >= 0");
  if (ctx->ensemble && capacity_entries > 0)
    return fail(ctx, TSBTS_ERR_ARG, "ensembles record no schedule log");
  try {
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    free_list(ctx->lg_allocs);
    Params& P = ctx->P;
    P.lg_cap = capacity_entries;
    P.lg_era = P.lg_pass = P.lg_nact = P.lg_i = nullptr;
    P.lg_tau = P.lg_dt = nullptr;
    if (capacity_entries > 0) {
      auto& L = ctx->lg_allocs;
      P.lg_era = dalloc<int>(L, capacity_entries);
      P.lg_pass = dalloc<int>(L, capacity_entries);
      P.lg_nact = dalloc<int>(L, capacity_entries);
      P.lg_tau = dalloc<long long>(L, capacity_entries);
      P.lg_i = dalloc<int>(L, capacity_entries);
      P.lg_dt = dalloc<long long>(L, capacity_entries);
    }
    const long long zero[3] = {0, 0, 0};
    ck(cudaMemcpyAsync(&ctx->d_ctl->log_steps, zero, sizeof zero,
                       cudaMemcpyHostToDevice, ctx->s), "reset log");
    ctx->graph_dirty = true;
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

int tsbts_schedule_size(tsbts_ctx* ctx, int64_t* steps, int64_t* entries,
                        int64_t* dropped) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  try {
    read_ctl(ctx);
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
  const long long cap = ctx->P.lg_cap;
  if (steps) *steps = std::min<long long>(ctx->h_ctl->log_steps, cap);
  if (entries) *entries = std::min<long long>(ctx->h_ctl->log_ent, cap);
  if (dropped)
    *dropped = ctx->h_ctl->log_drop +
               std::max<long long>(0, ctx->h_ctl->log_steps - cap);
  return TSBTS_OK;
}

int tsbts_schedule_get(tsbts_ctx* ctx, int32_t* step_era, int32_t* step_pass,
                       int64_t* step_tau, int32_t* step_nact, int32_t* ent_i,
                       int64_t* ent_dt) {
  int64_t ns = 0, ne = 0, dr = 0;
  int rc = tsbts_schedule_size(ctx, &ns, &ne, &dr);
  if (rc) return rc;
  try {
    const Params& P = ctx->P;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (dst && bytes)
        ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->s),
           "read log");
    };
    cp(step_era, P.lg_era, sizeof(int32_t) * ns);
    cp(step_pass, P.lg_pass, sizeof(int32_t) * ns);
    cp(step_tau, P.lg_tau, sizeof(int64_t) * ns);
    cp(step_nact, P.lg_nact, sizeof(int32_t) * ns);
    cp(ent_i, P.lg_i, sizeof(int32_t) * ne);
    cp(ent_dt, P.lg_dt, sizeof(int64_t) * ne);
    ck(cudaStreamSynchronize(ctx->s), "synchronize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    return cuda_fail(ctx, f);
  }
}

const char* tsbts_last_error(const tsbts_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

void tsbts_destroy(tsbts_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->cfg.device);
  adjoint_release(ctx);
  release_all(ctx);
  if (ctx->own_stream && ctx->s) cudaStreamDestroy(ctx->s);
  cudaGetLastError();
  delete ctx;
}

int tsbts_force(int precision, int exact_order, int64_t n, const double* m,
                const double* r, const double* v, double eps, int64_t n_act,
                const int32_t* idx, double* a, double* phi, double* q,
                void* stream) {
  if (precision != TSBTS_FP64 && precision != TSBTS_MIXED) return TSBTS_ERR_ARG;
  if (n < 1 || n > 0x7fffffffLL || n_act < 0 || n_act > 0x7fffffffLL)
    return TSBTS_ERR_ARG;
  if (!(eps >= 0.0) || !std::isfinite(eps)) return TSBTS_ERR_ARG;
  if (!m || !r || !v || (n_act > 0 && (!idx || !a || !phi || !q)))
    return TSBTS_ERR_ARG;
  if (n_act == 0) return TSBTS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    int dev = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    const ForceLaunch fl = force_launch_shape(precision, dev);
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if ((int)g_scratch.size() <= dev) g_scratch.resize(dev + 1);
    Scratch& S = g_scratch[dev];
    // partial sums of up to n active bodies: the plan tuner times active
    // counts up to n, whatever this call's n_act
    const long long need_part = std::max<long long>(
        force_partial_capacity(fl, n), 5LL * std::max<int64_t>(n_act, n));
    if (S.n_cap < n || S.part_cap < need_part) {
      ck(cudaDeviceSynchronize(), "synchronize before scratch growth");
      cudaFree(S.soa);
      cudaFree(S.j4);
      cudaFree(S.part);
      cudaFree(S.nsplit);
      cudaFree(S.iota);
      S = Scratch{};
      const int ncap = (int)std::max<int64_t>(n, S.n_cap);
      ck(cudaMalloc(&S.soa, sizeof(double) * 7 * (size_t)ncap), "scratch");
      ck(cudaMalloc(&S.j4, sizeof(float4) * 3 * (size_t)ncap), "scratch");
      ck(cudaMalloc(&S.part, sizeof(double) * need_part), "scratch");
      ck(cudaMalloc(&S.nsplit, sizeof(int)), "scratch");
      ck(cudaMalloc(&S.iota, sizeof(int) * (size_t)ncap), "scratch");
      std::vector<int> iota(ncap);
      for (int k = 0; k < ncap; ++k) iota[k] = k;
      ck(cudaMemcpy(S.iota, iota.data(), sizeof(int) * (size_t)ncap,
                    cudaMemcpyHostToDevice),
         "scratch");
      S.n_cap = ncap;
      S.part_cap = need_part;
    }
    const int ni = (int)n;
    double* x = S.soa;
    float4* j4 = S.j4;
    ck(launch_pack_aos(precision, ni, m, r, v, x, x + ni, x + 2LL * ni,
                       x + 3LL * ni, x + 4LL * ni, x + 5LL * ni, x + 6LL * ni,
                       j4, j4 + ni, j4 + 2LL * ni, s),
       "pack");
    ForceArgs fa{};
    fa.n = ni;
    fa.m = x + 6LL * ni;
    for (int d = 0; d < 3; ++d) {
      fa.x[d] = x + (long long)d * ni;
      fa.w[d] = x + (long long)(3 + d) * ni;
    }
    fa.jhi = j4;
    fa.jlo = j4 + ni;
    fa.jv = j4 + 2LL * ni;
    fa.idx = idx;
    fa.n_act_fixed = (int)n_act;
    fa.nsplit_out = S.nsplit;
    fa.part = S.part;
    fa.part_cap = S.part_cap;
    fa.eps2 = eps * eps;
    fa.eps2f = (float)(eps * eps);
    fa.exact = precision == TSBTS_FP64 &&
               (exact_order == 1 || (exact_order < 0 && n <= 8192));
    fa.plan = plan_force(precision, fa.exact, (int)n_act, ni, fl.grid,
                         S.part_cap);
    if (precision == TSBTS_MIXED && ni <= (1 << 20)) {
      // measured plans: the first call for a new n tunes them on these j
      // records and caches the table for the process
      const std::vector<Plan>* tp = tuned_plans(dev, ni, fl.grid);
      if (!tp) {
        std::vector<Plan> t;
        ForceArgs base = fa;
        base.idx = S.iota;
        // tuned for the capacity every caller with this n has
        base.part_cap = force_partial_capacity(fl, ni);
        ck(autotune_mixed_plans(dev, base, fl, S.nsplit, s, &t),
           "force plan autotuning");
        tp = tuned_plans(dev, ni, fl.grid);
      }
      if (tp && (long long)(*tp)[n_act].S * 5 * n_act <= S.part_cap)
        fa.plan = (*tp)[n_act];
    }
    fa.has_plan = 1;
    if (std::getenv("TSBTS_PRINT_PLANS"))
      std::fprintf(stderr, "tsbts_force n=%d n_act=%lld: ig %d n_g %d S %d "
                   "chunk %d %s\n", ni, (long long)n_act, fa.plan.ig,
                   fa.plan.n_g, fa.plan.S, fa.plan.chunk,
                   fa.plan.direct ? "direct" : "tiled");
    ck(launch_force(precision, fa, fl, s), "force");
    ck(launch_force_finalize(S.part, S.nsplit, (int)n_act, a, phi, q, s),
       "force finalize");
    return TSBTS_OK;
  } catch (const CudaFail& f) {
    std::fprintf(stderr, "tsbts_force: %s: %s\n", f.what,
                 cudaGetErrorString(f.e));
    return TSBTS_ERR_CUDA;
  }
}

int tsbts_release_scratch(void) {
  std::lock_guard<std::mutex> g(g_scratch_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSBTS_ERR_CUDA;
  if ((int)g_scratch.size() <= dev) return TSBTS_OK;
  Scratch& S = g_scratch[dev];
  cudaDeviceSynchronize();
  cudaFree(S.soa);
  cudaFree(S.j4);
  cudaFree(S.part);
  cudaFree(S.nsplit);
  cudaFree(S.iota);
  S = Scratch{};
  return TSBTS_OK;
}

const char* tsbts_version(void) { return kVersion; }

}  // extern "C"

// ---------------------------------------------------------------------
// tsbts_force_static: the stand-alone force with its scratch memory in a
// fixed device array instead of cudaMalloc'd buffers, for callers that
// cannot allocate device memory.
//
// The array lives in this file, so every GPU that loads the library holds
// it until the process exits. In host code `g_static_scratch` names a
// host-side stand-in, not the device array: its device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// only that address is handed to the kernels.
// ---------------------------------------------------------------------
namespace {

constexpr int kStaticMaxBodies = 65536;
// packed j records: 7 doubles per body (FP64) or 3 float4 (mixed, 48 B)
constexpr size_t kStaticJBytes = (size_t)7 * sizeof(double) * kStaticMaxBodies;
// j-split partial sums: room for two splits of 5 values per active body
constexpr long long kStaticPartDoubles = 2LL * 5 * kStaticMaxBodies;
constexpr size_t kStaticBytes =
    kStaticJBytes + sizeof(double) * kStaticPartDoubles + 256;
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticDev {
  unsigned char* ptr;   // device address of g_static_scratch
  ForceLaunch fl[2];    // launch shapes, FP64 and mixed
  bool ready;
};
std::mutex g_static_mu;
StaticDev g_static_dev[kStaticMaxDevices];

// once per device, with that device current: the array's device address
// and the launch shapes (no allocation on this path)
int static_setup(int dev, StaticDev** out) {
  std::lock_guard<std::mutex> g(g_static_mu);
  StaticDev& d = g_static_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      std::fprintf(stderr,
                   "tsbts_force_static: device address of the scratch "
                   "array: %s\n",
                   cudaGetErrorString(e));
      cudaGetLastError();
      return TSBTS_ERR_CUDA;
    }
    d.ptr = static_cast<unsigned char*>(p);
    d.fl[0] = force_launch_shape(0, dev);
    d.fl[1] = force_launch_shape(1, dev);
    d.ready = true;
  }
  *out = &d;
  return TSBTS_OK;
}

}  // namespace

extern "C" int tsbts_force_static(int precision, int exact_order, int64_t n,
                                  const double* m, const double* r,
                                  const double* v, double eps, int64_t n_act,
                                  const int32_t* idx, double* a, double* phi,
                                  double* q, void* stream) {
  if (precision != TSBTS_FP64 && precision != TSBTS_MIXED) return TSBTS_ERR_ARG;
  if (n < 1 || n > kStaticMaxBodies || n_act < 0 || n_act > kStaticMaxBodies)
    return TSBTS_ERR_ARG;
  if (!(eps >= 0.0) || !std::isfinite(eps)) return TSBTS_ERR_ARG;
  if (!m || !r || !v || (n_act > 0 && (!idx || !a || !phi || !q)))
    return TSBTS_ERR_ARG;
  if (n_act == 0) return TSBTS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 ||
      dev >= kStaticMaxDevices) {
    cudaGetLastError();
    return TSBTS_ERR_CUDA;
  }
  StaticDev* sd = nullptr;
  const int rc = static_setup(dev, &sd);
  if (rc != TSBTS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int ni = (int)n;
  const ForceLaunch& fl = sd->fl[precision ? 1 : 0];
  unsigned char* base = sd->ptr;
  double* x = reinterpret_cast<double*>(base);
  float4* j4 = reinterpret_cast<float4*>(base);
  double* part = reinterpret_cast<double*>(base + kStaticJBytes);
  int* nsplit = reinterpret_cast<int*>(base + kStaticJBytes +
                                       sizeof(double) * kStaticPartDoubles);
  // Every region is written before it is read in this call (the packed j
  // records, every (split, body) partial of the plan, the split count), so
  // nothing left by an earlier call needs clearing.
  // a failed launch is reported like tsbts_force's: the step and the CUDA
  // error on stderr
  auto failed = [](const char* what, cudaError_t e) {
    std::fprintf(stderr, "tsbts_force_static: %s: %s\n", what,
                 cudaGetErrorString(e));
    return TSBTS_ERR_CUDA;
  };
  cudaError_t e = launch_pack_aos(
      precision, ni, m, r, v, x, x + ni, x + 2LL * ni, x + 3LL * ni,
      x + 4LL * ni, x + 5LL * ni, x + 6LL * ni, j4, j4 + ni, j4 + 2LL * ni, s);
  if (e != cudaSuccess) return failed("pack", e);
  ForceArgs fa{};
  fa.n = ni;
  fa.m = x + 6LL * ni;
  for (int d = 0; d < 3; ++d) {
    fa.x[d] = x + (long long)d * ni;
    fa.w[d] = x + (long long)(3 + d) * ni;
  }
  fa.jhi = j4;
  fa.jlo = j4 + ni;
  fa.jv = j4 + 2LL * ni;
  fa.idx = idx;
  fa.n_act_fixed = (int)n_act;
  fa.nsplit_out = nsplit;
  fa.part = part;
  fa.part_cap = kStaticPartDoubles;
  fa.eps2 = eps * eps;
  fa.eps2f = (float)(eps * eps);
  fa.exact = precision == TSBTS_FP64 &&
             (exact_order == 1 || (exact_order < 0 && n <= 8192));
  fa.plan = plan_force(precision, fa.exact, (int)n_act, ni, fl.grid,
                       kStaticPartDoubles);
  fa.has_plan = 1;
  e = launch_force(precision, fa, fl, s);
  if (e != cudaSuccess) return failed("force", e);
  e = launch_force_finalize(part, nsplit, (int)n_act, a, phi, q, s);
  if (e != cudaSuccess) return failed("force finalize", e);
  return TSBTS_OK;
}
