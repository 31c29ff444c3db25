// Ensemble kernels: many independent clusters integrated together with the
// TSBTS scheme (Sec. 2 Alg. 2, fixed era of Sec. 3). All clusters' bodies
// share the Bodies arrays (cluster c owns off[c] .. off[c+1]-1); each
// cluster keeps its own block time and per-level body counts. One global
// block step advances every cluster that has not finished the pass by one
// of its own block steps, with five launches:
//   select   one warp per cluster: the cluster's next block time;
//   predict  every body to its cluster's block time, per-cluster
//            compaction of the active lists (local indices);
//   plan     one block: each cluster's force plan and the prefix sums that
//            lay the work items of all clusters out as one list;
//   force    a persistent grid over that list (the per-item code of the
//            single-system kernels, with j restricted to the cluster);
//   correct  Eq. 1, Eq. 4 / Alg. 1 and the history append per active body.
// Clusters of very different sizes and active counts share one launch, so
// small clusters do not pay a launch each and big ones keep the grid busy.
#include <climits>

#include "era_rule.h"
#include "force_device.cuh"
#include "step_device.cuh"
#include "tsbts_kernels.cuh"

namespace tsbts {

constexpr int kEnsMaxClusters = 4096;
constexpr int kPlanThreads = 1024;

// ---------------------------------------------------------------------
// pass set-up
// ---------------------------------------------------------------------
__global__ void ens_pass_begin_kernel(Ens E, long long tau_s) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < E.nc;
       c += gridDim.x * blockDim.x) {
    E.tau_c[c] = E.ts ? E.ts[c] : tau_s;
    E.tau_next[c] = 0;
    E.cnt[c] = 0;
    for (int k = 0; k < kMaxLevels; ++k) E.hist[c * kMaxLevels + k] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) E.totals[k] = 0;
}

__global__ void ens_pass_setup_kernel(Bodies B, Params P, Ens E,
                                      History cur) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x) {
    cur.tau[i] = B.tau[i];
    for (int c = 0; c < 3; ++c) {
      cur.r[c][i] = B.r[c][i];
      cur.v[c][i] = B.v[c][i];
      cur.a[c][i] = B.a[c][i];
    }
    cur.dts[i] = B.dts[i];
    cur.body[i] = i;
    cur.seq[i] = 0;
    B.hcnt[i] = 1;
    B.cursor[i] = B.hoff[i];
    B.seg_ta[i] = LLONG_MAX;
    atomicAdd(&E.hist[E.cl[i] * kMaxLevels + level_of(B.dt[i], P.k_max)], 1);
  }
}

// ---------------------------------------------------------------------
// dynamic eras, one per cluster (Alg. 3 with reading R11 on the cluster's
// own bodies): one block per cluster finds the earliest and latest next
// block time of its bodies and sets the era end, capped at the end of the
// integration; a cluster already there gets an empty era
// ---------------------------------------------------------------------
constexpr int kEraThreads = 256;

__global__ void __launch_bounds__(kEraThreads)
    ens_era_kernel(Bodies B, Ens E, long long dtmax_t, int dyn_min_log2,
                   long long tau_end) {
  const int c = blockIdx.x;
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int i = E.off[c] + threadIdx.x; i < E.off[c + 1]; i += kEraThreads) {
    const long long t = B.tau[i] + B.dt[i];
    lo = t < lo ? t : lo;
    hi = t > hi ? t : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long a = __shfl_xor_sync(kFull, lo, o);
    const long long b = __shfl_xor_sync(kFull, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  __shared__ long long s_lo[kEraThreads / 32], s_hi[kEraThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    s_lo[threadIdx.x >> 5] = lo;
    s_hi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < kEraThreads / 32; ++w) {
    lo = s_lo[w] < lo ? s_lo[w] : lo;
    hi = s_hi[w] > hi ? s_hi[w] : hi;
  }
  const long long ts = E.ts[c];
  if (ts >= tau_end) {
    E.te[c] = ts;
    return;
  }
  const long long len = tsbts_dynamic_era_ticks(lo, hi, dtmax_t, dyn_min_log2);
  E.te[c] = ts + len < tau_end ? ts + len : tau_end;
  atomicAdd(E.undone, 1);
}

// after the era: every cluster's system time is its era end
__global__ void ens_era_end_kernel(Ens E) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < E.nc;
       c += gridDim.x * blockDim.x)
    E.ts[c] = E.te[c];
}

// ---------------------------------------------------------------------
// select: one warp per cluster
// ---------------------------------------------------------------------
__global__ void ens_select_kernel(Ens E, Params P) {
  Ctl* ctl = P.ctl;
  if (ctl->done) return;
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (c >= E.nc) return;
  const int lane = threadIdx.x & 31;
  const int h0 = E.hist[c * kMaxLevels + lane];
  const int h1 = E.hist[c * kMaxLevels + lane + 32];
  const unsigned b0 = __ballot_sync(kFull, h0 > 0 && lane <= P.k_max);
  const unsigned b1 = __ballot_sync(kFull, h1 > 0 && lane + 32 <= P.k_max);
  if (lane == 0) {
    const int kk = b1 ? 63 - __clz(b1) : (b0 ? 31 - __clz(b0) : -1);
    E.cnt[c] = 0;
    if (kk < 0) {
      atomicOr(&ctl->err, kErrLevels);
      E.tau_next[c] = LLONG_MAX;
      return;
    }
    const long long D = 1LL << (P.k_max - kk);
    const long long tn = (E.tau_c[c] / D + 1) * D;
    if (tn > (E.te ? E.te[c] : ctl->tau_e)) {
      E.tau_next[c] = LLONG_MAX;  // finished this pass
    } else {
      E.tau_next[c] = tn;
      atomicAdd(&E.totals[2], 1);
    }
  }
}

// ---------------------------------------------------------------------
// predict + per-cluster compaction
// ---------------------------------------------------------------------
__global__ void ens_predict_kernel(Bodies B, Params P, Ens E, History prev) {
  Ctl* ctl = P.ctl;
  if (ctl->done) return;
  if (E.totals[2] == 0) {  // every cluster has finished the pass
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->done = 1;
    return;
  }
  const int pass = ctl->pass;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = false;
  int c = -1;
  if (j < B.n) {
    // the body's time and step are loaded alongside its cluster's block
    // time; the prediction reads the rest as its path needs it
    c = E.cl[j];
    const long long tj = B.tau[j];
    const long long dtj = B.dt[j];
    PredIn L;
    L.have_state = false;
    L.have_seg = false;
    const long long tn = E.tau_next[c];
    if (tn != LLONG_MAX) {
      const long long nt = tj + dtj;
      act = (nt == tn);
      if (nt < tn) atomicOr(&ctl->err, kErrInvariant);
      predict_body(B, P, prev, j, tj, tn, pass, act, L);
    }
  }
  // lanes of one cluster share one atomic on the cluster's counter
  const unsigned am = __ballot_sync(kFull, act);
  if (act) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(am, c);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&E.cnt[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int o = E.off[c];
    E.act[o + base + rank] = j - o;
  }
}

// ---------------------------------------------------------------------
// plan: per-cluster plans and the work-item layout (one block)
// ---------------------------------------------------------------------
// The work of one global step is spread over about kEnsTargetItems work
// items of similar size: a cluster with w = n_act * N_c interactions gets
// its i-groups (ig = n_act rounded up to a power of two, at most 128) and
// as many j-splits as w / (W / kEnsTargetItems) asks for (W = the step's
// total), within a floor of j per lane; so a large cluster's step spreads
// over the whole grid instead of a few blocks. Measured on the 512-cluster
// workload (t = 0..1/8): 912, 1824 and 3648 target items gave 167, 180 and
// 185 G interactions/s, a floor of 32 j per lane instead of 8 was slower.
#ifndef TSBTS_ENS_ITEMS
#define TSBTS_ENS_ITEMS 3648
#endif
#ifndef TSBTS_ENS_LANE_MIN
#define TSBTS_ENS_LANE_MIN 8
#endif
constexpr int kEnsTargetItems = TSBTS_ENS_ITEMS;
constexpr int kEnsLaneMin = TSBTS_ENS_LANE_MIN;
constexpr int kEnsSplitCap = 64;

__device__ __forceinline__ Plan ens_plan_for(int n_act, int n, int exact,
                                             double per_item) {
  Plan p;
  p.S = 1;
  p.chunk = (n + 1) & ~1;
  if (exact) {
    p.ig = 128;
    p.direct = 0;
  } else {
    int ig = 1;
    while (ig < n_act && ig < 128) ig <<= 1;
    p.ig = ig;
    p.direct = ig <= 16;
  }
  p.n_g = (n_act + p.ig - 1) / p.ig;
  if (!exact && n_act > 0 && per_item > 0.0) {
    const double w = (double)n_act * (double)n;
    int S = (int)ceil(w / per_item / p.n_g);
    const int jg = 128 / p.ig;
    int smax = n / (jg * kEnsLaneMin);
    smax = smax < 1 ? 1 : (smax > kEnsSplitCap ? kEnsSplitCap : smax);
    S = S < 1 ? 1 : (S > smax ? smax : S);
    p.S = S;
    p.chunk = (((n + S - 1) / S) + 1) & ~1;
  }
  return p;
}

// inclusive scan over a block of kPlanThreads threads
template <class T>
__device__ __forceinline__ T block_scan(T x, T* wt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = wt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    wt[lane] = w;
  }
  __syncthreads();
  const T r = wid ? x + wt[wid - 1] : x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kPlanThreads)
    ens_plan_kernel(Ens E, Params P, int init) {
  Ctl* ctl = P.ctl;
  if (!init && ctl->done) return;
  __shared__ int wti[32];
  __shared__ long long wtl[32];
  __shared__ int c_items, c_nact;
  __shared__ long long c_part;
  __shared__ unsigned long long s_inter;
  __shared__ int s_fallback;
  if (threadIdx.x == 0) {
    c_items = 0;
    c_nact = 0;
    c_part = 0;
    s_inter = 0;
    s_fallback = 0;
  }
  __syncthreads();
  // the step's total work sets the size of a work item
  for (int c = threadIdx.x; c < E.nc; c += blockDim.x)
    if (E.tau_next[c] != LLONG_MAX && E.cnt[c] > 0)
      atomicAdd(&s_inter, (unsigned long long)E.cnt[c] *
                              (unsigned long long)(E.off[c + 1] - E.off[c]));
  __syncthreads();
  const unsigned long long total_w = s_inter;
  double per_item = (double)total_w / kEnsTargetItems;
  // the split partials of the step must fit the partial-sum buffer
  // (else every cluster takes one split)
  {
    __shared__ unsigned long long s_parts;
    if (threadIdx.x == 0) s_parts = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < E.nc; c += blockDim.x) {
      if (E.tau_next[c] == LLONG_MAX) continue;
      const int na = E.cnt[c];
      const Plan p = ens_plan_for(na, E.off[c + 1] - E.off[c], P.exact,
                                  per_item);
      atomicAdd(&s_parts, 5ULL * p.S * (unsigned long long)na);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_parts > (unsigned long long)E.part_cap)
      s_fallback = 1;
    __syncthreads();
    if (s_fallback) per_item = 0.0;
  }
  for (int base = 0; base < E.nc; base += kPlanThreads) {
    const int c = base + threadIdx.x;
    const bool valid = c < E.nc;
    int n_act = 0, nb = 0, items = 0;
    long long parts = 0;
    if (valid) {
      nb = E.off[c + 1] - E.off[c];
      if (E.tau_next[c] != LLONG_MAX) n_act = E.cnt[c];
      const Plan p = ens_plan_for(n_act, nb, P.exact, per_item);
      E.plan[c] = p;
      items = n_act ? p.n_g * p.S : 0;
      parts = n_act ? 5LL * p.S * n_act : 0;
    }
    const int ci = c_items, cn = c_nact;
    const long long cp = c_part;
    const int inc_i = block_scan<int>(items, wti);
    const int inc_n = block_scan<int>(n_act, wti);
    const long long inc_p = block_scan<long long>(parts, wtl);
    if (valid) {
      E.item_off[c] = ci + inc_i - items;
      E.act_base[c] = cn + inc_n - n_act;
      E.part_off[c] = cp + inc_p - parts;
    }
    __syncthreads();
    if (threadIdx.x == kPlanThreads - 1) {
      c_items = ci + inc_i;
      c_nact = cn + inc_n;
      c_part = cp + inc_p;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    E.item_off[E.nc] = c_items;
    E.act_base[E.nc] = c_nact;
    E.part_off[E.nc] = c_part;
    E.totals[0] = c_items;
    E.totals[1] = c_nact;
    E.totals[4] = 0;  // the force launch's item counter
    if (!init) {
      E.totals[3] = (int)ctl->slot[0].nrec;
      ctl->slot[0].nrec += c_nact;
      E.totals[2] = 0;  // counted again by the next select
      ctl->steps += 1ULL;
      ctl->inter += s_inter;
    }
  }
}

// ---------------------------------------------------------------------
// force over the work items of all clusters
// ---------------------------------------------------------------------
__device__ __forceinline__ int find_cluster(const int* s_off, int nc, int w) {
  // last c with s_off[c] <= w (clusters without items have equal bounds)
  int lo = 0, hi = nc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// the block's next work item: one atomic per item on a counter the planner
// zeroes (items below gridDim.x are taken statically by their blocks)
__device__ __forceinline__ int next_item(const Ens& E, int& s_next) {
  __syncthreads();  // the previous item's shared-memory use is over
  if (threadIdx.x == 0) s_next = gridDim.x + atomicAdd(&E.totals[4], 1);
  __syncthreads();
  return s_next;
}

__device__ __forceinline__ ForceArgs cluster_args(const Bodies& B,
                                                  const Ens& E, int c,
                                                  double* part,
                                                  const Plan& p, int n_act,
                                                  int exact) {
  const int o = E.off[c];
  ForceArgs A{};
  A.n = E.off[c + 1] - o;
  A.m = B.m + o;
  for (int d = 0; d < 3; ++d) {
    A.x[d] = B.pr[d] + o;
    A.w[d] = B.pv[d] + o;
  }
  A.jhi = B.jhi + o;
  A.jlo = B.jlo + o;
  A.jv = B.jv + o;
  A.idx = E.act + o;
  A.part = part + E.part_off[c];
  A.part_cap = 5LL * p.S * n_act;
  A.eps2 = E.eps2[c];
  A.eps2f = E.eps2f[c];
  A.exact = exact;
  return A;
}

__global__ void __launch_bounds__(kThreads, kMixMinBlocks)
    ens_force_mixed_kernel(Bodies B, Ens E, const Ctl* ctl, double* part) {
  if (ctl->done) return;
  const int total = E.totals[0];
  if (total <= 0) return;
  __shared__ int s_off[kEnsMaxClusters + 1];
  __shared__ MixTile T;
  __shared__ float red[9][kThreads];
  for (int c = threadIdx.x; c <= E.nc; c += blockDim.x) s_off[c] = E.item_off[c];
  __syncthreads();
  __shared__ int s_next;
  // items of different clusters differ in cost: after its first item a
  // block takes the next free one from a counter (dynamic balance)
  for (int w = blockIdx.x; w < total; w = next_item(E, s_next)) {
    const int c = find_cluster(s_off, E.nc, w);
    const Plan p = E.plan[c];
    const int local = w - s_off[c];
    const int g = local / p.S, split = local - (local / p.S) * p.S;
    const int n_act = E.cnt[c];
    const ForceArgs A = cluster_args(B, E, c, part, p, n_act, 0);
    if (p.direct) {
      switch (p.ig) {
        case 16: mixed_direct_item<16, 1>(A, n_act, p, g, split, red); break;
        case 8: mixed_direct_item<8, 1>(A, n_act, p, g, split, red); break;
        case 4: mixed_direct_item<4, 1>(A, n_act, p, g, split, red); break;
        case 2: mixed_direct_item<2, 1>(A, n_act, p, g, split, red); break;
        default: mixed_direct_item<1, 1>(A, n_act, p, g, split, red); break;
      }
    } else {
      switch (p.ig) {
        case 128: mixed_item<128>(A, n_act, p, g, split, T, red); break;
        case 64: mixed_item<64>(A, n_act, p, g, split, T, red); break;
        default: mixed_item<32>(A, n_act, p, g, split, T, red); break;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    ens_force_fp64_kernel(Bodies B, Ens E, const Ctl* ctl, double* part,
                          int exact) {
  if (ctl->done) return;
  const int total = E.totals[0];
  if (total <= 0) return;
  __shared__ int s_off[kEnsMaxClusters + 1];
  __shared__ F64Tile T;
  __shared__ double red[5][kThreads];
  for (int c = threadIdx.x; c <= E.nc; c += blockDim.x) s_off[c] = E.item_off[c];
  __syncthreads();
  __shared__ int s_next;
  // items of different clusters differ in cost: after its first item a
  // block takes the next free one from a counter (dynamic balance)
  for (int w = blockIdx.x; w < total; w = next_item(E, s_next)) {
    const int c = find_cluster(s_off, E.nc, w);
    const Plan p = E.plan[c];
    const int local = w - s_off[c];
    const int g = local / p.S, split = local - (local / p.S) * p.S;
    const int n_act = E.cnt[c];
    const ForceArgs A = cluster_args(B, E, c, part, p, n_act, exact);
    switch (p.ig) {
      case 128: f64_item<128>(A, n_act, p, g, split, T, red); break;
      case 64: f64_item<64>(A, n_act, p, g, split, T, red); break;
      case 32: f64_item<32>(A, n_act, p, g, split, T, red); break;
      case 16: f64_item<16>(A, n_act, p, g, split, T, red); break;
      case 8: f64_item<8>(A, n_act, p, g, split, T, red); break;
      case 4: f64_item<4>(A, n_act, p, g, split, T, red); break;
      case 2: f64_item<2>(A, n_act, p, g, split, T, red); break;
      default: f64_item<1>(A, n_act, p, g, split, T, red); break;
    }
  }
}

// ---------------------------------------------------------------------
// correct: one thread per active-list slot
// ---------------------------------------------------------------------
__global__ void ens_correct_kernel(Bodies B, Params P, Ens E, History cur,
                                   History prev, const double* part) {
  Ctl* ctl = P.ctl;
  if (ctl->done) return;
  const int pass = ctl->pass;
  const long long rec0 = E.totals[3];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < B.n;
       t += gridDim.x * blockDim.x) {
    const int c = E.cl[t];
    const long long tn = E.tau_next[c];
    if (tn == LLONG_MAX) continue;
    const int o = E.off[c];
    const int k = t - o;
    const int n_act = E.cnt[c];
    if (k >= n_act) continue;
    const int i = o + E.act[t];
    double an[3], q;
    sum_partials(part + E.part_off[c], n_act, E.plan[c].S, k, an, q);
    const Corrected cr = correct_body(B, P, cur, prev, i, an, q, tn, pass,
                                      rec0 + E.act_base[c] + k, &ctl->err);
    if (cr.underflow) atomicAdd(&ctl->underflow, 1ULL);
    if (cr.d_new != cr.d_old) {
      atomicSub(&E.hist[c * kMaxLevels + level_of(cr.d_old, P.k_max)], 1);
      atomicAdd(&E.hist[c * kMaxLevels + level_of(cr.d_new, P.k_max)], 1);
    }
    if (k == 0) E.tau_c[c] = tn;
  }
}

// ---------------------------------------------------------------------
// initialisation (Alg. 2 step 1 for every cluster) and energy
// ---------------------------------------------------------------------
__global__ void ens_init_active_kernel(Ens E, int n) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += gridDim.x * blockDim.x)
    E.act[t] = t - E.off[E.cl[t]];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < E.nc;
       c += gridDim.x * blockDim.x) {
    E.cnt[c] = E.off[c + 1] - E.off[c];
    E.tau_next[c] = 0;
  }
}

__global__ void ens_init_finalize_kernel(Bodies B, Params P, Ens E,
                                         const double* part) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x) {
    const int c = E.cl[i];
    const int k = i - E.off[c];
    double an[3], q;
    sum_partials(part + E.part_off[c], E.cnt[c], E.plan[c].S, k, an, q);
    if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]) || isnan(q))
      atomicOr(&P.ctl->err, kErrNonFinite);
    for (int d = 0; d < 3; ++d) B.a[d][i] = an[d];
    const double dts = __ddiv_rn(P.eta, __dsqrt_rn(q));
    B.dts[i] = dts;
    int uf = 0;
    B.dt[i] = level_ticks(dts, P.k_min, P.k_max, &uf);
    if (uf) atomicAdd(&P.ctl->underflow, 1ULL);
    B.tau[i] = 0;
  }
}

// per body: sum over the other bodies of its cluster, ascending j
__global__ void ens_energy_pair_kernel(Bodies B, Ens E, double* w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x) {
    const int c = E.cl[i];
    const double eps2 = E.eps2[c];
    const double xi = B.pr[0][i], yi = B.pr[1][i], zi = B.pr[2][i];
    const double mi = B.m[i];
    double wi = 0.0;
    for (int j = E.off[c]; j < E.off[c + 1]; ++j) {
      if (j == i) continue;
      const double dx = __dsub_rn(B.pr[0][j], xi);
      const double dy = __dsub_rn(B.pr[1][j], yi);
      const double dz = __dsub_rn(B.pr[2][j], zi);
      const double s2 = __dadd_rn(
          __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                    __dmul_rn(dz, dz)),
          eps2);
      wi = __dadd_rn(wi, __ddiv_rn(__dmul_rn(mi, B.m[j]), __dsqrt_rn(s2)));
    }
    w[i] = wi;
  }
}

// per cluster: body sums in ascending order
__global__ void ens_energy_sum_kernel(Bodies B, Ens E, const double* w,
                                      double* ek, double* ep) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < E.nc;
       c += gridDim.x * blockDim.x) {
    double k = 0.0, p = 0.0;
    for (int i = E.off[c]; i < E.off[c + 1]; ++i) {
      const double vx = B.pv[0][i], vy = B.pv[1][i], vz = B.pv[2][i];
      const double v2 = __dadd_rn(
          __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
      k = __dadd_rn(k, __dmul_rn(__dmul_rn(0.5, B.m[i]), v2));
      p = __dsub_rn(p, __dmul_rn(0.5, w[i]));
    }
    ek[c] = k;
    ep[c] = p;
  }
}

// ---------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------
static inline int blocks_for(long long n, int threads, int cap) {
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

int ens_max_clusters() { return kEnsMaxClusters; }

ForceLaunch ens_force_launch_shape(int precision, int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (precision)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, ens_force_mixed_kernel, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, ens_force_fp64_kernel, kThreads, 0);
  ForceLaunch fl;
  fl.grid = (sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
  fl.threads = kThreads;
  fl.tile_i = kThreads;
  fl.part_cap = 0;
  return fl;
}

void launch_ens_era(const Bodies& B, const Ens& E, long long dtmax_t,
                    int dyn_min_log2, long long tau_end, cudaStream_t s) {
  ens_era_kernel<<<E.nc, kEraThreads, 0, s>>>(B, E, dtmax_t, dyn_min_log2,
                                              tau_end);
}

void launch_ens_era_end(const Ens& E, cudaStream_t s) {
  ens_era_end_kernel<<<blocks_for(E.nc, 128, 1024), 128, 0, s>>>(E);
}

void launch_ens_pass_begin(const Ens& E, long long tau_s, cudaStream_t s) {
  ens_pass_begin_kernel<<<blocks_for(E.nc, 128, 1024), 128, 0, s>>>(E, tau_s);
}

void launch_ens_pass_setup(const Bodies& B, const Params& P, const Ens& E,
                           const History& cur, cudaStream_t s) {
  ens_pass_setup_kernel<<<blocks_for(B.n, 256, 4096), 256, 0, s>>>(B, P, E,
                                                                  cur);
}

void launch_ens_step(const Bodies& B, const Params& P, const Ens& E,
                     const History& HA, const History& HB,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaEvent_t ev0, cudaEvent_t ev1, unsigned evflags,
                     cudaStream_t s) {
  ens_select_kernel<<<blocks_for(E.nc, 4, 1 << 20), 128, 0, s>>>(E, P);
  ens_predict_kernel<<<blocks_for(B.n, 64, 1 << 30), 64, 0, s>>>(B, P, E,
                                                                 HB);
  ens_plan_kernel<<<1, kPlanThreads, 0, s>>>(E, P, 0);
  if (ev0) cudaEventRecordWithFlags(ev0, s, evflags);
  if (precision)
    ens_force_mixed_kernel<<<fl.grid, kThreads, 0, s>>>(B, E, P.ctl, B.part);
  else
    ens_force_fp64_kernel<<<fl.grid, kThreads, 0, s>>>(B, E, P.ctl, B.part,
                                                       exact);
  if (ev1) cudaEventRecordWithFlags(ev1, s, evflags);
  ens_correct_kernel<<<blocks_for(B.n, 64, 1 << 20), 64, 0, s>>>(B, P, E, HA,
                                                                 HB, B.part);
}

void launch_ens_init(const Bodies& B, const Params& P, const Ens& E,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaStream_t s) {
  ens_init_active_kernel<<<blocks_for(B.n, 256, 4096), 256, 0, s>>>(E, B.n);
  ens_plan_kernel<<<1, kPlanThreads, 0, s>>>(E, P, 1);
  if (precision)
    ens_force_mixed_kernel<<<fl.grid, kThreads, 0, s>>>(B, E, P.ctl, B.part);
  else
    ens_force_fp64_kernel<<<fl.grid, kThreads, 0, s>>>(B, E, P.ctl, B.part,
                                                       exact);
  ens_init_finalize_kernel<<<blocks_for(B.n, 256, 4096), 256, 0, s>>>(
      B, P, E, B.part);
}

void launch_ens_energy(const Bodies& B, const Params& P, const Ens& E,
                       long long T, double* w, double* ek, double* ep,
                       cudaStream_t s) {
  launch_energy_predict(B, P, T, s);
  ens_energy_pair_kernel<<<blocks_for(B.n, 128, 1 << 20), 128, 0, s>>>(B, E,
                                                                       w);
  ens_energy_sum_kernel<<<blocks_for(E.nc, 64, 1 << 20), 64, 0, s>>>(B, E, w,
                                                                     ek, ep);
}

}  // namespace tsbts
