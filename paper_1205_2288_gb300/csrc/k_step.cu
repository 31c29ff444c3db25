// Block-step kernels of the TSBTS library (Sec. 2 Alg. 2 steps 3-8, Sec. 4
// Alg. 3): era/pass set-up, block selection fused with the prediction or
// time-symmetric interpolation of every body, correction (Eq. 1) with the
// next-step choice (Eq. 4, Alg. 1) and the era-history append, the history
// reorder between passes, energy. Each kernel of a block step waits
// (griddepcontrol.wait) before reading what its predecessor wrote, so the
// launches may also use programmatic stream serialization.
//
// The loop is device-resident: every kernel reads the block time, active
// count and pass state from the control block, so a whole chunk of block
// steps is launched (or replayed from a CUDA graph) without a host round
// trip; once the block time passes the era end every kernel returns.
//
// Block selection uses the commensurability of block steps: each body sits
// on a multiple of its own power-of-two step, so the next block time is the
// next multiple of the smallest populated step after the current block
// time, and a per-level body count (updated by the correction)
// replaces the paper's sort by block time.
#include "step_device.cuh"
#include "tsbts_kernels.cuh"

namespace tsbts {

// ---------------------------------------------------------------------
// Pass set-up
// ---------------------------------------------------------------------
__global__ void pass_begin_kernel(Ctl* ctl, long long tau_s, long long tau_e,
                                  int pass, int era, int n) {
  if (threadIdx.x < kMaxLevels) ctl->hist[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    const long long lg = ctl->log_ent;
    for (int p = 0; p < 2; ++p) {
      ctl->slot[p].tau_c = tau_s;
      ctl->slot[p].tau_next = 0;
      ctl->slot[p].nrec = n;
      ctl->slot[p].lg_base = lg;
      ctl->slot[p].cnt = 0;
      ctl->slot[p].nsplit = 0;
    }
    ctl->tau_e = tau_e;
    ctl->done = 0;
    ctl->pass = pass;
    ctl->era = era;
  }
}

// era-start record of every body, cursors, and the level histogram
__global__ void pass_setup_kernel(Bodies B, Params P, History cur) {
  __shared__ int h[kMaxLevels];
  for (int t = threadIdx.x; t < kMaxLevels; t += blockDim.x) h[t] = 0;
  __syncthreads();
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
    B.cursor[i] = B.hoff[i];  // first previous-pass record of body i
    B.seg_ta[i] = LLONG_MAX;
    atomicAdd(&h[level_of(B.dt[i], P.k_max)], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kMaxLevels; t += blockDim.x)
    if (h[t]) atomicAdd(&P.ctl->hist[t], h[t]);
}

// ---------------------------------------------------------------------
// Step A: block time, active list, prediction of every body (Alg. 2
// steps 3-4; Eq. 2; time-symmetric interpolation in passes >= 1).
// ---------------------------------------------------------------------

__global__ void select_predict_kernel(Bodies B, Params P, History HA,
                                      History HB, int p) {
  __shared__ long long s_tn;
  __shared__ int s_stop;
  Ctl* ctl = P.ctl;
  // everything below reads what the previous step's force launch wrote
  pdl_wait();
  pdl_launch_dependents();
  // this body's inputs, loaded before the block time and the pass are
  // known (the segment cache too: it is not used in the first pass), so
  // that every load of the kernel is in flight at once
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  long long tj = 0, dtj = 0;
  PredIn L;
  if (j < B.n) {
    tj = B.tau[j];
    dtj = B.dt[j];
    load_pred_in(B, j, true, L);
  }
  const int pass = ctl->pass;
  if (threadIdx.x < 32) {
    // smallest populated step = highest populated level, one warp-wide load
    const int lane = threadIdx.x;
    const int h0 = ctl->hist[lane], h1 = ctl->hist[lane + 32];
    const unsigned b0 = __ballot_sync(kFull, h0 > 0 && lane <= P.k_max);
    const unsigned b1 = __ballot_sync(kFull, h1 > 0 && lane + 32 <= P.k_max);
    if (lane == 0) {
      int stop = ctl->done ? 3 : 0;
      long long tn = 0;
      if (!stop) {
        const int kk = b1 ? 63 - __clz(b1) : (b0 ? 31 - __clz(b0) : -1);
        if (kk < 0) {
          stop = 1;
        } else {
          const long long D = 1LL << (P.k_max - kk);
          tn = (ctl->slot[p].tau_c / D + 1) * D;
          if (tn > ctl->tau_e) stop = 2;
        }
      }
      s_tn = tn;
      s_stop = stop;
    }
  }
  __syncthreads();
  if (s_stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && s_stop != 3) {
      if (s_stop == 1) atomicOr(&ctl->err, kErrLevels);
      ctl->done = 1;
    }
    return;
  }
  const long long tn = s_tn;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->slot[p].tau_next = tn;
  const History& prev = HB;
  bool act = false;
  if (j < B.n) {
    const long long nt = tj + dtj;
    act = (nt == tn);
    if (nt < tn) atomicOr(&ctl->err, kErrInvariant);
    predict_body(B, P, prev, j, tj, tn, pass, act, L);
  }
  // compaction of the active list (order within a step is arbitrary)
  const unsigned bal = __ballot_sync(kFull, act);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && bal) base = atomicAdd(&ctl->slot[p].cnt, __popc(bal));
  base = __shfl_sync(kFull, base, 0);
  if (act) B.act[base + __popc(bal & ((1u << lane) - 1u))] = j;
}

// ---------------------------------------------------------------------
// Step C: correction (Eq. 1), next step (pass 0: standard block step;
// passes >= 1: Alg. 1 with Eq. 4), history append, level counts.
//
// The force launch leaves S split partial sums per active body (S = 1 for
// FP64 sums in ascending j). With few splits one thread takes a body and
// adds its partials in split order. With many splits (a small active set
// spread over the whole grid) a warp takes a body: lane l adds the
// contiguous splits [l per, (l + 1) per) in order, a fixed shuffle tree
// combines the lanes, and lane 0 corrects the body; the partials then
// arrive in one round of loads instead of S. Every order is fixed, so the
// result does not depend on timing.
// ---------------------------------------------------------------------
constexpr int kWarpSumMinSplits = 9;  // S at or above this: a warp per body

// one body's correction after its force sums are known; level-count
// changes go to the block's dh
__device__ __forceinline__ void correct_one(const Bodies& B, const Params& P,
                                            const History& cur,
                                            const History& prev,
                                            const StepSlot& sl, int pass,
                                            int k, const double an[3],
                                            double q, int* dh) {
  Ctl* ctl = P.ctl;
  const int i = B.act[k];
  const Corrected cr = correct_body(B, P, cur, prev, i, an, q, sl.tau_next,
                                    pass, sl.nrec + k, &ctl->err);
  const long long c = cr.d_new;
  if (cr.underflow) atomicAdd(&ctl->underflow, 1ULL);
  if (c != cr.d_old) {
    atomicSub(&dh[level_of(cr.d_old, P.k_max)], 1);
    atomicAdd(&dh[level_of(c, P.k_max)], 1);
  }
  if (P.lg_cap > 0) {
    const long long e = sl.lg_base + k;
    if (e < P.lg_cap) {
      P.lg_i[e] = i;
      P.lg_dt[e] = c;
    }
  }
}

__global__ void correct_kernel(Bodies B, Params P, History HA, History HB,
                               int p) {
  // everything below reads what the force launch wrote
  pdl_wait();
  pdl_launch_dependents();
  Ctl* ctl = P.ctl;
  // the step's values and the pass-over flag in one round of loads
  const int done = ctl->done;
  const StepSlot sl = ctl->slot[p];
  const int pass = ctl->pass;
  if (done) return;
  __shared__ int dh[kMaxLevels];
  for (int t = threadIdx.x; t < kMaxLevels; t += blockDim.x) dh[t] = 0;
  __syncthreads();
  const int n_act = sl.cnt;
  const int S = sl.nsplit;
  const History& cur = HA;
  const History& prev = HB;
  const double* part = B.part;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  // a warp per body only while every body gets its own warp: the FP64
  // correction of one lane costs a whole warp's issue slots
  if (S >= kWarpSumMinSplits && n_act <= nw) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int per = (S + 31) >> 5;
    for (int k = w0; k < n_act; k += nw) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, q = 0.0;
      int have = 0;
      const int lo = lane * per, hi = min(S, lo + per);
      for (int b0 = lo; b0 < hi; b0 += 4) {
        double x[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (b0 + u < hi) {
            const double* pp = part + (long long)(b0 + u) * 5 * n_act;
            x[u][0] = pp[k];
            x[u][1] = pp[n_act + k];
            x[u][2] = pp[2LL * n_act + k];
            x[u][3] = pp[4LL * n_act + k];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (b0 + u < hi) {
            if (!have) {
              s0 = x[u][0];
              s1 = x[u][1];
              s2 = x[u][2];
              q = x[u][3];
              have = 1;
            } else {
              s0 = __dadd_rn(s0, x[u][0]);
              s1 = __dadd_rn(s1, x[u][1]);
              s2 = __dadd_rn(s2, x[u][2]);
              q = fmax(q, x[u][3]);
            }
          }
        }
      }
      for (int off = 16; off >= 1; off >>= 1) {
        const double o0 = __shfl_down_sync(kFull, s0, off);
        const double o1 = __shfl_down_sync(kFull, s1, off);
        const double o2 = __shfl_down_sync(kFull, s2, off);
        const double oq = __shfl_down_sync(kFull, q, off);
        const int oh = __shfl_down_sync(kFull, have, off);
        if (lane < off && oh) {
          if (have) {
            s0 = __dadd_rn(s0, o0);
            s1 = __dadd_rn(s1, o1);
            s2 = __dadd_rn(s2, o2);
            q = fmax(q, oq);
          } else {
            s0 = o0;
            s1 = o1;
            s2 = o2;
            q = oq;
            have = 1;
          }
        }
      }
      if (lane == 0) {
        const double an[3] = {s0, s1, s2};
        correct_one(B, P, cur, prev, sl, pass, k, an, q, dh);
      }
    }
  } else {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_act;
         k += gridDim.x * blockDim.x) {
      double an[3], q;
      sum_partials(part, n_act, S, k, an, q);
      correct_one(B, P, cur, prev, sl, pass, k, an, q, dh);
    }
  }
  // level-count changes of this block, one global atomic per changed level
  __syncthreads();
  for (int t = threadIdx.x; t <= P.k_max; t += blockDim.x)
    if (dh[t]) atomicAdd(&ctl->hist[t], dh[t]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    StepSlot& nx = ctl->slot[p ^ 1];
    nx.tau_c = sl.tau_next;
    nx.tau_next = 0;
    nx.nrec = sl.nrec + n_act;
    nx.lg_base = sl.lg_base + n_act;
    nx.cnt = 0;
    nx.nsplit = 0;
    ctl->steps += 1ULL;
    ctl->inter += (unsigned long long)n_act * (unsigned long long)B.n;
    if (P.lg_cap > 0) {
      const long long s = ctl->log_steps;
      if (s < P.lg_cap) {
        P.lg_era[s] = ctl->era;
        P.lg_pass[s] = pass;
        P.lg_tau[s] = sl.tau_next;
        P.lg_nact[s] = n_act;
      }
      ctl->log_steps = s + 1;
      const long long over = sl.lg_base + n_act - P.lg_cap;
      ctl->log_drop += over <= 0 ? 0 : (over < n_act ? over : n_act);
      ctl->log_ent = sl.lg_base + n_act;
    }
  }
}

// ---------------------------------------------------------------------
// Era helpers: snapshot/restore, next-time extrema (Alg. 3)
// ---------------------------------------------------------------------
// ---------------------------------------------------------------------
// Between passes: the running pass's appended records become the next
// pass's previous-pass records in body-major (CSR) order. hoff is the
// exclusive scan of the per-body record counts; each record then moves to
// hoff[body] + rank.
// ---------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

// block-wide inclusive scan of one value per thread (kScanThreads threads)
__device__ __forceinline__ int block_inclusive_scan(int x, int* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  return wid ? x + warp_tot[wid - 1] : x;
}

__global__ void scan_block_sums_kernel(const int* cnt, int n, int* bsum) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int s = 0;
  for (int e = 0; e < kScanPer; ++e)
    if (base + e < n) s += cnt[base + e];
  const int inc = block_inclusive_scan(s, wt);
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = inc;
}

// exclusive scan of the block sums in place, one block
__global__ void scan_bsum_kernel(int* bsum, int nblk) {
  __shared__ int wt[kScanThreads / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblk; b0 += kScanThreads) {
    const int b = b0 + threadIdx.x;
    const int x = b < nblk ? bsum[b] : 0;
    const int inc = block_inclusive_scan(x, wt);
    const int c = carry;
    if (b < nblk) bsum[b] = c + inc - x;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c + inc;
    __syncthreads();
  }
}

__global__ void scan_write_kernel(const int* cnt, int n, const int* bsum,
                                  int* off) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int v[kScanPer], s = 0;
  for (int e = 0; e < kScanPer; ++e) {
    v[e] = base + e < n ? cnt[base + e] : 0;
    s += v[e];
  }
  int run = block_inclusive_scan(s, wt) - s + bsum[blockIdx.x];
  for (int e = 0; e < kScanPer; ++e) {
    run += v[e];
    if (base + e < n) off[base + e + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
}

__global__ void history_scatter_kernel(History src, History dst,
                                       const int* off, const Ctl* ctl) {
  long long nrec = ctl->slot[0].nrec > ctl->slot[1].nrec ? ctl->slot[0].nrec
                                                         : ctl->slot[1].nrec;
  if (nrec > src.cap) nrec = src.cap;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       r < nrec; r += (long long)gridDim.x * blockDim.x) {
    const long long d = (long long)off[src.body[r]] + src.seq[r];
    dst.tau[d] = src.tau[r];
    for (int c = 0; c < 3; ++c) {
      dst.r[c][d] = src.r[c][r];
      dst.v[c][d] = src.v[c][r];
      dst.a[c][d] = src.a[c][r];
    }
    dst.dts[d] = src.dts[r];
  }
}

// ---------------------------------------------------------------------
// Converged iteration (reading R15): after pass p >= 1, the pass repeated
// pass p - 1 when every body has as many records at the same times (the
// running pass's append buffer against the previous pass's CSR records)
// and every body's position at the end of the pass is within tol of the
// end of pass p - 1 (rlast). Any difference sets ctl->notconv.
// ---------------------------------------------------------------------
__global__ void converged_kernel(Bodies B, History cur, History prev,
                                 const double* rl0, const double* rl1,
                                 const double* rl2, double tol,
                                 long long nrec, Ctl* ctl) {
  int bad = 0;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < B.n; i += stride) {
    if (B.hcnt[i] != B.hoff[i + 1] - B.hoff[i]) bad = 1;
    if (!(fabs(B.r[0][i] - rl0[i]) < tol) || !(fabs(B.r[1][i] - rl1[i]) < tol) ||
        !(fabs(B.r[2][i] - rl2[i]) < tol))
      bad = 1;
  }
  for (long long r = tid; r < nrec; r += stride) {
    const int b = cur.body[r], q = cur.seq[r];
    const int cnt = B.hoff[b + 1] - B.hoff[b];
    if (q >= cnt || cur.tau[r] != prev.tau[B.hoff[b] + q]) bad = 1;
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0)
    atomicOr(&ctl->notconv, 1);
}

__global__ void copy_state_kernel(Bodies dst, Bodies src) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dst.n;
       i += gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      dst.r[c][i] = src.r[c][i];
      dst.v[c][i] = src.v[c][i];
      dst.a[c][i] = src.a[c][i];
    }
    dst.dts[i] = src.dts[i];
    dst.tau[i] = src.tau[i];
    dst.dt[i] = src.dt[i];
  }
}

__global__ void next_time_extrema_kernel(Bodies B, Ctl* ctl) {
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x) {
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
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&ctl->first, lo);
    atomicMax(&ctl->last, hi);
  }
}

// ---------------------------------------------------------------------
// Initialisation (Alg. 2 step 1)
// ---------------------------------------------------------------------
__global__ void load_aos_kernel(Bodies B, const double* m, const double* r,
                                const double* v, Ctl* ctl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x) {
    B.m[i] = m[i];
    B.mf[i] = (float)m[i];
    bool ok = isfinite(m[i]);
    for (int c = 0; c < 3; ++c) {
      const double x = r[3LL * i + c], u = v[3LL * i + c];
      B.r[c][i] = x;
      B.v[c][i] = u;
      B.a[c][i] = 0.0;
      ok = ok && isfinite(x) && isfinite(u);
    }
    B.tau[i] = 0;
    B.dt[i] = 1;
    B.dts[i] = 0.0;
    B.act[i] = i;
    if (!ok) atomicOr(&ctl->err, kErrNonFinite);
  }
}

// float masses of the mixed j records from the FP64 masses
__global__ void masses_to_float_kernel(Bodies B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.n;
       i += gridDim.x * blockDim.x)
    B.mf[i] = (float)B.m[i];
}

// j data of the initial state (prediction to t = 0 is the state itself)
__global__ void init_jdata_kernel(Bodies B, Params P) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B.n;
       j += gridDim.x * blockDim.x) {
    double rp[3], vp[3];
    for (int c = 0; c < 3; ++c) {
      rp[c] = B.r[c][j];
      vp[c] = B.v[c][j];
    }
    store_prediction(B, P, j, rp, vp);
  }
}

__global__ void init_finalize_kernel(Bodies B, Params P, const int* nsplit) {
  const int S = *nsplit;
  const int n = B.n;
  Ctl* ctl = P.ctl;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    double an[3], q;
    an[0] = B.part[0 * n + i];
    an[1] = B.part[1 * n + i];
    an[2] = B.part[2 * n + i];
    q = B.part[4 * n + i];
    #pragma unroll 4
    for (int sp = 1; sp < S; ++sp) {
      const double* pp = B.part + (long long)sp * 5 * n;
      an[0] = __dadd_rn(an[0], pp[0 * n + i]);
      an[1] = __dadd_rn(an[1], pp[1 * n + i]);
      an[2] = __dadd_rn(an[2], pp[2 * n + i]);
      q = fmax(q, pp[4 * n + i]);
    }
    if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]) || isnan(q))
      atomicOr(&ctl->err, kErrNonFinite);
    for (int c = 0; c < 3; ++c) B.a[c][i] = an[c];
    const double dts = __ddiv_rn(P.eta, __dsqrt_rn(q));
    B.dts[i] = dts;
    int uf = 0;
    B.dt[i] = level_ticks(dts, P.k_min, P.k_max, &uf);
    if (uf) atomicAdd(&ctl->underflow, 1ULL);
    B.tau[i] = 0;
  }
}

// ---------------------------------------------------------------------
// Energy at the system time (Sec. 3): Eq. 2 prediction of every body,
// per-body pair sums over ascending j, body sums over ascending i.
// ---------------------------------------------------------------------
__global__ void energy_predict_kernel(Bodies B, Params P, long long T) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B.n;
       j += gridDim.x * blockDim.x) {
    const double h = __dmul_rn((double)(T - B.tau[j]), P.inv_ticks);
    for (int c = 0; c < 3; ++c) {
      double rp, vp;
      taylor1(B.r[c][j], B.v[c][j], B.a[c][j], h, rp, vp);
      B.pr[c][j] = rp;
      B.pv[c][j] = vp;
    }
  }
}

template <int NT, int TJ>
__global__ void __launch_bounds__(NT) energy_pair_kernel(Bodies B, double eps2,
                                                         double* w) {
  __shared__ double sx[TJ], sy[TJ], sz[TJ], sm[TJ];
  const int n = B.n;
  for (int i0 = blockIdx.x * NT; i0 < n; i0 += gridDim.x * NT) {
    const int i = i0 + threadIdx.x;
    const bool valid = i < n;
    const double xi = valid ? B.pr[0][i] : 0.0;
    const double yi = valid ? B.pr[1][i] : 0.0;
    const double zi = valid ? B.pr[2][i] : 0.0;
    const double mi = valid ? B.m[i] : 0.0;
    double wi = 0.0;
    for (int jt = 0; jt < n; jt += TJ) {
      const int cnt = min(TJ, n - jt);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += NT) {
        sx[t] = B.pr[0][jt + t];
        sy[t] = B.pr[1][jt + t];
        sz[t] = B.pr[2][jt + t];
        sm[t] = B.m[jt + t];
      }
      __syncthreads();
      for (int t = 0; t < cnt; ++t) {
        if (jt + t == i) continue;
        const double dx = __dsub_rn(sx[t], xi);
        const double dy = __dsub_rn(sy[t], yi);
        const double dz = __dsub_rn(sz[t], zi);
        const double s2 = __dadd_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                      __dmul_rn(dz, dz)),
            eps2);
        wi = __dadd_rn(wi, __ddiv_rn(__dmul_rn(mi, sm[t]), __dsqrt_rn(s2)));
      }
    }
    if (valid) w[i] = wi;
  }
}

__global__ void energy_sum_kernel(Bodies B, const double* w, double* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double k = 0.0, p = 0.0;
  for (int i = 0; i < B.n; ++i) {
    const double vx = B.pv[0][i], vy = B.pv[1][i], vz = B.pv[2][i];
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)),
                                __dmul_rn(vz, vz));
    k = __dadd_rn(k, __dmul_rn(__dmul_rn(0.5, B.m[i]), v2));
    p = __dsub_rn(p, __dmul_rn(0.5, w[i]));
  }
  out[0] = k;
  out[1] = p;
}

// ---------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------
static inline int grid_for(int n, int threads, int cap = 1 << 16) {
  int g = (n + threads - 1) / threads;
  return g < 1 ? 1 : (g > cap ? cap : g);
}

void launch_pass_begin(Ctl* ctl, long long tau_s, long long tau_e, int pass,
                       int era, int n, cudaStream_t s) {
  pass_begin_kernel<<<1, kMaxLevels, 0, s>>>(ctl, tau_s, tau_e, pass, era, n);
}

void launch_history_to_csr(const Bodies& B, const History& append,
                           const History& csr, const Ctl* ctl, int sms,
                           cudaStream_t s) {
  const int nblk = (B.n + kScanBlock - 1) / kScanBlock;
  scan_block_sums_kernel<<<nblk, kScanThreads, 0, s>>>(B.hcnt, B.n,
                                                       B.scan_tmp);
  scan_bsum_kernel<<<1, kScanThreads, 0, s>>>(B.scan_tmp, nblk);
  scan_write_kernel<<<nblk, kScanThreads, 0, s>>>(B.hcnt, B.n, B.scan_tmp,
                                                  B.hoff);
  history_scatter_kernel<<<sms * 8, 256, 0, s>>>(append, csr, B.hoff, ctl);
}

void launch_pass_setup(const Bodies& B, const Params& P, const History& cur,
                       cudaStream_t s) {
  pass_setup_kernel<<<grid_for(B.n, 256, 2048), 256, 0, s>>>(B, P, cur);
}

cudaError_t launch_select_predict(const Bodies& B, const Params& P,
                                  const History& HA, const History& HB, int p,
                                  bool pdl, cudaStream_t s) {
  // 64-thread blocks spread the FP64 prediction over more SMs
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_for(B.n, 64, 1 << 30));
  cfg.blockDim = dim3(64);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, select_predict_kernel, B, P, HA, HB, p);
}

cudaError_t launch_correct(const Bodies& B, const Params& P,
                           const History& HA, const History& HB, int p,
                           int grid, bool pdl, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, correct_kernel, B, P, HA, HB, p);
}

void launch_converged(const Bodies& B, const History& cur,
                      const History& prev, double* const rlast[3], double tol,
                      long long nrec, Ctl* ctl, int sms, cudaStream_t s) {
  converged_kernel<<<sms * 4, 256, 0, s>>>(B, cur, prev, rlast[0], rlast[1],
                                           rlast[2], tol, nrec, ctl);
}

void launch_copy_state(const Bodies& dst, const Bodies& src, cudaStream_t s) {
  copy_state_kernel<<<grid_for(dst.n, 256, 4096), 256, 0, s>>>(dst, src);
}

void launch_next_time_extrema(const Bodies& B, Ctl* ctl, cudaStream_t s) {
  next_time_extrema_kernel<<<grid_for(B.n, 256, 1024), 256, 0, s>>>(B, ctl);
}

void launch_load_aos(const Bodies& B, const double* m, const double* r,
                     const double* v, Ctl* ctl, cudaStream_t s) {
  load_aos_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B, m, r, v, ctl);
}

void launch_masses_to_float(const Bodies& B, cudaStream_t s) {
  masses_to_float_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B);
}

void launch_init_jdata(const Bodies& B, const Params& P, cudaStream_t s) {
  init_jdata_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B, P);
}

void launch_init_finalize(const Bodies& B, const Params& P, const int* nsplit,
                          cudaStream_t s) {
  init_finalize_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B, P, nsplit);
}

void launch_energy(const Bodies& B, const Params& P, long long T, double* w,
                   double* out, int sms, cudaStream_t s) {
  energy_predict_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B, P, T);
  constexpr int NT = 128, TJ = 64;
  int g = grid_for(B.n, NT);
  energy_pair_kernel<NT, TJ><<<g, NT, 0, s>>>(B, P.eps2, w);
  energy_sum_kernel<<<1, 32, 0, s>>>(B, w, out);
  (void)sms;
}

void launch_energy_predict(const Bodies& B, const Params& P, long long T,
                           cudaStream_t s) {
  energy_predict_kernel<<<grid_for(B.n, 256), 256, 0, s>>>(B, P, T);
}

}  // namespace tsbts
