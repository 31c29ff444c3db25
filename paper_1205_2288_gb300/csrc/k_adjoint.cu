// Kernels of the adjoint of a frozen block schedule: the replay of an era's
// passes as plain block steps (prediction of every body, Eq. 3 force sums
// on the active bodies, Eq. 1 correction) and its reverse mode, one block
// step at a time in reverse order. In the first pass (or a lone pass) every
// body is predicted with Eq. 2 from its own state; in a later pass a body
// that is not active is placed from the previous pass's records (Sec. 2:
// the record on an exact hit, the cubic Hermite between the records that
// bracket the block time, else Eq. 2).
//
// Reverse step at block time T with active set A, given the cotangents
// (gr, gv, ga) of the post-step state:
//  - Eq. 1 (r_i' = p_i, v_i' = v_i + (a_i + f_i) h_i / 2, a_i' = f_i) gives
//    for i in A: lam_i = dL/df_i = ga_i + h_i gv_i / 2, the cotangent gr_i
//    of p_i, and ga_i <- h_i gv_i / 2, gr_i <- 0 for the pre-step state;
//  - the force f_i = sum_{j != i} m_j d_ij / s^3 (d_ij = p_j - p_i,
//    s^2 = |d_ij|^2 + eps^2) contributes, per pair,
//      g_ij = m_j (lam_i / s^3 - 3 (lam_i . d_ij) d_ij / s^5)
//    to p_j and -g_ij to p_i, and lam_i . d_ij / s^3 to m_j. The i side
//    (sum over j of g_ij for each active i) and the j side (sum over active
//    i for each body j) are two pair sums run by one launch;
//  - Eq. 2 (p_j = r_j + v_j h_j + a_j h_j^2 / 2) passes the position
//    cotangent to gr, gv and ga of every body.
// The pre-step state of each active body is restored from the tape written
// by the forward replay (or by the recomputation of a checkpointed
// segment), so no arithmetic is run backwards.
//
// Through several passes: a position cotangent of a body placed from
// records goes to those records (Hermite weights h00 and h10 h on record
// A's r and v, h01 and h11 h on record B's); when the step that wrote a
// record is reversed, the record's cotangent joins that of the body's
// post-step state. Every pass starts from the era-start state, so the
// passes' era-start cotangents add up (adj_pass_end_kernel).
//
// The FP64 replay uses the integrator's op-by-op FP64 expressions and force
// kernels, so it reproduces a sequential FP64 replay bit for bit when the
// force sums run in ascending j. The mixed pair terms of the reverse sweep
// are FP32 on double-single relative coordinates, two sources per packed
// f32x2 instruction, summed in FP32 over one shared-memory tile of sources
// and then in FP64.
#include <algorithm>

#include "force_device.cuh"
#include "tsbts_kernels.cuh"

namespace tsbts {

namespace {

constexpr int kAdjThreads = 128;

// tuning of the force vector-Jacobian product and the replay force
// (compile-time; defaults measured on GB300): lanes per target, threads in
// flight per SM that the split count aims at, most splits, sources per
// shared-memory tile, unroll of the packed pair loop, register budget hint
#ifndef TSBTS_VJP_TPT
#define TSBTS_VJP_TPT 4
#endif
#ifndef TSBTS_VJP_WANT
#define TSBTS_VJP_WANT 512
#endif
#ifndef TSBTS_VJP_SMAX
#define TSBTS_VJP_SMAX 16
#endif
#ifndef TSBTS_VJP_TILE
#define TSBTS_VJP_TILE 512
#endif
#ifndef TSBTS_VJP_UNROLL
#define TSBTS_VJP_UNROLL 2
#endif
#ifndef TSBTS_VJP_MINB
#define TSBTS_VJP_MINB 1
#endif
constexpr int kVjpTpt = TSBTS_VJP_TPT;
constexpr int kVjpWant = TSBTS_VJP_WANT;
constexpr int kVjpSmax = TSBTS_VJP_SMAX;
constexpr int kVjpMinBlocks = TSBTS_VJP_MINB;
constexpr int kVjpUnroll = TSBTS_VJP_UNROLL;

__device__ __forceinline__ void pack_ds(double x, double y, double z, float w,
                                        float4& hi, float4& lo) {
  const float xh = (float)x, yh = (float)y, zh = (float)z;
  hi = make_float4(xh, yh, zh, w);
  lo = make_float4((float)(x - (double)xh), (float)(y - (double)yh),
                   (float)(z - (double)zh), 0.f);
}

__device__ __forceinline__ double tick_h(long long T, long long tau,
                                         double inv_ticks) {
  return __dmul_rn((double)(T - tau), inv_ticks);
}

// predicted position of body j at block time T (Eq. 2) into P
__device__ __forceinline__ void predict_into(int j, long long T,
                                             double inv_ticks, int mixed,
                                             const AdjState& St,
                                             const AdjPred& P, double p[3]) {
  const double h = tick_h(T, St.tau[j], inv_ticks);
  for (int c = 0; c < 3; ++c) {
    double vp;
    taylor1(St.r[c][j], St.v[c][j], St.a[c][j], h, p[c], vp);
    P.p[c][j] = p[c];
  }
  if (mixed) {
    float4 hi, lo;
    pack_ds(p[0], p[1], p[2], (float)P.m[j], hi, lo);
    P.jhi[j] = hi;
    P.jlo[j] = lo;
  }
}

// packed j records of a predicted position
__device__ __forceinline__ void store_pred(int j, const double p[3], float w,
                                           int mixed, const AdjPred& P) {
  for (int c = 0; c < 3; ++c) P.p[c][j] = p[c];
  if (mixed) {
    float4 hi, lo;
    pack_ds(p[0], p[1], p[2], w, hi, lo);
    P.jhi[j] = hi;
    P.jlo[j] = lo;
  }
}

// ---------------------------------------------------------------------
// Records of the previous pass
// ---------------------------------------------------------------------

// Move body j's record cursor forward to its last record in Q at or before
// tick T (block ticks increase within a pass); each step follows the entry
// links to a later entry, below Q.hi, so the loop ends.
__device__ __forceinline__ long long q_advance(const AdjRecs& R,
                                               const AdjPass& Q, int j,
                                               long long T) {
  const long long c0 = Q.cur[j];
  long long cur = c0;
  for (;;) {
    const long long nx = cur < 0 ? Q.first[j] : R.next_e[cur];
    if (nx >= Q.hi || R.tau[nx] > T) break;
    cur = nx;
  }
  if (cur != c0) Q.cur[j] = cur;
  return cur;
}

// The same cursor moved backward (the reverse sweep's ticks decrease);
// each step follows the links to an earlier entry, or to -1 below Q.lo.
__device__ __forceinline__ long long q_retreat(const AdjRecs& R,
                                               const AdjPass& Q, int j,
                                               long long T) {
  const long long c0 = Q.cur[j];
  long long cur = c0;
  while (cur >= 0 && R.tau[cur] > T) {
    const long long pe = R.prev_e[cur];
    cur = pe >= Q.lo ? pe : -1;
  }
  if (cur != c0) Q.cur[j] = cur;
  return cur;
}

// Position of body j at tick T from Q's records, cur being its last record
// at or before T: the record on an exact hit (kind 1), the cubic Hermite
// between cur and the next record (kind 2), or nothing past the last
// record (kind 0: the caller uses Eq. 2). ra, rb: the records used.
__device__ __forceinline__ int q_place(const AdjRecs& R, const AdjPass& Q,
                                       int j, long long cur, long long T,
                                       double inv_ticks, double p[3],
                                       long long& ra, long long& rb) {
  ra = cur;
  rb = -1;
  const long long ta = cur < 0 ? R.tau0[j] : R.tau[cur];
  if (cur >= 0 && ta == T) {
    for (int c = 0; c < 3; ++c) p[c] = R.r[c][cur];
    return 1;
  }
  const long long nx = cur < 0 ? Q.first[j] : R.next_e[cur];
  if (nx >= Q.hi) return 0;
  rb = nx;
  const HermiteW w = hermite_weights(ta, R.tau[nx], T, inv_ticks);
  for (int c = 0; c < 3; ++c) {
    const double ya = cur < 0 ? R.r0[c][j] : R.r[c][cur];
    const double da = cur < 0 ? R.v0[c][j] : R.v[c][cur];
    p[c] = hermite1(w, ya, da, R.r[c][nx], R.v[c][nx]);
  }
  return 2;
}

// ---------------------------------------------------------------------
// Forward replay
// ---------------------------------------------------------------------

// a_in / tau_in: the era-start accelerations and ticks of a general start
// state (nullptr: zero, the initial force following)
__global__ void adj_load_kernel(int n, const double* m_in, const double* r_in,
                                const double* v_in, const double* a_in,
                                const long long* tau_in, int mixed,
                                double* m_out, AdjState St, AdjPred P,
                                int* err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    const double m = m_in[j];
    bool ok = isfinite(m);
    m_out[j] = m;
    double p[3];
    for (int c = 0; c < 3; ++c) {
      const double r = r_in[3LL * j + c], v = v_in[3LL * j + c];
      const double a = a_in ? a_in[3LL * j + c] : 0.0;
      ok = ok && isfinite(r) && isfinite(v) && isfinite(a);
      St.r[c][j] = r;
      St.v[c][j] = v;
      St.a[c][j] = a;
      P.p[c][j] = r;
      p[c] = r;
    }
    St.tau[j] = tau_in ? tau_in[j] : 0;
    if (mixed) {
      float4 hi, lo;
      pack_ds(p[0], p[1], p[2], (float)m, hi, lo);
      P.jhi[j] = hi;
      P.jlo[j] = lo;
    }
    if (!ok) atomicOr(err, 1);
  }
}

// sum of the force kernel's j-split partials of active slot k
__device__ __forceinline__ void partial_sum(const double* part, int n_act,
                                            int S, int k, double an[3]) {
  for (int c = 0; c < 3; ++c) an[c] = part[(long long)c * n_act + k];
  for (int sp = 1; sp < S; ++sp) {
    const double* pp = part + (long long)sp * 5 * n_act;
    for (int c = 0; c < 3; ++c)
      an[c] = __dadd_rn(an[c], pp[(long long)c * n_act + k]);
  }
}

// Initial accelerations (the force on every body at r0) and the Eq. 2
// prediction of every body to the first block time T_next (< 0: none).
// new accelerations of a step: from the replay force kernel's sums (F.f)
// when given, else from the integrator force kernel's j-split partials
struct FSum {
  const double* f[3];
};
__device__ __forceinline__ void force_of(const FSum& F, const double* part,
                                         int n_act, int S, int k,
                                         double an[3]) {
  if (F.f[0]) {
    for (int c = 0; c < 3; ++c) an[c] = F.f[c][k];
  } else {
    partial_sum(part, n_act, S, k, an);
  }
}

__global__ void adj_init_accel_kernel(int n, const double* part,
                                      const int* nsplit, FSum F,
                                      long long T_next, double inv_ticks,
                                      int mixed, AdjState St, AdjPred P,
                                      int* err) {
  const int S = F.f[0] ? 1 : *nsplit;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    double an[3];
    force_of(F, part, n, S, j, an);
    if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]))
      atomicOr(err, 1);
    for (int c = 0; c < 3; ++c) St.a[c][j] = an[c];
    if (T_next >= 0) {
      double p[3];
      predict_into(j, T_next, inv_ticks, mixed, St, P, p);
    }
  }
}

__global__ void adj_predict_kernel(int n, long long T, double inv_ticks,
                                   int mixed, AdjState St, AdjPred P,
                                   const long long* fwd_e, long long e_hi,
                                   AdjRecs R, AdjPass Q) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    double p[3];
    if (Q.on && fwd_e[j] >= e_hi) {
      long long ra, rb;
      const long long cur = q_advance(R, Q, j, T);
      if (q_place(R, Q, j, cur, T, inv_ticks, p, ra, rb)) {
        store_pred(j, p, mixed ? (float)P.m[j] : 0.f, mixed, P);
        continue;
      }
    }
    predict_into(j, T, inv_ticks, mixed, St, P, p);
  }
}

// The per-body kernels below are latency-bound: each body's loads are all
// issued before any of its stores (the state and cotangent arrays are
// reached through pointers the compiler must assume may alias), so that a
// body waits for at most two dependent rounds of memory accesses.

// Per body: Eq. 1 if the body is active in the step [e_lo, e_hi) of the
// schedule (fwd_e[j] is its next entry not yet replayed; the tape receives
// its pre-step state), then Eq. 2 prediction to the next block time T_next
// (< 0: none).
__global__ void adj_correct_predict_kernel(
    int n, int n_act, long long T, long long e_lo, long long e_hi,
    long long T_next, long long e_hi_next, double inv_ticks, int mixed,
    const double* part, const int* nsplit, FSum F, AdjState St, AdjPred P,
    AdjTape Tp, long long* fwd_e, const long long* next_e, AdjRecs R,
    AdjPass Q, int* err) {
  const int S = F.f[0] ? 1 : *nsplit;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    // loads
    const long long e = fwd_e[j];
    long long tau = St.tau[j];
    double r[3], v[3], a[3], p[3];
    for (int c = 0; c < 3; ++c) {
      r[c] = St.r[c][j];
      v[c] = St.v[c][j];
      a[c] = St.a[c][j];
      p[c] = P.p[c][j];
    }
    const float mf = mixed ? (float)P.m[j] : 0.f;
    const bool active = e < e_hi;
    double an[3] = {0.0, 0.0, 0.0};
    long long ne = 0;
    if (active) {
      force_of(F, part, n_act, S, (int)(e - e_lo), an);
      ne = next_e[e];
    }
    if (active) {
      if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]))
        atomicOr(err, 1);
      if (Tp.tau) {
        const long long t = e - Tp.base;
        for (int c = 0; c < 3; ++c) {
          Tp.x[c][t] = r[c];
          Tp.x[3 + c][t] = v[c];
          Tp.x[6 + c][t] = a[c];
        }
        Tp.tau[t] = tau;
      }
      // Eq. 1 over the body's own step
      const double h = tick_h(T, tau, inv_ticks);
      for (int c = 0; c < 3; ++c) {
        v[c] = __dadd_rn(v[c],
                         __dmul_rn(__dmul_rn(0.5, __dadd_rn(a[c], an[c])), h));
        r[c] = p[c];
        a[c] = an[c];
        St.r[c][j] = r[c];
        St.v[c][j] = v[c];
        St.a[c][j] = a[c];
      }
      tau = T;
      St.tau[j] = T;
      fwd_e[j] = ne;
      if (Q.write)
        for (int c = 0; c < 3; ++c) {
          R.r[c][e] = r[c];
          R.v[c][e] = v[c];
        }
    }
    if (T_next >= 0) {
      double q[3];
      int kind = 0;
      if (Q.on && (active ? ne : e) >= e_hi_next) {
        long long ra, rb;
        const long long cur = q_advance(R, Q, j, T_next);
        kind = q_place(R, Q, j, cur, T_next, inv_ticks, q, ra, rb);
      }
      if (!kind) {
        const double h = tick_h(T_next, tau, inv_ticks);
        for (int c = 0; c < 3; ++c) {
          double vp;
          taylor1(r[c], v[c], a[c], h, q[c], vp);
        }
      }
      store_pred(j, q, mf, mixed, P);
    }
  }
}

// ---------------------------------------------------------------------
// Reverse sweep
// ---------------------------------------------------------------------

// One kernel ends a reverse step and starts the step before it, body by
// body (each body's two halves touch only its own state and cotangents;
// the two steps use different slot arrays).
//
// End of the reverse step at block time F.T: the body's position cotangent
// (m_j G_j from the j side; for a body active in slot k also the cotangent
// of its new position minus u_k) passed through Eq. 2 to gr, gv, ga, and
// its mass cotangent Z_j.
//
// Start of the reverse step at block time R.T: restore the pre-step state
// of an active body from the tape (cur_e[j] is its latest entry not yet
// reversed), the Eq. 1 part of the reverse step, and the Eq. 2 prediction.
// With R.all every body is active at T = 0 (the initial force): its
// cotangent ga becomes lam and nothing is restored.
__global__ void adj_back_step_kernel(int n, double inv_ticks, int mixed,
                                     AdjBackFin F, AdjBackPrep R, AdjState St,
                                     AdjTape Tp, long long* cur_e,
                                     const long long* prev_e, AdjCot C,
                                     AdjPred P, VjpOut O, AdjRecs Rc,
                                     AdjPass Q, int* err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    // first round of loads
    const long long tau0 = St.tau[j];
    double gr[3], gv[3], ga[3];
    for (int c = 0; c < 3; ++c) {
      gr[c] = C.gr[c][j];
      gv[c] = C.gv[c][j];
      ga[c] = C.ga[c][j];
    }
    double gm = 0.0, G[4] = {0.0, 0.0, 0.0, 0.0}, mj = 0.0;
    int kf = -1;
    if (F.active) {
      gm = C.gm[j];
      kf = F.Sl.slot[j];
      for (int c = 0; c < 4; ++c) G[c] = O.g[c][j];
      mj = P.m[j];
    }
    long long e = -1;
    double r[3], v[3], a[3];
    long long tau1 = tau0;
    float mf = 0.f;
    if (R.active) {
      if (!R.all) e = cur_e[j];
      for (int c = 0; c < 3; ++c) {
        r[c] = St.r[c][j];
        v[c] = St.v[c][j];
        a[c] = St.a[c][j];
      }
      if (mixed) mf = (float)P.m[j];
    }
    // second round: the slot's values and the tape
    double gp0[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
    if (kf >= 0)
      for (int c = 0; c < 3; ++c) {
        gp0[c] = F.Sl.gp0[c][kf];
        u[c] = O.u[c][kf];
      }
    int kr = -1;
    long long pe = 0;
    if (R.active) {
      if (R.all) {
        kr = j;
      } else if (e >= R.e_lo) {
        kr = (int)(e - R.e_lo);
        const long long t = e - Tp.base;
        for (int c = 0; c < 3; ++c) {
          r[c] = Tp.x[c][t];
          v[c] = Tp.x[3 + c][t];
          a[c] = Tp.x[6 + c][t];
        }
        tau1 = Tp.tau[t];
        pe = prev_e[e];
      }
    }
    // end of the step at F.T
    if (F.active) {
      double gp[3];
      for (int c = 0; c < 3; ++c) {
        gp[c] = mj * G[c];
        if (kf >= 0) gp[c] = gp0[c] + (gp[c] - u[c]);
      }
      if (!isfinite(gp[0]) || !isfinite(gp[1]) || !isfinite(gp[2]) ||
          !isfinite(G[3]))
        atomicOr(err, 1);
      gm += G[3];
      const int kind = kf < 0 && Q.on ? Rc.kind[j] : 0;
      if (kind == 0) {
        const double h = tick_h(F.T, tau0, inv_ticks);
        const double hh2 = 0.5 * h * h;
        for (int c = 0; c < 3; ++c) {
          gr[c] += gp[c];
          gv[c] += h * gp[c];
          ga[c] += hh2 * gp[c];
        }
      } else {
        // placed from the previous pass's records: their cotangents
        const long long ra = Rc.ra[j];
        double* ar[3];
        for (int c = 0; c < 3; ++c) ar[c] = ra < 0 ? Q.g0r[c] + j : Rc.gr[c] + ra;
        if (kind == 1) {
          for (int c = 0; c < 3; ++c) *ar[c] += gp[c];
        } else {
          const long long rb = Rc.rb[j];
          const long long ta = ra < 0 ? Rc.tau0[j] : Rc.tau[ra];
          const HermiteW w = hermite_weights(ta, Rc.tau[rb], F.T, inv_ticks);
          for (int c = 0; c < 3; ++c) {
            double* av = ra < 0 ? Q.g0v[c] + j : Rc.gv[c] + ra;
            *ar[c] += w.h00 * gp[c];
            *av += w.h10h * gp[c];
            Rc.gr[c][rb] += w.h01 * gp[c];
            Rc.gv[c][rb] += w.h11h * gp[c];
          }
        }
      }
      C.gm[j] = gm;
    }
    // an active body's record cotangent (written when the next pass was
    // reversed) joins its post-step state's
    if (kr >= 0 && !R.all && Q.inject)
      for (int c = 0; c < 3; ++c) {
        gr[c] += Rc.gr[c][e];
        gv[c] += Rc.gv[c][e];
      }
    // start of the step at R.T
    if (R.active) {
      const AdjSlots& Sl = R.Sl;
      const double h = tick_h(R.T, tau1, inv_ticks);
      double p[3];
      int kind = 0;
      if (kr < 0 && Q.on) {
        long long ra, rb;
        const long long cur = q_retreat(Rc, Q, j, R.T);
        kind = q_place(Rc, Q, j, cur, R.T, inv_ticks, p, ra, rb);
        Rc.kind[j] = kind;
        Rc.ra[j] = ra;
        Rc.rb[j] = rb;
      }
      if (!kind)
        for (int c = 0; c < 3; ++c) {
          double vp;
          taylor1(r[c], v[c], a[c], h, p[c], vp);
        }
      if (kr >= 0 && !R.all) {
        for (int c = 0; c < 3; ++c) {
          St.r[c][j] = r[c];
          St.v[c][j] = v[c];
          St.a[c][j] = a[c];
        }
        St.tau[j] = tau1;
        cur_e[j] = pe;
      }
      Sl.slot[j] = kr;
      store_pred(j, p, mf, mixed, P);
      if (kr >= 0) {
        const double hh = __dmul_rn(0.5, h);
        double lam[3];
        for (int c = 0; c < 3; ++c) {
          const double gv_h = __dmul_rn(hh, gv[c]);
          lam[c] = R.all ? ga[c] : __dadd_rn(ga[c], gv_h);
          Sl.lam[c][kr] = lam[c];
          Sl.gp0[c][kr] = R.all ? 0.0 : gr[c];
          Sl.ap[c][kr] = p[c];
          ga[c] = R.all ? 0.0 : gv_h;
          if (!R.all) gr[c] = 0.0;
        }
        if (mixed) {
          float4 hi, lo;
          pack_ds(p[0], p[1], p[2], 0.f, hi, lo);
          Sl.ahi[kr] = hi;
          Sl.alo[kr] = lo;
          Sl.alam[kr] =
              make_float4((float)lam[0], (float)lam[1], (float)lam[2], 0.f);
        }
      }
    }
    for (int c = 0; c < 3; ++c) {
      C.gr[c][j] = gr[c];
      C.gv[c][j] = gv[c];
      C.ga[c][j] = ga[c];
    }
  }
}

// End of one pass's reverse sweep (every pass starts from the era-start
// state): G0 += the state's cotangents plus those of the pass's era-start
// records (cleared for the pass two earlier); the state's cotangents then
// restart from zero for the pass before, or become G0 after the first pass.
__global__ void adj_pass_end_kernel(int n, AdjCot C, AdjCot G0,
                                    AdjPass Qp, int last) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double sr = C.gr[c][j] + Qp.g0r[c][j];
      const double sv = C.gv[c][j] + Qp.g0v[c][j];
      const double r = G0.gr[c][j] + sr;
      const double v = G0.gv[c][j] + sv;
      const double a = G0.ga[c][j] + C.ga[c][j];
      G0.gr[c][j] = r;
      G0.gv[c][j] = v;
      G0.ga[c][j] = a;
      Qp.g0r[c][j] = 0.0;
      Qp.g0v[c][j] = 0.0;
      C.gr[c][j] = last ? r : 0.0;
      C.gv[c][j] = last ? v : 0.0;
      C.ga[c][j] = last ? a : 0.0;
    }
  }
}

// ---------------------------------------------------------------------
// Force vector-Jacobian product
// ---------------------------------------------------------------------
//
// i side: for active slot k (body i), u_k = sum_{j != i} g_ij
//   = lam_i W_i - 3 U_i,  W_i = sum m_j / s^3,
//   U_i = sum m_j (lam_i . d_ij) d_ij / s^5.
// j side: for body j, G_j = sum_{i in A, i != j} (lam_i / s^3
//   - 3 (lam_i . d_ij) d_ij / s^5) and Z_j = sum lam_i . d_ij / s^3, with
// d_ij = p_j - p_i; body j's position cotangent gets m_j G_j, its mass
// cotangent Z_j.
//
// Work split (both sides): a block holds IG = 128 / tpt targets with tpt
// lanes each and runs one of S chunks of the sources. Lane sums are added
// in a fixed shuffle tree; with S > 1 each block writes one partial per
// target and the last block of the group to finish (counted with an
// atomic) adds the S partials in split order, so the result does not
// depend on which block finished first.

struct VjpArgs {
  int n, n_act;
  const int* idx;   // body of each active slot
  double eps2;
  float eps2f;
  AdjPred P;
  AdjSlots Sl;
  VjpShape V;
  int iblocks;
  VjpOut O;
};

struct VjpSm {
  int last;
  double sums[4][kAdjThreads];
};

template <int kN>
__device__ __forceinline__ void lane_reduce(double (&x)[kN], int tpt) {
  for (int o = tpt >> 1; o > 0; o >>= 1)
    for (int c = 0; c < kN; ++c) x[c] += __shfl_xor_sync(kFull, x[c], o);
}

struct VjpBlock {
  int g;        // target group
  int sp;       // source split
  int t0;       // first target of the group
  int tl;       // this thread's target within the group
  int tgt;      // its target
  int lane;     // its lane among the target's tpt threads
  int beg, end; // source range of the split
  bool live;
};

__device__ __forceinline__ VjpBlock vjp_block(const VjpSide& V, int b,
                                              int n_targets, int n_sources) {
  VjpBlock B;
  const int ig = kAdjThreads / V.tpt;
  B.g = b / V.S;
  B.sp = b - B.g * V.S;
  B.t0 = B.g * ig;
  B.tl = threadIdx.x / V.tpt;
  B.tgt = B.t0 + B.tl;
  B.lane = threadIdx.x & (V.tpt - 1);
  B.live = B.tgt < n_targets;
  B.beg = B.sp * V.chunk;
  B.end = min(n_sources, B.beg + V.chunk);
  return B;
}

// the reduced sums of one target: i side (kSide 0) u = lam W - 3 U into
// O.u; j side (kSide 1) G, Z into O.g; replay force (kSide 2) into O.f
template <int kSide>
__device__ __forceinline__ void vjp_store(const VjpArgs& A, int t,
                                          const double (&x)[4]) {
  if (kSide == 0) {
    for (int c = 0; c < 3; ++c)
      A.O.u[c][t] = A.Sl.lam[c][t] * x[0] - 3.0 * x[1 + c];
  } else if (kSide == 1) {
    for (int c = 0; c < 4; ++c) A.O.g[c][t] = x[c];
  } else {
    for (int c = 0; c < 3; ++c) A.O.f[c][t] = x[c];
  }
}

template <int kSide>
__device__ __forceinline__ void vjp_finish(const VjpArgs& A, const VjpSide& V,
                                           const VjpBlock& B, int n_targets,
                                           double (&acc)[4], double* part,
                                           int* cnt, VjpSm& sm) {
  lane_reduce(acc, V.tpt);
  if (V.S == 1) {
    if (B.live && B.lane == 0) vjp_store<kSide>(A, B.tgt, acc);
    return;
  }
  const int ig = kAdjThreads / V.tpt;
  double* gp = part + (long long)B.g * V.S * 4 * ig;
  if (B.lane == 0)
    for (int c = 0; c < 4; ++c) gp[((long long)B.sp * 4 + c) * ig + B.tl] = acc[c];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sm.last = atomicAdd(&cnt[B.g], 1) == V.S - 1;
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  for (int o = threadIdx.x; o < 4 * ig; o += kAdjThreads) {
    const int c = o / ig, t = o - c * ig;
    const double* q = gp + (long long)c * ig + t;
    const long long stride = 4LL * ig;
    double x = 0.0;
    int sp = 0;
    // eight loads in flight, then added in split order
    for (; sp + 8 <= V.S; sp += 8) {
      double y[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) y[w] = __ldcg(q + (sp + w) * stride);
#pragma unroll
      for (int w = 0; w < 8; ++w) x += y[w];
    }
    for (; sp < V.S; ++sp) x += __ldcg(q + sp * stride);
    sm.sums[c][t] = x;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ig; t += kAdjThreads) {
    if (B.t0 + t < n_targets) {
      const double x[4] = {sm.sums[0][t], sm.sums[1][t], sm.sums[2][t],
                           sm.sums[3][t]};
      vjp_store<kSide>(A, B.t0 + t, x);
    }
  }
  if (threadIdx.x == 0) cnt[B.g] = 0;  // ready for the next launch
}

// FP64: plain loops over the sources, FP64 sums.
__device__ __forceinline__ void vjp_i_f64(const VjpArgs& A, int b, VjpSm& sm) {
  const VjpSide& V = A.V.si;
  const VjpBlock B = vjp_block(V, b, A.n_act, A.n);
  const int k = B.tgt;
  const int end = B.live ? B.end : B.beg;
  const int bi = B.live ? A.idx[k] : -1;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // W, U
  double ix = 0, iy = 0, iz = 0, lx = 0, ly = 0, lz = 0;
  if (B.live) {
    ix = A.Sl.ap[0][k];
    iy = A.Sl.ap[1][k];
    iz = A.Sl.ap[2][k];
    lx = A.Sl.lam[0][k];
    ly = A.Sl.lam[1][k];
    lz = A.Sl.lam[2][k];
  }
  for (int j = B.beg + B.lane; j < end; j += V.tpt) {
    const double dx = A.P.p[0][j] - ix;
    const double dy = A.P.p[1][j] - iy;
    const double dz = A.P.p[2][j] - iz;
    const double s2 = dx * dx + dy * dy + dz * dz + A.eps2;
    const double rs = (j == bi) ? 0.0 : rsqrt(s2);
    const double rs2 = rs * rs;
    const double mr3 = A.P.m[j] * rs2 * rs;
    const double cc = mr3 * rs2 * (lx * dx + ly * dy + lz * dz);
    acc[0] += mr3;
    acc[1] += cc * dx;
    acc[2] += cc * dy;
    acc[3] += cc * dz;
  }
  vjp_finish<0>(A, V, B, A.n_act, acc, A.O.part_i, A.O.cnt_i, sm);
}

__device__ __forceinline__ void vjp_j_f64(const VjpArgs& A, int b, VjpSm& sm) {
  const VjpSide& V = A.V.sj;
  const VjpBlock B = vjp_block(V, b, A.n, A.n_act);
  const int j = B.tgt;
  const int end = B.live ? B.end : B.beg;
  const int sj = B.live ? A.Sl.slot[j] : -1;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // G, Z
  double px = 0, py = 0, pz = 0;
  if (B.live) {
    px = A.P.p[0][j];
    py = A.P.p[1][j];
    pz = A.P.p[2][j];
  }
  for (int k = B.beg + B.lane; k < end; k += V.tpt) {
    const double lx = A.Sl.lam[0][k], ly = A.Sl.lam[1][k],
                 lz = A.Sl.lam[2][k];
    const double dx = px - A.Sl.ap[0][k];
    const double dy = py - A.Sl.ap[1][k];
    const double dz = pz - A.Sl.ap[2][k];
    const double s2 = dx * dx + dy * dy + dz * dz + A.eps2;
    const double rs = (k == sj) ? 0.0 : rsqrt(s2);
    const double rs2 = rs * rs;
    const double rs3 = rs2 * rs;
    const double t = (lx * dx + ly * dy + lz * dz) * rs3;
    const double cc = -3.0 * t * rs2;
    acc[0] += rs3 * lx + cc * dx;
    acc[1] += rs3 * ly + cc * dy;
    acc[2] += rs3 * lz + cc * dz;
    acc[3] += t;
  }
  vjp_finish<1>(A, V, B, A.n, acc, A.O.part_j, A.O.cnt_j, sm);
}

// Mixed: sources staged in shared memory by tiles of kVjpTile, structure of
// arrays, and taken four at a time (128-bit shared loads) as two packed
// pairs; every FMA-pipe operation works on two sources at once (f32x2).
// A tile is padded to a multiple of 4 tpt with neutral sources (zero mass
// or zero lam, far away), so every lane runs the same packed loop. A warp
// whose target sits in the tile runs the masked loop, where the target's
// own pair gets 1/s = 0 and adds exact zeros.
constexpr int kVjpTile = TSBTS_VJP_TILE;
constexpr float kFar = 1.0e18f;

struct __align__(16) VjpTileI {
  float xh[kVjpTile], yh[kVjpTile], zh[kVjpTile], m[kVjpTile];
  float xl[kVjpTile], yl[kVjpTile], zl[kVjpTile];
};
struct __align__(16) VjpTileJ {
  float xh[kVjpTile], yh[kVjpTile], zh[kVjpTile];
  float xl[kVjpTile], yl[kVjpTile], zl[kVjpTile];
  float lx[kVjpTile], ly[kVjpTile], lz[kVjpTile];
};
union VjpSmem {
  VjpTileI i;
  VjpTileJ j;
};

__device__ __forceinline__ ulonglong2 ld4(const float* p) {
  return *reinterpret_cast<const ulonglong2*>(p);
}

// two sources (tile slots c, c + 1) on one active body: ii holds the
// target's hi (0..2), lo (3..5) and lam (6..8), each broadcast to a pair
template <bool kMask>
__device__ __forceinline__ void pair_vjp_i2(const f2 (&ii)[9], f2 xh, f2 yh,
                                            f2 zh, f2 m, f2 xl, f2 yl, f2 zl,
                                            int c, int self, f2 e2, f2& W,
                                            f2& Ux, f2& Uy, f2& Uz) {
  const f2 dx = add2(sub2(xh, ii[0]), sub2(xl, ii[3]));
  const f2 dy = add2(sub2(yh, ii[1]), sub2(yl, ii[4]));
  const f2 dz = add2(sub2(zh, ii[2]), sub2(zl, ii[5]));
  const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
  float s0, s1;
  upk(s2, s0, s1);
  float r0 = rsqrtf(s0), r1 = rsqrtf(s1);
  if (kMask) {
    if (c == self) r0 = 0.f;
    if (c + 1 == self) r1 = 0.f;
  }
  const f2 rs = pk(r0, r1);
  const f2 rs2 = mul2(rs, rs);
  const f2 mr3 = mul2(mul2(m, rs), rs2);
  const f2 ld = fma2(ii[6], dx, fma2(ii[7], dy, mul2(ii[8], dz)));
  const f2 cc = mul2(mul2(mr3, rs2), ld);
  W = add2(W, mr3);
  Ux = fma2(cc, dx, Ux);
  Uy = fma2(cc, dy, Uy);
  Uz = fma2(cc, dz, Uz);
}

// two active sources (tile slots c, c + 1) on one body: jj holds the
// target's hi (0..2) and lo (3..5)
template <bool kMask>
__device__ __forceinline__ void pair_vjp_j2(const f2 (&jj)[6], f2 xh, f2 yh,
                                            f2 zh, f2 xl, f2 yl, f2 zl, f2 lx,
                                            f2 ly, f2 lz, int c, int self,
                                            f2 e2, f2 m3, f2& G0, f2& G1,
                                            f2& G2, f2& Z) {
  const f2 dx = add2(sub2(jj[0], xh), sub2(jj[3], xl));
  const f2 dy = add2(sub2(jj[1], yh), sub2(jj[4], yl));
  const f2 dz = add2(sub2(jj[2], zh), sub2(jj[5], zl));
  const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
  float s0, s1;
  upk(s2, s0, s1);
  float r0 = rsqrtf(s0), r1 = rsqrtf(s1);
  if (kMask) {
    if (c == self) r0 = 0.f;
    if (c + 1 == self) r1 = 0.f;
  }
  const f2 rs = pk(r0, r1);
  const f2 rs2 = mul2(rs, rs);
  const f2 rs3 = mul2(rs2, rs);
  const f2 t = mul2(fma2(lx, dx, fma2(ly, dy, mul2(lz, dz))), rs3);
  Z = add2(Z, t);
  const f2 cc = mul2(mul2(t, rs2), m3);
  G0 = fma2(cc, dx, fma2(rs3, lx, G0));
  G1 = fma2(cc, dy, fma2(rs3, ly, G1));
  G2 = fma2(cc, dz, fma2(rs3, lz, G2));
}

__device__ __forceinline__ float hsum(f2 x) {
  float a, b;
  upk(x, a, b);
  return a + b;
}

__device__ __forceinline__ void vjp_i_mixed(const VjpArgs& A, int b,
                                            VjpSmem& T0, VjpSm& sm) {
  const VjpSide& V = A.V.si;
  const VjpBlock B = vjp_block(V, b, A.n_act, A.n);
  const int k = B.tgt;
  const int bi = B.live ? A.idx[k] : -1;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 ih = B.live ? A.Sl.ahi[k] : z4;
  const float4 il = B.live ? A.Sl.alo[k] : z4;
  const float4 lm = B.live ? A.Sl.alam[k] : z4;
  const f2 ii[9] = {pk(ih.x, ih.x), pk(ih.y, ih.y), pk(ih.z, ih.z),
                    pk(il.x, il.x), pk(il.y, il.y), pk(il.z, il.z),
                    pk(lm.x, lm.x), pk(lm.y, lm.y), pk(lm.z, lm.z)};
  const f2 e2 = pk(A.eps2f, A.eps2f);
  const int step = 4 * V.tpt;
  DS dacc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // W, U
  VjpTileI& T = T0.i;
  for (int jt = B.beg; jt < B.end; jt += kVjpTile) {
    const int cnt = min(kVjpTile, B.end - jt);
    const int cntp = (cnt + step - 1) / step * step;
    __syncthreads();
    for (int c = threadIdx.x; c < cntp; c += kAdjThreads) {
      if (c < cnt) {
        const float4 h = A.P.jhi[jt + c], l = A.P.jlo[jt + c];
        T.xh[c] = h.x; T.yh[c] = h.y; T.zh[c] = h.z; T.m[c] = h.w;
        T.xl[c] = l.x; T.yl[c] = l.y; T.zl[c] = l.z;
      } else {
        T.xh[c] = kFar; T.yh[c] = kFar; T.zh[c] = kFar; T.m[c] = 0.f;
        T.xl[c] = 0.f; T.yl[c] = 0.f; T.zl[c] = 0.f;
      }
    }
    __syncthreads();
    const bool self_here = B.live && bi >= jt && bi < jt + cnt;
    const int sc = self_here ? bi - jt : -1;
    f2 W = pk(0.f, 0.f), Ux = W, Uy = W, Uz = W;
    if (__any_sync(kFull, self_here)) {
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), m = ld4(&T.m[c]),
                         xl = ld4(&T.xl[c]), yl = ld4(&T.yl[c]),
                         zl = ld4(&T.zl[c]);
        pair_vjp_i2<true>(ii, xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, c, sc,
                          e2, W, Ux, Uy, Uz);
        pair_vjp_i2<true>(ii, xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, c + 2,
                          sc, e2, W, Ux, Uy, Uz);
      }
    } else {
#pragma unroll kVjpUnroll
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), m = ld4(&T.m[c]),
                         xl = ld4(&T.xl[c]), yl = ld4(&T.yl[c]),
                         zl = ld4(&T.zl[c]);
        pair_vjp_i2<false>(ii, xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, c,
                           -1, e2, W, Ux, Uy, Uz);
        pair_vjp_i2<false>(ii, xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, c + 2,
                           -1, e2, W, Ux, Uy, Uz);
      }
    }
    ds_add(dacc[0], hsum(W));
    ds_add(dacc[1], hsum(Ux));
    ds_add(dacc[2], hsum(Uy));
    ds_add(dacc[3], hsum(Uz));
  }
  double acc[4];
  for (int c = 0; c < 4; ++c) acc[c] = (double)dacc[c].hi + (double)dacc[c].lo;
  vjp_finish<0>(A, V, B, A.n_act, acc, A.O.part_i, A.O.cnt_i, sm);
}

__device__ __forceinline__ void vjp_j_mixed(const VjpArgs& A, int b,
                                            VjpSmem& T0, VjpSm& sm) {
  const VjpSide& V = A.V.sj;
  const VjpBlock B = vjp_block(V, b, A.n, A.n_act);
  const int j = B.tgt;
  const int sj = B.live ? A.Sl.slot[j] : -1;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 th = B.live ? A.P.jhi[j] : z4;
  const float4 tl = B.live ? A.P.jlo[j] : z4;
  const f2 jj[6] = {pk(th.x, th.x), pk(th.y, th.y), pk(th.z, th.z),
                    pk(tl.x, tl.x), pk(tl.y, tl.y), pk(tl.z, tl.z)};
  const f2 e2 = pk(A.eps2f, A.eps2f);
  const f2 m3 = pk(-3.f, -3.f);
  const int step = 4 * V.tpt;
  DS dacc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // G, Z
  VjpTileJ& T = T0.j;
  for (int kt = B.beg; kt < B.end; kt += kVjpTile) {
    const int cnt = min(kVjpTile, B.end - kt);
    const int cntp = (cnt + step - 1) / step * step;
    __syncthreads();
    for (int c = threadIdx.x; c < cntp; c += kAdjThreads) {
      if (c < cnt) {
        const float4 h = A.Sl.ahi[kt + c], l = A.Sl.alo[kt + c],
                     lm = A.Sl.alam[kt + c];
        T.xh[c] = h.x; T.yh[c] = h.y; T.zh[c] = h.z;
        T.xl[c] = l.x; T.yl[c] = l.y; T.zl[c] = l.z;
        T.lx[c] = lm.x; T.ly[c] = lm.y; T.lz[c] = lm.z;
      } else {
        T.xh[c] = kFar; T.yh[c] = kFar; T.zh[c] = kFar;
        T.xl[c] = 0.f; T.yl[c] = 0.f; T.zl[c] = 0.f;
        T.lx[c] = 0.f; T.ly[c] = 0.f; T.lz[c] = 0.f;
      }
    }
    __syncthreads();
    const bool self_here = sj >= kt && sj < kt + cnt;
    const int sc = self_here ? sj - kt : -1;
    f2 G0 = pk(0.f, 0.f), G1 = G0, G2 = G0, Z = G0;
    if (__any_sync(kFull, self_here)) {
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), xl = ld4(&T.xl[c]),
                         yl = ld4(&T.yl[c]), zl = ld4(&T.zl[c]),
                         lx = ld4(&T.lx[c]), ly = ld4(&T.ly[c]),
                         lz = ld4(&T.lz[c]);
        pair_vjp_j2<true>(jj, xh.x, yh.x, zh.x, xl.x, yl.x, zl.x, lx.x, ly.x,
                          lz.x, c, sc, e2, m3, G0, G1, G2, Z);
        pair_vjp_j2<true>(jj, xh.y, yh.y, zh.y, xl.y, yl.y, zl.y, lx.y, ly.y,
                          lz.y, c + 2, sc, e2, m3, G0, G1, G2, Z);
      }
    } else {
#pragma unroll kVjpUnroll
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), xl = ld4(&T.xl[c]),
                         yl = ld4(&T.yl[c]), zl = ld4(&T.zl[c]),
                         lx = ld4(&T.lx[c]), ly = ld4(&T.ly[c]),
                         lz = ld4(&T.lz[c]);
        pair_vjp_j2<false>(jj, xh.x, yh.x, zh.x, xl.x, yl.x, zl.x, lx.x,
                           ly.x, lz.x, c, -1, e2, m3, G0, G1, G2, Z);
        pair_vjp_j2<false>(jj, xh.y, yh.y, zh.y, xl.y, yl.y, zl.y, lx.y,
                           ly.y, lz.y, c + 2, -1, e2, m3, G0, G1, G2, Z);
      }
    }
    ds_add(dacc[0], hsum(G0));
    ds_add(dacc[1], hsum(G1));
    ds_add(dacc[2], hsum(G2));
    ds_add(dacc[3], hsum(Z));
  }
  double acc[4];
  for (int c = 0; c < 4; ++c) acc[c] = (double)dacc[c].hi + (double)dacc[c].lo;
  vjp_finish<1>(A, V, B, A.n, acc, A.O.part_j, A.O.cnt_j, sm);
}

// Replay force (mixed): a_i = sum_{j != i} m_j d_ij / s^3 for the active
// bodies at the predicted positions, with the i side's work split, tiles
// and packed pair loop; the sums are double-single per lane, FP64 after.
template <bool kMask>
__device__ __forceinline__ void pair_force2(const f2 (&ii)[6], f2 xh, f2 yh,
                                            f2 zh, f2 m, f2 xl, f2 yl, f2 zl,
                                            int c, int self, f2 e2, f2& ax,
                                            f2& ay, f2& az) {
  const f2 dx = add2(sub2(xh, ii[0]), sub2(xl, ii[3]));
  const f2 dy = add2(sub2(yh, ii[1]), sub2(yl, ii[4]));
  const f2 dz = add2(sub2(zh, ii[2]), sub2(zl, ii[5]));
  const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
  float s0, s1;
  upk(s2, s0, s1);
  float r0 = rsqrtf(s0), r1 = rsqrtf(s1);
  if (kMask) {
    if (c == self) r0 = 0.f;
    if (c + 1 == self) r1 = 0.f;
  }
  const f2 rs = pk(r0, r1);
  const f2 mr3 = mul2(mul2(m, rs), mul2(rs, rs));
  ax = fma2(mr3, dx, ax);
  ay = fma2(mr3, dy, ay);
  az = fma2(mr3, dz, az);
}

__device__ __forceinline__ void force_mixed(const VjpArgs& A, int b,
                                            VjpSmem& T0, VjpSm& sm) {
  const VjpSide& V = A.V.si;
  const VjpBlock B = vjp_block(V, b, A.n_act, A.n);
  const int bi = B.live ? A.idx[B.tgt] : -1;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 ih = B.live ? A.P.jhi[bi] : z4;
  const float4 il = B.live ? A.P.jlo[bi] : z4;
  const f2 ii[6] = {pk(ih.x, ih.x), pk(ih.y, ih.y), pk(ih.z, ih.z),
                    pk(il.x, il.x), pk(il.y, il.y), pk(il.z, il.z)};
  const f2 e2 = pk(A.eps2f, A.eps2f);
  const int step = 4 * V.tpt;
  DS dacc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  VjpTileI& T = T0.i;
  for (int jt = B.beg; jt < B.end; jt += kVjpTile) {
    const int cnt = min(kVjpTile, B.end - jt);
    const int cntp = (cnt + step - 1) / step * step;
    __syncthreads();
    for (int c = threadIdx.x; c < cntp; c += kAdjThreads) {
      if (c < cnt) {
        const float4 h = A.P.jhi[jt + c], l = A.P.jlo[jt + c];
        T.xh[c] = h.x; T.yh[c] = h.y; T.zh[c] = h.z; T.m[c] = h.w;
        T.xl[c] = l.x; T.yl[c] = l.y; T.zl[c] = l.z;
      } else {
        T.xh[c] = kFar; T.yh[c] = kFar; T.zh[c] = kFar; T.m[c] = 0.f;
        T.xl[c] = 0.f; T.yl[c] = 0.f; T.zl[c] = 0.f;
      }
    }
    __syncthreads();
    const bool self_here = B.live && bi >= jt && bi < jt + cnt;
    const int sc = self_here ? bi - jt : -1;
    f2 ax = pk(0.f, 0.f), ay = ax, az = ax;
    if (__any_sync(kFull, self_here)) {
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), m = ld4(&T.m[c]),
                         xl = ld4(&T.xl[c]), yl = ld4(&T.yl[c]),
                         zl = ld4(&T.zl[c]);
        pair_force2<true>(ii, xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, c, sc,
                          e2, ax, ay, az);
        pair_force2<true>(ii, xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, c + 2,
                          sc, e2, ax, ay, az);
      }
    } else {
#pragma unroll kVjpUnroll
      for (int c = 4 * B.lane; c < cntp; c += step) {
        const ulonglong2 xh = ld4(&T.xh[c]), yh = ld4(&T.yh[c]),
                         zh = ld4(&T.zh[c]), m = ld4(&T.m[c]),
                         xl = ld4(&T.xl[c]), yl = ld4(&T.yl[c]),
                         zl = ld4(&T.zl[c]);
        pair_force2<false>(ii, xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, c, -1,
                           e2, ax, ay, az);
        pair_force2<false>(ii, xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, c + 2,
                           -1, e2, ax, ay, az);
      }
    }
    ds_add(dacc[0], hsum(ax));
    ds_add(dacc[1], hsum(ay));
    ds_add(dacc[2], hsum(az));
  }
  double acc[4];
  for (int c = 0; c < 3; ++c) acc[c] = (double)dacc[c].hi + (double)dacc[c].lo;
  acc[3] = 0.0;
  vjp_finish<2>(A, V, B, A.n_act, acc, A.O.part_i, A.O.cnt_i, sm);
}

__global__ void __launch_bounds__(kAdjThreads, kVjpMinBlocks)
    adj_force_kernel(VjpArgs A) {
  __shared__ VjpSm sm;
  __shared__ VjpSmem tile;
  force_mixed(A, blockIdx.x, tile, sm);
}

template <int kMixed>
__global__ void __launch_bounds__(kAdjThreads, kVjpMinBlocks)
    adj_vjp_kernel(VjpArgs A) {
  const int b = blockIdx.x;
  __shared__ VjpSm sm;
  if (kMixed) {
    __shared__ VjpSmem tile;
    if (b < A.iblocks)
      vjp_i_mixed(A, b, tile, sm);
    else
      vjp_j_mixed(A, b - A.iblocks, tile, sm);
  } else {
    if (b < A.iblocks)
      vjp_i_f64(A, b, sm);
    else
      vjp_j_f64(A, b - A.iblocks, sm);
  }
}

// ---------------------------------------------------------------------
// Loss, seeds, output
// ---------------------------------------------------------------------

constexpr int kLossThreads = 1024;

__global__ void __launch_bounds__(kLossThreads)
    adj_loss_kernel(int n, const double* m, AdjState St, double* out) {
  __shared__ double sm[kLossThreads], sr[kLossThreads];
  double M = 0.0, S = 0.0;
  for (int i = threadIdx.x; i < n; i += kLossThreads) {
    const double x = St.r[0][i], y = St.r[1][i], z = St.r[2][i];
    M += m[i];
    S += m[i] * (x * x + y * y + z * z);
  }
  sm[threadIdx.x] = M;
  sr[threadIdx.x] = S;
  __syncthreads();
  for (int o = kLossThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sm[threadIdx.x] += sm[threadIdx.x + o];
      sr[threadIdx.x] += sr[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sr[0] / sm[0];
    out[1] = sm[0];
  }
}

__global__ void adj_loss_seed_kernel(int n, const double* m, AdjState St,
                                     const double* out, AdjCot C) {
  const double L = out[0], M = out[1];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    const double x = St.r[0][j], y = St.r[1][j], z = St.r[2][j];
    const double r2 = x * x + y * y + z * z;
    const double w = 2.0 * m[j] / M;
    for (int c = 0; c < 3; ++c) {
      C.gr[c][j] = w * St.r[c][j];
      C.gv[c][j] = 0.0;
      C.ga[c][j] = 0.0;
    }
    C.gm[j] = (r2 - L) / M;
  }
}

__global__ void adj_seed_kernel(int n, const double* gr, const double* gv,
                                const double* ga, AdjCot C) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      C.gr[c][j] = gr ? gr[3LL * j + c] : 0.0;
      C.gv[c][j] = gv ? gv[3LL * j + c] : 0.0;
      C.ga[c][j] = ga ? ga[3LL * j + c] : 0.0;
    }
    C.gm[j] = 0.0;
  }
}

__global__ void soa_to_aos_kernel(int n, const double* x, const double* y,
                                  const double* z, double* dst) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    dst[3LL * j] = x[j];
    dst[3LL * j + 1] = y[j];
    dst[3LL * j + 2] = z[j];
  }
}

int grid_for(int n) { return std::max(1, std::min((n + 255) / 256, 4096)); }

// per-body kernels of the step loop are latency-bound: small blocks spread
// them over every SM
constexpr int kBodyThreads = 64;
int body_grid(int n) {
  return std::max(1, std::min((n + kBodyThreads - 1) / kBodyThreads, 16384));
}

// Both sides: kVjpTpt lanes per target (more, up to 32, when the targets
// are few; fewer when the sources are few), 128 / tpt targets per block
// sharing each source tile, and as many source
// splits (at most kVjpSmax, each lane at least 16 sources) as fill about
// kVjpWant threads per SM.
VjpSide choose_side(long long nt, long long ns, int sms) {
  const long long want = (long long)sms * kVjpWant;
  int tpt = kVjpTpt;
  // few targets: more lanes each, so that the block's threads are used
  while (tpt < 32 && (kAdjThreads / (2 * tpt)) >= nt) tpt *= 2;
  while (tpt > 1 && ns < 16LL * tpt) tpt >>= 1;
  const int ig = kAdjThreads / tpt;
  VjpSide v{};
  const long long groups = std::max<long long>(1, (nt + ig - 1) / ig);
  long long S = (want + groups * kAdjThreads - 1) / (groups * kAdjThreads);
  S = std::min<long long>(S, kVjpSmax);
  S = std::min<long long>(S, std::max<long long>(1, ns / (16LL * tpt)));
  S = std::max<long long>(S, 1);
  long long chunk = std::max<long long>(1, (ns + S - 1) / S);
  S = std::max<long long>(1, (ns + chunk - 1) / chunk);
  v.tpt = tpt;
  v.S = (int)S;
  v.chunk = (int)chunk;
  v.groups = (int)groups;
  return v;
}

}  // namespace

VjpShape vjp_shape(int n, int n_act, int sms) {
  VjpShape s;
  s.si = choose_side(n_act, n, sms);
  s.sj = choose_side(n, n_act, sms);
  return s;
}

void launch_adj_load(int n, const double* m_in, const double* r_in,
                     const double* v_in, const double* a_in,
                     const long long* tau_in, int mixed, double* m_out,
                     const AdjState& St, const AdjPred& P, int* err,
                     cudaStream_t s) {
  adj_load_kernel<<<grid_for(n), 256, 0, s>>>(n, m_in, r_in, v_in, a_in,
                                              tau_in, mixed, m_out, St, P,
                                              err);
}

void launch_adj_init_accel(int n, const double* part, const int* nsplit,
                           double* const fsum[3], long long T_next,
                           double inv_ticks, int mixed, const AdjState& St,
                           const AdjPred& P, int* err, cudaStream_t s) {
  const FSum F{{fsum[0], fsum[1], fsum[2]}};
  adj_init_accel_kernel<<<body_grid(n), kBodyThreads, 0, s>>>(
      n, part, nsplit, F, T_next, inv_ticks, mixed, St, P, err);
}

void launch_adj_predict(int n, long long T, double inv_ticks, int mixed,
                        const AdjState& St, const AdjPred& P,
                        const long long* fwd_e, long long e_hi,
                        const AdjRecs& R, const AdjPass& Q, cudaStream_t s) {
  adj_predict_kernel<<<body_grid(n), kBodyThreads, 0, s>>>(
      n, T, inv_ticks, mixed, St, P, fwd_e, e_hi, R, Q);
}

void launch_adj_correct_predict(int n, int n_act, long long T, long long e_lo,
                                long long e_hi, long long T_next,
                                long long e_hi_next, double inv_ticks,
                                int mixed, const double* part,
                                const int* nsplit, double* const fsum[3],
                                const AdjState& St, const AdjPred& P,
                                const AdjTape& Tp, long long* fwd_e,
                                const long long* next_e, const AdjRecs& R,
                                const AdjPass& Q, int* err, cudaStream_t s) {
  const FSum F{{fsum[0], fsum[1], fsum[2]}};
  adj_correct_predict_kernel<<<body_grid(n), kBodyThreads, 0, s>>>(
      n, n_act, T, e_lo, e_hi, T_next, e_hi_next, inv_ticks, mixed, part,
      nsplit, F, St, P, Tp, fwd_e, next_e, R, Q, err);
}

void launch_adj_force(int n, int n_act, const int* idx, double eps2,
                      const AdjPred& P, const VjpSide& si, const VjpOut& O,
                      cudaStream_t s) {
  VjpArgs A{};
  A.n = n;
  A.n_act = n_act;
  A.idx = idx;
  A.eps2 = eps2;
  A.eps2f = (float)eps2;
  A.P = P;
  A.V.si = si;
  A.O = O;
  adj_force_kernel<<<si.groups * si.S, kAdjThreads, 0, s>>>(A);
}

void launch_adj_back_step(int n, double inv_ticks, int mixed,
                          const AdjBackFin& F, const AdjBackPrep& R,
                          const AdjState& St, const AdjTape& Tp,
                          long long* cur_e, const long long* prev_e,
                          const AdjCot& C, const AdjPred& P, const VjpOut& O,
                          const AdjRecs& Rc, const AdjPass& Q, int* err,
                          cudaStream_t s) {
  adj_back_step_kernel<<<body_grid(n), kBodyThreads, 0, s>>>(
      n, inv_ticks, mixed, F, R, St, Tp, cur_e, prev_e, C, P, O, Rc, Q, err);
}

void launch_adj_pass_end(int n, const AdjCot& C, const AdjCot& G0,
                         double* const g0r[3], double* const g0v[3], int last,
                         cudaStream_t s) {
  AdjPass Qp{};
  for (int c = 0; c < 3; ++c) {
    Qp.g0r[c] = g0r[c];
    Qp.g0v[c] = g0v[c];
  }
  adj_pass_end_kernel<<<body_grid(n), kBodyThreads, 0, s>>>(n, C, G0, Qp,
                                                            last);
}

void launch_adj_vjp(int mixed, int n, int n_act, const int* idx, double eps2,
                    const AdjPred& P, const AdjSlots& Sl, const VjpShape& V,
                    const VjpOut& O, cudaStream_t s) {
  VjpArgs A;
  A.n = n;
  A.n_act = n_act;
  A.idx = idx;
  A.eps2 = eps2;
  A.eps2f = (float)eps2;
  A.P = P;
  A.Sl = Sl;
  A.V = V;
  A.iblocks = V.si.groups * V.si.S;
  A.O = O;
  const int grid = A.iblocks + V.sj.groups * V.sj.S;
  if (mixed)
    adj_vjp_kernel<1><<<grid, kAdjThreads, 0, s>>>(A);
  else
    adj_vjp_kernel<0><<<grid, kAdjThreads, 0, s>>>(A);
}

void launch_adj_loss(int n, const double* m, const AdjState& St, double* out,
                     const AdjCot& C, cudaStream_t s) {
  adj_loss_kernel<<<1, kLossThreads, 0, s>>>(n, m, St, out);
  adj_loss_seed_kernel<<<grid_for(n), 256, 0, s>>>(n, m, St, out, C);
}

void launch_adj_seed(int n, const double* gr, const double* gv,
                     const double* ga, const AdjCot& C, cudaStream_t s) {
  adj_seed_kernel<<<grid_for(n), 256, 0, s>>>(n, gr, gv, ga, C);
}

void launch_soa_to_aos(int n, double* const src[3], double* dst,
                       cudaStream_t s) {
  soa_to_aos_kernel<<<grid_for(n), 256, 0, s>>>(n, src[0], src[1], src[2],
                                                dst);
}

}  // namespace tsbts
