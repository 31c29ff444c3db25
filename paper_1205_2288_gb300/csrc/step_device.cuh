// Per-body device code of the block step (Sec. 2 Alg. 2 steps 4, 6, 7),
// shared by the single-system kernels (k_step.cu) and the ensemble kernels
// (k_ensemble.cu): prediction or time-symmetric interpolation of one body,
// and the correction, next-step choice and history append of one active
// body. The FP64 arithmetic is the op-by-op form of tsbts_internal.cuh.
#pragma once

#include <climits>

#include "tsbts_internal.cuh"

namespace tsbts {

// j data of the force kernels at the block time: FP64 arrays or the packed
// double-single records of the mixed path
__device__ __forceinline__ void store_prediction(const Bodies& B,
                                                 const Params& P, int j,
                                                 const double rp[3],
                                                 const double vp[3]) {
  if (P.precision == 0) {
    for (int c = 0; c < 3; ++c) {
      B.pr[c][j] = rp[c];
      B.pv[c][j] = vp[c];
    }
  } else {
    const float xh = (float)rp[0], yh = (float)rp[1], zh = (float)rp[2];
    B.jhi[j] = make_float4(xh, yh, zh, (float)B.m[j]);
    B.jlo[j] = make_float4((float)(rp[0] - (double)xh),
                           (float)(rp[1] - (double)yh),
                           (float)(rp[2] - (double)zh), 0.f);
    B.jv[j] = make_float4((float)vp[0], (float)vp[1], (float)vp[2], 0.f);
  }
}

// Body j (time tj) at block time tn: Taylor (Eq. 2) in the first pass and
// for active bodies; otherwise cubic Hermite between the previous pass's
// records that bracket tn, the record itself on an exact hit, Taylor where
// the records do not reach tn. The bracketing records are kept in the
// body's segment cache and refilled from its contiguous (CSR) records when
// tn leaves the segment.
__device__ __forceinline__ void predict_body(const Bodies& B, const Params& P,
                                             const History& prev, int j,
                                             long long tj, long long tn,
                                             int pass, bool act) {
  double rp[3], vp[3];
  bool have = false;
  if (pass > 0 && !act) {
    const int n = B.n;
    long long ta = B.seg_ta[j], tb = B.seg_tb[j];
    if (!(ta <= tn && (tb < 0 || tn < tb))) {
      int c = B.cursor[j];
      const int end = B.hoff[j + 1];
      if (prev.tau[c] <= tn) {
        while (c + 1 < end && prev.tau[c + 1] <= tn) ++c;
        B.cursor[j] = c;
        const int nx = c + 1 < end ? c + 1 : -1;
        ta = prev.tau[c];
        tb = nx >= 0 ? prev.tau[nx] : -1;
        for (int d = 0; d < 3; ++d) {
          B.seg[(d + 0) * n + j] = prev.r[d][c];
          B.seg[(d + 3) * n + j] = prev.v[d][c];
          B.seg[(d + 6) * n + j] = prev.a[d][c];
          if (nx >= 0) {
            B.seg[(d + 9) * n + j] = prev.r[d][nx];
            B.seg[(d + 12) * n + j] = prev.v[d][nx];
            B.seg[(d + 15) * n + j] = prev.a[d][nx];
          }
        }
      } else {
        ta = LLONG_MAX;  // no record at or before tn: Taylor
        tb = -1;
      }
      B.seg_ta[j] = ta;
      B.seg_tb[j] = tb;
    }
    if (ta == tn) {
      for (int d = 0; d < 3; ++d) {
        rp[d] = B.seg[(d + 0) * n + j];
        vp[d] = B.seg[(d + 3) * n + j];
      }
      have = true;
    } else if (ta < tn && tb > tn) {
      const HermiteW w = hermite_weights(ta, tb, tn, P.inv_ticks);
      for (int d = 0; d < 3; ++d) {
        rp[d] = hermite1(w, B.seg[(d + 0) * n + j], B.seg[(d + 3) * n + j],
                         B.seg[(d + 9) * n + j], B.seg[(d + 12) * n + j]);
        vp[d] = hermite1(w, B.seg[(d + 3) * n + j], B.seg[(d + 6) * n + j],
                         B.seg[(d + 12) * n + j], B.seg[(d + 15) * n + j]);
      }
      have = true;
    }
  }
  if (!have) {
    const double h = __dmul_rn((double)(tn - tj), P.inv_ticks);
    for (int d = 0; d < 3; ++d)
      taylor1(B.r[d][j], B.v[d][j], B.a[d][j], h, rp[d], vp[d]);
  }
  store_prediction(B, P, j, rp, vp);
}

// S split partial sums of active position k (layout [split][5][n_act]),
// added in split order
__device__ __forceinline__ void sum_partials(const double* part, int n_act,
                                             int S, int k, double an[3],
                                             double& q) {
  const double* pp = part;
  an[0] = pp[0 * n_act + k];
  an[1] = pp[1 * n_act + k];
  an[2] = pp[2 * n_act + k];
  q = pp[4 * n_act + k];
#pragma unroll 4
  for (int sp = 1; sp < S; ++sp) {
    pp = part + (long long)sp * 5 * n_act;
    an[0] = __dadd_rn(an[0], pp[0 * n_act + k]);
    an[1] = __dadd_rn(an[1], pp[1 * n_act + k]);
    an[2] = __dadd_rn(an[2], pp[2 * n_act + k]);
    q = fmax(q, pp[4 * n_act + k]);
  }
}

struct Corrected {
  long long d_old, d_new;
  int underflow;
};

// Active body i at block time tn with new acceleration an and criterion q:
// Eq. 1 (position from Eq. 2, velocity kick), step estimate eta / sqrt(q),
// the history record `rec`, and the next step (pass 0: standard block step;
// passes >= 1: Alg. 1 with Eq. 4 against the previous pass's records).
__device__ __forceinline__ Corrected correct_body(const Bodies& B,
                                                  const Params& P,
                                                  const History& cur,
                                                  const History& prev, int i,
                                                  const double an[3], double q,
                                                  long long tn, int pass,
                                                  long long rec, int* err) {
  if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]) ||
      !(q >= 0.0) || isnan(q))
    atomicOr(err, kErrNonFinite);
  const long long d = B.dt[i];
  const double h = __dmul_rn((double)d, P.inv_ticks);
  double rn[3], vn[3];
  for (int c = 0; c < 3; ++c) {
    double rp, vp;
    taylor1(B.r[c][i], B.v[c][i], B.a[c][i], h, rp, vp);
    rn[c] = rp;
    vn[c] = __dadd_rn(B.v[c][i],
                      __dmul_rn(__dmul_rn(0.5, __dadd_rn(B.a[c][i], an[c])),
                                h));
    B.r[c][i] = rn[c];
    B.v[c][i] = vn[c];
    B.a[c][i] = an[c];
  }
  B.tau[i] = tn;
  const double dts = __ddiv_rn(P.eta, __dsqrt_rn(q));
  B.dts[i] = dts;
  if (rec < cur.cap) {
    cur.tau[rec] = tn;
    for (int c = 0; c < 3; ++c) {
      cur.r[c][rec] = rn[c];
      cur.v[c][rec] = vn[c];
      cur.a[c][rec] = an[c];
    }
    cur.dts[rec] = dts;
    cur.body[rec] = i;
    const int sq = B.hcnt[i];
    cur.seq[rec] = sq;
    B.hcnt[i] = sq + 1;
  } else {
    atomicOr(err, kErrHistory);
  }
  Corrected out;
  out.d_old = d;
  out.underflow = 0;
  if (pass == 0) {
    out.d_new = forward_step(tn, d, dts, P.k_min, P.k_max, &out.underflow);
  } else {
    // advance the body's previous-pass cursor to the block time; the
    // lookups below then read the few records that follow it
    int start = B.cursor[i];
    const int end = B.hoff[i + 1];
    if (prev.tau[start] <= tn) {
      while (start + 1 < end && prev.tau[start + 1] <= tn) ++start;
      B.cursor[i] = start;
    }
    const double e2 = history_dts_at(prev, start, end, tn + 2 * d, dts);
    const double e1 = history_dts_at(prev, start, end, tn + d, dts);
    out.d_new = symmetric_step(tn, d, dts, e2, e1, P.k_min, P.k_max,
                               P.dtmax_t, &out.underflow);
  }
  B.dt[i] = out.d_new;
  return out;
}

}  // namespace tsbts
