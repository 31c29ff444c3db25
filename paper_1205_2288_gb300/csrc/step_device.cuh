// Per-body device code of the block step (Sec. 2 Alg. 2 steps 4, 6, 7),
// shared by the single-system kernels (k_step.cu) and the ensemble kernels
// (k_ensemble.cu): prediction or time-symmetric interpolation of one body,
// and the correction, next-step choice and history append of one active
// body. The FP64 arithmetic is the op-by-op form of tsbts_internal.cuh.
#pragma once

#include <climits>

#include "tsbts_internal.cuh"

namespace tsbts {

// Double-single split with integer operations only (the FP64 pipe of this
// GPU is 64 times narrower than the FP32 one, and a conversion costs as
// much as an FP64 add): hi is x with its significand cut to the leading 24
// bits, lo the exact remainder rounded to float, so hi + lo equals x to
// about 2^-48 relative. Doubles outside 2^-70 .. 2^100 in magnitude (and
// zeros, non-finite values) take the conversion path.
__device__ __forceinline__ void split_ds(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 1023 - 70 || e > 1023 + 100) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
    return;
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & ((1ULL << 52) - 1);
  hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) |
                       (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & ((1u << 29) - 1));
  const float scale = __uint_as_float((unsigned)(e - 1023 - 52 + 127) << 23);
  lo = __uint_as_float(__float_as_uint(__uint2float_rn(r) * scale) | sign);
}

// x rounded to float (to nearest, ties away) with integer operations; same
// range rule as split_ds
__device__ __forceinline__ float to_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 1023 - 70 || e > 1023 + 100) return __double2float_rn(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & ((1ULL << 52) - 1);
  // exponent and significand as one integer: the rounding carry may
  // propagate into the exponent, which is the correct result
  const unsigned mag = ((unsigned)(e - 1023 + 127) << 23) +
                       (unsigned)((m + (1ULL << 28)) >> 29);
  return __uint_as_float(sign | mag);
}

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
    float h[3], l[3];
    for (int c = 0; c < 3; ++c) split_ds(rp[c], h[c], l[c]);
    B.jhi[j] = make_float4(h[0], h[1], h[2], B.mf[j]);
    B.jlo[j] = make_float4(l[0], l[1], l[2], 0.f);
    B.jv[j] = make_float4(to_float(vp[0]), to_float(vp[1]), to_float(vp[2]),
                          0.f);
  }
}

// Body j's prediction inputs, loaded in one batch before the block time is
// known: its state (for Eq. 2) and its segment cache (the previous-pass
// records bracketing the last block time: times ta, tb and r, v, a of both
// ends, 18 values).
// Fields not preloaded (have_state / have_seg false) are read by
// predict_body when its path needs them, which keeps the memory traffic of
// very large body counts (ensembles) at what each path reads.
struct PredIn {
  double r[3], v[3], a[3];
  long long ta, tb;
  double seg[18];
  bool have_state, have_seg;
};

__device__ __forceinline__ void load_pred_state(const Bodies& B, int j,
                                                PredIn& L) {
  for (int d = 0; d < 3; ++d) {
    L.r[d] = B.r[d][j];
    L.v[d] = B.v[d][j];
    L.a[d] = B.a[d][j];
  }
  L.have_state = true;
}

__device__ __forceinline__ void load_pred_seg(const Bodies& B, int j,
                                              PredIn& L) {
  const int n = B.n;
  L.ta = B.seg_ta[j];
  L.tb = B.seg_tb[j];
#pragma unroll
  for (int q = 0; q < 18; ++q) L.seg[q] = B.seg[(long long)q * n + j];
  L.have_seg = true;
}

__device__ __forceinline__ void load_pred_in(const Bodies& B, int j,
                                             bool with_seg, PredIn& L) {
  load_pred_state(B, j, L);
  L.have_seg = false;
  if (with_seg) load_pred_seg(B, j, L);
}

// Body j (time tj) at block time tn: Taylor (Eq. 2) in the first pass and
// for active bodies; otherwise cubic Hermite between the previous pass's
// records that bracket tn, the record itself on an exact hit, Taylor where
// the records do not reach tn. The bracketing records are kept in the
// body's segment cache and refilled from its contiguous (CSR) records when
// tn leaves the segment. L holds the body's preloaded inputs.
__device__ __forceinline__ void predict_body(const Bodies& B, const Params& P,
                                             const History& prev, int j,
                                             long long tj, long long tn,
                                             int pass, bool act, PredIn& L) {
  double rp[3], vp[3];
  bool have = false;
  if (pass > 0 && !act) {
    const int n = B.n;
    if (!L.have_seg) load_pred_seg(B, j, L);
    long long ta = L.ta, tb = L.tb;
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
          L.seg[d + 0] = prev.r[d][c];
          L.seg[d + 3] = prev.v[d][c];
          L.seg[d + 6] = prev.a[d][c];
          if (nx >= 0) {
            L.seg[d + 9] = prev.r[d][nx];
            L.seg[d + 12] = prev.v[d][nx];
            L.seg[d + 15] = prev.a[d][nx];
          }
        }
#pragma unroll
        for (int q = 0; q < 18; ++q) B.seg[(long long)q * n + j] = L.seg[q];
      } else {
        ta = LLONG_MAX;  // no record at or before tn: Taylor
        tb = -1;
      }
      B.seg_ta[j] = ta;
      B.seg_tb[j] = tb;
    }
    if (ta == tn) {
      for (int d = 0; d < 3; ++d) {
        rp[d] = L.seg[d + 0];
        vp[d] = L.seg[d + 3];
      }
      have = true;
    } else if (ta < tn && tb > tn) {
      const HermiteW w = hermite_weights(ta, tb, tn, P.inv_ticks);
      if (P.precision == 0) {
        for (int d = 0; d < 3; ++d) {
          rp[d] = hermite1(w, L.seg[d + 0], L.seg[d + 3], L.seg[d + 9],
                           L.seg[d + 12]);
          vp[d] = hermite1(w, L.seg[d + 3], L.seg[d + 6], L.seg[d + 12],
                           L.seg[d + 15]);
        }
      } else {
        // mixed path: the same cubic with fused multiply-adds (the FP32
        // force reads only the double-single rounding of it)
        for (int d = 0; d < 3; ++d) {
          rp[d] = fma(w.h00, L.seg[d + 0],
                      fma(w.h10h, L.seg[d + 3],
                          fma(w.h01, L.seg[d + 9], w.h11h * L.seg[d + 12])));
          vp[d] = fma(w.h00, L.seg[d + 3],
                      fma(w.h10h, L.seg[d + 6],
                          fma(w.h01, L.seg[d + 12], w.h11h * L.seg[d + 15])));
        }
      }
      have = true;
    }
  }
  if (!have) {
    if (!L.have_state) load_pred_state(B, j, L);
    const double h = __dmul_rn((double)(tn - tj), P.inv_ticks);
    if (P.precision == 0) {
      for (int d = 0; d < 3; ++d)
        taylor1(L.r[d], L.v[d], L.a[d], h, rp[d], vp[d]);
    } else {
      // mixed path: Eq. 2 in Horner form with fused multiply-adds
      for (int d = 0; d < 3; ++d) {
        rp[d] = fma(fma(0.5 * L.a[d], h, L.v[d]), h, L.r[d]);
        vp[d] = fma(L.a[d], h, L.v[d]);
      }
    }
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

// The step estimate of Eq. 3, eta / sqrt(q). FP64 path: correctly rounded
// square root and division, as the plain definition. Mixed path (q is a
// maximum of FP32 pair terms): the FP32 reciprocal square root refined by
// one Newton-Raphson step for 1/sqrt(q) in FP64, about 2^-40 relative,
// with a third of the dependent FP64 latency; q outside 1e-30 .. 1e30 (and
// 0, inf, NaN) takes the FP64 form.
__device__ __forceinline__ double step_estimate(const Params& P, double q) {
  if (P.precision != 0 && q > 1e-30 && q < 1e30) {
    const double y0 = (double)rsqrtf((float)q);
    const double y1 = y0 * fma(-0.5 * q * y0, y0, 1.5);
    return P.eta * y1;
  }
  return __ddiv_rn(P.eta, __dsqrt_rn(q));
}

struct Corrected {
  long long d_old, d_new;
  int underflow;
};

// The body's next previous-pass records (time and step estimate), loaded
// in one batch so that the cursor advance and the two Eq. 4 lookups of
// Alg. 1 read registers instead of chaining dependent loads; records past
// the window are read from memory.
constexpr int kHistWin = 8;
struct HistWin {
  int base;
  long long t[kHistWin];
  double d[kHistWin];
};

__device__ __forceinline__ void load_hist_win(HistWin& W, const History& H,
                                              int base, int end) {
  W.base = base;
#pragma unroll
  for (int q = 0; q < kHistWin; ++q) {
    const int c = base + q;
    const bool in = c < end;
    W.t[q] = in ? H.tau[c] : LLONG_MAX;
    W.d[q] = in ? H.dts[c] : 0.0;
  }
}

__device__ __forceinline__ long long win_tau(const HistWin& W,
                                             const History& H, int c) {
  const int q = c - W.base;
  if (q < 0 || q >= kHistWin) return H.tau[c];
  long long v = W.t[0];
#pragma unroll
  for (int k = 1; k < kHistWin; ++k)
    if (q == k) v = W.t[k];
  return v;
}

__device__ __forceinline__ double win_dts(const HistWin& W, const History& H,
                                          int c) {
  const int q = c - W.base;
  if (q < 0 || q >= kHistWin) return H.dts[c];
  double v = W.d[0];
#pragma unroll
  for (int k = 1; k < kHistWin; ++k)
    if (q == k) v = W.d[k];
  return v;
}

// history_dts_at on the window (same values, same arithmetic)
__device__ __forceinline__ double history_dts_at_w(const HistWin& W,
                                                   const History& H,
                                                   int start, int end,
                                                   long long t,
                                                   double fallback) {
  int c = start;
  if (win_tau(W, H, c) > t) return fallback;
  while (c + 1 < end && win_tau(W, H, c + 1) <= t) ++c;
  const long long tc = win_tau(W, H, c);
  if (tc == t) return win_dts(W, H, c);
  if (c + 1 >= end) return fallback;
  const long long tc1 = win_tau(W, H, c + 1);
  const double dc = win_dts(W, H, c), dc1 = win_dts(W, H, c + 1);
  const double w = __ddiv_rn((double)(t - tc), (double)(tc1 - tc));
  return __dadd_rn(dc, __dmul_rn(__dsub_rn(dc1, dc), w));
}

// Active body i at block time tn with new acceleration an and criterion q:
// Eq. 1 (position from Eq. 2, velocity kick), step estimate eta / sqrt(q),
// the history record `rec`, and the next step (pass 0: standard block step;
// passes >= 1: Alg. 1 with Eq. 4 against the previous pass's records).
// Every load of the body comes before its stores (the arrays are reached
// through pointers the compiler must assume may alias), so the body waits
// for few dependent rounds of memory accesses.
__device__ __forceinline__ Corrected correct_body(const Bodies& B,
                                                  const Params& P,
                                                  const History& cur,
                                                  const History& prev, int i,
                                                  const double an[3], double q,
                                                  long long tn, int pass,
                                                  long long rec, int* err) {
  // loads
  const long long d = B.dt[i];
  double r0[3], v0[3], a0[3];
  for (int c = 0; c < 3; ++c) {
    r0[c] = B.r[c][i];
    v0[c] = B.v[c][i];
    a0[c] = B.a[c][i];
  }
  const bool fits = rec < cur.cap;
  const int sq = fits ? B.hcnt[i] : 0;
  int start = 0, end = 0;
  HistWin W;
  if (pass != 0) {
    start = B.cursor[i];
    end = B.hoff[i + 1];
    load_hist_win(W, prev, start, end);
  }
  if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]) ||
      !(q >= 0.0) || isnan(q))
    atomicOr(err, kErrNonFinite);
  // Eq. 1
  const double h = __dmul_rn((double)d, P.inv_ticks);
  double rn[3], vn[3];
  if (P.precision == 0) {
    for (int c = 0; c < 3; ++c) {
      double rp, vp;
      taylor1(r0[c], v0[c], a0[c], h, rp, vp);
      rn[c] = rp;
      vn[c] = __dadd_rn(
          v0[c], __dmul_rn(__dmul_rn(0.5, __dadd_rn(a0[c], an[c])), h));
    }
  } else {
    // mixed path: the same update with fused multiply-adds (half the
    // dependent FP64 operations; the forces carry FP32 pair terms)
    const double hh = 0.5 * h;
    for (int c = 0; c < 3; ++c) {
      rn[c] = fma(fma(hh, a0[c], v0[c]), h, r0[c]);
      vn[c] = fma(a0[c] + an[c], hh, v0[c]);
    }
  }
  const double dts = step_estimate(P, q);
  Corrected out;
  out.d_old = d;
  out.underflow = 0;
  int new_cursor = -1;
  if (pass == 0) {
    out.d_new = forward_step(tn, d, dts, P.k_min, P.k_max, &out.underflow);
  } else {
    // advance the body's previous-pass cursor to the block time; the
    // lookups below then read the few records that follow it
    if (win_tau(W, prev, start) <= tn) {
      while (start + 1 < end && win_tau(W, prev, start + 1) <= tn) ++start;
      new_cursor = start;
    }
    const double e2 = history_dts_at_w(W, prev, start, end, tn + 2 * d, dts);
    const double e1 = history_dts_at_w(W, prev, start, end, tn + d, dts);
    out.d_new = symmetric_step(tn, d, dts, e2, e1, P.k_min, P.k_max,
                               P.dtmax_t, &out.underflow);
  }
  // stores
  for (int c = 0; c < 3; ++c) {
    B.r[c][i] = rn[c];
    B.v[c][i] = vn[c];
    B.a[c][i] = an[c];
  }
  B.tau[i] = tn;
  B.dts[i] = dts;
  if (fits) {
    cur.tau[rec] = tn;
    for (int c = 0; c < 3; ++c) {
      cur.r[c][rec] = rn[c];
      cur.v[c][rec] = vn[c];
      cur.a[c][rec] = an[c];
    }
    cur.dts[rec] = dts;
    cur.body[rec] = i;
    cur.seq[rec] = sq;
    B.hcnt[i] = sq + 1;
  } else {
    atomicOr(err, kErrHistory);
  }
  if (new_cursor >= 0) B.cursor[i] = new_cursor;
  B.dt[i] = out.d_new;
  return out;
}

}  // namespace tsbts
