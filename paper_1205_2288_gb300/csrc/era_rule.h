// Host arithmetic at era boundaries: the length of a dynamic era (Alg. 3
// with reading R11) and the check of a state to resume from.
//
// first and last are the earliest and latest next block times of all bodies
// (tau_i + dt_i, in ticks) at the era start; dt_max_ticks is the largest
// step, a power of two. The span last - first is clamped to
// [dt_max 2^-dyn_min_log2 (at least one tick), dt_max] and the era is the
// smallest power of two at least that long. Rounding down instead would
// leave most eras shorter than the largest steps in use, which the paper's
// comparison of dynamic and fixed eras (Sec. 4) rules out.
//
// Plain C++ with no CUDA dependence, so that the host test suite can
// compile and check it on its own (the era length is also callable from
// device code when nvcc compiles it, for ensembles whose clusters each
// take their own dynamic era).
#ifndef TSBTS_ERA_RULE_H
#define TSBTS_ERA_RULE_H

#include <cmath>
#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define TSBTS_HOST_DEVICE __host__ __device__
#else
#define TSBTS_HOST_DEVICE
#endif

inline TSBTS_HOST_DEVICE long long tsbts_dynamic_era_ticks(
    long long first, long long last, long long dt_max_ticks,
    int dyn_min_log2) {
  long long lo = dyn_min_log2 < 63 ? dt_max_ticks >> dyn_min_log2 : 0;
  if (lo < 1) lo = 1;
  long long e = last - first;
  if (e < lo) e = lo;
  if (e > dt_max_ticks) e = dt_max_ticks;
  long long p2 = 1;
  while (p2 < e) p2 *= 2;  // dt_max is a power of two >= e
  return p2;
}

// Whether bodies 0..n-1 (host arrays: m[n]; r, v, a as n x 3 rows; tau,
// dt in ticks; dts step estimates) could end an era at system time T
// (ticks): every step a power of two in [1, dt_max_ticks], every tau a
// multiple of its step with tau <= T < tau + dt, every value finite and
// every dts > 0 (+inf allowed). Returns -1 when they could, else the first
// body that could not. An era starts from these fields alone (Alg. 2 steps
// 2 and 10), and each step later indexes the level histogram, so nothing
// may be copied before the check passes.
inline long long tsbts_first_bad_body(long long T, long long dt_max_ticks,
                                      long long n, const double* m,
                                      const double* r, const double* v,
                                      const double* a, const int64_t* tau,
                                      const int64_t* dt, const double* dts) {
  for (long long i = 0; i < n; ++i) {
    const long long d = dt[i], ti = tau[i];
    bool ok = d >= 1 && d <= dt_max_ticks && (d & (d - 1)) == 0 && ti >= 0 &&
              ti % d == 0 && ti <= T && T - ti < d;
    ok = ok && std::isfinite(m[i]) && dts[i] > 0.0;
    for (int c = 0; c < 3; ++c)
      ok = ok && std::isfinite(r[3 * (size_t)i + c]) &&
           std::isfinite(v[3 * (size_t)i + c]) &&
           std::isfinite(a[3 * (size_t)i + c]);
    if (!ok) return i;
  }
  return -1;
}

#endif  // TSBTS_ERA_RULE_H
