// Length of a dynamic era (Alg. 3 with reading R11), host arithmetic only.
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
// compile and check it on its own.
#ifndef TSBTS_ERA_RULE_H
#define TSBTS_ERA_RULE_H

inline long long tsbts_dynamic_era_ticks(long long first, long long last,
                                         long long dt_max_ticks,
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

#endif  // TSBTS_ERA_RULE_H
