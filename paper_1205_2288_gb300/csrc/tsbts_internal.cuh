// Internal declarations of the GB300 TSBTS library: device data layout,
// control block of the device-resident block-step loop, and the FP64 step
// arithmetic (Eq. 1, Eq. 2, Eq. 4, Alg. 1, time-symmetric interpolation).
//
// Every FP64 expression on the step path is written with explicit
// round-to-nearest intrinsics (__dadd_rn, __dmul_rn, ...), which the
// compiler never contracts into FMAs, in the order of the plain definition.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tsbts {

constexpr int kMaxLevels = 64;
constexpr unsigned kFull = 0xffffffffu;

// device error bits (Ctl::err)
constexpr int kErrHistory = 1;    // history buffer full: era must re-run
constexpr int kErrNonFinite = 2;  // non-finite force, potential or q
constexpr int kErrInvariant = 4;  // block-time invariant broken (bug)
constexpr int kErrLevels = 8;     // level histogram empty (bug)

// One pass's era history (Sec. 2: the state of every body at each of its
// steps within the era). Two buffers with fixed roles:
//  - the append buffer of the running pass: records 0..n-1 are the bodies'
//    era-start records, later ones are appended in block-step order, each
//    tagged with its body and its rank among that body's records;
//  - the previous pass's records in body-major order (CSR): body b owns
//    records hoff[b] .. hoff[b+1]-1 in time order, so a body's records are
//    contiguous and walking them reads consecutive memory.
// Between two passes the append buffer is scattered into CSR order.
struct History {
  long long* tau;
  double* r[3];
  double* v[3];
  double* a[3];
  double* dts;
  int* body;  // append buffer only
  int* seq;   // append buffer only
  long long cap;
};

// Values of one block step. Two slots alternate between consecutive steps
// so that no kernel reads a field that another block of the same kernel
// writes.
struct StepSlot {
  long long tau_c;     // block time before this step
  long long tau_next;  // this step's block time
  long long nrec;      // records in the current history before this step
  long long lg_base;   // schedule-log entries before this step
  int cnt;             // active bodies (compaction counter)
  int nsplit;          // j-split count chosen by the force kernel
};

struct Ctl {
  StepSlot slot[2];
  long long tau_e;          // era end (ticks)
  long long first, last;    // next-time extrema for the dynamic era
  unsigned long long steps;       // block steps taken (all passes)
  unsigned long long inter;       // sum n_act * n
  unsigned long long underflow;   // steps clamped to one tick
  long long log_steps, log_ent, log_drop;
  int done;     // pass finished: every kernel of the step loop returns
  int pass;     // pass index within the era
  int era;      // era index (schedule log)
  int err;      // kErr* bits
  int notconv;  // converged-iteration check: nonzero if the pass differs
  int hist[kMaxLevels];  // bodies per level k (dt = 2^-k)
};

// Body arrays in HBM, structure of arrays, all length n.
struct Bodies {
  int n;
  double* m;
  float* mf;         // masses rounded to float (the mixed j records)
  double* r[3];
  double* v[3];
  double* a[3];
  double* dts;       // last step estimate eta / sqrt(q)
  long long* tau;    // body time (ticks)
  long long* dt;     // current step (ticks)
  // prediction at the block time (FP64 path reads these for all j)
  double* pr[3];
  double* pv[3];
  // packed j records for the mixed path: (x_hi, y_hi, z_hi, m),
  // (x_lo, y_lo, z_lo, 0), (vx, vy, vz, 0) as float4, 48 B per body
  float4* jhi;
  float4* jlo;
  float4* jv;
  int* act;          // active list of the step
  int* cursor;       // per body: its last previous-pass record (CSR index)
                     // with tau <= the current block time
  int* hcnt;         // per body: records appended in the running pass
  int* hoff;         // n + 1 CSR offsets of the previous pass's records
  int* scan_tmp;     // block sums of the offset scan
  // per body: the previous-pass records bracketing the block time, copied
  // out of the history so that prediction reads them coalesced. seg_ta is
  // the time of record A (LLONG_MAX: not loaded), seg_tb that of record B
  // (-1: A is the body's last record). seg holds 18 arrays of n doubles:
  // r, v, a of A (components 0..8) and of B (9..17).
  long long* seg_ta;
  long long* seg_tb;
  double* seg;
  double* part;      // force partials [nsplit][5][n_act]
  long long part_cap;  // doubles in part
};

struct Params {
  double eps2;
  double eta;
  double inv_ticks;  // 2^-k_max (exact)
  long long dtmax_t;
  int k_min, k_max;
  int precision;     // 0 FP64, 1 MIXED
  int exact;         // FP64 single-thread ascending-j sums
  Ctl* ctl;
  // schedule log (device), cap == 0: off
  int* lg_era;
  int* lg_pass;
  long long* lg_tau;
  int* lg_nact;
  int* lg_i;
  long long* lg_dt;
  long long lg_cap;
};

// An ensemble of independent clusters integrated together: bodies of
// cluster c are off[c] .. off[c+1]-1 in the Bodies arrays; each cluster
// keeps its own block time and level counts, and every global block step
// advances every cluster that has not finished the pass by one of its own
// block steps.
struct Ens {
  int nc;
  const int* off;        // nc + 1 body offsets
  const int* cl;         // cluster of each body
  const double* eps2;    // per cluster
  const float* eps2f;
  long long* tau_c;      // per cluster: block time before this step
  long long* tau_next;   // per cluster: this step's block time, or
                         // LLONG_MAX when the cluster has finished the pass
  int* cnt;              // per cluster: active bodies this step
  int* hist;             // nc * kMaxLevels level counts
  int* act;              // n: active list of cluster c at off[c] (local ids)
  struct Plan* plan;     // per cluster: force plan this step
  int* item_off;         // nc + 1: prefix of force work items
  int* act_base;         // nc + 1: prefix of active counts
  long long* part_off;   // nc + 1: prefix of partial sums (doubles)
  int* totals;           // [0] items, [1] active bodies, [2] clusters
                         // still stepping, [3] record base of this step,
                         // [4] items taken by the force launch
  long long part_cap;    // doubles in the partial-sum buffer
  // dynamic eras (each cluster its own, Alg. 3 on its own bodies): per
  // cluster the era start and end in ticks, and the count of clusters that
  // have not reached the end of the integration; nullptr with a fixed era
  // (one era for all clusters)
  long long* ts;
  long long* te;
  int* undone;
};

// Work plan of one force launch: IG active bodies per work item (128 / IG
// threads per body), n_g i-groups, S j-splits of `chunk` j each; direct = 1
// reads j records straight from global memory instead of staging tiles in
// shared memory (for narrow groups, where a tile would be reused by few
// bodies).
struct Plan {
  int ig;
  int n_g;
  int S;
  int chunk;
  int direct;
};

// Arguments of the force kernels (shared by the integrator and the
// stand-alone force entry point).
struct ForceArgs {
  const Plan* plans;   // plan per active count 0..n (nullable)
  Plan plan;           // used when has_plan
  int has_plan;
  int n;
  // FP64 structure-of-arrays j data
  const double* m;
  const double* x[3];
  const double* w[3];  // velocities
  // mixed packed j records
  const float4* jhi;
  const float4* jlo;
  const float4* jv;
  const int* idx;      // active list
  int n_act_fixed;     // >= 0: active count; < 0: read *n_act_ptr
  const int* n_act_ptr;
  int* nsplit_out;     // block 0 writes the chosen split count (nullable)
  const int* done;     // nullable; the kernel returns when *done != 0
  double* part;        // [nsplit][5][n_act]
  long long part_cap;  // doubles available in part
  double eps2;
  float eps2f;
  int exact;           // FP64: no j-split
};

// Measured work plans of the integrator's force launch, one per power-of-two
// bucket of active counts (bucket b holds counts in (2^(b-1), 2^b], the last
// bucket ends at n); passed by value so that choosing the plan costs no
// memory access once the active count is known.
constexpr int kMaxBuckets = 26;
struct PlanTable {
  Plan b[kMaxBuckets];
  int nb;
};

__host__ __device__ inline int plan_bucket(int n_act, int nb) {
  int b = 0;
  while (b + 1 < nb && (1 << b) < n_act) ++b;
  return b;
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor in
// the stream still runs; it must wait before reading what the predecessor
// writes. Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------
// FP64 step arithmetic, op by op.
// ---------------------------------------------------------------------

// Largest 2^-k <= x with k_min <= k <= k_max, in ticks (Eq. 4). The
// largest power of two <= x is 2^e with e the unbiased exponent field of x,
// so no floating-point arithmetic is needed. x <= 0, NaN and x < 2^-k_max
// give one tick and set *underflow; x >= 2^-k_min (and +inf) give dt_max.
__host__ __device__ inline long long level_ticks(double x, int k_min,
                                                 int k_max, int* underflow) {
  if (!(x > 0.0)) {
    if (underflow) *underflow = 1;
    return 1;
  }
#ifdef __CUDA_ARCH__
  const long long bits = __double_as_longlong(x);
#else
  long long bits;
  __builtin_memcpy(&bits, &x, sizeof bits);
#endif
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  if (e >= -k_min) return 1LL << (k_max - k_min);
  if (-e > k_max) {
    if (underflow) *underflow = 1;
    return 1;
  }
  return 1LL << (k_max + e);
}

__host__ __device__ inline int level_of(long long dt_ticks, int k_max) {
  int k = k_max;
  while (dt_ticks > 1) {
    dt_ticks >>= 1;
    --k;
  }
  return k;
}

// first pass (standard block step): largest commensurate power of two
// <= min(L(dts), 2d)
__device__ inline long long forward_step(long long tau, long long d,
                                         double dts, int k_min, int k_max,
                                         int* uf) {
  long long c = level_ticks(dts, k_min, k_max, uf);
  if (c > 2 * d) c = 2 * d;
  while (tau % c != 0) c >>= 1;
  return c;
}

// Alg. 1 as described in its prose: even time tries 2d, d, then d/2; odd
// time tries d, then d/2; a candidate c passes Eq. 4 when
// c <= L((dts + dte(tau + c)) / 2).
__device__ inline long long symmetric_step(long long tau, long long d,
                                           double dts, double dte2,
                                           double dte1, int k_min, int k_max,
                                           long long dtmax_t, int* uf) {
  const bool even = (tau % (2 * d)) == 0;
  if (even && 2 * d <= dtmax_t &&
      2 * d <= level_ticks(__dmul_rn(__dadd_rn(dts, dte2), 0.5), k_min,
                           k_max, nullptr))
    return 2 * d;
  if (d <= level_ticks(__dmul_rn(__dadd_rn(dts, dte1), 0.5), k_min, k_max,
                       nullptr))
    return d;
  if (d == 1) {
    *uf = 1;
    return 1;
  }
  return d >> 1;
}

// Eq. 2 for one component: r + v h + (0.5 a) h h and v + a h
__device__ inline void taylor1(double r, double v, double a, double h,
                               double& rp, double& vp) {
  rp = __dadd_rn(__dadd_rn(r, __dmul_rn(v, h)),
                 __dmul_rn(__dmul_rn(__dmul_rn(0.5, a), h), h));
  vp = __dadd_rn(v, __dmul_rn(a, h));
}

// time-symmetric cubic Hermite basis on [ta, tb] at t
struct HermiteW {
  double h00, h10h, h01, h11h;
};

// t / D in FP64 for whole numbers of ticks t and D > 0. Record times of one
// body differ by its power-of-two steps, so D is almost always a power of
// two; then the quotient is an exact scaling by 2^-log2(D), which equals the
// correctly rounded division bit for bit and costs one multiply instead of
// the FP64 division sequence.
__device__ inline double ticks_ratio(long long t, long long D) {
  if ((D & (D - 1)) == 0) {
    const int e = 63 - __clzll(D);
    const double inv = __longlong_as_double((long long)(1023 - e) << 52);
    return __dmul_rn((double)t, inv);
  }
  return __ddiv_rn((double)t, (double)D);
}

__device__ inline HermiteW hermite_weights(long long ta, long long tb,
                                           long long t, double inv_ticks) {
  const double x = ticks_ratio(t - ta, tb - ta);
  const double h = __dmul_rn((double)(tb - ta), inv_ticks);
  const double omx = __dsub_rn(1.0, x);
  HermiteW w;
  w.h00 = __dmul_rn(__dmul_rn(__dadd_rn(1.0, __dmul_rn(2.0, x)), omx), omx);
  const double h10 = __dmul_rn(__dmul_rn(x, omx), omx);
  w.h01 = __dmul_rn(__dmul_rn(x, x), __dsub_rn(3.0, __dmul_rn(2.0, x)));
  const double h11 = __dmul_rn(__dmul_rn(x, x), __dsub_rn(x, 1.0));
  w.h10h = __dmul_rn(h10, h);
  w.h11h = __dmul_rn(h11, h);
  return w;
}

__device__ inline double hermite1(const HermiteW& w, double ya, double da,
                                  double yb, double db) {
  return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(w.h00, ya),
                                       __dmul_rn(w.h10h, da)),
                             __dmul_rn(w.h01, yb)),
                   __dmul_rn(w.h11h, db));
}

// previous pass's step estimate of a body at tick t (linear between the
// bracketing records; fallback past the stored records)
// Previous pass's step estimate of a body at tick t, from its CSR records
// [start, end) (start has tau <= the current block time <= t): linear
// between the bracketing records, `fallback` past the last record.
__device__ inline double history_dts_at(const History& H, int start, int end,
                                        long long t, double fallback) {
  int c = start;
  if (H.tau[c] > t) return fallback;
  while (c + 1 < end && H.tau[c + 1] <= t) ++c;
  if (H.tau[c] == t) return H.dts[c];
  if (c + 1 >= end) return fallback;
  const double w = ticks_ratio(t - H.tau[c], H.tau[c + 1] - H.tau[c]);
  return __dadd_rn(H.dts[c], __dmul_rn(__dsub_rn(H.dts[c + 1], H.dts[c]), w));
}

// ---------------------------------------------------------------------
// Host-side launch helpers implemented in the .cu files.
// ---------------------------------------------------------------------

// grid size and threads of the force kernels on the current device
struct ForceLaunch {
  int grid;
  int threads;
  int tile_i;          // active bodies per work item
  long long part_cap;  // doubles of partials the grid can produce
};

ForceLaunch force_launch_shape(int precision, int device);
// Doubles of split partial sums a force launch over n bodies may write: room
// for every body of n with up to twice the tiled split cap (at most 2^27,
// at least the grid's own floor). Every caller of one body count uses the
// same capacity, so plans tuned by one fit the buffers of another.
long long force_partial_capacity(const ForceLaunch& fl, long long n);
Plan plan_force(int precision, int exact, int n_act, int n, int grid,
                long long part_cap);
// measured plans of the mixed force kernel per active count 0..n (cached
// per device, n and grid for the life of the process)
const std::vector<Plan>* tuned_plans(int device, int n, int grid);
cudaError_t autotune_mixed_plans(int device, const ForceArgs& base,
                                 const ForceLaunch& fl, int* d_nsplit,
                                 cudaStream_t s, std::vector<Plan>* table);
// pt (nullable): plans per bucket of active counts; pdl: launch with
// programmatic stream serialization
cudaError_t launch_force(int precision, const ForceArgs& fa,
                         const ForceLaunch& fl, cudaStream_t s,
                         const PlanTable* pt = nullptr, bool pdl = false);
// sum nsplit partials per active body into AoS a, phi, q
cudaError_t launch_force_finalize(const double* part, const int* nsplit,
                                  int n_act, double* a, double* phi,
                                  double* q, cudaStream_t s);
// AoS (n, 3) -> packed j records for either precision
cudaError_t launch_pack_aos(int precision, int n, const double* m,
                            const double* r, const double* v, double* sx,
                            double* sy, double* sz, double* sw0, double* sw1,
                            double* sw2, double* sm, float4* jhi, float4* jlo,
                            float4* jv, cudaStream_t s);

}  // namespace tsbts
