// Force kernels of the TSBTS library (Sec. 2 Alg. 2 step 5; Eq. 3; Plummer
// softening of Sec. 3): for each active body i and all j != i
//   a_i   = sum m_j d_ij / s^3,   phi_i = -sum m_j / s,
//   q_i   = max max(|v_ij|^2 / s^2, m_j / s^3),   s^2 = |d_ij|^2 + eps^2.
//
// Work decomposition (the GB300 analogue of the paper's Alg. 4 data/work
// partition). A persistent grid walks work items (i-group, j-chunk). The
// launch reads the active count from device memory and picks, on the
// device, the i-group width IG (bodies per 128-thread block):
//  - IG = 128: one body per thread, every thread sweeps the j-chunk (data
//    partition); the mixed path runs two j per packed f32x2 instruction.
//  - IG < 128 (fewer than 128 active bodies): 128 / IG threads share each
//    body's j-chunk and their partial sums are combined by a fixed-order
//    tree in shared memory (work partition inside a block).
// The j range is further split across blocks so that the grid stays full;
// split partial sums go to a scratch buffer and are added in split order by
// the consumer. Every order is fixed, so results are deterministic.
//
// j records are staged tile by tile in shared memory with coalesced loads
// and read back as broadcasts; the pair loop is FMA-pipe bound.
#include <algorithm>
#include <iterator>
#include <map>
#include <mutex>
#include <vector>

#include "tsbts_internal.cuh"

namespace tsbts {

constexpr int kThreads = 128;   // threads per block
constexpr int kTileF64 = 64;    // j per shared-memory tile, FP64
constexpr int kTileMix = 256;   // j per shared-memory tile, mixed
constexpr int kLaneMinMix = 16; // fewest j per thread in a split item
constexpr int kLaneMinF64 = 8;
constexpr int kSplitCap = 16;   // most j-splits of one active body

// tuning of the mixed pair loop (compile-time; defaults measured on GB300)
#ifndef TSBTS_MIX_UNROLL
#define TSBTS_MIX_UNROLL 4
#endif
#ifndef TSBTS_MIX_QUAD
#define TSBTS_MIX_QUAD 1
#endif
#ifndef TSBTS_MIX_MINB
#define TSBTS_MIX_MINB 3
#endif
constexpr int kMixUnroll = TSBTS_MIX_UNROLL;  // unroll of the j-pair loop
constexpr bool kMixQuad = TSBTS_MIX_QUAD;     // 128-bit loads of four j
constexpr int kMixMinBlocks = TSBTS_MIX_MINB; // register budget hint

// Host choice of the work plan for n_act active bodies: over i-group widths
// IG = 128 .. 1 and split counts S = 1 .. kSplitCap, minimise a cost model
// of waves of the grid times the per-item time (j per thread plus a fixed
// item overhead and the block's reduction tree) plus the consumer's cost of
// reading S partial sums. Wave quantisation is what the search is for: 256
// items on a 456-block grid leave 44% of the GPU idle.
Plan plan_force(int precision, int exact, int n_act, int n, int grid,
                long long part_cap) {
  Plan best = {kThreads, (n_act + kThreads - 1) / kThreads, 1, n};
  if (exact || n_act <= 0) return best;
  const int lane_min = precision ? kLaneMinMix : kLaneMinF64;
  double best_cost = 1e300;
  for (int ig = kThreads; ig >= 1; ig >>= 1) {
    if (ig > 2 * n_act && ig > 1) continue;
    const int jg = kThreads / ig;
    int lg = 0;
    while ((1 << lg) < jg) ++lg;
    const long long n_g = (n_act + ig - 1) / ig;
    long long smax = n / ((long long)jg * lane_min);
    smax = std::max<long long>(1, std::min<long long>(smax, kSplitCap));
    for (int S = 1; S <= smax; ++S) {
      if (S > 1 && (long long)S * 5 * n_act > part_cap) break;
      long long chunk = (n + S - 1) / S;
      chunk = (chunk + 1) & ~1LL;
      const long long items = n_g * S;
      const long long waves = (items + grid - 1) / grid;
      const double per_item = (double)((chunk + jg - 1) / jg) + 96.0 + 8.0 * lg;
      const double cost = waves * per_item + 16.0 * S * (1 + n_act / 4096);
      if (cost < best_cost) {
        best_cost = cost;
        best = Plan{ig, (int)n_g, S, (int)chunk};
      }
    }
  }
  return best;
}

__device__ __forceinline__ Plan make_plan(int n_act, int n, int grid,
                                          int exact, long long part_cap,
                                          int lane_min, int tile) {
  Plan p;
  p.direct = 0;
  if (exact) {
    p.ig = kThreads;
    p.n_g = (n_act + kThreads - 1) / kThreads;
    p.S = 1;
    p.chunk = n;
    return p;
  }
  // Narrow the i-groups until about kSplitCap splits fill the grid: j-lanes
  // inside a block are combined by a cheap shared-memory tree, whereas
  // every extra split adds a partial sum that the consumer must read.
  long long want = (long long)kSplitCap * n_act / grid;
  int ig = 1;
  while (ig < kThreads && 2LL * ig <= want) ig <<= 1;
  const int jg = kThreads / ig;
  const int n_g = (n_act + ig - 1) / ig;
  int S = grid / n_g;
  int smax = n / (jg * lane_min);
  if (smax > kSplitCap) smax = kSplitCap;
  if (smax < 1) smax = 1;
  if (S > smax) S = smax;
  if (S < 1) S = 1;
  while (S > 1 && (long long)S * 5 * n_act > part_cap) --S;
  int chunk = (n + S - 1) / S;
  chunk = (chunk + 1) & ~1;  // packed loops take j in pairs
  p.ig = ig;
  p.n_g = n_g;
  p.S = S;
  p.chunk = chunk;
  (void)tile;
  return p;
}

__device__ __forceinline__ void write_partial(const ForceArgs& A, int n_act,
                                              int split, int k, double ax,
                                              double ay, double az, double ph,
                                              double q) {
  // a plan whose partial sums do not fit the buffer writes nothing (every
  // plan the library makes fits; this guards the buffer, not the result)
  if ((long long)(split + 1) * 5 * n_act > A.part_cap) return;
  double* p = A.part + (long long)split * 5 * n_act;
  p[0 * n_act + k] = ax;
  p[1 * n_act + k] = ay;
  p[2 * n_act + k] = az;
  p[3 * n_act + k] = ph;
  p[4 * n_act + k] = q;
}

// ---------------------------------------------------------------------
// FP64: each pair term rounded op by op in the order of the definition.
// ---------------------------------------------------------------------
struct F64Tile {
  double x[kTileF64], y[kTileF64], z[kTileF64];
  double u[kTileF64], v[kTileF64], w[kTileF64], m[kTileF64];
};

struct F64Acc {
  double ax, ay, az, ph, q;
};

__device__ __forceinline__ void pair_f64(const F64Tile& T, int t, double xi,
                                         double yi, double zi, double ui,
                                         double vi, double wi, double eps2,
                                         F64Acc& s) {
  const double dx = __dsub_rn(T.x[t], xi);
  const double dy = __dsub_rn(T.y[t], yi);
  const double dz = __dsub_rn(T.z[t], zi);
  const double s2 = __dadd_rn(
      __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                __dmul_rn(dz, dz)),
      eps2);
  const double sq = __dsqrt_rn(s2);
  const double f = __ddiv_rn(T.m[t], __dmul_rn(s2, sq));
  s.ax = __dadd_rn(s.ax, __dmul_rn(f, dx));
  s.ay = __dadd_rn(s.ay, __dmul_rn(f, dy));
  s.az = __dadd_rn(s.az, __dmul_rn(f, dz));
  s.ph = __dsub_rn(s.ph, __ddiv_rn(T.m[t], sq));
  const double wx = __dsub_rn(T.u[t], ui);
  const double wy = __dsub_rn(T.v[t], vi);
  const double wz = __dsub_rn(T.w[t], wi);
  const double c = __ddiv_rn(
      __dadd_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)),
                __dmul_rn(wz, wz)),
      s2);
  if (c > s.q) s.q = c;
  if (f > s.q) s.q = f;
}

template <int IG>
__device__ void f64_items(const ForceArgs& A, int n_act, const Plan& P,
                          F64Tile& T, double (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  constexpr int TJ = kTileF64;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const double eps2 = A.eps2;
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x) {
    const int g = w / P.S;
    const int split = w - g * P.S;
    const int k = g * IG + il;
    const bool valid = k < n_act;
    const int i = valid ? A.idx[k] : -1;
    double xi = 0, yi = 0, zi = 0, ui = 0, vi = 0, wi = 0;
    if (valid) {
      xi = A.x[0][i];
      yi = A.x[1][i];
      zi = A.x[2][i];
      ui = A.w[0][i];
      vi = A.w[1][i];
      wi = A.w[2][i];
    }
    F64Acc s = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int j0 = split * P.chunk;
    const int j1 = min(A.n, j0 + P.chunk);
    for (int jt = j0; jt < j1; jt += TJ) {
      const int cnt = min(TJ, j1 - jt);
      __syncthreads();
      for (int q = t; q < cnt; q += kThreads) {
        const int j = jt + q;
        T.x[q] = A.x[0][j];
        T.y[q] = A.x[1][j];
        T.z[q] = A.x[2][j];
        T.u[q] = A.w[0][j];
        T.v[q] = A.w[1][j];
        T.w[q] = A.w[2][j];
        T.m[q] = A.m[j];
      }
      __syncthreads();
      for (int q = jl; q < cnt; q += JG) {
        if (jt + q == i) continue;
        pair_f64(T, q, xi, yi, zi, ui, vi, wi, eps2, s);
      }
    }
    if constexpr (JG > 1) {
      red[0][t] = s.ax;
      red[1][t] = s.ay;
      red[2][t] = s.az;
      red[3][t] = s.ph;
      red[4][t] = s.q;
      __syncthreads();
      for (int half = JG / 2; half >= 1; half >>= 1) {
        if (jl < half) {
          const int o = t + half * IG;
          for (int c = 0; c < 4; ++c) red[c][t] = __dadd_rn(red[c][t], red[c][o]);
          red[4][t] = fmax(red[4][t], red[4][o]);
        }
        __syncthreads();
      }
      if (jl == 0) {
        s.ax = red[0][t];
        s.ay = red[1][t];
        s.az = red[2][t];
        s.ph = red[3][t];
        s.q = red[4][t];
      }
    }
    if (jl == 0 && valid)
      write_partial(A, n_act, split, k, s.ax, s.ay, s.az, s.ph, s.q);
  }
}

__global__ void __launch_bounds__(kThreads) force_fp64_kernel(ForceArgs A) {
  if (A.done && *A.done) return;
  const int n_act = A.n_act_fixed >= 0 ? A.n_act_fixed : *A.n_act_ptr;
  if (n_act <= 0) return;
  const Plan P = A.has_plan ? A.plan
                 : A.plans  ? A.plans[n_act]
                            : make_plan(n_act, A.n, gridDim.x, A.exact,
                                        A.part_cap, kLaneMinF64, kTileF64);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.nsplit_out)
    *A.nsplit_out = P.S;
  __shared__ F64Tile T;
  __shared__ double red[5][kThreads];
  switch (P.ig) {
    case 128: f64_items<128>(A, n_act, P, T, red); break;
    case 64: f64_items<64>(A, n_act, P, T, red); break;
    case 32: f64_items<32>(A, n_act, P, T, red); break;
    case 16: f64_items<16>(A, n_act, P, T, red); break;
    case 8: f64_items<8>(A, n_act, P, T, red); break;
    case 4: f64_items<4>(A, n_act, P, T, red); break;
    case 2: f64_items<2>(A, n_act, P, T, red); break;
    default: f64_items<1>(A, n_act, P, T, red); break;
  }
}

// ---------------------------------------------------------------------
// Mixed: FP32 pair terms on double-single relative coordinates
// d = (x_hi,j - x_hi,i) + (x_lo,j - x_lo,i); FP32 sums per j tile folded
// into hi/lo compensated accumulators; q is an exact FP32 max.
// ---------------------------------------------------------------------
struct MixTile {  // structure of arrays: consecutive j pair up for f32x2
  float xh[kTileMix], yh[kTileMix], zh[kTileMix], m[kTileMix];
  float xl[kTileMix], yl[kTileMix], zl[kTileMix];
  float u[kTileMix], v[kTileMix], w[kTileMix];
};

struct MixI {
  float xh, yh, zh, xl, yl, zl, u, v, w;
};

// compensated accumulator: value = hi + lo
struct DS {
  float hi, lo;
};

__device__ __forceinline__ void ds_add(DS& a, float t) {
  const float s = __fadd_rn(a.hi, t);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)),
                              __fsub_rn(t, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

__device__ __forceinline__ void ds_add(DS& a, DS b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)),
                              __fsub_rn(b.hi, bb));
  a.hi = s;
  a.lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

__device__ __forceinline__ void pair_mixed(const MixI& I, const MixTile& T,
                                           int t, float eps2, float& ax,
                                           float& ay, float& az, float& ph,
                                           float& q) {
  const float dx = __fsub_rn(T.xh[t], I.xh) + __fsub_rn(T.xl[t], I.xl);
  const float dy = __fsub_rn(T.yh[t], I.yh) + __fsub_rn(T.yl[t], I.yl);
  const float dz = __fsub_rn(T.zh[t], I.zh) + __fsub_rn(T.zl[t], I.zl);
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  const float rinv = rsqrtf(s2);
  const float rinv2 = rinv * rinv;
  const float mr = T.m[t] * rinv;
  const float mr3 = mr * rinv2;
  ax = fmaf(mr3, dx, ax);
  ay = fmaf(mr3, dy, ay);
  az = fmaf(mr3, dz, az);
  ph += mr;
  const float wx = T.u[t] - I.u;
  const float wy = T.v[t] - I.v;
  const float wz = T.w[t] - I.w;
  const float w2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
  q = max3(q, w2 * rinv2, mr3);
}

// packed pairs of floats (two j per instruction)
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 x, float& a, float& b) {
  asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 ld2(const float* p) {
  return *reinterpret_cast<const f2*>(p);
}

// the j operands of two interactions, one packed pair per component
struct J2 {
  f2 xh, yh, zh, m, xl, yl, zl, u, v, w;
};

// j = t, t + 1 (t even): one 64-bit shared load per component
__device__ __forceinline__ J2 load_j2(const MixTile& T, int t) {
  J2 J;
  J.xh = ld2(&T.xh[t]); J.yh = ld2(&T.yh[t]); J.zh = ld2(&T.zh[t]);
  J.m = ld2(&T.m[t]);
  J.xl = ld2(&T.xl[t]); J.yl = ld2(&T.yl[t]); J.zl = ld2(&T.zl[t]);
  J.u = ld2(&T.u[t]); J.v = ld2(&T.v[t]); J.w = ld2(&T.w[t]);
  return J;
}

// j = t .. t + 3 (t a multiple of 4): one 128-bit shared load per component
__device__ __forceinline__ void load_j4(const MixTile& T, int t, J2& a, J2& b) {
  const ulonglong2 xh = *reinterpret_cast<const ulonglong2*>(&T.xh[t]);
  const ulonglong2 yh = *reinterpret_cast<const ulonglong2*>(&T.yh[t]);
  const ulonglong2 zh = *reinterpret_cast<const ulonglong2*>(&T.zh[t]);
  const ulonglong2 m = *reinterpret_cast<const ulonglong2*>(&T.m[t]);
  const ulonglong2 xl = *reinterpret_cast<const ulonglong2*>(&T.xl[t]);
  const ulonglong2 yl = *reinterpret_cast<const ulonglong2*>(&T.yl[t]);
  const ulonglong2 zl = *reinterpret_cast<const ulonglong2*>(&T.zl[t]);
  const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(&T.u[t]);
  const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(&T.v[t]);
  const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&T.w[t]);
  a = J2{xh.x, yh.x, zh.x, m.x, xl.x, yl.x, zl.x, u.x, v.x, w.x};
  b = J2{xh.y, yh.y, zh.y, m.y, xl.y, yl.y, zl.y, u.y, v.y, w.y};
}

// two interactions (j = t, t + 1) on one body, all FMA-pipe work packed.
// MASK: the pair with tile index `self` is the body itself; its 1/s is set
// to 0, so it adds exact zeros and the sums equal those of the unmasked
// loop over the other j.
template <bool MASK>
__device__ __forceinline__ void pair_mixed2(const f2 (&ii)[9], const J2& J,
                                            int t, f2 eps2, f2& ax, f2& ay,
                                            f2& az, f2& ph, float& q,
                                            int self = -1) {
  const f2 dx = add2(sub2(J.xh, ii[0]), sub2(J.xl, ii[3]));
  const f2 dy = add2(sub2(J.yh, ii[1]), sub2(J.yl, ii[4]));
  const f2 dz = add2(sub2(J.zh, ii[2]), sub2(J.zl, ii[5]));
  const f2 s2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
  float s0, s1;
  upk(s2, s0, s1);
  float r0 = rsqrtf(s0), r1 = rsqrtf(s1);
  if (MASK) {
    if (t == self) r0 = 0.f;
    if (t + 1 == self) r1 = 0.f;
  }
  const f2 rinv = pk(r0, r1);
  const f2 rinv2 = mul2(rinv, rinv);
  const f2 mr = mul2(J.m, rinv);
  const f2 mr3 = mul2(mr, rinv2);
  ax = fma2(mr3, dx, ax);
  ay = fma2(mr3, dy, ay);
  az = fma2(mr3, dz, az);
  ph = add2(ph, mr);
  const f2 wx = sub2(J.u, ii[6]);
  const f2 wy = sub2(J.v, ii[7]);
  const f2 wz = sub2(J.w, ii[8]);
  const f2 w2 = fma2(wx, wx, fma2(wy, wy, mul2(wz, wz)));
  const f2 c = mul2(w2, rinv2);
  float c0, c1, m0, m1;
  upk(c, c0, c1);
  upk(mr3, m0, m1);
  q = max3(max3(q, c0, m0), c1, m1);
}

template <int IG>
__device__ __forceinline__ void finish_mixed_item(const ForceArgs& A,
                                                  int n_act, int split, int k,
                                                  bool valid, DS sx, DS sy,
                                                  DS sz, DS sp, float q,
                                                  float (*red)[kThreads]);

template <int IG>
__device__ void mixed_items(const ForceArgs& A, int n_act, const Plan& P,
                            MixTile& T, float (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  constexpr int TJ = kTileMix;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const float eps2 = A.eps2f;
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x) {
    const int g = w / P.S;
    const int split = w - g * P.S;
    const int k = g * IG + il;
    const bool valid = k < n_act;
    const int i = valid ? A.idx[k] : -1;
    MixI I = {};
    if (valid) {
      const float4 h = A.jhi[i], l = A.jlo[i], vv = A.jv[i];
      I.xh = h.x; I.yh = h.y; I.zh = h.z;
      I.xl = l.x; I.yl = l.y; I.zl = l.z;
      I.u = vv.x; I.v = vv.y; I.w = vv.z;
    }
    DS sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sp = {0, 0};
    float q = 0.f;
    const int j0 = split * P.chunk;
    const int j1 = min(A.n, j0 + P.chunk);
    // FP32 running sums over about kTileMix j per thread, then folded
    float ax = 0, ay = 0, az = 0, ph = 0;
    int tiles = 0;
    for (int jt = j0; jt < j1; jt += TJ) {
      const int cnt = min(TJ, j1 - jt);
      __syncthreads();
      for (int c = t; c < cnt; c += kThreads) {
        const float4 h = A.jhi[jt + c], l = A.jlo[jt + c], vv = A.jv[jt + c];
        T.xh[c] = h.x; T.yh[c] = h.y; T.zh[c] = h.z; T.m[c] = h.w;
        T.xl[c] = l.x; T.yl[c] = l.y; T.zl[c] = l.z;
        T.u[c] = vv.x; T.v[c] = vv.y; T.w[c] = vv.z;
      }
      __syncthreads();
      const bool self_here = valid && i >= jt && i < jt + cnt;
      if (cnt == TJ) {
        // thread jl takes the j pairs (2 jl, 2 jl + 1) + 2 JG m; a warp with
        // a body inside the tile runs the same arithmetic with that pair
        // masked, so each body's sums do not depend on its warp-mates
        const f2 ii[9] = {pk(I.xh, I.xh), pk(I.yh, I.yh), pk(I.zh, I.zh),
                          pk(I.xl, I.xl), pk(I.yl, I.yl), pk(I.zl, I.zl),
                          pk(I.u, I.u),   pk(I.v, I.v),   pk(I.w, I.w)};
        const f2 e2 = pk(eps2, eps2);
        f2 pax = pk(0.f, 0.f), pay = pax, paz = pax, pph = pax;
        const bool any_self = __any_sync(kFull, self_here);
        const int sc = self_here ? i - jt : -1;
        if constexpr (kMixQuad && 4 * JG <= TJ) {
          // thread jl takes the j quads 4 jl + 4 JG m (128-bit loads)
          if (any_self) {
            for (int c = 4 * jl; c < TJ; c += 4 * JG) {
              J2 a, b;
              load_j4(T, c, a, b);
              pair_mixed2<true>(ii, a, c, e2, pax, pay, paz, pph, q, sc);
              pair_mixed2<true>(ii, b, c + 2, e2, pax, pay, paz, pph, q, sc);
            }
          } else {
#pragma unroll kMixUnroll
            for (int c = 4 * jl; c < TJ; c += 4 * JG) {
              J2 a, b;
              load_j4(T, c, a, b);
              pair_mixed2<false>(ii, a, c, e2, pax, pay, paz, pph, q);
              pair_mixed2<false>(ii, b, c + 2, e2, pax, pay, paz, pph, q);
            }
          }
        } else {
          if (any_self) {
            for (int c = 2 * jl; c < TJ; c += 2 * JG)
              pair_mixed2<true>(ii, load_j2(T, c), c, e2, pax, pay, paz, pph,
                                q, sc);
          } else {
#pragma unroll kMixUnroll
            for (int c = 2 * jl; c < TJ; c += 2 * JG)
              pair_mixed2<false>(ii, load_j2(T, c), c, e2, pax, pay, paz, pph,
                                 q);
          }
        }
        float a0, a1;
        upk(pax, a0, a1);
        ax += a0 + a1;
        upk(pay, a0, a1);
        ay += a0 + a1;
        upk(paz, a0, a1);
        az += a0 + a1;
        upk(pph, a0, a1);
        ph += a0 + a1;
      } else {
        for (int c = jl; c < cnt; c += JG) {
          if (jt + c == i) continue;
          pair_mixed(I, T, c, eps2, ax, ay, az, ph, q);
        }
      }
      if (++tiles == JG) {
        tiles = 0;
        ds_add(sx, ax);
        ds_add(sy, ay);
        ds_add(sz, az);
        ds_add(sp, ph);
        ax = ay = az = ph = 0.f;
      }
    }
    ds_add(sx, ax);
    ds_add(sy, ay);
    ds_add(sz, az);
    ds_add(sp, ph);
    finish_mixed_item<IG>(A, n_act, split, k, valid, sx, sy, sz, sp, q, red);
  }
}

// Reduce the JG j-lane partial sums of each body in a fixed-order tree in
// shared memory and write the item's partial sums.
template <int IG>
__device__ __forceinline__ void finish_mixed_item(const ForceArgs& A,
                                                  int n_act, int split, int k,
                                                  bool valid, DS sx, DS sy,
                                                  DS sz, DS sp, float q,
                                                  float (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  const int t = threadIdx.x;
  const int jl = t / IG;
  {
    if constexpr (JG > 1) {
      red[0][t] = sx.hi; red[1][t] = sx.lo;
      red[2][t] = sy.hi; red[3][t] = sy.lo;
      red[4][t] = sz.hi; red[5][t] = sz.lo;
      red[6][t] = sp.hi; red[7][t] = sp.lo;
      red[8][t] = q;
      __syncthreads();
      for (int half = JG / 2; half >= 1; half >>= 1) {
        if (jl < half) {
          const int o = t + half * IG;
          for (int c = 0; c < 8; c += 2) {
            DS a = {red[c][t], red[c + 1][t]};
            ds_add(a, DS{red[c][o], red[c + 1][o]});
            red[c][t] = a.hi;
            red[c + 1][t] = a.lo;
          }
          red[8][t] = fmaxf(red[8][t], red[8][o]);
        }
        __syncthreads();
      }
      if (jl == 0) {
        sx = DS{red[0][t], red[1][t]};
        sy = DS{red[2][t], red[3][t]};
        sz = DS{red[4][t], red[5][t]};
        sp = DS{red[6][t], red[7][t]};
        q = red[8][t];
      }
    }
    if (jl == 0 && valid)
      write_partial(A, n_act, split, k, (double)sx.hi + (double)sx.lo,
                    (double)sy.hi + (double)sy.lo,
                    (double)sz.hi + (double)sz.lo,
                    -((double)sp.hi + (double)sp.lo), (double)q);
    __syncthreads();  // red is reused by the next item
  }
}

__device__ __forceinline__ void pair_mixed_g(const MixI& I, const float4 h,
                                             const float4 l, const float4 vv,
                                             float eps2, float& ax, float& ay,
                                             float& az, float& ph, float& q) {
  const float dx = __fsub_rn(h.x, I.xh) + __fsub_rn(l.x, I.xl);
  const float dy = __fsub_rn(h.y, I.yh) + __fsub_rn(l.y, I.yl);
  const float dz = __fsub_rn(h.z, I.zh) + __fsub_rn(l.z, I.zl);
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  const float rinv = rsqrtf(s2);
  const float rinv2 = rinv * rinv;
  const float mr = h.w * rinv;
  const float mr3 = mr * rinv2;
  ax = fmaf(mr3, dx, ax);
  ay = fmaf(mr3, dy, ay);
  az = fmaf(mr3, dz, az);
  ph += mr;
  const float wx = vv.x - I.u;
  const float wy = vv.y - I.v;
  const float wz = vv.z - I.w;
  const float w2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
  q = max3(q, w2 * rinv2, mr3);
}

// Narrow groups without shared-memory staging: j-lane jl of a body reads
// j = j0 + jl, j0 + jl + JG, ... straight from global memory (the j records
// are L2-resident), so a small active set costs no block-wide tile loads.
template <int IG>
__device__ void mixed_items_direct(const ForceArgs& A, int n_act,
                                   const Plan& P, float (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const float eps2 = A.eps2f;
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x) {
    const int g = w / P.S;
    const int split = w - g * P.S;
    const int k = g * IG + il;
    const bool valid = k < n_act;
    const int i = valid ? A.idx[k] : -1;
    MixI I = {};
    if (valid) {
      const float4 h = A.jhi[i], l = A.jlo[i], vv = A.jv[i];
      I.xh = h.x; I.yh = h.y; I.zh = h.z;
      I.xl = l.x; I.yl = l.y; I.zl = l.z;
      I.u = vv.x; I.v = vv.y; I.w = vv.z;
    }
    DS sx = {0, 0}, sy = {0, 0}, sz = {0, 0}, sp = {0, 0};
    float q = 0.f;
    float ax = 0, ay = 0, az = 0, ph = 0;
    const int j0 = split * P.chunk;
    const int j1 = min(A.n, j0 + P.chunk);
    int cnt = 0;
#pragma unroll 4
    for (int j = j0 + jl; j < j1; j += JG) {
      const float4 h = A.jhi[j], l = A.jlo[j], vv = A.jv[j];
      if (j != i) pair_mixed_g(I, h, l, vv, eps2, ax, ay, az, ph, q);
      if (++cnt == kTileMix) {
        cnt = 0;
        ds_add(sx, ax);
        ds_add(sy, ay);
        ds_add(sz, az);
        ds_add(sp, ph);
        ax = ay = az = ph = 0.f;
      }
    }
    ds_add(sx, ax);
    ds_add(sy, ay);
    ds_add(sz, az);
    ds_add(sp, ph);
    finish_mixed_item<IG>(A, n_act, split, k, valid, sx, sy, sz, sp, q, red);
  }
}

__global__ void __launch_bounds__(kThreads, kMixMinBlocks)
    force_mixed_kernel(ForceArgs A) {
  if (A.done && *A.done) return;
  const int n_act = A.n_act_fixed >= 0 ? A.n_act_fixed : *A.n_act_ptr;
  if (n_act <= 0) return;
  const Plan P = A.has_plan ? A.plan
                 : A.plans  ? A.plans[n_act]
                            : make_plan(n_act, A.n, gridDim.x, 0, A.part_cap,
                                        kLaneMinMix, kTileMix);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.nsplit_out)
    *A.nsplit_out = P.S;
  __shared__ MixTile T;
  __shared__ float red[9][kThreads];
  if (P.direct) {
    switch (P.ig) {
      case 128: mixed_items_direct<128>(A, n_act, P, red); break;
      case 64: mixed_items_direct<64>(A, n_act, P, red); break;
      case 32: mixed_items_direct<32>(A, n_act, P, red); break;
      case 16: mixed_items_direct<16>(A, n_act, P, red); break;
      case 8: mixed_items_direct<8>(A, n_act, P, red); break;
      case 4: mixed_items_direct<4>(A, n_act, P, red); break;
      case 2: mixed_items_direct<2>(A, n_act, P, red); break;
      default: mixed_items_direct<1>(A, n_act, P, red); break;
    }
    return;
  }
  switch (P.ig) {
    case 128: mixed_items<128>(A, n_act, P, T, red); break;
    case 64: mixed_items<64>(A, n_act, P, T, red); break;
    case 32: mixed_items<32>(A, n_act, P, T, red); break;
    case 16: mixed_items<16>(A, n_act, P, T, red); break;
    case 8: mixed_items<8>(A, n_act, P, T, red); break;
    case 4: mixed_items<4>(A, n_act, P, T, red); break;
    case 2: mixed_items<2>(A, n_act, P, T, red); break;
    default: mixed_items<1>(A, n_act, P, T, red); break;
  }
}

// ---------------------------------------------------------------------
// Consumers of the partial sums, packing, launch shapes.
// ---------------------------------------------------------------------
__global__ void force_finalize_kernel(const double* part, const int* nsplit,
                                      int n_act, double* a, double* phi,
                                      double* q) {
  const int S = *nsplit;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_act;
       k += gridDim.x * blockDim.x) {
    double s[4];
    for (int c = 0; c < 4; ++c) s[c] = part[c * n_act + k];
    double qq = part[4 * n_act + k];
    #pragma unroll 4
    for (int sp = 1; sp < S; ++sp) {
      const double* p = part + (long long)sp * 5 * n_act;
      for (int c = 0; c < 4; ++c) s[c] = __dadd_rn(s[c], p[c * n_act + k]);
      qq = fmax(qq, p[4 * n_act + k]);
    }
    a[3 * (long long)k + 0] = s[0];
    a[3 * (long long)k + 1] = s[1];
    a[3 * (long long)k + 2] = s[2];
    phi[k] = s[3];
    q[k] = qq;
  }
}

__global__ void pack_aos_kernel(int precision, int n, const double* m,
                                const double* r, const double* v, double* sx,
                                double* sy, double* sz, double* sw0,
                                double* sw1, double* sw2, double* sm,
                                float4* jhi, float4* jlo, float4* jv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    const double x = r[3LL * j], y = r[3LL * j + 1], z = r[3LL * j + 2];
    const double u = v[3LL * j], vv = v[3LL * j + 1], w = v[3LL * j + 2];
    if (precision == 0) {
      sx[j] = x; sy[j] = y; sz[j] = z;
      sw0[j] = u; sw1[j] = vv; sw2[j] = w;
      sm[j] = m[j];
    } else {
      const float xh = (float)x, yh = (float)y, zh = (float)z;
      jhi[j] = make_float4(xh, yh, zh, (float)m[j]);
      jlo[j] = make_float4((float)(x - (double)xh), (float)(y - (double)yh),
                           (float)(z - (double)zh), 0.f);
      jv[j] = make_float4((float)u, (float)vv, (float)w, 0.f);
    }
  }
}

ForceLaunch force_launch_shape(int precision, int device) {
  // fixed table per device (this path allocates nothing)
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static ForceLaunch cache[2][kMaxDevices];
  std::lock_guard<std::mutex> g(mu);
  ForceLaunch* c = cache[precision ? 1 : 0];
  const bool cached = device >= 0 && device < kMaxDevices;
  if (cached && c[device].grid > 0) return c[device];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (precision)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_mixed_kernel,
                                                  kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_fp64_kernel,
                                                  kThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  ForceLaunch fl;
  fl.grid = sms * per_sm;
  fl.threads = kThreads;
  fl.tile_i = kThreads;
  fl.part_cap = 5LL * fl.grid * kThreads;
  if (cached) c[device] = fl;
  return fl;
}

cudaError_t launch_force(int precision, const ForceArgs& fa,
                         const ForceLaunch& fl, cudaStream_t s) {
  if (precision)
    force_mixed_kernel<<<fl.grid, kThreads, 0, s>>>(fa);
  else
    force_fp64_kernel<<<fl.grid, kThreads, 0, s>>>(fa);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Autotuner of the mixed force plans.
// ---------------------------------------------------------------------
namespace {

struct TuneKey {
  int device, n, grid;
  bool operator<(const TuneKey& o) const {
    return device != o.device ? device < o.device
           : n != o.n         ? n < o.n
                              : grid < o.grid;
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, std::vector<Plan>> g_tuned;

// candidate plans for b active bodies: every i-group width, staged tiles for
// the wider groups and direct loads for the narrower ones, split counts
// {1, 2, 3, 4, 6, 8, 12, 16} within the per-thread work floor and the
// partial-sum buffer, plus for each width the split count with the best
// wave fill of the grid
std::vector<Plan> candidates(int b, int n, int grid, long long part_cap) {
  static const int kS[] = {1, 2, 3, 4, 6, 8, 12, 16};
  std::vector<Plan> out;
  for (int ig = kThreads; ig >= 1; ig >>= 1) {
    if (ig > 2 * b && ig > 1) continue;
    const int jg = kThreads / ig;
    const int n_g = (b + ig - 1) / ig;
    long long smax = n / ((long long)jg * kLaneMinMix);
    smax = std::max<long long>(1, std::min<long long>(smax, kSplitCap));
    std::vector<int> ss(std::begin(kS), std::end(kS));
    int best_s = 1;
    double best_fill = 0;
    for (int S = 1; S <= smax; ++S) {
      const long long items = (long long)n_g * S;
      const double fill =
          (double)items / (double)(((items + grid - 1) / grid) * grid);
      if (fill > best_fill + 1e-9) {
        best_fill = fill;
        best_s = S;
      }
    }
    ss.push_back(best_s);
    std::sort(ss.begin(), ss.end());
    ss.erase(std::unique(ss.begin(), ss.end()), ss.end());
    for (int direct = 0; direct <= 1; ++direct) {
      if (direct && ig > 32) continue;
      if (!direct && ig < 8) continue;
      for (int S : ss) {
        if (S > smax) continue;
        if ((long long)S * 5 * b > part_cap) continue;
        long long chunk = (n + S - 1) / S;
        chunk = (chunk + 1) & ~1LL;
        out.push_back(Plan{ig, n_g, S, (int)chunk, direct});
      }
    }
  }
  return out;
}

}  // namespace

const std::vector<Plan>* tuned_plans(int device, int n, int grid) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned.find(TuneKey{device, n, grid});
  return it == g_tuned.end() ? nullptr : &it->second;
}

// Time the candidate plans of every power-of-two active count up to n on
// the j records in `base` (bodies idx[0..b) active) and keep the fastest;
// an active count between two buckets takes the plan of the larger one.
// The table is cached per (device, n, grid) for the life of the process.
cudaError_t autotune_mixed_plans(int device, const ForceArgs& base,
                                 const ForceLaunch& fl, int* d_nsplit,
                                 cudaStream_t s, std::vector<Plan>* table) {
  const int n = base.n;
  if (const std::vector<Plan>* t = tuned_plans(device, n, fl.grid)) {
    *table = *t;
    return cudaSuccess;
  }
  std::vector<int> buckets;
  for (long long b = 1; b < n; b *= 2) buckets.push_back((int)b);
  buckets.push_back(n);
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  std::vector<Plan> best(buckets.size());
  for (size_t bi = 0; bi < buckets.size() && err == cudaSuccess; ++bi) {
    const int b = buckets[bi];
    float best_ms = 1e30f;
    for (const Plan& p : candidates(b, n, fl.grid, base.part_cap)) {
      ForceArgs fa = base;
      fa.n_act_fixed = b;
      fa.n_act_ptr = nullptr;
      fa.nsplit_out = d_nsplit;
      fa.done = nullptr;
      fa.plans = nullptr;
      fa.plan = p;
      fa.has_plan = 1;
      launch_force(1, fa, fl, s);
      cudaEventRecord(e0, s);
      const int reps = 3;
      for (int r = 0; r < reps; ++r) launch_force(1, fa, fl, s);
      cudaEventRecord(e1, s);
      err = cudaEventSynchronize(e1);
      if (err != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best[bi] = p;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  table->assign(n + 1, Plan{kThreads, 0, 1, n, 0});
  size_t bi = 0;
  for (int k = 1; k <= n; ++k) {
    while (buckets[bi] < k) ++bi;
    Plan p = best[bi];
    p.n_g = (k + p.ig - 1) / p.ig;
    if ((long long)p.S * 5 * k > base.part_cap) {
      p.S = 1;
      p.chunk = (n + 1) & ~1;
    }
    (*table)[k] = p;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned[TuneKey{device, n, fl.grid}] = *table;
  return cudaSuccess;
}

cudaError_t launch_force_finalize(const double* part, const int* nsplit,
                                  int n_act, double* a, double* phi,
                                  double* q, cudaStream_t s) {
  if (n_act <= 0) return cudaSuccess;
  const int threads = 256;
  const int grid = std::min((n_act + threads - 1) / threads, 4096);
  force_finalize_kernel<<<grid, threads, 0, s>>>(part, nsplit, n_act, a, phi,
                                                 q);
  return cudaGetLastError();
}

cudaError_t launch_pack_aos(int precision, int n, const double* m,
                            const double* r, const double* v, double* sx,
                            double* sy, double* sz, double* sw0, double* sw1,
                            double* sw2, double* sm, float4* jhi, float4* jlo,
                            float4* jv, cudaStream_t s) {
  const int threads = 256;
  const int grid = std::min((n + threads - 1) / threads, 8192);
  pack_aos_kernel<<<grid, threads, 0, s>>>(precision, n, m, r, v, sx, sy, sz,
                                           sw0, sw1, sw2, sm, jhi, jlo, jv);
  return cudaGetLastError();
}

}  // namespace tsbts
