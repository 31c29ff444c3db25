// Device code of the force kernels (Sec. 2 Alg. 2 step 5; Eq. 3; Plummer
// softening of Sec. 3), shared by the single-system kernels (k_force.cu)
// and the ensemble kernels (k_ensemble.cu). One work item is an i-group of
// IG active bodies against one j-chunk; *_item computes one item, *_items
// walks the items of a plan over a persistent grid.
#pragma once

#include "tsbts_internal.cuh"

namespace tsbts {

constexpr int kThreads = 128;   // threads per block
constexpr int kTileF64 = 64;    // j per shared-memory tile, FP64
constexpr int kTileMix = 256;   // j per shared-memory tile, mixed
constexpr int kLaneMinMix = 16; // fewest j per thread in a split item
constexpr int kLaneMinF64 = 8;
constexpr int kSplitCap = 16;   // most j-splits of one active body
constexpr int kSplitCapDirect = 128;  // most j-splits of a direct-load plan
constexpr int kDirectBatch = 4;  // j records per lane loaded in one batch

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
struct __align__(16) F64Tile {
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

// 1/sqrt(s2) in FP64 for the j-split path: the FP32 reciprocal square root
// refined by two Newton-Raphson steps for 1/sqrt (y <- y + y (1 - s2 y^2)/2,
// each squaring the relative error: 2^-22 -> 2^-44 -> below FP64 rounding),
// ten FP64 operations instead of a correctly rounded square root and
// division (the FP64 pipe of this GPU is narrow). s2 outside 1e-36 .. 1e36
// takes the correctly rounded form.
__device__ __forceinline__ double rsqrt_f64(double s2) {
  if (!(s2 > 1e-36 && s2 < 1e36)) return __ddiv_rn(1.0, __dsqrt_rn(s2));
  double y = (double)rsqrtf((float)s2);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-(s2 * y), y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}

// The same pair term with the reciprocal square root and fused
// multiply-adds (j-split path: the sums are not in the oracle's order
// anyway, and each term agrees with the rounded definition to ~1e-16).
__device__ __forceinline__ void pair_f64_fast(const F64Tile& T, int t,
                                              double xi, double yi, double zi,
                                              double ui, double vi, double wi,
                                              double eps2, F64Acc& s) {
  const double dx = T.x[t] - xi;
  const double dy = T.y[t] - yi;
  const double dz = T.z[t] - zi;
  const double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  const double rinv = rsqrt_f64(s2);
  const double rinv2 = rinv * rinv;
  const double mr = T.m[t] * rinv;
  const double f = mr * rinv2;
  s.ax = fma(f, dx, s.ax);
  s.ay = fma(f, dy, s.ay);
  s.az = fma(f, dz, s.az);
  s.ph -= mr;
  const double wx = T.u[t] - ui;
  const double wy = T.v[t] - vi;
  const double wz = T.w[t] - wi;
  const double c = fma(wx, wx, fma(wy, wy, wz * wz)) * rinv2;
  s.q = fmax(s.q, fmax(c, f));
}

template <int IG>
__device__ void f64_item(const ForceArgs& A, int n_act, const Plan& P,
    int g, int split, F64Tile& T, double (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  constexpr int TJ = kTileF64;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const double eps2 = A.eps2;
  {
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
      if (A.exact) {
        for (int q = jl; q < cnt; q += JG) {
          if (jt + q == i) continue;
          pair_f64(T, q, xi, yi, zi, ui, vi, wi, eps2, s);
        }
      } else {
        for (int q = jl; q < cnt; q += JG) {
          if (jt + q == i) continue;
          pair_f64_fast(T, q, xi, yi, zi, ui, vi, wi, eps2, s);
        }
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

// FP64 with ascending-j sums for a few active bodies, one body per block:
// the block's threads compute the pair terms of kThreads consecutive j in
// parallel (the correctly rounded square root and divisions are the long
// latency) and thread 0 then adds them in ascending j, the same rounded
// operations in the same order as one thread running the whole loop. The
// self pair contributes exact zeros (a sum that starts at +0 is never -0,
// so adding +0 leaves it unchanged). q is a maximum, exact in any order.
__device__ inline void f64_item_exact1(const ForceArgs& A, int n_act, int k,
                                double (*red)[kThreads]) {
  const int t = threadIdx.x;
  const int i = A.idx[k];
  const double xi = A.x[0][i], yi = A.x[1][i], zi = A.x[2][i];
  const double ui = A.w[0][i], vi = A.w[1][i], wi = A.w[2][i];
  const double eps2 = A.eps2;
  F64Acc s = {0.0, 0.0, 0.0, 0.0, 0.0};
  double ql = 0.0;
  for (int jt = 0; jt < A.n; jt += kThreads) {
    const int j = jt + t;
    double tx = 0.0, ty = 0.0, tz = 0.0, tp = 0.0;
    if (j < A.n && j != i) {
      const double dx = __dsub_rn(A.x[0][j], xi);
      const double dy = __dsub_rn(A.x[1][j], yi);
      const double dz = __dsub_rn(A.x[2][j], zi);
      const double s2 = __dadd_rn(
          __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                    __dmul_rn(dz, dz)),
          eps2);
      const double sq = __dsqrt_rn(s2);
      const double mj = A.m[j];
      const double f = __ddiv_rn(mj, __dmul_rn(s2, sq));
      tx = __dmul_rn(f, dx);
      ty = __dmul_rn(f, dy);
      tz = __dmul_rn(f, dz);
      tp = __ddiv_rn(mj, sq);
      const double wx = __dsub_rn(A.w[0][j], ui);
      const double wy = __dsub_rn(A.w[1][j], vi);
      const double wz = __dsub_rn(A.w[2][j], wi);
      const double c = __ddiv_rn(
          __dadd_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)),
                    __dmul_rn(wz, wz)),
          s2);
      if (c > ql) ql = c;
      if (f > ql) ql = f;
    }
    __syncthreads();  // the previous tile's terms have been added
    red[0][t] = tx;
    red[1][t] = ty;
    red[2][t] = tz;
    red[3][t] = tp;
    __syncthreads();
    if (t == 0) {
      const int cnt = min(kThreads, A.n - jt);
      for (int q = 0; q < cnt; ++q) {
        s.ax = __dadd_rn(s.ax, red[0][q]);
        s.ay = __dadd_rn(s.ay, red[1][q]);
        s.az = __dadd_rn(s.az, red[2][q]);
        s.ph = __dsub_rn(s.ph, red[3][q]);
      }
    }
  }
  __syncthreads();
  red[4][t] = ql;
  __syncthreads();
  for (int half = kThreads / 2; half >= 1; half >>= 1) {
    if (t < half) red[4][t] = fmax(red[4][t], red[4][t + half]);
    __syncthreads();
  }
  if (t == 0) write_partial(A, n_act, 0, k, s.ax, s.ay, s.az, s.ph, red[4][0]);
  __syncthreads();  // red is reused by the block's next body
}

template <int IG>
__device__ void f64_items(const ForceArgs& A, int n_act, const Plan& P,
                          F64Tile& T, double (*red)[kThreads]) {
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x)
    f64_item<IG>(A, n_act, P, w / P.S, w % P.S, T, red);
}

// ---------------------------------------------------------------------
// Mixed: FP32 pair terms on double-single relative coordinates
// d = (x_hi,j - x_hi,i) + (x_lo,j - x_lo,i); FP32 sums per j tile folded
// into hi/lo compensated accumulators; q is an exact FP32 max.
// ---------------------------------------------------------------------
// structure of arrays: consecutive j pair up for f32x2. The tile is read
// with 8- and 16-byte shared loads, so it must start on a 16-byte boundary
// wherever the kernel places it among its other shared variables.
struct __align__(16) MixTile {
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
__device__ void mixed_item(const ForceArgs& A, int n_act, const Plan& P,
    int g, int split, MixTile& T, float (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  constexpr int TJ = kTileMix;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const float eps2 = A.eps2f;
  {
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

template <int IG>
__device__ void mixed_items(const ForceArgs& A, int n_act, const Plan& P,
                            MixTile& T, float (*red)[kThreads]) {
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x)
    mixed_item<IG>(A, n_act, P, w / P.S, w % P.S, T, red);
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
// BATCH j records per lane are loaded in one batch before any is used, so
// a small item waits for a few round trips to L2, not one per j; BATCH = 1
// keeps the register budget of kernels that hold more state (ensembles).
template <int IG, int BATCH = kDirectBatch>
__device__ void mixed_direct_item(const ForceArgs& A, int n_act, const Plan& P,
    int g, int split, float (*red)[kThreads]) {
  constexpr int JG = kThreads / IG;
  const int t = threadIdx.x;
  const int il = t % IG, jl = t / IG;
  const float eps2 = A.eps2f;
  {
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
    if constexpr (BATCH == 1) {
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
    }
    for (int jb = j0 + jl; BATCH > 1 && jb < j1; jb += JG * BATCH) {
      float4 h[BATCH], l[BATCH], vv[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int j = jb + u * JG;
        if (j < j1) {
          h[u] = __ldg(A.jhi + j);
          l[u] = __ldg(A.jlo + j);
          vv[u] = __ldg(A.jv + j);
        }
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int j = jb + u * JG;
        if (j < j1 && j != i)
          pair_mixed_g(I, h[u], l[u], vv[u], eps2, ax, ay, az, ph, q);
      }
      cnt += BATCH;
      if (cnt >= kTileMix) {
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

template <int IG>
__device__ void mixed_items_direct(const ForceArgs& A, int n_act,
                                   const Plan& P, float (*red)[kThreads]) {
  for (int w = blockIdx.x; w < P.n_g * P.S; w += gridDim.x)
    mixed_direct_item<IG>(A, n_act, P, w / P.S, w % P.S, red);
}

}  // namespace tsbts
