// Kernels of the adjoint of a frozen block schedule: the replay of an era's
// final-pass schedule as plain block steps (Eq. 2 prediction of every body,
// Eq. 3 force sums on the active bodies, Eq. 1 correction) and its reverse
// mode, one block step at a time in reverse order.
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
// The FP64 replay uses the integrator's op-by-op FP64 expressions and force
// kernels, so it reproduces a sequential FP64 replay bit for bit when the
// force sums run in ascending j. The mixed pair terms of the reverse sweep
// are FP32 on double-single relative coordinates, summed in FP32 over at
// most kFold sources and then in FP64.
#include <algorithm>

#include "tsbts_kernels.cuh"

namespace tsbts {

namespace {

constexpr int kAdjThreads = 128;
constexpr int kFold = 64;  // FP32 pair terms per FP64 fold, per lane

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

// ---------------------------------------------------------------------
// Forward replay
// ---------------------------------------------------------------------

__global__ void adj_load_kernel(int n, const double* m_in, const double* r_in,
                                const double* v_in, int mixed, double* m_out,
                                AdjState St, AdjPred P, int* err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    const double m = m_in[j];
    bool ok = isfinite(m);
    m_out[j] = m;
    double p[3];
    for (int c = 0; c < 3; ++c) {
      const double r = r_in[3LL * j + c], v = v_in[3LL * j + c];
      ok = ok && isfinite(r) && isfinite(v);
      St.r[c][j] = r;
      St.v[c][j] = v;
      St.a[c][j] = 0.0;
      P.p[c][j] = r;
      p[c] = r;
    }
    St.tau[j] = 0;
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

__global__ void adj_init_accel_kernel(int n, const double* part,
                                      const int* nsplit, AdjState St,
                                      int* err) {
  const int S = *nsplit;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    double an[3];
    partial_sum(part, n, S, j, an);
    if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]))
      atomicOr(err, 1);
    for (int c = 0; c < 3; ++c) St.a[c][j] = an[c];
  }
}

__global__ void adj_predict_kernel(int n, long long T, double inv_ticks,
                                   int mixed, AdjState St, AdjPred P) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    double p[3];
    predict_into(j, T, inv_ticks, mixed, St, P, p);
  }
}

// Eq. 1 for the active bodies; the tape receives their pre-step state
__global__ void adj_correct_kernel(int n_act, const int* idx, long long T,
                                   double inv_ticks, const double* part,
                                   const int* nsplit, AdjState St, AdjPred P,
                                   AdjTape Tp, long long e0, int* err) {
  const int S = *nsplit;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_act;
       k += gridDim.x * blockDim.x) {
    const int i = idx[k];
    double an[3];
    partial_sum(part, n_act, S, k, an);
    if (!isfinite(an[0]) || !isfinite(an[1]) || !isfinite(an[2]))
      atomicOr(err, 1);
    if (Tp.tau) {
      const long long t = e0 + k - Tp.base;
      for (int c = 0; c < 3; ++c) {
        Tp.x[c][t] = St.r[c][i];
        Tp.x[3 + c][t] = St.v[c][i];
        Tp.x[6 + c][t] = St.a[c][i];
      }
      Tp.tau[t] = St.tau[i];
    }
    const double h = tick_h(T, St.tau[i], inv_ticks);
    for (int c = 0; c < 3; ++c) {
      St.v[c][i] = __dadd_rn(
          St.v[c][i],
          __dmul_rn(__dmul_rn(0.5, __dadd_rn(St.a[c][i], an[c])), h));
      St.r[c][i] = P.p[c][i];
      St.a[c][i] = an[c];
    }
    St.tau[i] = T;
  }
}

// ---------------------------------------------------------------------
// Reverse sweep
// ---------------------------------------------------------------------

// Per body: restore the pre-step state of the active bodies from the tape
// (cur_e[j] is body j's latest entry not yet reversed), the Eq. 1 part of
// the reverse step for them, and the Eq. 2 prediction of every body. With
// `all` every body is active at T = 0 (the initial force): its cotangent
// ga becomes lam and nothing is restored.
__global__ void adj_back_prep_kernel(int n, long long T, double inv_ticks,
                                     long long e_lo, int all, int mixed,
                                     AdjState St, AdjTape Tp,
                                     long long* cur_e, const long long* prev_e,
                                     AdjCot C, AdjPred P, AdjSlots Sl) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    int k = -1;
    if (all) {
      k = j;
    } else {
      const long long e = cur_e[j];
      if (e >= e_lo) {
        k = (int)(e - e_lo);
        const long long t = e - Tp.base;
        for (int c = 0; c < 3; ++c) {
          St.r[c][j] = Tp.x[c][t];
          St.v[c][j] = Tp.x[3 + c][t];
          St.a[c][j] = Tp.x[6 + c][t];
        }
        St.tau[j] = Tp.tau[t];
        cur_e[j] = prev_e[e];
      }
    }
    Sl.slot[j] = k;
    double p[3];
    predict_into(j, T, inv_ticks, mixed, St, P, p);
    if (k < 0) continue;
    const double h = tick_h(T, St.tau[j], inv_ticks);
    const double hh = __dmul_rn(0.5, h);
    double lam[3];
    for (int c = 0; c < 3; ++c) {
      const double ga = C.ga[c][j];
      const double gv_h = __dmul_rn(hh, C.gv[c][j]);
      lam[c] = all ? ga : __dadd_rn(ga, gv_h);
      Sl.lam[c][k] = lam[c];
      Sl.gp0[c][k] = all ? 0.0 : C.gr[c][j];
      C.ga[c][j] = all ? 0.0 : gv_h;
      if (!all) C.gr[c][j] = 0.0;
      Sl.ap[c][k] = p[c];
    }
    if (mixed) {
      float4 hi, lo;
      pack_ds(p[0], p[1], p[2], 0.f, hi, lo);
      Sl.ahi[k] = hi;
      Sl.alo[k] = lo;
      Sl.alam[k] = make_float4((float)lam[0], (float)lam[1], (float)lam[2], 0.f);
    }
  }
}

struct VjpArgs {
  int n, n_act;
  const int* idx;
  const int* slot;
  double eps2;
  float eps2f;
  AdjPred P;
  AdjSlots Sl;
  VjpShape V;
  int iblocks;
  double* part_i;  // [S_i][3][n_act]
  double* part_j;  // [S_j][4][n]
};

template <int kN>
__device__ __forceinline__ void lane_reduce(double (&x)[kN], int tpt) {
  for (int o = tpt >> 1; o > 0; o >>= 1)
    for (int c = 0; c < kN; ++c) x[c] += __shfl_xor_sync(kFull, x[c], o);
}

// i side: for active slot k (body i), u_k = sum_{j != i} g_ij
//   = lam_i W_i - 3 U_i,  W_i = sum m_j / s^3,
//   U_i = sum m_j (lam_i . d_ij) d_ij / s^5.
template <int kMixed>
__device__ __forceinline__ void vjp_i_side(const VjpArgs& A, int b) {
  const VjpSide& V = A.V.si;
  const int tpb = kAdjThreads / V.tpt;
  const int g = b / V.S, sp = b - g * V.S;
  const int k = g * tpb + threadIdx.x / V.tpt;
  const int lane = threadIdx.x & (V.tpt - 1);
  const bool live = k < A.n_act;
  const int beg = sp * V.chunk;
  const int end = live ? min(A.n, beg + V.chunk) : beg;
  const int bi = live ? A.idx[k] : -1;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // W, U
  if (kMixed) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ih = live ? A.Sl.ahi[k] : z4;
    const float4 il = live ? A.Sl.alo[k] : z4;
    const float4 lm = live ? A.Sl.alam[k] : z4;
    for (int j0 = beg + lane; j0 < end; j0 += V.tpt * kFold) {
      const int j1 = min(end, j0 + V.tpt * kFold);
      float w = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f;
      for (int j = j0; j < j1; j += V.tpt) {
        const float4 jh = A.P.jhi[j], jl = A.P.jlo[j];
        const float dx = (jh.x - ih.x) + (jl.x - il.x);
        const float dy = (jh.y - ih.y) + (jl.y - il.y);
        const float dz = (jh.z - ih.z) + (jl.z - il.z);
        const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, A.eps2f)));
        const float rs = (j == bi) ? 0.f : rsqrtf(s2);
        const float rs2 = rs * rs;
        const float mr3 = jh.w * rs2 * rs;
        const float ld = fmaf(lm.x, dx, fmaf(lm.y, dy, lm.z * dz));
        const float cc = mr3 * rs2 * ld;
        w += mr3;
        u0 = fmaf(cc, dx, u0);
        u1 = fmaf(cc, dy, u1);
        u2 = fmaf(cc, dz, u2);
      }
      acc[0] += w;
      acc[1] += u0;
      acc[2] += u1;
      acc[3] += u2;
    }
  } else {
    double ix = 0, iy = 0, iz = 0, lx = 0, ly = 0, lz = 0;
    if (live) {
      ix = A.Sl.ap[0][k];
      iy = A.Sl.ap[1][k];
      iz = A.Sl.ap[2][k];
      lx = A.Sl.lam[0][k];
      ly = A.Sl.lam[1][k];
      lz = A.Sl.lam[2][k];
    }
    for (int j = beg + lane; j < end; j += V.tpt) {
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
  }
  lane_reduce(acc, V.tpt);
  if (live && lane == 0) {
    for (int c = 0; c < 3; ++c)
      A.part_i[((long long)sp * 3 + c) * A.n_act + k] =
          A.Sl.lam[c][k] * acc[0] - 3.0 * acc[1 + c];
  }
}

// j side: for body j, G_j = sum_{i in A, i != j} (lam_i / s^3
//   - 3 (lam_i . d_ij) d_ij / s^5) and Z_j = sum lam_i . d_ij / s^3, with
// d_ij = p_j - p_i; body j's position cotangent gets m_j G_j, its mass
// cotangent Z_j.
template <int kMixed>
__device__ __forceinline__ void vjp_j_side(const VjpArgs& A, int b) {
  const VjpSide& V = A.V.sj;
  const int tpb = kAdjThreads / V.tpt;
  const int g = b / V.S, sp = b - g * V.S;
  const int j = g * tpb + threadIdx.x / V.tpt;
  const int lane = threadIdx.x & (V.tpt - 1);
  const bool live = j < A.n;
  const int beg = sp * V.chunk;
  const int end = live ? min(A.n_act, beg + V.chunk) : beg;
  const int sj = live ? A.slot[j] : -1;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // G, Z
  if (kMixed) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 jh = live ? A.P.jhi[j] : z4;
    const float4 jl = live ? A.P.jlo[j] : z4;
    for (int k0 = beg + lane; k0 < end; k0 += V.tpt * kFold) {
      const int k1 = min(end, k0 + V.tpt * kFold);
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, zz = 0.f;
      for (int k = k0; k < k1; k += V.tpt) {
        const float4 ah = A.Sl.ahi[k], al = A.Sl.alo[k], lm = A.Sl.alam[k];
        const float dx = (jh.x - ah.x) + (jl.x - al.x);
        const float dy = (jh.y - ah.y) + (jl.y - al.y);
        const float dz = (jh.z - ah.z) + (jl.z - al.z);
        const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, A.eps2f)));
        const float rs = (k == sj) ? 0.f : rsqrtf(s2);
        const float rs2 = rs * rs;
        const float rs3 = rs2 * rs;
        const float t = fmaf(lm.x, dx, fmaf(lm.y, dy, lm.z * dz)) * rs3;
        const float cc = -3.f * t * rs2;
        zz += t;
        g0 = fmaf(cc, dx, fmaf(rs3, lm.x, g0));
        g1 = fmaf(cc, dy, fmaf(rs3, lm.y, g1));
        g2 = fmaf(cc, dz, fmaf(rs3, lm.z, g2));
      }
      acc[0] += g0;
      acc[1] += g1;
      acc[2] += g2;
      acc[3] += zz;
    }
  } else {
    double px = 0, py = 0, pz = 0;
    if (live) {
      px = A.P.p[0][j];
      py = A.P.p[1][j];
      pz = A.P.p[2][j];
    }
    for (int k = beg + lane; k < end; k += V.tpt) {
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
  }
  lane_reduce(acc, V.tpt);
  if (live && lane == 0) {
    for (int c = 0; c < 4; ++c)
      A.part_j[((long long)sp * 4 + c) * A.n + j] = acc[c];
  }
}

template <int kMixed>
__global__ void __launch_bounds__(kAdjThreads) adj_vjp_kernel(VjpArgs A) {
  const int b = blockIdx.x;
  if (b < A.iblocks)
    vjp_i_side<kMixed>(A, b);
  else
    vjp_j_side<kMixed>(A, b - A.iblocks);
}

// Sum the splits, assemble the position cotangent of every body and pass
// it through Eq. 2 to gr, gv, ga; add the mass cotangent.
__global__ void adj_back_finalize_kernel(int n, int n_act, long long T,
                                         double inv_ticks, int Si, int Sj,
                                         const double* part_i,
                                         const double* part_j, AdjPred P,
                                         AdjSlots Sl, AdjState St, AdjCot C,
                                         int* err) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    double G[4];
    for (int c = 0; c < 4; ++c) G[c] = part_j[(long long)c * n + j];
    for (int sp = 1; sp < Sj; ++sp)
      for (int c = 0; c < 4; ++c)
        G[c] += part_j[((long long)sp * 4 + c) * n + j];
    const double m = P.m[j];
    double gp[3];
    for (int c = 0; c < 3; ++c) gp[c] = m * G[c];
    const int k = Sl.slot[j];
    if (k >= 0) {
      for (int c = 0; c < 3; ++c) {
        double u = part_i[(long long)c * n_act + k];
        for (int sp = 1; sp < Si; ++sp)
          u += part_i[((long long)sp * 3 + c) * n_act + k];
        gp[c] = Sl.gp0[c][k] + (gp[c] - u);
      }
    }
    if (!isfinite(gp[0]) || !isfinite(gp[1]) || !isfinite(gp[2]) ||
        !isfinite(G[3]))
      atomicOr(err, 1);
    C.gm[j] += G[3];
    const double h = tick_h(T, St.tau[j], inv_ticks);
    const double hh2 = 0.5 * h * h;
    for (int c = 0; c < 3; ++c) {
      C.gr[c][j] += gp[c];
      C.gv[c][j] += h * gp[c];
      C.ga[c][j] += hh2 * gp[c];
    }
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
                                AdjCot C) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      C.gr[c][j] = gr ? gr[3LL * j + c] : 0.0;
      C.gv[c][j] = gv ? gv[3LL * j + c] : 0.0;
      C.ga[c][j] = 0.0;
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

VjpSide choose_side(long long nt, long long ns, int sms) {
  const long long want = (long long)sms * 1024;  // threads in flight
  const long long min_chunk = 64;
  VjpSide v{};
  long long S = (want + nt - 1) / nt;
  const long long smax = std::max<long long>(1, ns / min_chunk);
  int tpt = 1;
  if (S > smax) {
    // too few sources to split further: several threads per target
    const long long f = want / (nt * smax);
    while (tpt < 32 && 2 * tpt <= f && ns / smax >= 32LL * tpt) tpt *= 2;
    S = smax;
  }
  S = std::max<long long>(1, std::min<long long>(S, 1024));
  long long chunk = (ns + S - 1) / S;
  if (chunk < 1) chunk = 1;
  S = (ns + chunk - 1) / chunk;
  v.tpt = tpt;
  v.S = (int)std::max<long long>(1, S);
  v.chunk = (int)chunk;
  const int tpb = kAdjThreads / tpt;
  v.groups = (int)((nt + tpb - 1) / tpb);
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
                     const double* v_in, int mixed, double* m_out,
                     const AdjState& St, const AdjPred& P, int* err,
                     cudaStream_t s) {
  adj_load_kernel<<<grid_for(n), 256, 0, s>>>(n, m_in, r_in, v_in, mixed,
                                              m_out, St, P, err);
}

void launch_adj_init_accel(int n, const double* part, const int* nsplit,
                           const AdjState& St, int* err, cudaStream_t s) {
  adj_init_accel_kernel<<<grid_for(n), 256, 0, s>>>(n, part, nsplit, St, err);
}

void launch_adj_predict(int n, long long T, double inv_ticks, int mixed,
                        const AdjState& St, const AdjPred& P, cudaStream_t s) {
  adj_predict_kernel<<<grid_for(n), 256, 0, s>>>(n, T, inv_ticks, mixed, St,
                                                 P);
}

void launch_adj_correct(int n_act, const int* idx, long long T,
                        double inv_ticks, const double* part,
                        const int* nsplit, const AdjState& St,
                        const AdjPred& P, const AdjTape& Tp, long long e0,
                        int* err, cudaStream_t s) {
  // 32-thread blocks spread the FP64 work of small active sets over SMs
  const int grid = std::max(1, std::min((n_act + 31) / 32, 8192));
  adj_correct_kernel<<<grid, 32, 0, s>>>(n_act, idx, T, inv_ticks, part,
                                         nsplit, St, P, Tp, e0, err);
}

void launch_adj_back_prep(int n, long long T, double inv_ticks, long long e_lo,
                          int all, int mixed, const AdjState& St,
                          const AdjTape& Tp, long long* cur_e,
                          const long long* prev_e, const AdjCot& C,
                          const AdjPred& P, const AdjSlots& Sl,
                          cudaStream_t s) {
  adj_back_prep_kernel<<<grid_for(n), 256, 0, s>>>(
      n, T, inv_ticks, e_lo, all, mixed, St, Tp, cur_e, prev_e, C, P, Sl);
}

void launch_adj_vjp(int mixed, int n, int n_act, const int* idx, double eps2,
                    const AdjPred& P, const AdjSlots& Sl, const VjpShape& V,
                    double* part_i, double* part_j, cudaStream_t s) {
  VjpArgs A;
  A.n = n;
  A.n_act = n_act;
  A.idx = idx;
  A.slot = Sl.slot;
  A.eps2 = eps2;
  A.eps2f = (float)eps2;
  A.P = P;
  A.Sl = Sl;
  A.V = V;
  A.iblocks = V.si.groups * V.si.S;
  A.part_i = part_i;
  A.part_j = part_j;
  const int grid = A.iblocks + V.sj.groups * V.sj.S;
  if (mixed)
    adj_vjp_kernel<1><<<grid, kAdjThreads, 0, s>>>(A);
  else
    adj_vjp_kernel<0><<<grid, kAdjThreads, 0, s>>>(A);
}

void launch_adj_back_finalize(int n, int n_act, long long T, double inv_ticks,
                              const VjpShape& V, const double* part_i,
                              const double* part_j, const AdjPred& P,
                              const AdjSlots& Sl, const AdjState& St,
                              const AdjCot& C, int* err, cudaStream_t s) {
  adj_back_finalize_kernel<<<grid_for(n), 256, 0, s>>>(
      n, n_act, T, inv_ticks, V.si.S, V.sj.S, part_i, part_j, P, Sl, St, C,
      err);
}

void launch_adj_loss(int n, const double* m, const AdjState& St, double* out,
                     const AdjCot& C, cudaStream_t s) {
  adj_loss_kernel<<<1, kLossThreads, 0, s>>>(n, m, St, out);
  adj_loss_seed_kernel<<<grid_for(n), 256, 0, s>>>(n, m, St, out, C);
}

void launch_adj_seed(int n, const double* gr, const double* gv,
                     const AdjCot& C, cudaStream_t s) {
  adj_seed_kernel<<<grid_for(n), 256, 0, s>>>(n, gr, gv, C);
}

void launch_soa_to_aos(int n, double* const src[3], double* dst,
                       cudaStream_t s) {
  soa_to_aos_kernel<<<grid_for(n), 256, 0, s>>>(n, src[0], src[1], src[2],
                                                dst);
}

}  // namespace tsbts
