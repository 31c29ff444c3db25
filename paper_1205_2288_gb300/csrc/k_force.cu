// Force kernels of the TSBTS library (Sec. 2 Alg. 2 step 5; Eq. 3; Plummer
// softening of Sec. 3): for each active body i and all j != i
//   a_i   = sum m_j d_ij / s^3,   phi_i = -sum m_j / s,
//   q_i   = max max(|v_ij|^2 / s^2, m_j / s^3),   s^2 = |d_ij|^2 + eps^2.
//
// Work decomposition (the GB300 analogue of the paper's Alg. 4 data/work
// partition): a persistent grid walks work items (i-tile, j-chunk). When
// the active set is large every item covers all j (data partition); when
// it is small the j range is split so that the grid stays full (work
// partition), and the split partial sums are added in fixed split order
// by the consumer, so results are deterministic.
//
// j records are staged tile by tile in shared memory with coalesced loads
// and read back as broadcasts. The pairwise loop is FMA-pipe bound.
#include <algorithm>
#include <mutex>
#include <vector>

#include "tsbts_internal.cuh"

namespace tsbts {

constexpr int kJMin = 512;      // shortest j chunk of a split work item
constexpr int kThreads = 128;   // threads per block = active bodies per item
constexpr int kTileF64 = 64;    // j per shared-memory tile, FP64
constexpr int kTileMix = 256;   // j per shared-memory tile, mixed

__device__ __forceinline__ int choose_split(int n_tiles, int grid, int n,
                                            int exact, int n_act,
                                            long long part_cap) {
  if (exact) return 1;
  int s = grid / n_tiles;
  int smax = n / kJMin;
  if (smax < 1) smax = 1;
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  while (s > 1 && (long long)s * 5 * n_act > part_cap) --s;
  return s;
}

// ---------------------------------------------------------------------
// FP64: each pair term rounded op by op in the order of the definition.
// ---------------------------------------------------------------------
template <int NT, int TJ>
__global__ void __launch_bounds__(NT) force_fp64_kernel(ForceArgs A) {
  if (A.done && *A.done) return;
  const int n_act = A.n_act_fixed >= 0 ? A.n_act_fixed : *A.n_act_ptr;
  if (n_act <= 0) return;
  const int n = A.n;
  const int n_tiles = (n_act + NT - 1) / NT;
  const int S = choose_split(n_tiles, gridDim.x, n, A.exact, n_act,
                             A.part_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.nsplit_out)
    *A.nsplit_out = S;
  const int chunk = ((n + S - 1) / S + TJ - 1) / TJ * TJ;
  __shared__ double sx[TJ], sy[TJ], sz[TJ], su[TJ], sv[TJ], sw[TJ], sm[TJ];
  const double eps2 = A.eps2;
  const int items = n_tiles * S;
  for (int w = blockIdx.x; w < items; w += gridDim.x) {
    const int tile = w / S;
    const int split = w - tile * S;
    const int k = tile * NT + threadIdx.x;
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
    double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0, q = 0.0;
    const int j0 = split * chunk;
    const int j1 = min(n, j0 + chunk);
    for (int jt = j0; jt < j1; jt += TJ) {
      const int cnt = min(TJ, j1 - jt);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += NT) {
        const int j = jt + t;
        sx[t] = A.x[0][j];
        sy[t] = A.x[1][j];
        sz[t] = A.x[2][j];
        su[t] = A.w[0][j];
        sv[t] = A.w[1][j];
        sw[t] = A.w[2][j];
        sm[t] = A.m[j];
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
        const double s = __dsqrt_rn(s2);
        const double f = __ddiv_rn(sm[t], __dmul_rn(s2, s));
        ax = __dadd_rn(ax, __dmul_rn(f, dx));
        ay = __dadd_rn(ay, __dmul_rn(f, dy));
        az = __dadd_rn(az, __dmul_rn(f, dz));
        ph = __dsub_rn(ph, __ddiv_rn(sm[t], s));
        const double wx = __dsub_rn(su[t], ui);
        const double wy = __dsub_rn(sv[t], vi);
        const double wz = __dsub_rn(sw[t], wi);
        const double c = __ddiv_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)),
                      __dmul_rn(wz, wz)),
            s2);
        if (c > q) q = c;
        if (f > q) q = f;
      }
    }
    if (valid) {
      double* p = A.part + (long long)split * 5 * n_act;
      p[0 * n_act + k] = ax;
      p[1 * n_act + k] = ay;
      p[2 * n_act + k] = az;
      p[3 * n_act + k] = ph;
      p[4 * n_act + k] = q;
    }
  }
}

// ---------------------------------------------------------------------
// Mixed: FP32 pair terms on double-single relative coordinates
// d = (x_hi,j - x_hi,i) + (x_lo,j - x_lo,i); FP32 sums per j tile folded
// into hi/lo compensated accumulators; q is an exact FP32 max.
// ---------------------------------------------------------------------
__device__ __forceinline__ void two_sum_fold(float& hi, float& lo, float t) {
  const float s = __fadd_rn(hi, t);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)),
                              __fsub_rn(t, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

struct MixI {
  float xh, yh, zh, xl, yl, zl, u, v, w;
};

__device__ __forceinline__ void pair_mixed(const MixI& I, const float4 h,
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
  q = fmaxf(q, fmaxf(w2 * rinv2, mr3));
}

template <int NT, int TJ>
__global__ void __launch_bounds__(NT) force_mixed_kernel(ForceArgs A) {
  if (A.done && *A.done) return;
  const int n_act = A.n_act_fixed >= 0 ? A.n_act_fixed : *A.n_act_ptr;
  if (n_act <= 0) return;
  const int n = A.n;
  const int n_tiles = (n_act + NT - 1) / NT;
  const int S = choose_split(n_tiles, gridDim.x, n, 0, n_act, A.part_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.nsplit_out)
    *A.nsplit_out = S;
  const int chunk = ((n + S - 1) / S + TJ - 1) / TJ * TJ;
  __shared__ float4 shh[TJ], shl[TJ], shv[TJ];
  const float eps2 = A.eps2f;
  const int items = n_tiles * S;
  for (int w = blockIdx.x; w < items; w += gridDim.x) {
    const int tile = w / S;
    const int split = w - tile * S;
    const int k = tile * NT + threadIdx.x;
    const bool valid = k < n_act;
    const int i = valid ? A.idx[k] : -1;
    MixI I = {};
    if (valid) {
      const float4 h = A.jhi[i], l = A.jlo[i], vv = A.jv[i];
      I.xh = h.x; I.yh = h.y; I.zh = h.z;
      I.xl = l.x; I.yl = l.y; I.zl = l.z;
      I.u = vv.x; I.v = vv.y; I.w = vv.z;
    }
    float axh = 0, axl = 0, ayh = 0, ayl = 0, azh = 0, azl = 0;
    float phh = 0, phl = 0, q = 0;
    const int j0 = split * chunk;
    const int j1 = min(n, j0 + chunk);
    for (int jt = j0; jt < j1; jt += TJ) {
      const int cnt = min(TJ, j1 - jt);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += NT) {
        shh[t] = A.jhi[jt + t];
        shl[t] = A.jlo[jt + t];
        shv[t] = A.jv[jt + t];
      }
      __syncthreads();
      float ax = 0, ay = 0, az = 0, ph = 0;
      const bool self_here = valid && i >= jt && i < jt + cnt;
      if (__any_sync(kFull, self_here)) {
        for (int t = 0; t < cnt; ++t) {
          if (jt + t == i) continue;
          pair_mixed(I, shh[t], shl[t], shv[t], eps2, ax, ay, az, ph, q);
        }
      } else if (cnt == TJ) {
#pragma unroll 8
        for (int t = 0; t < TJ; ++t)
          pair_mixed(I, shh[t], shl[t], shv[t], eps2, ax, ay, az, ph, q);
      } else {
        for (int t = 0; t < cnt; ++t)
          pair_mixed(I, shh[t], shl[t], shv[t], eps2, ax, ay, az, ph, q);
      }
      two_sum_fold(axh, axl, ax);
      two_sum_fold(ayh, ayl, ay);
      two_sum_fold(azh, azl, az);
      two_sum_fold(phh, phl, ph);
    }
    if (valid) {
      double* p = A.part + (long long)split * 5 * n_act;
      p[0 * n_act + k] = (double)axh + (double)axl;
      p[1 * n_act + k] = (double)ayh + (double)ayl;
      p[2 * n_act + k] = (double)azh + (double)azl;
      p[3 * n_act + k] = -((double)phh + (double)phl);
      p[4 * n_act + k] = (double)q;
    }
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
    double s[4] = {0, 0, 0, 0};
    double qq = 0.0;
    for (int sp = 0; sp < S; ++sp) {
      const double* p = part + (long long)sp * 5 * n_act;
      if (sp == 0) {
        for (int c = 0; c < 4; ++c) s[c] = p[c * n_act + k];
        qq = p[4 * n_act + k];
      } else {
        for (int c = 0; c < 4; ++c) s[c] = __dadd_rn(s[c], p[c * n_act + k]);
        qq = fmax(qq, p[4 * n_act + k]);
      }
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
  static std::mutex mu;
  static std::vector<ForceLaunch> cache[2];
  std::lock_guard<std::mutex> g(mu);
  auto& c = cache[precision ? 1 : 0];
  if ((int)c.size() > device && c[device].grid > 0) return c[device];
  if ((int)c.size() <= device) c.resize(device + 1, ForceLaunch{0, 0, 0, 0});
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (precision)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, force_mixed_kernel<kThreads, kTileMix>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, force_fp64_kernel<kThreads, kTileF64>, kThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  ForceLaunch fl;
  fl.grid = sms * per_sm;
  fl.threads = kThreads;
  fl.tile_i = kThreads;
  fl.part_cap = 5LL * fl.grid * kThreads;
  c[device] = fl;
  return fl;
}

cudaError_t launch_force(int precision, const ForceArgs& fa,
                         const ForceLaunch& fl, cudaStream_t s) {
  if (precision)
    force_mixed_kernel<kThreads, kTileMix><<<fl.grid, kThreads, 0, s>>>(fa);
  else
    force_fp64_kernel<kThreads, kTileF64><<<fl.grid, kThreads, 0, s>>>(fa);
  return cudaGetLastError();
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
