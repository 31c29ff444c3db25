// Pipe-throughput probe: the measured peaks that the rooflines of the
// force kernels are quoted against. The pairwise force of Eq. 3 is not a
// dense contraction, so its bound is the FP32 (mixed path) or FP64 (plain
// path) FMA pipe, not the tensor cores; this probe measures what those
// pipes sustain on the device at hand.
//
// Each kind runs independent dependency chains of one operation in every
// thread of a grid several blocks deep per SM, so the pipe, not latency,
// sets the rate:
//   0  FP32 fma.rn.f32 (one FMA-pipe op per lane per instruction)
//   1  FP32 fma.rn.f32x2 (two FMA-pipe ops per lane per instruction)
//   2  FP64 fma.rn.f64
//   3  rsqrt.approx.f32 (the special-function unit)
// The result is lane operations per second, timed with CUDA events around
// one launch after a warm-up launch.
#include <cuda_runtime.h>

#include "../../include/tsbts.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

typedef unsigned long long f2;

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float rsq(float x) {
  float y;
  asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a, b are runtime values close to 1 and 0 so that the chains neither
// overflow nor collapse to constants
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads)
    probe_kernel(long long iters, float a, float b, float* sink) {
  if constexpr (KIND == 0) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = b * (threadIdx.x + k);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains; ++k)
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[k]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;
  } else if constexpr (KIND == 1) {
    f2 x[kChains];
    f2 A, B;
    asm("mov.b64 %0, {%1,%1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1,%1};" : "=l"(B) : "f"(b));
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const float u = b * (threadIdx.x + k);
      asm("mov.b64 %0, {%1,%1};" : "=l"(x[k]) : "f"(u));
    }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma2(x[k], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float lo, hi;
      asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
      s += lo + hi;
    }
    if (s == 1234.5f) sink[0] = s;
  } else if constexpr (KIND == 2) {
    double x[kChains];
    const double A = a, B = b;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = B * (threadIdx.x + k);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains; ++k)
        asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[k]) : "d"(A), "d"(B));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5) sink[0] = (float)s;
  } else {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0f + b * (threadIdx.x + k);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = rsq(x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) sink[0] = s;
  }
}

template <int KIND>
cudaError_t run_probe(int grid, long long iters, float* sink, cudaStream_t s,
                      float* ms) {
  const float a = 0.999999f, b = 1e-7f;
  probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(iters / 8, a, b, sink);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  cudaEventRecord(e0, s);
  probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(iters, a, b, sink);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" int tsbts_pipe_peak(int kind, int64_t iters, double* ops_per_s,
                               double* ms_out) {
  if (kind < 0 || kind > 3 || iters < 1 || iters > (1LL << 30) || !ops_per_s)
    return TSBTS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return TSBTS_ERR_CUDA;
  }
  // eight 256-thread blocks per SM: 64 warps, enough independent chains to
  // keep every pipe busy
  const int grid = sms * 8;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return TSBTS_ERR_CUDA;
  }
  cudaStream_t s = nullptr;
  float ms = 0.f;
  cudaError_t e;
  switch (kind) {
    case 0: e = run_probe<0>(grid, iters, sink, s, &ms); break;
    case 1: e = run_probe<1>(grid, iters, sink, s, &ms); break;
    case 2: e = run_probe<2>(grid, iters, sink, s, &ms); break;
    default: e = run_probe<3>(grid, iters, sink, s, &ms); break;
  }
  cudaFree(sink);
  if (e != cudaSuccess || !(ms > 0.f)) {
    cudaGetLastError();
    return TSBTS_ERR_CUDA;
  }
  const double lanes_per_inst = kind == 1 ? 2.0 : 1.0;
  const double ops = (double)grid * kProbeThreads * (double)iters * kChains *
                     lanes_per_inst;
  *ops_per_s = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return TSBTS_OK;
}
