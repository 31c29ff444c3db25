// Host-side context of the TSBTS library and the helpers shared by the
// host translation units (engine.cu: integrator and ensembles; adjoint.cu:
// frozen-schedule adjoint).
#pragma once
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tsbts.h"
#include "tsbts_kernels.cuh"

namespace tsbts {
struct AdjCtx;  // adjoint state (adjoint.cu)
}

using namespace tsbts;

struct CudaFail {
  cudaError_t e;
  const char* what;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaFail{e, what};
}

struct tsbts_ctx {
  tsbts_config cfg{};
  std::string err;
  bool poisoned = false;
  bool inited = false;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int sms = 1;
  // problem
  int n = 0;
  double eps = 0, eta = 0;
  int k_min = 0;
  long long dtmax_t = 0;
  long long t_sys = 0;
  int exact = 0;
  // device memory
  std::vector<void*> allocs;
  Bodies B{}, snap{};
  History H[2]{};
  std::vector<void*> hist_allocs[2];
  Params P{};
  Ctl* d_ctl = nullptr;
  double* rlast[3] = {nullptr, nullptr, nullptr};  // positions after the
                                                   // last pass (R15)
  Ctl* h_ctl = nullptr;  // pinned mirror
  double* d_w = nullptr;
  double* d_eout = nullptr;
  int* d_nsplit = nullptr;  // scratch for init's split count
  PlanTable pt{};            // force work plan per bucket of active counts
  ForceLaunch fl{};
  int correct_grid = 1;
  // counters
  long long eras = 0, passes = 0, restarts = 0;
  long long max_rec = 0;
  // timing
  int timing = 0;            // time every timing-th chunk of steps (0: off)
  long long chunk_no = 0;    // chunks of block steps launched since init
  long long force_inter = 0; // interactions of the timed steps
  std::vector<cudaEvent_t> ev;
  double force_ms = 0;
  long long force_launches = 0;
  long long launches = 0;  // kernels launched since init
  // schedule log
  long long lg_cap = 0;
  std::vector<void*> lg_allocs;
  // CUDA graph of graph_steps block steps
  cudaGraphExec_t gexec = nullptr;    // without timing events
  cudaGraphExec_t gexec_t = nullptr;  // with events around each force
  bool graph_dirty = true;
  // ensemble of independent clusters (tsbts_init_ensemble)
  bool ensemble = false;
  int nc = 0;
  Ens E{};
  ForceLaunch efl{};
  double* d_ek = nullptr;
  double* d_ep = nullptr;
  // adjoint of a frozen block schedule (tsbts_adjoint_init)
  tsbts::AdjCtx* adj = nullptr;
};

template <class T>
T* dalloc(std::vector<void*>& list, size_t count) {
  void* p = nullptr;
  ck(cudaMalloc(&p, sizeof(T) * (count ? count : 1)), "cudaMalloc");
  list.push_back(p);
  return static_cast<T*>(p);
}

inline void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

inline int fail(tsbts_ctx* c, int code, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (code == TSBTS_ERR_CUDA || code == TSBTS_ERR_NONFINITE ||
        code == TSBTS_ERR_TIMEOUT)
      c->poisoned = true;
  }
  return code;
}

inline int cuda_fail(tsbts_ctx* c, const CudaFail& f) {
  return fail(c, TSBTS_ERR_CUDA,
              std::string(f.what) + ": " + cudaGetErrorString(f.e));
}

// frees the adjoint state of a context (adjoint.cu)
void adjoint_release(tsbts_ctx* c);
