// Launchers of the block-step kernels (k_step.cu) used by the host engine.
#pragma once

#include <climits>

#include "tsbts_internal.cuh"

namespace tsbts {

void launch_pass_begin(Ctl* ctl, long long tau_s, long long tau_e, int pass,
                       int era, int n, cudaStream_t s);
void launch_pass_setup(const Bodies& B, const Params& P, const History& cur,
                       cudaStream_t s);
void launch_select_predict(const Bodies& B, const Params& P, const History& HA,
                           const History& HB, int p, cudaStream_t s);
void launch_correct(const Bodies& B, const Params& P, const History& HA,
                    const History& HB, int p, int grid, cudaStream_t s);
void launch_copy_state(const Bodies& dst, const Bodies& src, cudaStream_t s);
// the running pass's appended records -> previous-pass records in CSR order
void launch_history_to_csr(const Bodies& B, const History& append,
                           const History& csr, const Ctl* ctl, int sms,
                           cudaStream_t s);
void launch_next_time_extrema(const Bodies& B, Ctl* ctl, cudaStream_t s);
void launch_load_aos(const Bodies& B, const double* m, const double* r,
                     const double* v, Ctl* ctl, cudaStream_t s);
void launch_init_jdata(const Bodies& B, const Params& P, cudaStream_t s);
void launch_init_finalize(const Bodies& B, const Params& P, const int* nsplit,
                          cudaStream_t s);
void launch_energy(const Bodies& B, const Params& P, long long T, double* w,
                   double* out, int sms, cudaStream_t s);
// Eq. 2 prediction of every body to tick T into the FP64 j arrays
void launch_energy_predict(const Bodies& B, const Params& P, long long T,
                           cudaStream_t s);

// ensembles of independent clusters (k_ensemble.cu)
int ens_max_clusters();
ForceLaunch ens_force_launch_shape(int precision, int device);
void launch_ens_pass_begin(const Ens& E, long long tau_s, cudaStream_t s);
void launch_ens_pass_setup(const Bodies& B, const Params& P, const Ens& E,
                           const History& cur, cudaStream_t s);
// one global block step (five launches); ev0/ev1 (nullable) bracket the
// force launch
void launch_ens_step(const Bodies& B, const Params& P, const Ens& E,
                     const History& HA, const History& HB,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaEvent_t ev0, cudaEvent_t ev1, unsigned evflags,
                     cudaStream_t s);
void launch_ens_init(const Bodies& B, const Params& P, const Ens& E,
                     const ForceLaunch& fl, int precision, int exact,
                     cudaStream_t s);
void launch_ens_energy(const Bodies& B, const Params& P, const Ens& E,
                       long long T, double* w, double* ek, double* ep,
                       cudaStream_t s);

}  // namespace tsbts
