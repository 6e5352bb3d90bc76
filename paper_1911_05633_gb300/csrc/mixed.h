// Mixed-precision (FP32 arithmetic, FP32 accumulation) contraction kernels of Eqs. P_MM and S_MM on
// the CUDA cores: the fallback of the queue kernels (contract.h) when their configuration does not fit.
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace gw {

struct MixedPlan {
  bool ready = false;
  float* d_Cf = nullptr;  // product-basis coefficients in FP32
  size_t smem_P = 0, smem_S = 0;
};

gw_status mixed_init(MixedPlan& m, const HostPlan& h, const std::vector<DevEntry>& ent);
void mixed_free(MixedPlan& m);
gw_status mixed_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                               const double2* G_R, double2* P_R, int* d_status, cudaStream_t st);
gw_status mixed_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                            const double2* G_R, const double2* Wt_R, double2* Sig_R, int* d_status, cudaStream_t st);

}  // namespace gw
