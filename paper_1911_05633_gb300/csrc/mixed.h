// Mixed-precision (BF16 split, FP32 accumulate) contraction path of Eqs. P_MM and S_MM.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace gw {

struct MixedPlan {
  bool ready = false;
};

gw_status mixed_init(MixedPlan& m, const HostPlan& h, const std::vector<DevEntry>& ent);
void mixed_free(MixedPlan& m);
gw_status mixed_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                               const double2* G_R, double2* P_R, cudaStream_t st);
gw_status mixed_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                            const double2* G_R, const double2* Wt_R, double2* Sig_R, cudaStream_t st);

}  // namespace gw
