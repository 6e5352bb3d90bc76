// Mixed-precision (FP32 arithmetic, FP32 accumulation) contraction path of Eqs. P_MM and S_MM.
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
  // tensor-core P path (eligible shapes only)
  bool tc_ready = false;
  uint16_t* d_Bsplit = nullptr;  // C^b in three BF16 planes per species
  int* d_Bsplit_off = nullptr;
  int* d_species = nullptr;
  size_t smem_tc = 0;
  // tensor-core Sigma path
  bool tc_s_ready = false;
  uint16_t* d_BsplitT = nullptr;  // (C^b)^T in three BF16 planes per species
  int* d_BsplitT_off = nullptr;
  size_t smem_tc_s = 0;
};

gw_status mixed_init(MixedPlan& m, const HostPlan& h, const std::vector<DevEntry>& ent);
void mixed_free(MixedPlan& m);
gw_status mixed_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                               const double2* G_R, double2* P_R, int* d_status, cudaStream_t st);
gw_status mixed_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double* d_C,
                            const double2* G_R, const double2* Wt_R, double2* Sig_R, int* d_status, cudaStream_t st);

bool tc_eligible(const HostPlan& h, size_t* smem_out);
gw_status tc_init(MixedPlan& m, const HostPlan& h);
void tc_free(MixedPlan& m);
gw_status tc_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double2* G_R, double2* P_R,
                            int* d_status, cudaStream_t st);
gw_status tc_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double2* G_R,
                         const double2* Wt_R, double2* Sig_R, int* d_status, cudaStream_t st);

}  // namespace gw
