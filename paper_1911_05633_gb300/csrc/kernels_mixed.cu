// Mixed-precision contraction path (tcgen05 tensor cores).  Not built yet:
// every entry point reports GW_ERR_UNSUPPORTED so that no caller silently gets FP64.
#include "mixed.h"

namespace gw {

gw_status mixed_init(MixedPlan& m, const HostPlan&, const std::vector<DevEntry>&) {
  m.ready = false;
  return GW_OK;
}

void mixed_free(MixedPlan& m) { m.ready = false; }

gw_status mixed_polarizability(MixedPlan&, const HostPlan&, const DevEntry*, const double*, const double2*, double2*,
                               cudaStream_t) {
  set_last_error("mixed-precision polarizability not available in this build");
  return GW_ERR_UNSUPPORTED;
}

gw_status mixed_self_energy(MixedPlan&, const HostPlan&, const DevEntry*, const double*, const double2*,
                            const double2*, double2*, cudaStream_t) {
  set_last_error("mixed-precision self-energy not available in this build");
  return GW_ERR_UNSUPPORTED;
}

}  // namespace gw
