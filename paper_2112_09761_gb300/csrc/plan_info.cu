// plan_info.cu — how many kernels a plan's evaluation enqueues.
#include <string>

#include "gpm_internal.cuh"

namespace gpm {
gpm_status api_fail(gpm_status st, const std::string& msg);
}  // namespace gpm

extern "C" gpm_status gpm_plan_launches(const gpm_plan_t* p, uint32_t* n) {
  if (!p || !n) return gpm::api_fail(GPM_E_INVALID_ARG, "gpm_plan_launches: NULL argument");
  uint32_t c = 1;  // one enumeration kernel, or the wedge kernel of a full 4-cycle count
  if (p->lgs) {
    // one launch per non-empty size class, plus the arc roots and their overflow pass
    c = 0;
    for (int i = 0; i < 4; i++) c += p->lgs_count[i] ? 1u : 0u;
    if (p->heavy_count) c += 2;
  }
  *n = c;
  return GPM_OK;
}
