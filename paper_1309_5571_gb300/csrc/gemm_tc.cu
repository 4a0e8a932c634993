// Low-precision (tensor-core) projection: placeholder until the tcgen05 path lands.
#include "internal.h"

namespace dmrg {

dmrg_status launch_project_tc(dmrg_plan*, dmrg_precision, const double*, double*, cudaStream_t) {
  set_error("low-precision projection is not built yet");
  return DMRG_ERR_UNSUPPORTED;
}

void destroy_tc(dmrg_plan*) {}

bool tc_available(dmrg_precision) { return false; }

}  // namespace dmrg
