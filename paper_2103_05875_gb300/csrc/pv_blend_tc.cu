// K1 (tensor-core form) -- placeholder until the tcgen05 kernel lands.
#include "pv_internal.h"

bool pv_tc_supported(const pv_desc*, const char** why) {
  if (why) *why = "not built yet";
  return false;
}
cudaError_t pv_tc_plan_create(pv_volume*) { return cudaErrorNotSupported; }
void pv_tc_plan_destroy(pv_volume*) {}
cudaError_t pv_launch_blend_tc(pv_volume*, const void*, const void*, cudaStream_t) {
  return cudaErrorNotSupported;
}
