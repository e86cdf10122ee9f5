// Tensor-core (tcgen05) BF16 hi/lo form of the full-rank iteration: not built yet.
#include "ssm_internal.cuh"

namespace ssm {

ssm_status tc_prepare(ssm_plan_s* pl, cudaStream_t s) {
  (void)pl;
  (void)s;
  set_error("the BF16X3 tensor-core form is not available in this build");
  return SSM_EUNSUPPORTED;
}
ssm_status tc_iteration(ssm_plan_s*, int, bool, double*, int*, cudaStream_t) {
  set_error("the BF16X3 tensor-core form is not available in this build");
  return SSM_EUNSUPPORTED;
}
void tc_release(ssm_plan_s*) {}
int tc_max_partials(const ssm_plan_s*) { return 1; }

}  // namespace ssm
