// Tensor-core products (tcgen05 / TMEM / TMA) -- placeholder until the
// kernels land; the float plan rejects BF16 / BF16X3 products for now.
#include "internal.cuh"
#include "plan.h"

namespace mp {
cudaError_t tc_init(matpow_plan_s*) { return cudaSuccess; }
void tc_free(matpow_plan_s*) {}
matpow_status tc_fill_desc(matpow_plan_s* p, GemmDesc*, int*) {
  return fail(p, MATPOW_EUNSUPPORTED, "tensor-core products are not built yet");
}
matpow_status tc_launch_pair(matpow_plan_s* p, const GemmPair&, cudaStream_t) {
  return fail(p, MATPOW_EUNSUPPORTED, "tensor-core products are not built yet");
}
matpow_status tc_launch_group(matpow_plan_s* p, const GemmDesc*, int, int, Scale*, cudaStream_t) {
  return fail(p, MATPOW_EUNSUPPORTED, "tensor-core products are not built yet");
}
}  // namespace mp
