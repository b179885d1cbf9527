// tcgen05 controlled-U GEMM (complex64, split-TF32 on the 5th-generation tensor cores).
#include "hhl_common.cuh"

namespace hhl {

bool tc_supported(const Plan&) { return false; }
hhl_status tc_prepare_operands(Plan&, const double2*, int, cudaStream_t) {
  return fail(HHL_ERR_UNSUPPORTED, "tcgen05 GEMM not built");
}
hhl_status launch_ctrl_u_tc(const Plan&, void*, int, bool, cudaStream_t) {
  return fail(HHL_ERR_UNSUPPORTED, "tcgen05 GEMM not built");
}
void tc_free(Plan&) {}

}  // namespace hhl
