// Tensor-core form of the fused stage kernel (not built yet in this file).
#include "../../include/dgmx.h"
#include "tc_api.h"

namespace dgmx {
int tc_prepare(dg_ctx *ctx) {
  ctx->err = "tensor-core precisions are not available in this build";
  return DG_ERR_UNSUPPORTED;
}
void tc_free(dg_ctx *ctx) { ctx->tc = nullptr; }
cudaError_t launch_stage_tc(dg_ctx *, int, const StageArgs &) { return cudaErrorNotSupported; }
} // namespace dgmx
