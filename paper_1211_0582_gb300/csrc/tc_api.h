// Tensor-core (split-precision) form of the fused stage kernel: host interface.
#pragma once
#include "common.cuh"

namespace dgmx {
// Builds the hi/lo operator copies for ctx->precision; returns a dg_status.
int tc_prepare(dg_ctx *ctx);
// Releases what tc_prepare allocated.
void tc_free(dg_ctx *ctx);
// Launches the tensor-core stage kernel on ctx->stream.
cudaError_t launch_stage_tc(dg_ctx *ctx, int mode, const StageArgs &a);
} // namespace dgmx
