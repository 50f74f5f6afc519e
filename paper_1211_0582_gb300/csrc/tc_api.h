// Tensor-core (split-precision) form of the fused stage kernel: host interface.
#pragma once
#include "common.cuh"
#include "grid_sync.cuh"

namespace dgmx {
// Builds the hi/lo operator copies for ctx->precision; returns a dg_status.
int tc_prepare(dg_ctx *ctx);
// Releases what tc_prepare allocated.
void tc_free(dg_ctx *ctx);
// Launches the tensor-core stage kernel on ctx->stream, or on stream s.
// MODE_LSERK_STORE (the LSERK stage that also writes the E rows of the
// right-hand side to a.rhs, [3][K][Np_pad]) is supported at N <= 5.
cudaError_t launch_stage_tc(dg_ctx *ctx, int mode, const StageArgs &a);
cudaError_t launch_stage_tc(dg_ctx *ctx, int mode, const StageArgs &a, cudaStream_t s);
// Orders the persistent multi-step tensor-core kernel supports (N <= 5).
bool tc_ensemble_supported(const dg_ctx *ctx);
// Persistent multi-step form for ensembles: nsteps LSERK4 steps in one
// cooperative launch (grid barrier between stages, per-element time step from
// the geometry record); u_a holds the state at entry and the stages alternate
// u_a -> u_b -> u_a ...; a.res is the residual.
cudaError_t launch_tc_ensemble(dg_ctx *ctx, const StageArgs &a, const StageCoeffs &rk, float *u_a, float *u_b,
                               int nsteps, GridBarrier *gb, cudaStream_t s);
} // namespace dgmx
