// LSERK4 stepping that performs no device allocation.
//
// dg_step() ping-pongs the stage state through a scratch field vector that
// dg_mesh_upload() allocates. Some callers cannot have the library allocate
// device memory at all: applications whose device memory is owned up front by
// their own allocator (a framework's caching allocator or a fixed arena that
// reserves nearly all of the GPU), and callers that must not risk a
// cudaMalloc stall or failure in the middle of a time loop. For them,
// dg_step_noalloc() runs the same stage kernels with the ping-pong buffer taken
// from a fixed-size array that is part of the library's device image, so the
// call itself allocates nothing.
//
// The array holds kNoAllocFloats FP32 values (16 MiB); every GPU on which the
// library is loaded keeps it until the process exits. All calls share it and
// it keeps whatever the last call left in it; the stage kernel overwrites every
// entry it later reads, so nothing needs clearing. Calls whose work overlaps on
// the GPU (two streams, two contexts) race on the array.
#include <cmath>
#include <string>

#include "../../include/dgmx.h"
#include "common.cuh"
#include "tc_api.h"

namespace dgmx {
namespace {

constexpr size_t kNoAllocFloats = size_t(4) << 20; // 16 MiB of FP32

static __device__ __align__(256) float g_stage_scratch[kNoAllocFloats];

// Device address of the array in the current context. The array's name is a
// host-side stand-in and must never reach a kernel; its device address is
// looked up on every call (cheap next to the stage launches), so a device
// reset or another context on the same device never sees a stale address.
cudaError_t scratch_for_current_device(float **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_stage_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<float *>(p);
  return cudaSuccess;
}

int fail(dg_ctx *ctx, int code, const std::string &msg) {
  ctx->err = msg;
  return code;
}

} // namespace
} // namespace dgmx

using namespace dgmx;

extern "C" int dg_step_noalloc(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha) {
  if (!ctx) return DG_ERR_ARG;
  if (ctx->K <= 0) return fail(ctx, DG_ERR_ARG, "dg_step_noalloc: no mesh uploaded");
  if (!u || !res) return fail(ctx, DG_ERR_ARG, "dg_step_noalloc: null field pointer");
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(res)) & 15u)
    return fail(ctx, DG_ERR_ARG, "dg_step_noalloc: fields must be 16-byte aligned");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(alpha))
    return fail(ctx, DG_ERR_ARG, "dg_step_noalloc: bad dt/nsteps/alpha");
  const size_t floats = size_t(6) * size_t(ctx->K) * size_t(ctx->ops.Npad);
  if (floats > kNoAllocFloats)
    return fail(ctx, DG_ERR_ARG,
                "dg_step_noalloc: the field vector has " + std::to_string(floats) +
                    " floats, more than the fixed scratch of " + std::to_string(kNoAllocFloats) +
                    " floats (16 MiB); use dg_step for larger meshes");
  const size_t bytes = floats * sizeof(float);
  const uintptr_t pu = reinterpret_cast<uintptr_t>(u), pr = reinterpret_cast<uintptr_t>(res);
  if (pu < pr + bytes && pr < pu + bytes) return fail(ctx, DG_ERR_ARG, "dg_step_noalloc: u and res overlap");
  float *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_step_noalloc: ") + cudaGetErrorString(e));
  return lserk_drive(ctx, u, res, dt, nsteps, alpha, scratch, "dg_step_noalloc");
}
