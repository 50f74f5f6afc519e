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
#include <mutex>
#include <string>

#include "../../include/dgmx.h"
#include "common.cuh"
#include "tc_api.h"

namespace dgmx {
namespace {

constexpr size_t kNoAllocFloats = size_t(4) << 20; // 16 MiB of FP32
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_stage_scratch[kNoAllocFloats];

std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the name is a host-side stand-in and must never reach a kernel).
cudaError_t scratch_for_current_device(float **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stage_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_ptr[dev];
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

  StageArgs a{};
  a.geo = ctx->d_geo;
  a.fgeo = ctx->d_fgeo;
  a.fconn = ctx->d_fconn;
  a.fmat = ctx->d_fmat;
  a.wait_limit = ctx->wait_limit;
  a.DT = ctx->d_DT;
  a.LT = ctx->d_LT;
  a.fmask = ctx->d_tab;
  a.nbrtab = ctx->d_tab + 4 * ctx->ops.Nfp;
  a.K = ctx->K;
  a.alpha = alpha;
  a.dt = float(dt);
  a.res = res;
  const float *cur = u;
  float *nxt = scratch;
  for (int step = 0; step < nsteps; ++step)
    for (int st = 0; st < 5; ++st) {
      a.u = cur;
      a.u_out = nxt;
      a.rk_a = float(kLserkA[st]);
      a.rk_b = float(kLserkB[st]);
      e = ctx->precision == DG_FP32 ? launch_stage_simt(ctx->N, MODE_LSERK, a, ctx->stream)
                                    : launch_stage_tc(ctx, MODE_LSERK, a);
      if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_step_noalloc: ") + cudaGetErrorString(e));
      float *prev = const_cast<float *>(cur);
      cur = nxt;
      nxt = prev;
    }
  if (cur != u) {
    e = cudaMemcpyAsync(u, cur, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_step_noalloc: ") + cudaGetErrorString(e));
  }
  return DG_OK;
}
