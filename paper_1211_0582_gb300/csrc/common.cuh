// Internal definitions shared by the CUDA translation units of libdgmx.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>

#include "refops.h"

struct dg_ctx;

namespace dgmx {

// Per-element FP32 record (64 bytes): metric terms, material factors, Jacobian.
enum GeoSlot {
  G_RX = 0, G_RY, G_RZ, G_SX, G_SY, G_SZ, G_TX, G_TY, G_TZ,
  G_IEPS = 9, G_IMU = 10, G_Z = 11, G_Y = 12, G_J = 13, G_DT = 14, // G_DT: per-element step (ensembles)
  G_STRIDE = 16
};

// Stage kinds of the fused kernels.
// MODE_LSERK_STORE: LSERK update that also writes the E components of the rhs
enum StageMode { MODE_RHS = 0, MODE_LSERK = 1, MODE_LSERK_STORE = 2 };

// Arguments of one fused right-hand-side / LSERK-stage launch.
struct StageArgs {
  const float *u;      // [6][K][Npad] state the right-hand side is evaluated at
  float *rhs;          // MODE_RHS: output [6][K][Npad]
  float *res;          // MODE_LSERK: residual, updated in place
  float *u_out;        // MODE_LSERK: u + b * res (must not alias u)
  const float *geo;    // [K][16]
  const float4 *fgeo;  // [K][4] {nx, ny, nz, Fscale}
  const int2 *fconn;   // [K][4] {neighbour element, connection kind}
  const float4 *fmat;  // [K][4] {Fscale/(Z-+Z+), -Fscale/(Y-+Y+), Z+, Y+} flux weights per face
  long long wait_limit; // device waits give up after this many SM cycles (0 = default, ~1 s)
  const float *DT;     // [3][Np][Npad]  transposed Dr, Ds, Dt
  const float *LT;     // [4Nfp][Npad]   transposed LIFT
  const uint8_t *fmask;  // [4Nfp]  volume node of each face node
  const uint8_t *nbrtab; // [96][Nfp] neighbour volume node per connection kind
  int64_t K;
  float alpha;         // 1 upwind, 0 central
  float rk_a, rk_b, dt;
  int dt_geo;          // 1: take the time step of each element from geo[k][G_DT] instead of dt
};

// Launchers, one per kernel family (defined in the .cu files).
cudaError_t launch_stage_simt(int N, int mode, const StageArgs &a, cudaStream_t s);
template <int N>
cudaError_t launch_simt_order(int mode, const StageArgs &a, cudaStream_t s);

struct GeometryArgs {
  int64_t K;
  const double *VX, *VY, *VZ;
  const int32_t *EToV;
  const float *eps, *mu;
  float *geo;
  float4 *fgeo;
  int *bad;  // first element index with J <= 0 (atomicMin), K if none
};
cudaError_t launch_geometry(const GeometryArgs &a, cudaStream_t s);
cudaError_t launch_set_eps(int64_t K, const float *eps, float *geo, int *bad, cudaStream_t s);
cudaError_t launch_face_weights(int64_t K, const float *geo, const float4 *fgeo, const int2 *fconn, float4 *fmat,
                                cudaStream_t s);
void ensemble_free(dg_ctx *ctx);
// Releases the adjoint work buffers.
void adjoint_free(dg_ctx *ctx);
// Re-arms the ensemble grid barrier after a timed-out launch (blocks that gave
// up leave its arrival count behind).
cudaError_t ensemble_reset_barrier(dg_ctx *ctx);
// Drops the captured graph of the ensemble step (its arguments changed).
void ensemble_drop_graph(dg_ctx *ctx);
cudaError_t launch_energy(int N, int64_t K, int Npad, const float *u, const float *geo, const double *M,
                          double *out, cudaStream_t s);
// Sets *flag (device int) to 1 if any of the nfloats values at u (16-byte
// aligned, nfloats a multiple of 4) is a NaN or an infinity; never clears it.
cudaError_t launch_nonfinite_check(const float *u, int64_t nfloats, int *flag, cudaStream_t s);
// The LSERK4 driver shared by dg_step and dg_step_noalloc: nsteps steps of the
// fused stage kernel on ctx's stream with the stage ping-pong through
// `pingpong` (a device field vector distinct from u and res), the final state
// copied back into u, and, when ctx->check_nonfinite is set, the non-finite
// check of u and res (synchronising). `who` names the entry point in errors.
// Arguments are validated by the caller. Returns a dg_status.
int lserk_drive(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha, float *pingpong,
                const char *who);

// Five-stage fourth-order low-storage Runge-Kutta coefficients (Carpenter &
// Kennedy 1994, 2N storage).
extern const double kLserkA[5];
extern const double kLserkB[5];
extern const double kLserkC[5];

// Programmatic dependent launch for kernels launched back to back on one
// stream (the stages of a step). A kernel waits for the previous kernel to
// complete, with its writes visible, before it reads or writes any data that
// kernel touches (pdl_wait, after its own setup), and lets the next kernel be
// launched once each of its blocks has started its last piece of work
// (pdl_launch_next), so that the next kernel's setup (shared-memory tables,
// operators, tensor-memory allocation) runs on SMs that free up at the end
// without holding SMs idle for long while other streams have work. Kernels
// launched without the attribute are serialised as usual and both return at
// once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next_and_wait() {
  pdl_launch_next();
  pdl_wait();
}

// NVTX range over one C-ABI call (profilers can select the launches of a
// call by it, e.g. ncu --nvtx --nvtx-include "dg_step/"); header-only NVTX 3,
// inert unless a tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

} // namespace dgmx

// Library context (opaque to callers).
struct dg_ctx {
  int N = 0;
  int precision = 0;
  cudaStream_t stream = nullptr;
  dgmx::RefOps ops;
  std::string err;
  int64_t K = 0;
  int64_t Nv = 0;
  // device data owned by the context
  float *d_geo = nullptr;
  float4 *d_fgeo = nullptr;
  float4 *d_fmat = nullptr;
  int2 *d_fconn = nullptr;
  float *d_DT = nullptr;
  float *d_LT = nullptr;
  uint8_t *d_tab = nullptr;  // fmask (4Nfp), neighbour volume-node table (96 Nfp), neighbour face-node table (96 Nfp)
  float *d_Dn = nullptr;     // [3][Np][Npad] D_d[i][j] row-major (transposed-operator kernels)
  float *d_LF = nullptr;     // [Np][4Nfp] LIFT row-major (transposed-operator kernels)
  double *d_M = nullptr;
  float *d_scratch = nullptr;  // field vector for the LSERK stage ping-pong
  double *d_red = nullptr;     // reduction outputs
  int *d_flag = nullptr;
  long long wait_limit = 0;    // device-wait limit in SM cycles for the stage kernels (0 = default)
  int check_nonfinite = 0;     // dg_step: check u and res for NaN/Inf after the last stage
  void *tc = nullptr;          // tensor-core operator buffers (precision != DG_FP32)
  void *ens = nullptr;         // ensemble state (dg_ensemble_upload)
  void *adj = nullptr;         // adjoint / receiver-trace work buffers (grown on demand)
  void *adj_tc = nullptr;      // operators of the tensor-core reverse stage (built on first use)
  int adj_form = -1;           // reverse stage: 0 CUDA cores, 1 tensor cores, -1 tensor cores where supported
  int adj_segment = 0;         // steps per segment of the last dg_adjoint_step call
  std::vector<double> host_vert;   // VX, VY, VZ (kept for node coordinates)
  std::vector<int32_t> host_EToV;
};
