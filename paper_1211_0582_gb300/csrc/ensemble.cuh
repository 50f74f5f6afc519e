// Persistent multi-step form of the FP32 fused stage, for ensembles of meshes.
//
// An ensemble of independent meshes is stored as one disjoint union (elements
// of mesh i contiguous, neighbours always inside the same mesh, each element
// carrying its mesh's time step in geo[k][G_DT]). One cooperative launch then
// advances every mesh by `nsteps` LSERK4 steps: each block loops over
// element tiles of EB elements (EB is picked by the autotuner), and a
// grid-wide barrier separates the five stages of every step, because a stage
// reads the neighbours' states written by the previous stage. Field loads go
// through L2 (the L1 of another SM may hold a stale copy from two stages ago).
#pragma once
#include "grid_sync.cuh"
#include "simt_stage.cuh"

namespace dgmx {

// u_a holds the state at entry; stages alternate u_a -> u_b -> u_a ...
template <int N, int EB>
__global__ void __launch_bounds__(SimtCfg<N, EB>::NT)
    k_ensemble_persistent(StageArgs a, StageCoeffs rk, float *u_a, float *u_b, int nsteps, GridBarrier *gb,
                          int *err_flag) {
  extern __shared__ float4 smem4[];
  const int64_t ntiles = (a.K + EB - 1) / EB;
  bool flip = false;
  for (int step = 0; step < nsteps; ++step)
    for (int st = 0; st < 5; ++st) {
      a.u = flip ? u_b : u_a;
      a.u_out = flip ? u_a : u_b;
      a.rk_a = rk.a[st];
      a.rk_b = rk.b[st];
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads(); // shared memory of the previous tile is no longer read
        simt_stage_tile<N, MODE_LSERK, EB, true>(a, t * EB, smem4);
      }
      if (!grid_barrier(gb, a.wait_limit > 0 ? a.wait_limit : (1ll << 31))) {
        if (threadIdx.x == 0) atomicExch(err_flag, 1);
        return;
      }
      flip = !flip;
    }
}

} // namespace dgmx

namespace dgmx {

// Elements-per-block candidates of the autotuner for order N (0 = unused slot).
template <int N>
struct EnsembleCandidates {
  static constexpr int NQ = Dims<N>::NQ;
  static constexpr int c(int i) {
    const int v = (i == 0 ? 240 : i == 1 ? 176 : i == 2 ? 128 : 80) / NQ;
    return v < 1 ? 1 : v;
  }
};

// occ = 0: as many blocks per SM as fit; occ = 1: half as many (rounded up),
// a second tuning axis (fewer blocks take part in each grid barrier, more
// tiles per block); the blocks per SM launched go to *used (may be null)
template <int N, int EB>
cudaError_t launch_ensemble_eb(const StageArgs &a, const StageCoeffs &rk, float *ua, float *ub, int nsteps,
                               GridBarrier *gb, int *flag, cudaStream_t s, int sms, int occ, int *used) {
  using Cfg = SimtCfg<N, EB>;
  auto kern = k_ensemble_persistent<N, EB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::SMEM));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (occ == 1) per_sm = (per_sm + 1) / 2;
  if (used) *used = per_sm;
  const int64_t ntiles = (a.K + EB - 1) / EB;
  const int64_t cap = int64_t(per_sm) * sms;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Cfg::NT);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, rk, ua, ub, nsteps, gb, flag);
}

// Candidate cand: elements per block C::c(cand % 4), occupancy level cand / 4.
template <int N>
cudaError_t launch_ensemble_order(int cand, const StageArgs &a, const StageCoeffs &rk, float *ua, float *ub,
                                  int nsteps, GridBarrier *gb, int *flag, cudaStream_t s, int sms, int *used) {
  using C = EnsembleCandidates<N>;
  const int occ = cand / 4;
  switch (cand % 4) {
  case 0: return launch_ensemble_eb<N, C::c(0)>(a, rk, ua, ub, nsteps, gb, flag, s, sms, occ, used);
  case 1: return launch_ensemble_eb<N, C::c(1)>(a, rk, ua, ub, nsteps, gb, flag, s, sms, occ, used);
  case 2: return launch_ensemble_eb<N, C::c(2)>(a, rk, ua, ub, nsteps, gb, flag, s, sms, occ, used);
  default: return launch_ensemble_eb<N, C::c(3)>(a, rk, ua, ub, nsteps, gb, flag, s, sms, occ, used);
  }
}

} // namespace dgmx
