// FP32 CUDA-core form of the fused right-hand side / LSERK stage.
//
// One block owns EB consecutive elements and runs the paper's four subtasks
// (Section 2, Fig. dg-subtasks) on them without leaving the SM:
//   1. stage the block's fields u[6][EB][Npad] in shared memory (float4 loads,
//      coalesced because each field's element rows are contiguous);
//   2. local differentiation: thread (element e, node quad q) forms
//      u_r, u_s, u_t = D_{r,s,t} u for its four nodes and six fields, then the
//      chain rule (eq. dg-reference-matrices) and the curls;
//   3. flux gather (eq. num-flux): interior trace from shared memory,
//      exterior trace from the neighbour's row (L2), PEC mirror on walls,
//      upwind flux with the face's precomputed impedance weights (Fscale
//      included), into shared memory;
//   4. flux lifting: LIFT (Np x 4Nfp) times the face fluxes, added to the
//      curls and scaled by 1/eps, 1/mu;
// then either stores the right-hand side or applies the low-storage RK
// update res = a res + dt rhs, u_out = u + b res (operator assembly).
// The transposed operators D^T[j][i], LIFT^T[m][i] are read as float4 along i
// through the read-only cache; they are small and stay cache resident. The
// launch is persistent (blocks loop over element tiles) with the elements per
// block picked per order from measurements: 128 / (Np_pad / 4), 80 / (...) at
// N = 4.
#pragma once
#include <atomic>

#include "common.cuh"
#include "flux.cuh"

namespace dgmx {

// Elements per block of the single-mesh launch (measured best on GB300).
template <int N>
constexpr int simt_default_eb() {
  return (N == 4 ? 80 : 128) / Dims<N>::NQ > 0 ? (N == 4 ? 80 : 128) / Dims<N>::NQ : 1;
}

template <int N, int EB_ = simt_default_eb<N>()>
struct SimtCfg {
  using D = Dims<N>;
  static constexpr int EB = EB_;                         // elements per block
  static constexpr int NT = (EB * D::NQ + 31) / 32 * 32; // threads per block
  static constexpr size_t SMEM =
      (size_t(6) * EB * D::NPP + size_t(6) * EB * D::NFF) * 4 + ((100 * D::NFP + 15) / 16) * 16;
};

// Field loads: from L2, bypassing L1 (fields are streamed once and the
// neighbour traces hit L2 anyway; L1 stays with the operator matrices), or
// through the read-only path (measured slower). Persistent multi-stage kernels
// need the L2 path for coherence: other blocks wrote the data in an earlier stage.
template <bool COHERENT>
__device__ __forceinline__ float4 load_field4(const float *p) {
  if constexpr (COHERENT) return __ldcg(reinterpret_cast<const float4 *>(p));
  else return ldg4(p);
}
template <bool COHERENT>
__device__ __forceinline__ float load_field(const float *p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

// One block-tile of EB elements starting at k0 (all threads of the block call it).
template <int N, int MODE, int EB, bool COHERENT>
__device__ __forceinline__ void simt_stage_tile(const StageArgs &a, int64_t k0, float4 *smem4) {
  using D = Dims<N>;
  using Cfg = SimtCfg<N, EB>;
  constexpr int NP = D::NP, NFP = D::NFP, NPP = D::NPP, NQ = D::NQ, NFF = D::NFF;
  constexpr int NT = Cfg::NT;
  float *s_u = reinterpret_cast<float *>(smem4);             // [6][EB][NPP]
  float *s_fl = s_u + 6 * EB * NPP;                          // [6][EB][NFF]
  uint8_t *s_fm = reinterpret_cast<uint8_t *>(s_fl + 6 * EB * NFF); // [NFF]
  uint8_t *s_nb = s_fm + NFF;                                // [96][NFP]

  const int tid = threadIdx.x;
  const int64_t KN = a.K * NPP;

  for (int idx = tid; idx < 6 * EB * NQ; idx += NT) {
    int c = idx / (EB * NQ), rem = idx - c * (EB * NQ);
    int e = rem / NQ, q = rem - e * NQ;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k0 + e < a.K) v = load_field4<COHERENT>(a.u + c * KN + (k0 + e) * NPP + 4 * q);
    reinterpret_cast<float4 *>(s_u)[(c * EB + e) * NQ + q] = v;
  }
  for (int idx = tid; idx < NFF + kConnKinds * NFP; idx += NT)
    s_fm[idx] = idx < NFF ? a.fmask[idx] : a.nbrtab[idx - NFF];
  __syncthreads();

  const int e = tid / NQ, q = tid - (tid / NQ) * NQ;
  const bool owner = tid < EB * NQ;
  const int64_t k = k0 + (owner ? e : 0);
  const bool live = owner && k < a.K;
  float vol[6][4];

  // ---- local differentiation + chain rule + curl
  if (owner) {
    float acc[3][6][4];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[d][c][n] = 0.f;
    const float *su = s_u + e * NPP;
#pragma unroll 2
    for (int j = 0; j < NP; ++j) {
      float4 dr = ldg4(a.DT + (0 * NP + j) * NPP + 4 * q);
      float4 ds = ldg4(a.DT + (1 * NP + j) * NPP + 4 * q);
      float4 dt = ldg4(a.DT + (2 * NP + j) * NPP + 4 * q);
      const float dv[3][4] = {{dr.x, dr.y, dr.z, dr.w}, {ds.x, ds.y, ds.z, ds.w}, {dt.x, dt.y, dt.z, dt.w}};
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float uj = su[c * EB * NPP + j];
        // packed FP32 pairs: two output nodes per instruction
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int n = 0; n < 4; n += 2) {
            const float2 r = f2fma(make_float2(dv[d][n], dv[d][n + 1]), f2(uj), make_float2(acc[d][c][n], acc[d][c][n + 1]));
            acc[d][c][n] = r.x;
            acc[d][c][n + 1] = r.y;
          }
      }
    }
    const float *g = a.geo + (live ? k : 0) * G_STRIDE;
    float m[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) m[i] = __ldg(g + i);
    // m = {rx ry rz sx sy sz tx ty tz}: d/dx_l = m[l] d/dr + m[3+l] d/ds + m[6+l] d/dt
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      float dd[6][3];
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int l = 0; l < 3; ++l) dd[c][l] = m[l] * acc[0][c][n] + m[3 + l] * acc[1][c][n] + m[6 + l] * acc[2][c][n];
      vol[0][n] = dd[5][1] - dd[4][2];    // (curl H)_x
      vol[1][n] = dd[3][2] - dd[5][0];    // (curl H)_y
      vol[2][n] = dd[4][0] - dd[3][1];    // (curl H)_z
      vol[3][n] = -(dd[2][1] - dd[1][2]); // -(curl E)_x
      vol[4][n] = -(dd[0][2] - dd[2][0]); // -(curl E)_y
      vol[5][n] = -(dd[1][0] - dd[0][1]); // -(curl E)_z
    }
  }

  // ---- flux gather
  for (int it = tid; it < EB * NFF; it += NT) {
    int ee = it / NFF, fm = it - ee * NFF;
    int f = fm / NFP, mm = fm - f * NFP;
    int64_t kk = k0 + ee;
    float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (kk < a.K) {
      int vm = s_fm[fm];
      float qm[6], qp[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) qm[c] = s_u[(c * EB + ee) * NPP + vm];
      const int2 cn = __ldg(a.fconn + kk * 4 + f);
      const float4 nf = __ldg(a.fgeo + kk * 4 + f);
      const float4 wf = __ldg(a.fmat + kk * 4 + f); // face weights (neighbour or mirror impedances)
      if (cn.y == kBoundaryConn) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          qp[c] = -qm[c];
          qp[c + 3] = qm[c + 3];
        }
      } else {
        int vn = s_nb[cn.y * NFP + mm];
        const float *up = a.u + int64_t(cn.x) * NPP + vn;
#pragma unroll
        for (int c = 0; c < 6; ++c) qp[c] = load_field<COHERENT>(up + c * KN);
      }
      maxwell_flux_w(nf, qm, qp, wf, a.alpha, fl);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) s_fl[(c * EB + ee) * NFF + fm] = fl[c];
  }
  __syncthreads();

  if (!owner) return;
  // ---- flux lifting
  {
    const float *sf = s_fl + e * NFF;
#pragma unroll 4
    for (int fm = 0; fm < NFF; ++fm) {
      float4 L = ldg4(a.LT + fm * NPP + 4 * q);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float gv = sf[c * EB * NFF + fm];
        const float2 v01 = f2fma(make_float2(L.x, L.y), f2(gv), make_float2(vol[c][0], vol[c][1]));
        const float2 v23 = f2fma(make_float2(L.z, L.w), f2(gv), make_float2(vol[c][2], vol[c][3]));
        vol[c][0] = v01.x, vol[c][1] = v01.y, vol[c][2] = v23.x, vol[c][3] = v23.y;
      }
    }
  }
  if (!live) return;
  // ---- material scaling and output / operator assembly
  const float ie = __ldg(a.geo + k * G_STRIDE + G_IEPS), im = __ldg(a.geo + k * G_STRIDE + G_IMU);
  const float dtk = a.dt_geo ? __ldg(a.geo + k * G_STRIDE + G_DT) : a.dt;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const float w = c < 3 ? ie : im;
    float r4[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) r4[n] = (4 * q + n < NP) ? vol[c][n] * w : 0.f;
    const int64_t off = c * KN + k * NPP + 4 * q;
    if (MODE == MODE_RHS) {
      *reinterpret_cast<float4 *>(a.rhs + off) = make_float4(r4[0], r4[1], r4[2], r4[3]);
    } else {
      // the first LSERK4 stage has a = 0: the residual it overwrites is not read
      float4 rs = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.rk_a != 0.f)
        rs = COHERENT ? __ldcg(reinterpret_cast<const float4 *>(a.res + off))
                      : *reinterpret_cast<const float4 *>(a.res + off);
      float4 uo = reinterpret_cast<const float4 *>(s_u)[(c * EB + e) * NQ + q];
      float rv[4] = {rs.x, rs.y, rs.z, rs.w}, uv[4] = {uo.x, uo.y, uo.z, uo.w};
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        bool pad = 4 * q + n >= NP;
        rv[n] = pad ? 0.f : fmaf(a.rk_a, rv[n], dtk * r4[n]);
        uv[n] = pad ? 0.f : fmaf(a.rk_b, rv[n], uv[n]);
      }
      *reinterpret_cast<float4 *>(a.res + off) = make_float4(rv[0], rv[1], rv[2], rv[3]);
      *reinterpret_cast<float4 *>(a.u_out + off) = make_float4(uv[0], uv[1], uv[2], uv[3]);
      // the adjoint's eps gradient reads only the E components of the stage right-hand side
      if (MODE == MODE_LSERK_STORE && c < 3)
        *reinterpret_cast<float4 *>(a.rhs + off) = make_float4(r4[0], r4[1], r4[2], r4[3]);
    }
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(SimtCfg<N>::NT) k_stage_simt(StageArgs a) {
  extern __shared__ float4 smem4[];
  constexpr int EB = SimtCfg<N>::EB;
  const int64_t ntiles = (a.K + EB - 1) / EB;
  pdl_wait(); // stage after stage: fields of the previous stage from here on
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (t + int64_t(gridDim.x) >= ntiles) pdl_launch_next(); // this block's last tile
    __syncthreads(); // shared memory of the previous tile is no longer read
    simt_stage_tile<N, MODE, EB, true>(a, t * EB, smem4);
  }
}

template <int N>
cudaError_t launch_simt_order(int mode, const StageArgs &a, cudaStream_t s) {
  using Cfg = SimtCfg<N>;
  const void *kern = mode == MODE_RHS ? (const void *)k_stage_simt<N, MODE_RHS>
                     : mode == MODE_LSERK ? (const void *)k_stage_simt<N, MODE_LSERK>
                                          : (const void *)k_stage_simt<N, MODE_LSERK_STORE>;
  // the shared-memory opt-in is a per-device function attribute: set it on every launch
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::SMEM));
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // persistent grid: as many blocks as fit on the GPU at once (at most one per
  // tile); blocks per SM of each kernel cached per device
  constexpr int kDevCache = 64;
  static std::atomic<int> per_sm_cache[3][kDevCache];
  int per_sm = dev < kDevCache ? per_sm_cache[mode][dev].load(std::memory_order_relaxed) : 0;
  if (per_sm == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (dev < kDevCache) per_sm_cache[mode][dev].store(per_sm, std::memory_order_relaxed);
  }
  const int64_t ntiles = (a.K + Cfg::EB - 1) / Cfg::EB, cap = int64_t(per_sm) * sms;
  const unsigned blocks = unsigned(ntiles < cap ? ntiles : cap);
  if (mode == MODE_RHS) return launch_pdl(k_stage_simt<N, MODE_RHS>, dim3(blocks), dim3(Cfg::NT), Cfg::SMEM, s, a);
  if (mode == MODE_LSERK) return launch_pdl(k_stage_simt<N, MODE_LSERK>, dim3(blocks), dim3(Cfg::NT), Cfg::SMEM, s, a);
  return launch_pdl(k_stage_simt<N, MODE_LSERK_STORE>, dim3(blocks), dim3(Cfg::NT), Cfg::SMEM, s, a);
}

} // namespace dgmx
