// Tensor-core form of the fused right-hand side / LSERK stage (sm_103a).
//
// The two dense contractions of the DG operator run on the fifth-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), in split
// precision: every operand x is stored as a 16-bit pair hi = rn(x),
// lo = rn(x - hi), and each product is formed as hi*hi + hi*lo + lo*hi with
// FP32 accumulation (BF16, or FP16 with a power-of-two scale per row).
//
// Section 2, Fig. (el-local-ops): the field data of many elements is treated
// as one matrix so that local differentiation and lifting become
// matrix-matrix products. Here the rows are (element, field) pairs of a tile
// of 20 elements (5 per 32-lane TMEM quarter, 30 of 32 lanes used):
//   GEMM1  V[(e,f), (d,i)] = sum_j u[(e,f), j] D_d[i, j]        (d = r, s, t)
//   GEMM2  S[(e,f), i]     = sum_m flux[(e,f), m] LIFT[i, m]
// The operators (B operands) stay resident in shared memory for the whole
// persistent kernel ("store the matrices, stream the vector data", Section 3).
// The epilogue reads V and S from TMEM with one thread per row, applies the
// chain rule (eq. dg-reference-matrices), exchanges the two needed physical
// derivatives between the six field lanes of an element with warp shuffles to
// form curl H and -curl E, adds the lifted flux, scales by 1/eps, 1/mu and
// either stores the right-hand side or applies the LSERK update.
//
// Supported orders: N = 1..5 (the operators of N >= 6 do not fit in shared
// memory next to the tiles; those orders use the CUDA-core kernel).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include "../../include/dgmx.h"
#include "flux.cuh"
#include "tc_api.h"
#include "umma.cuh"

namespace dgmx {

namespace {

constexpr int kThreads = 512;
constexpr int kTileElems = 20; // 4 TMEM lane quarters x 5 elements
constexpr int kRows = 120;     // (element, field) rows actually used per tile
constexpr int kMaxTcOrder = 5;

__host__ __device__ constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int tmem_cols(int x) {
  return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512;
}

template <int N>
struct TC {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NFP = D::NFP, NPP = D::NPP, NFF = D::NFF, NQ = D::NQ;
  static constexpr int K1 = rup(NP, 16);  // GEMM1 reduction length (input nodes)
  static constexpr int NB = rup(NP, 16);  // output columns per derivative direction
  static constexpr int N1 = 3 * NB;       // GEMM1 output columns
  static constexpr int K2 = rup(NFF, 16); // GEMM2 reduction length (face nodes)
  static constexpr int N2 = NB;           // GEMM2 output columns
  static constexpr int TCOLS = tmem_cols(N1 + N2);
  static constexpr int A1B = 128 * K1 * 2, A2B = 128 * K2 * 2, B1B = N1 * K1 * 2, B2B = N2 * K2 * 2;
  static constexpr int OFF_A1H = 0, OFF_A1L = OFF_A1H + A1B;
  static constexpr int OFF_A2H = OFF_A1L + A1B, OFF_A2L = OFF_A2H + A2B;
  static constexpr int OFF_B1H = OFF_A2L + A2B, OFF_B1L = OFF_B1H + B1B;
  static constexpr int OFF_B2H = OFF_B1L + B1B, OFF_B2L = OFF_B2H + B2B;
  static constexpr int OPS_BYTES = 2 * B1B + 2 * B2B; // contiguous from OFF_B1H
  static constexpr int OFF_U = OFF_B2L + B2B;          // fp32 [kRows][NPP]
  static constexpr int OFF_FL = OFF_U + kRows * NPP * 4; // fp32 [kRows][NFF]
  static constexpr int OFF_TAB = OFF_FL + kRows * NFF * 4;
  static constexpr int OFF_SC = OFF_TAB + rup(NFF + kConnKinds * NFP, 16); // float [4][128]
  static constexpr int OFF_BAR = OFF_SC + 4 * 128 * 4;
  static constexpr int SMEM = OFF_BAR + 16;
};

struct TcState {
  void *d_ops = nullptr;
  int sms = 0;
};

template <bool BF16>
__device__ __forceinline__ void split4(float4 v, uint2 &hi, uint2 &lo) {
  if constexpr (BF16) {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y), l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
    hi = make_uint2(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1));
    lo = make_uint2(*reinterpret_cast<uint32_t *>(&l0), *reinterpret_cast<uint32_t *>(&l1));
  } else {
    __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
    float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    __half2 l0 = __floats2half2_rn(v.x - f0.x, v.y - f0.y), l1 = __floats2half2_rn(v.z - f1.x, v.w - f1.y);
    hi = make_uint2(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1));
    lo = make_uint2(*reinterpret_cast<uint32_t *>(&l0), *reinterpret_cast<uint32_t *>(&l1));
  }
}

// Warm L2 with [p, p + bytes) (bytes a multiple of 16, p 16-byte aligned).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  if (bytes == 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Operand row (32 * quarter + lane) -> compact row (6 e + f), or -1 for the
// two unused lanes of each quarter.
__device__ __forceinline__ int compact_row(int r) {
  const int l = r & 31;
  return l < 30 ? (r >> 5) * 30 + l : -1;
}

// Split the FP32 staging rows [120][ld] (first `cols` columns) into the hi/lo
// K-major operands, scaled per row. Work items are ordered so that each
// half-warp writes one 128-byte core matrix (8 rows x 16 bytes): conflict-free
// shared stores. Padding positions are never written (they stay zero).
template <bool BF16>
__device__ __forceinline__ void convert_rows(const float *src, int ld, int cols, int Kp, const float *scale,
                                             uint8_t *dst_hi, uint8_t *dst_lo, int tid) {
  const int kgroups = Kp / 8;
  const int units = 128 * kgroups * 2;
  for (int u = tid; u < units; u += kThreads) {
    const int rr = u & 7, qh = (u >> 3) & 1;
    const int rest = u >> 4;
    const int kg = rest % kgroups, g = rest / kgroups;
    const int r = 8 * g + rr, k = 8 * kg + 4 * qh;
    const int cr = compact_row(r);
    if (cr < 0 || k >= cols) continue;
    float4 v = *reinterpret_cast<const float4 *>(src + cr * ld + k);
    if constexpr (!BF16) {
      const float sc = scale[cr];
      v.x *= sc, v.y *= sc, v.z *= sc, v.w *= sc;
    }
    uint2 hi, lo;
    split4<BF16>(v, hi, lo);
    const uint32_t off = umma::kmajor_offset(uint32_t(r), uint32_t(k), uint32_t(Kp));
    *reinterpret_cast<uint2 *>(dst_hi + off) = hi;
    *reinterpret_cast<uint2 *>(dst_lo + off) = lo;
  }
}

// Power-of-two scale bringing a row maximum mx (>= 0) into [0.5, 1) and its
// inverse, from the exponent field of mx (FP16 range guard). Zero, subnormal
// or non-finite maxima give scale 1.
__device__ __forceinline__ void row_scale(float mx, float &scale, float &inv) {
  const uint32_t ex = (__float_as_uint(mx) >> 23) & 0xFFu;
  if (ex == 0u || ex >= 253u) {
    scale = 1.f;
    inv = 1.f;
    return;
  }
  scale = __uint_as_float((253u - ex) << 23);
  inv = __uint_as_float((ex + 1u) << 23);
}

// Maximum of |row| over `len` FP32 values, 4 threads per row (row = tid / 4
// for tid < 4 * kRows), combined with shuffles inside the 4-lane group.
__device__ __forceinline__ float row_absmax4(const float *rows, int ld, int len, int tid) {
  const int r = tid >> 2, part = tid & 3;
  float mx = 0.f;
  if (r < kRows)
    for (int j = part; j < len; j += 4) mx = fmaxf(mx, fabsf(rows[r * ld + j]));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  return mx;
}

// Three split products per K step: hi*hi, hi*lo, lo*hi, FP32 accumulation.
template <bool BF16>
__device__ __forceinline__ void issue_split_gemm(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                                 uint32_t b_lo, int Kp, int Nrows) {
  const uint32_t sbo = uint32_t(Kp) * 16u;
  for (int n0 = 0; n0 < Nrows; n0 += 256) {
    const int nl = Nrows - n0 < 256 ? Nrows - n0 : 256;
    const uint32_t idesc = umma::make_idesc(BF16, 128, uint32_t(nl));
    const uint32_t boff = uint32_t(n0 / 8) * sbo;
    for (int kk = 0; kk < Kp / 16; ++kk) {
      const uint32_t ko = uint32_t(kk) * 256u;
      const uint64_t ah = umma::make_desc(a_hi + ko, 128, sbo), al = umma::make_desc(a_lo + ko, 128, sbo);
      const uint64_t bh = umma::make_desc(b_hi + boff + ko, 128, sbo), bl = umma::make_desc(b_lo + boff + ko, 128, sbo);
      umma::mma_f16(d_tmem + uint32_t(n0), ah, bh, idesc, kk > 0 ? 1u : 0u);
      umma::mma_f16(d_tmem + uint32_t(n0), ah, bl, idesc, 1u);
      umma::mma_f16(d_tmem + uint32_t(n0), al, bh, idesc, 1u);
    }
  }
}

template <int N, int MODE, bool BF16>
__global__ void __launch_bounds__(kThreads, 1)
    k_stage_tc(StageArgs a, const uint4 *__restrict__ ops, int ntiles, int *err_flag) {
  using T = TC<N>;
  constexpr int NP = T::NP, NFP = T::NFP, NPP = T::NPP, NFF = T::NFF, NQ = T::NQ;
  extern __shared__ __align__(1024) uint8_t smem[];
  float *s_u = reinterpret_cast<float *>(smem + T::OFF_U);
  float *s_fl = reinterpret_cast<float *>(smem + T::OFF_FL);
  uint8_t *s_fm = smem + T::OFF_TAB;
  uint8_t *s_nb = s_fm + NFF;
  float *s_sc1 = reinterpret_cast<float *>(smem + T::OFF_SC); // [128] scale, inverse at +128
  float *s_sc2 = s_sc1 + 256;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + T::OFF_BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + T::OFF_BAR + 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t KN = a.K * NPP;
  const uint32_t sbase = umma::smem_u32(smem);

  // warm L2 with everything a tile streams from HBM (fields, residual, geometry)
  auto prefetch_tile = [&](int t) {
    if (t >= ntiles) return;
    const int64_t kb = int64_t(t) * kTileElems;
    const int64_t ne = a.K - kb < kTileElems ? a.K - kb : kTileElems;
    const uint32_t rowbytes = uint32_t(ne * NPP * 4);
    for (int f = 0; f < 6; ++f) {
      prefetch_l2(a.u + f * KN + kb * NPP, rowbytes);
      if (MODE == MODE_LSERK) prefetch_l2(a.res + f * KN + kb * NPP, rowbytes);
    }
    prefetch_l2(a.fconn + kb * 4, uint32_t(ne * 4 * sizeof(int2)));
    prefetch_l2(a.fgeo + kb * 4, uint32_t(ne * 4 * sizeof(float4)));
    prefetch_l2(a.geo + kb * G_STRIDE, uint32_t(ne * G_STRIDE * 4));
  };

  // ---- one-time setup: zero the A operands (padding rows/columns stay zero),
  // load the resident operators and the face tables, allocate TMEM.
  for (int i = tid; i < (2 * T::A1B + 2 * T::A2B) / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < T::OPS_BYTES / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem + T::OFF_B1H)[i] = __ldg(ops + i);
  for (int i = tid; i < NFF + kConnKinds * NFP; i += kThreads)
    s_fm[i] = i < NFF ? a.fmask[i] : a.nbrtab[i - NFF];
  for (int i = tid; i < 512; i += kThreads) s_sc1[i] = 1.f;
  if (tid == 0) {
    umma::mbar_init(bar, 1);
    umma::fence_mbar_init();
    prefetch_tile(blockIdx.x);
  }
  if (warp == 0) umma::tmem_alloc(tslot, T::TCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;

  // epilogue roles: TMEM lane quarter (warp % 4) and node-chunk part (warp / 4)
  const int quarter = warp & 3, part = warp >> 2;
  const bool lane_used = lane < 30;
  const int ep = lane_used ? lane / 6 : 4;
  const int fld = lane_used ? lane % 6 : 5;
  const int comp = fld % 3;
  const bool isE = fld < 3;
  const int src1 = ep * 6 + (isE ? 3 : 0) + (comp + 2) % 3;
  const int src2 = ep * 6 + (isE ? 3 : 0) + (comp + 1) % 3;
  const int dl1 = (comp + 2) % 3, dl2 = (comp + 1) % 3;
  const int e_loc = quarter * 5 + ep;
  const int ridx = e_loc * 6 + fld;
  const uint32_t lane_taddr = tmem + (uint32_t(quarter * 32) << 16);
  constexpr int NCH = (NP + 7) / 8; // 8-node chunks per row
  constexpr int CPP = (NCH + 3) / 4; // chunks per part
  const int ch0 = part * CPP;
  const int ch1 = (part + 1) * CPP < NCH ? (part + 1) * CPP : NCH;

  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t k0 = int64_t(tile) * kTileElems;
    if (tid == 0) prefetch_tile(tile + gridDim.x);

    // ---- 1. stage the tile's fields in shared memory (FP32, pads zeroed);
    // all loads of a thread are issued before any store
    {
      constexpr int TOT = 6 * kTileElems * NQ;
      constexpr int IT = (TOT + kThreads - 1) / kThreads;
      float4 v[IT];
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int idx = tid + s * kThreads;
        v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < TOT) {
          const int f = idx / (kTileElems * NQ), rem = idx - f * (kTileElems * NQ);
          const int e = rem / NQ, q = rem - e * NQ;
          if (k0 + e < a.K) v[s] = ldg4(a.u + f * KN + (k0 + e) * NPP + 4 * q);
        }
      }
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int idx = tid + s * kThreads;
        if (idx < TOT) {
          const int f = idx / (kTileElems * NQ), rem = idx - f * (kTileElems * NQ);
          const int e = rem / NQ, q = rem - e * NQ;
          float4 w = v[s];
          if (4 * q + 3 >= NP) {
            if (4 * q + 0 >= NP) w.x = 0.f;
            if (4 * q + 1 >= NP) w.y = 0.f;
            if (4 * q + 2 >= NP) w.z = 0.f;
            if (4 * q + 3 >= NP) w.w = 0.f;
          }
          reinterpret_cast<float4 *>(s_u)[(e * 6 + f) * NQ + q] = w;
        }
      }
    }
    __syncthreads();

    // ---- 2. split into the A1 operand (hi/lo), row-scaled for FP16
    if constexpr (!BF16) {
      const float mx = row_absmax4(s_u, NPP, NP, tid);
      if ((tid & 3) == 0 && (tid >> 2) < kRows) row_scale(mx, s_sc1[tid >> 2], s_sc1[128 + (tid >> 2)]);
      __syncthreads();
    }
    convert_rows<BF16>(s_u, NPP, NPP, T::K1, s_sc1, smem + T::OFF_A1H, smem + T::OFF_A1L, tid);
    umma::fence_proxy_async();
    __syncthreads();

    // ---- 3. local differentiation on the tensor cores (asynchronous)
    if (tid == 0) {
      umma::fence_after_sync();
      issue_split_gemm<BF16>(tmem, sbase + T::OFF_A1H, sbase + T::OFF_A1L, sbase + T::OFF_B1H, sbase + T::OFF_B1L,
                             T::K1, T::N1);
    }

    // ---- 4. flux gather (overlaps GEMM1): interior trace from shared memory,
    // exterior trace from the neighbour's row, PEC mirror on walls. Loads of
    // all items of a thread are issued before the arithmetic.
    {
      constexpr int TOT = kTileElems * NFF;
      constexpr int IT = (TOT + kThreads - 1) / kThreads;
      int2 cn[IT];
      float4 nf[IT];
      float zm[IT], ym[IT];
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int it = tid + s * kThreads;
        const int e = it / NFF, fm = it - e * NFF, f = fm / NFP;
        const int64_t k = k0 + e;
        cn[s] = make_int2(0, kBoundaryConn);
        nf[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        zm[s] = 1.f, ym[s] = 1.f;
        if (it < TOT && k < a.K) {
          cn[s] = __ldg(a.fconn + k * 4 + f);
          nf[s] = __ldg(a.fgeo + k * 4 + f);
          zm[s] = __ldg(a.geo + k * G_STRIDE + G_Z);
          ym[s] = __ldg(a.geo + k * G_STRIDE + G_Y);
        }
      }
      float qp[IT][6], zp[IT], yp[IT];
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int it = tid + s * kThreads;
        const int e = it / NFF, fm = it - e * NFF, f = fm / NFP, mm = fm - f * NFP;
        zp[s] = zm[s], yp[s] = ym[s];
        if (it < TOT && k0 + e < a.K && cn[s].y != kBoundaryConn) {
          const int vn = s_nb[cn[s].y * NFP + mm];
          const float *up = a.u + int64_t(cn[s].x) * NPP + vn;
#pragma unroll
          for (int c = 0; c < 6; ++c) qp[s][c] = __ldg(up + c * KN);
          zp[s] = __ldg(a.geo + int64_t(cn[s].x) * G_STRIDE + G_Z);
          yp[s] = __ldg(a.geo + int64_t(cn[s].x) * G_STRIDE + G_Y);
        } else {
#pragma unroll
          for (int c = 0; c < 6; ++c) qp[s][c] = 0.f;
        }
      }
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int it = tid + s * kThreads;
        if (it >= TOT) continue;
        const int e = it / NFF, fm = it - e * NFF;
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (k0 + e < a.K) {
          const int vm = s_fm[fm];
          float qm[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) qm[c] = s_u[(e * 6 + c) * NPP + vm];
          if (cn[s].y == kBoundaryConn) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              qp[s][c] = -qm[c];
              qp[s][c + 3] = qm[c + 3];
            }
          }
          maxwell_flux(nf[s], qm, qp[s], zm[s], zp[s], ym[s], yp[s], a.alpha, fl);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) s_fl[(e * 6 + c) * NFF + fm] = fl[c];
      }
    }
    __syncthreads();

    // ---- 5. split the face fluxes into the A2 operand
    if constexpr (!BF16) {
      const float mx = row_absmax4(s_fl, NFF, NFF, tid);
      if ((tid & 3) == 0 && (tid >> 2) < kRows) row_scale(mx, s_sc2[tid >> 2], s_sc2[128 + (tid >> 2)]);
      __syncthreads();
    }
    convert_rows<BF16>(s_fl, NFF, NFF, T::K2, s_sc2, smem + T::OFF_A2H, smem + T::OFF_A2L, tid);
    umma::fence_proxy_async();
    __syncthreads();

    // ---- 6. flux lifting on the tensor cores, then wait for both products
    if (tid == 0) {
      umma::fence_after_sync();
      issue_split_gemm<BF16>(tmem + uint32_t(T::N1), sbase + T::OFF_A2H, sbase + T::OFF_A2L, sbase + T::OFF_B2H,
                             sbase + T::OFF_B2L, T::K2, T::N2);
      umma::commit(bar);
    }
    // residual of this thread's chunks, loaded while the products run
    const int64_t k = k0 + e_loc;
    const bool live = lane_used && k < a.K;
    float4 rres[2 * CPP];
#pragma unroll
    for (int c = 0; c < CPP; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        rres[2 * c + h] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int i = (ch0 + c) * 8 + 4 * h;
        if (MODE == MODE_LSERK && live && ch0 + c < ch1 && i < NPP)
          rres[2 * c + h] = *reinterpret_cast<const float4 *>(a.res + fld * KN + k * NPP + i);
      }
    float g1r = 0.f, g1s = 0.f, g1t = 0.f, g2r = 0.f, g2s = 0.f, g2t = 0.f, w = 0.f;
    if (live) {
      const float *g = a.geo + k * G_STRIDE;
      // d/dx_l = (dr/dx_l) d/dr + (ds/dx_l) d/ds + (dt/dx_l) d/dt
      g1r = __ldg(g + G_RX + dl1), g1s = __ldg(g + G_SX + dl1), g1t = __ldg(g + G_TX + dl1);
      g2r = __ldg(g + G_RX + dl2), g2s = __ldg(g + G_SX + dl2), g2t = __ldg(g + G_TX + dl2);
      w = __ldg(g + (isE ? G_IEPS : G_IMU));
    }
    const float inv1 = BF16 ? 1.f : s_sc1[128 + (lane_used ? ridx : 0)];
    const float inv2 = BF16 ? 1.f : s_sc2[128 + (lane_used ? ridx : 0)];
    const bool ok = umma::mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err_flag, 1);
      break;
    }
    umma::fence_after_sync();

    // ---- 7. epilogue: chain rule, curls, lifting, material scale, update
#pragma unroll
    for (int c = 0; c < CPP; ++c) {
      const int ch = ch0 + c;
      if (ch >= ch1) break;
      const int i0 = ch * 8;
      float ur[8], us[8], ut[8], lf[8];
      umma::tmem_ld8(lane_taddr + uint32_t(i0), ur);
      umma::tmem_ld8(lane_taddr + uint32_t(T::NB + i0), us);
      umma::tmem_ld8(lane_taddr + uint32_t(2 * T::NB + i0), ut);
      umma::tmem_ld8(lane_taddr + uint32_t(T::N1 + i0), lf);
      umma::tmem_wait_ld();
      float rv[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const float dr = ur[n] * inv1, ds = us[n] * inv1, dt = ut[n] * inv1;
        const float p1 = g1r * dr + g1s * ds + g1t * dt;
        const float p2 = g2r * dr + g2s * ds + g2t * dt;
        const float v1 = __shfl_sync(0xffffffffu, p1, src1);
        const float v2 = __shfl_sync(0xffffffffu, p2, src2);
        const float vol = isE ? (v1 - v2) : (v2 - v1);
        rv[n] = (vol + lf[n] * inv2) * w;
      }
      if (live) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = i0 + 4 * h;
          if (i < NPP) {
            float r4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) r4[q] = (i + q < NP) ? rv[4 * h + q] : 0.f;
            const int64_t off = fld * KN + k * NPP + i;
            if (MODE == MODE_RHS) {
              *reinterpret_cast<float4 *>(a.rhs + off) = make_float4(r4[0], r4[1], r4[2], r4[3]);
            } else {
              const float4 rs = rres[2 * c + h];
              const float4 uo = *reinterpret_cast<const float4 *>(s_u + ridx * NPP + i);
              const float rsv[4] = {rs.x, rs.y, rs.z, rs.w}, uov[4] = {uo.x, uo.y, uo.z, uo.w};
              float nr[4], nu[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const bool pad = i + q >= NP;
                nr[q] = pad ? 0.f : fmaf(a.rk_a, rsv[q], a.dt * r4[q]);
                nu[q] = pad ? 0.f : fmaf(a.rk_b, nr[q], uov[q]);
              }
              *reinterpret_cast<float4 *>(a.res + off) = make_float4(nr[0], nr[1], nr[2], nr[3]);
              *reinterpret_cast<float4 *>(a.u_out + off) = make_float4(nu[0], nu[1], nu[2], nu[3]);
            }
          }
        }
      }
    }
    umma::fence_before_sync();
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, T::TCOLS);
}

// Host: the operators in the canonical K-major operand layout, hi then lo.
template <int N>
std::vector<uint8_t> build_operand_block(const RefOps &o, bool bf16) {
  using T = TC<N>;
  std::vector<uint8_t> blk(T::OPS_BYTES, 0);
  auto put = [&](int base_hi, int base_lo, int row, int col, int Kp, double v) {
    uint16_t hb, lb;
    if (bf16) {
      __nv_bfloat16 h = __float2bfloat16_rn(float(v));
      __nv_bfloat16 l = __float2bfloat16_rn(float(v - double(__bfloat162float(h))));
      std::memcpy(&hb, &h, 2);
      std::memcpy(&lb, &l, 2);
    } else {
      __half h = __float2half_rn(float(v));
      __half l = __float2half_rn(float(v - double(__half2float(h))));
      std::memcpy(&hb, &h, 2);
      std::memcpy(&lb, &l, 2);
    }
    uint32_t off = umma::kmajor_offset(uint32_t(row), uint32_t(col), uint32_t(Kp));
    std::memcpy(&blk[base_hi + off], &hb, 2);
    std::memcpy(&blk[base_lo + off], &lb, 2);
  };
  const int b1h = 0, b1l = T::B1B, b2h = 2 * T::B1B, b2l = 2 * T::B1B + T::B2B;
  const std::vector<double> *Ds[3] = {&o.Dr, &o.Ds, &o.Dt};
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < T::NP; ++i)
      for (int j = 0; j < T::NP; ++j) put(b1h, b1l, d * T::NB + i, j, T::K1, (*Ds[d])[i * T::NP + j]);
  for (int i = 0; i < T::NP; ++i)
    for (int m = 0; m < T::NFF; ++m) put(b2h, b2l, i, m, T::K2, o.LIFT[i * T::NFF + m]);
  return blk;
}

template <int N, int MODE, bool BF16>
cudaError_t launch_tc_kernel(const StageArgs &a, const TcState &st, int *flag, cudaStream_t s) {
  using T = TC<N>;
  static_assert(T::SMEM <= 232448, "tensor-core tile does not fit in shared memory");
  auto kern = k_stage_tc<N, MODE, BF16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  const int ntiles = int((a.K + kTileElems - 1) / kTileElems);
  const int grid = ntiles < st.sms ? ntiles : st.sms;
  kern<<<grid, kThreads, T::SMEM, s>>>(a, reinterpret_cast<const uint4 *>(st.d_ops), ntiles, flag);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_tc_order(int mode, bool bf16, const StageArgs &a, const TcState &st, int *flag, cudaStream_t s) {
  if (mode == MODE_RHS)
    return bf16 ? launch_tc_kernel<N, MODE_RHS, true>(a, st, flag, s) : launch_tc_kernel<N, MODE_RHS, false>(a, st, flag, s);
  return bf16 ? launch_tc_kernel<N, MODE_LSERK, true>(a, st, flag, s)
              : launch_tc_kernel<N, MODE_LSERK, false>(a, st, flag, s);
}

} // namespace

int tc_prepare(dg_ctx *ctx) {
  if (ctx->N > kMaxTcOrder) {
    ctx->err = "tensor-core precisions support N <= 5 (operators of higher orders do not fit in shared memory)";
    return DG_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    ctx->err = "tc_prepare: cannot query the device";
    return DG_ERR_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    ctx->err = "tensor-core precisions need a GB300 (sm_103) device";
    return DG_ERR_UNSUPPORTED;
  }
  const bool bf16 = ctx->precision == DG_BF16X3;
  std::vector<uint8_t> blk;
  switch (ctx->N) {
  case 1: blk = build_operand_block<1>(ctx->ops, bf16); break;
  case 2: blk = build_operand_block<2>(ctx->ops, bf16); break;
  case 3: blk = build_operand_block<3>(ctx->ops, bf16); break;
  case 4: blk = build_operand_block<4>(ctx->ops, bf16); break;
  default: blk = build_operand_block<5>(ctx->ops, bf16); break;
  }
  TcState *st = new TcState();
  st->sms = prop.multiProcessorCount;
  if (cudaMalloc(&st->d_ops, blk.size()) != cudaSuccess) {
    delete st;
    ctx->err = "tc_prepare: device allocation failed";
    return DG_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(st->d_ops, blk.data(), blk.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  ctx->tc = st;
  if (e != cudaSuccess) {
    ctx->err = std::string("tc_prepare: ") + cudaGetErrorString(e);
    return DG_ERR_CUDA;
  }
  return DG_OK;
}

void tc_free(dg_ctx *ctx) {
  TcState *st = static_cast<TcState *>(ctx->tc);
  if (st) {
    if (st->d_ops) cudaFree(st->d_ops);
    delete st;
  }
  ctx->tc = nullptr;
}

cudaError_t launch_stage_tc(dg_ctx *ctx, int mode, const StageArgs &a) {
  const TcState *st = static_cast<const TcState *>(ctx->tc);
  if (!st) return cudaErrorNotReady;
  const bool bf16 = ctx->precision == DG_BF16X3;
  int *flag = ctx->d_flag + 1;
  switch (ctx->N) {
  case 1: return launch_tc_order<1>(mode, bf16, a, *st, flag, ctx->stream);
  case 2: return launch_tc_order<2>(mode, bf16, a, *st, flag, ctx->stream);
  case 3: return launch_tc_order<3>(mode, bf16, a, *st, flag, ctx->stream);
  case 4: return launch_tc_order<4>(mode, bf16, a, *st, flag, ctx->stream);
  case 5: return launch_tc_order<5>(mode, bf16, a, *st, flag, ctx->stream);
  default: return cudaErrorNotSupported;
  }
}

} // namespace dgmx
