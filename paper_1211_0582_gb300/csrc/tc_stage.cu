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
  static constexpr int OFF_FL = OFF_U + (kRows * NPP + 24) * 4; // fp32 [kRows][NFF]
  static constexpr int OFF_TAB = OFF_FL + kRows * NFF * 4;
  static constexpr int OFF_SC = OFF_TAB + rup(NFF + kConnKinds * NFP, 16); // float [4][128]
  static constexpr int OFF_BAR = OFF_SC + 4 * 128 * 4;   // mbarriers: MMA done, residual landed; TMEM slot
  static constexpr int OFF_FACE = OFF_BAR + 32;          // per-tile face table [80] x 12 words
  static constexpr int SMEM = OFF_FACE + kTileElems * 4 * 48;
  // the residual tile [6][kTileElems * NPP + 4] reuses the flux staging
  static_assert(6 * (kTileElems * NPP + 4) <= kRows * NFF, "residual tile does not fit in the flux staging");
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

// Compact row (6 e + f) -> float offset of that row in the field-major
// staging, whose field blocks are padded by 4 floats so that the six field
// rows of one element fall in different shared-memory banks.
template <int NPP>
__device__ __forceinline__ int staged_off(int cr) { return (cr % 6) * (kTileElems * NPP + 4) + (cr / 6) * NPP; }

// Split the FP32 staging rows (compact rows 0..119; row-major with stride ld,
// or the field-major staging) into the hi/lo K-major operands, scaled per row.
// Work items are ordered so that each half-warp writes one 128-byte core matrix
// (8 rows x 16 bytes): conflict-free shared stores. Padding positions are never
// written (they stay zero).
template <bool BF16, bool FIELD_MAJOR, int NPP = 4>
__device__ __forceinline__ void convert_rows(const float *src, int ld, int cols, int Kp, const float *scale,
                                             uint8_t *dst_hi, uint8_t *dst_lo, int tid, int valid) {
  const int kgroups = Kp / 8;
  const int units = 128 * kgroups * 2;
  for (int u = tid; u < units; u += kThreads) {
    const int rr = u & 7, qh = (u >> 3) & 1;
    const int rest = u >> 4;
    const int kg = rest % kgroups, g = rest / kgroups;
    const int r = 8 * g + rr, k = 8 * kg + 4 * qh;
    const int cr = compact_row(r);
    if (cr < 0 || k >= cols) continue;
    const int sr = cr; // scales are indexed by compact row
    float4 v = *reinterpret_cast<const float4 *>(src + (FIELD_MAJOR ? staged_off<NPP>(cr) : cr * ld) + k);
    if (k + 3 >= valid) {
      if (k + 0 >= valid) v.x = 0.f;
      if (k + 1 >= valid) v.y = 0.f;
      if (k + 2 >= valid) v.z = 0.f;
      if (k + 3 >= valid) v.w = 0.f;
    }
    if constexpr (!BF16) {
      const float sc = scale[sr];
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
  // field-major staging [6][kTileElems][NPP]: the tile's fields, updated in place
  float *s_u = reinterpret_cast<float *>(smem + T::OFF_U);
  // flux staging [120][NFF] (compact rows), then the residual (or rhs) tile [6][kTileElems][NPP]
  float *s_fl = reinterpret_cast<float *>(smem + T::OFF_FL);
  float *s_res = s_fl;
  uint8_t *s_fm = smem + T::OFF_TAB;
  uint8_t *s_nb = s_fm + NFF;
  float *s_sc1 = reinterpret_cast<float *>(smem + T::OFF_SC); // staged rows: scale, inverse at +128
  float *s_sc2 = s_sc1 + 256;                                 // compact rows
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + T::OFF_BAR); // MMA completion
  uint64_t *barR = bar + 1;                                        // residual tile landed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + T::OFF_BAR + 16);
  float4 *s_face = reinterpret_cast<float4 *>(smem + T::OFF_FACE); // [80][3]: {n, Fs}, {wE, wH, Z+, Y+}, {k2, conn}

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t KN = a.K * NPP;
  const uint32_t sbase = umma::smem_u32(smem);

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
    prefetch_l2(a.fmat + kb * 4, uint32_t(ne * 4 * sizeof(float4)));
    prefetch_l2(a.geo + kb * G_STRIDE, uint32_t(ne * G_STRIDE * 4));
  };

  // ---- one-time setup
  for (int i = tid; i < (2 * T::A1B + 2 * T::A2B) / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < T::OPS_BYTES / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem + T::OFF_B1H)[i] = __ldg(ops + i);
  for (int i = tid; i < NFF + kConnKinds * NFP; i += kThreads)
    s_fm[i] = i < NFF ? a.fmask[i] : a.nbrtab[i - NFF];
  for (int i = tid; i < 512; i += kThreads) s_sc1[i] = 1.f;
  if (tid == 0) {
    umma::mbar_init(bar, 1);
    umma::mbar_init(barR, 1);
    umma::fence_mbar_init();
    prefetch_tile(blockIdx.x);
  }
  if (warp == 0) umma::tmem_alloc(tslot, T::TCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;

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
  constexpr int FS = kTileElems * NPP + 4; // padded field-block stride of the staging
  const int soff = fld * FS + e_loc * NPP; // this lane's row in the staging
  const uint32_t lane_taddr = tmem + (uint32_t(quarter * 32) << 16);
  constexpr int NCH = (NP + 7) / 8;
  constexpr int CPP = (NCH + 3) / 4;
  const int ch0 = part * CPP;
  const int ch1 = (part + 1) * CPP < NCH ? (part + 1) * CPP : NCH;

  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t k0 = int64_t(tile) * kTileElems;
    const int ne = int(a.K - k0 < kTileElems ? a.K - k0 : kTileElems);
    if (tid == 0) prefetch_tile(tile + gridDim.x);

    // ---- 1. face table and fields of the tile (loads first, then, once the
    // previous tile's bulk stores have read shared memory, the stores)
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
          if (e < ne) v[s] = ldg4(a.u + f * KN + (k0 + e) * NPP + 4 * q);
        }
      }
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, 0.f, 1.f, 1.f);
      int2 cn = make_int2(0, kBoundaryConn);
      if (tid < kTileElems * 4 && (tid >> 2) < ne) {
        const int64_t q = (k0 + (tid >> 2)) * 4 + (tid & 3);
        cn = __ldg(a.fconn + q);
        r0 = __ldg(a.fgeo + q);
        r1 = __ldg(a.fmat + q);
      }
      if (tid == 0) umma::bulk_wait_read_all();
      __syncthreads();
      if (tid < kTileElems * 4) {
        s_face[tid * 3 + 0] = r0;
        s_face[tid * 3 + 1] = r1;
        s_face[tid * 3 + 2] = make_float4(__int_as_float(cn.x), __int_as_float(cn.y), 0.f, 0.f);
      }
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int idx = tid + s * kThreads;
        if (idx < TOT) {
          const int q = idx % NQ;
          float4 w = v[s];
          if (4 * q + 3 >= NP) {
            if (4 * q + 0 >= NP) w.x = 0.f;
            if (4 * q + 1 >= NP) w.y = 0.f;
            if (4 * q + 2 >= NP) w.z = 0.f;
            if (4 * q + 3 >= NP) w.w = 0.f;
          }
          const int f = idx / (kTileElems * NQ), eq = idx - f * (kTileElems * NQ);
          *reinterpret_cast<float4 *>(s_u + f * FS + 4 * eq) = w;
        }
      }
    }
    __syncthreads();

    // ---- 2. split into the A1 operand (hi/lo), row-scaled for FP16
    if constexpr (!BF16) {
      const int r = tid >> 2, pt = tid & 3;
      float mx = 0.f;
      if (r < kRows)
        for (int j = pt; j < NP; j += 4) mx = fmaxf(mx, fabsf(s_u[staged_off<NPP>(r) + j]));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      if (pt == 0 && r < kRows) row_scale(mx, s_sc1[r], s_sc1[128 + r]);
      __syncthreads();
    }
    convert_rows<BF16, true, NPP>(s_u, NPP, NPP, T::K1, s_sc1, smem + T::OFF_A1H, smem + T::OFF_A1L, tid, NP);
    umma::fence_proxy_async();
    __syncthreads();

    // ---- 3. local differentiation on the tensor cores (asynchronous)
    if (tid == 0) {
      umma::fence_after_sync();
      issue_split_gemm<BF16>(tmem, sbase + T::OFF_A1H, sbase + T::OFF_A1L, sbase + T::OFF_B1H, sbase + T::OFF_B1L,
                             T::K1, T::N1);
    }

    // ---- 4. flux gather (overlaps GEMM1)
    {
      constexpr int TOT = kTileElems * NFF;
      constexpr int IT = (TOT + kThreads - 1) / kThreads;
      float qp[IT][6];
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int it = tid + s * kThreads;
        const int e = it / NFF, fm = it - e * NFF, f = fm / NFP, mm = fm - f * NFP;
#pragma unroll
        for (int c = 0; c < 6; ++c) qp[s][c] = 0.f;
        if (it < TOT && e < ne) {
          const float4 r2 = s_face[(e * 4 + f) * 3 + 2];
          const int conn = __float_as_int(r2.y);
          if (conn != kBoundaryConn) {
            const float *up = a.u + int64_t(__float_as_int(r2.x)) * NPP + s_nb[conn * NFP + mm];
#pragma unroll
            for (int c = 0; c < 6; ++c) qp[s][c] = __ldg(up + c * KN);
          }
        }
      }
#pragma unroll
      for (int s = 0; s < IT; ++s) {
        const int it = tid + s * kThreads;
        if (it >= TOT) continue;
        const int e = it / NFF, fm = it - e * NFF, f = fm / NFP;
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (e < ne) {
          const float4 r0 = s_face[(e * 4 + f) * 3 + 0], r1 = s_face[(e * 4 + f) * 3 + 1];
          const bool wall = __float_as_int(s_face[(e * 4 + f) * 3 + 2].y) == kBoundaryConn;
          const int vm = s_fm[fm];
          float qm[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) qm[c] = s_u[c * FS + e * NPP + vm];
          if (wall) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              qp[s][c] = -qm[c];
              qp[s][c + 3] = qm[c + 3];
            }
          }
          const float nx = r0.x, ny = r0.y, nz = r0.z;
          const float dEx = qp[s][0] - qm[0], dEy = qp[s][1] - qm[1], dEz = qp[s][2] - qm[2];
          const float dHx = qp[s][3] - qm[3], dHy = qp[s][4] - qm[4], dHz = qp[s][5] - qm[5];
          const float cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
          const float cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
          float vx = r1.z * dHx - a.alpha * cEx, vy = r1.z * dHy - a.alpha * cEy, vz = r1.z * dHz - a.alpha * cEz;
          fl[0] = r1.x * (ny * vz - nz * vy);
          fl[1] = r1.x * (nz * vx - nx * vz);
          fl[2] = r1.x * (nx * vy - ny * vx);
          vx = r1.w * dEx + a.alpha * cHx, vy = r1.w * dEy + a.alpha * cHy, vz = r1.w * dEz + a.alpha * cHz;
          fl[3] = r1.y * (ny * vz - nz * vy);
          fl[4] = r1.y * (nz * vx - nx * vz);
          fl[5] = r1.y * (nx * vy - ny * vx);
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
    convert_rows<BF16, false>(s_fl, NFF, NFF, T::K2, s_sc2, smem + T::OFF_A2H, smem + T::OFF_A2L, tid, NFF);
    umma::fence_proxy_async();
    __syncthreads();
    // the flux staging is free: the residual tile lands there during GEMM2
    if (MODE == MODE_LSERK && tid == 0) {
      const uint32_t rowbytes = uint32_t(ne * NPP * 4);
      umma::mbar_arrive_expect_tx(barR, 6u * rowbytes);
      for (int f = 0; f < 6; ++f)
        umma::bulk_g2s(s_res + f * FS, a.res + f * KN + k0 * NPP, rowbytes, barR);
    }

    // ---- 6. flux lifting on the tensor cores, then wait for both products
    if (tid == 0) {
      umma::fence_after_sync();
      issue_split_gemm<BF16>(tmem + uint32_t(T::N1), sbase + T::OFF_A2H, sbase + T::OFF_A2L, sbase + T::OFF_B2H,
                             sbase + T::OFF_B2L, T::K2, T::N2);
      umma::commit(bar);
    }
    const int64_t k = k0 + e_loc;
    const bool live = lane_used && e_loc < ne;
    float g1r = 0.f, g1s = 0.f, g1t = 0.f, g2r = 0.f, g2s = 0.f, g2t = 0.f, w = 0.f;
    if (live) {
      const float *g = a.geo + k * G_STRIDE;
      g1r = __ldg(g + G_RX + dl1), g1s = __ldg(g + G_SX + dl1), g1t = __ldg(g + G_TX + dl1);
      g2r = __ldg(g + G_RX + dl2), g2s = __ldg(g + G_SX + dl2), g2t = __ldg(g + G_TX + dl2);
      w = __ldg(g + (isE ? G_IEPS : G_IMU));
    }
    const float inv1 = BF16 ? 1.f : s_sc1[128 + (lane_used ? ridx : 0)];
    const float inv2 = BF16 ? 1.f : s_sc2[128 + (lane_used ? ridx : 0)];
    bool ok = umma::mbar_wait_bounded(bar, phase);
    if (MODE == MODE_LSERK) ok = umma::mbar_wait_bounded(barR, phase) && ok;
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err_flag, 1);
        // give the products and the residual copy in flight one more bounded
        // wait before tensor and shared memory are released
        umma::mbar_wait_bounded(bar, phase ^ 1u);
        if (MODE == MODE_LSERK) umma::mbar_wait_bounded(barR, phase ^ 1u);
      }
      break;
    }
    umma::fence_after_sync();

    // ---- 7. epilogue: chain rule, curls, lifting, material scale; the update
    // is written in place into the staged tiles
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
            float4 *rp = reinterpret_cast<float4 *>(s_res + soff + i);
            if (MODE == MODE_RHS) {
              *rp = make_float4(r4[0], r4[1], r4[2], r4[3]);
            } else {
              float4 *up = reinterpret_cast<float4 *>(s_u + soff + i);
              const float4 rs = *rp, uo = *up;
              const float rsv[4] = {rs.x, rs.y, rs.z, rs.w}, uov[4] = {uo.x, uo.y, uo.z, uo.w};
              float nr[4], nu[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const bool pad = i + q >= NP;
                nr[q] = pad ? 0.f : fmaf(a.rk_a, rsv[q], a.dt * r4[q]);
                nu[q] = pad ? 0.f : fmaf(a.rk_b, nr[q], uov[q]);
              }
              *rp = make_float4(nr[0], nr[1], nr[2], nr[3]);
              *up = make_float4(nu[0], nu[1], nu[2], nu[3]);
            }
          }
        }
      }
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    // ---- 8. write the tile back with asynchronous bulk stores
    if (tid == 0) {
      const uint32_t rowbytes = uint32_t(ne * NPP * 4);
      for (int f = 0; f < 6; ++f) {
        if (MODE == MODE_RHS) {
          umma::bulk_s2g(a.rhs + f * KN + k0 * NPP, s_res + f * FS, rowbytes);
        } else {
          umma::bulk_s2g(a.res + f * KN + k0 * NPP, s_res + f * FS, rowbytes);
          umma::bulk_s2g(a.u_out + f * KN + k0 * NPP, s_u + f * FS, rowbytes);
        }
      }
      umma::bulk_commit();
    }
  }
  if (tid == 0) umma::bulk_wait_all();
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
