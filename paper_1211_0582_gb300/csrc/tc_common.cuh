// Shared pieces of the tensor-core (split-precision) stage kernels: operand
// splitting, FP16 range scaling and the TMEM row layout of an element tile.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <vector>

#include "common.cuh"
#include "f32x2.cuh"
#include "umma.cuh"

namespace dgmx {
namespace tcc {

__host__ __device__ constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int tmem_cols(int x) {
  return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512;
}


struct TcState {
  void *d_ops = nullptr;
  int sms = 0;
  int form = 1; // N <= 5 stage: 1 single-tile resident form (default), 0 warp-specialised
};

// hi/lo split of two FP32 values into packed 16-bit pairs (x0 in the low half).
// BF16: hi by a rounding conversion, widened back by a shift (BF16 is the top
// half of FP32); lo = x - hi is exact in FP32 and converted with rounding.
// FP16: hi by a rounding conversion and widened back exactly; lo = x - hi is
// exact in FP32 and converted with rounding.
template <bool BF16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  if constexpr (BF16) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<const uint32_t *>(&hh);
    const float2 r = f2sub(make_float2(x0, x1), make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xFFFF0000u)));
    const __nv_bfloat162 ll = __floats2bfloat162_rn(r.x, r.y);
    lo = *reinterpret_cast<const uint32_t *>(&ll);
  } else {
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 r = f2sub(make_float2(x0, x1), __half22float2(hh));
    const __half2 ll = __floats2half2_rn(r.x, r.y);
    hi = *reinterpret_cast<const uint32_t *>(&hh);
    lo = *reinterpret_cast<const uint32_t *>(&ll);
  }
}

// Operand row (32 * quarter + lane) -> compact row (6 e + f), or -1 for the
// two unused lanes of each quarter.
__host__ __device__ constexpr int compact_row(int r) { return (r & 31) < 30 ? (r >> 5) * 30 + (r & 31) : -1; }

// Power-of-two scale bringing a maximum mx (>= 0) into [0.5, 1) and its
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

__device__ __forceinline__ float absmax4(float m, float4 v) {
  return fmaxf(fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y))), fmaxf(fabsf(v.z), fabsf(v.w)));
}

// Three split products per K step (hi*hi, hi*lo, lo*hi, FP32 accumulation in
// tensor memory) with the A operand (hi and lo) in tensor memory: one N
// chunk; a K step of 16 advances the A address by 8 columns.
template <bool BF16, int KP, int NR>
__device__ __forceinline__ void issue_split_gemm_ta(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                                    uint32_t b_lo) {
  constexpr uint32_t sbo = uint32_t(KP) * 16u;
  static_assert(NR <= 256, "one N chunk");
  const uint32_t idesc = umma::make_idesc(BF16, 128, uint32_t(NR));
  const uint64_t dbh = umma::make_desc(b_hi, 128, sbo), dbl = umma::make_desc(b_lo, 128, sbo);
#pragma unroll
  for (int kk = 0; kk < KP / 16; ++kk) {
    const uint64_t ko = uint64_t(kk) * 16u;
    const uint32_t ac = uint32_t(8 * kk);
    umma::mma_f16_ta(d_tmem, a_hi + ac, dbh + ko, idesc, kk > 0 ? 1u : 0u);
    umma::mma_f16_ta(d_tmem, a_hi + ac, dbl + ko, idesc, 1u);
    umma::mma_f16_ta(d_tmem, a_lo + ac, dbh + ko, idesc, 1u);
  }
}

// Orders 6 and 7: the operator slices in stream order (hi/lo), and the
// launch of the streamed-operator stage kernel.
std::vector<uint8_t> build_streamed_operators(int N, const RefOps &o, bool bf16);
cudaError_t launch_tc_streamed(int N, int mode, bool bf16, const StageArgs &a, const TcState &st, int *flag,
                               cudaStream_t s);

} // namespace tcc
} // namespace dgmx
