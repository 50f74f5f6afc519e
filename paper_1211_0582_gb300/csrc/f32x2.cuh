// Packed FP32 pairs: per-element IEEE fp32 add, sub, mul and fma with
// round-to-nearest on two values in one instruction each (PTX .f32x2, sm_100
// family). Results are those of the scalar operations, bit for bit.
#pragma once
#include <cuda_runtime.h>

namespace dgmx {

#define DGMX_F2OP(name, op)                                                                                          \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                                                       \
    float2 d;                                                                                                        \
    asm("{\n .reg .b64 A, B, D;\n mov.b64 A, {%2, %3};\n mov.b64 B, {%4, %5};\n " op                            \
        " D, A, B;\n mov.b64 {%0, %1}, D;\n}"                                                                        \
        : "=f"(d.x), "=f"(d.y)                                                                                       \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                                   \
    return d;                                                                                                        \
  }
DGMX_F2OP(f2add, "add.rn.f32x2")
DGMX_F2OP(f2sub, "sub.rn.f32x2")
DGMX_F2OP(f2mul, "mul.rn.f32x2")
#undef DGMX_F2OP
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 A, B, C, D;\n mov.b64 A, {%2, %3};\n mov.b64 B, {%4, %5};\n mov.b64 C, {%6, %7};\n"
      " fma.rn.f32x2 D, A, B, C;\n mov.b64 {%0, %1}, D;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

} // namespace dgmx
