// Device-side pieces shared by the fused right-hand-side kernels: sizes per
// polynomial order and the Maxwell numerical flux at one face node.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "f32x2.cuh"

namespace dgmx {

template <int N>
struct Dims {
  static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6; // nodes per element
  static constexpr int NFP = (N + 1) * (N + 2) / 2;          // nodes per face
  static constexpr int NPP = (NP + 3) / 4 * 4;               // padded row length
  static constexpr int NQ = NPP / 4;                         // float4 per row
  static constexpr int NFF = 4 * NFP;                        // face nodes per element
};

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// Flux difference n.(F - F*) at one face node, times Fscale (Section 5,
// Fig. flux-code a, with jumps dq = q+ - q- and impedance weights for
// material jumps):
//   flux_E = n x (Z+ dH - alpha n x dE) / (Z- + Z+)
//   flux_H = -n x (Y+ dE + alpha n x dH) / (Y- + Y+)
// qm/qp: Ex Ey Ez Hx Hy Hz on the interior/exterior side; out: 6 values;
// nf: the face normal; w: the face's precomputed weights
// {Fscale/(Z- + Z+), -Fscale/(Y- + Y+), Z+, Y+}.
__device__ __forceinline__ void maxwell_flux_w(float4 nf, const float *qm, const float *qp, float4 w, float alpha,
                                               float *out) {
  const float nx = nf.x, ny = nf.y, nz = nf.z;
  const float dEx = qp[0] - qm[0], dEy = qp[1] - qm[1], dEz = qp[2] - qm[2];
  const float dHx = qp[3] - qm[3], dHy = qp[4] - qm[4], dHz = qp[5] - qm[5];
  const float cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
  const float cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
  float vx = w.z * dHx - alpha * cEx, vy = w.z * dHy - alpha * cEy, vz = w.z * dHz - alpha * cEz;
  out[0] = w.x * (ny * vz - nz * vy);
  out[1] = w.x * (nz * vx - nx * vz);
  out[2] = w.x * (nx * vy - ny * vx);
  vx = w.w * dEx + alpha * cHx;
  vy = w.w * dEy + alpha * cHy;
  vz = w.w * dEz + alpha * cHz;
  out[3] = w.y * (ny * vz - nz * vy);
  out[4] = w.y * (nz * vx - nx * vz);
  out[5] = w.y * (nx * vy - ny * vx);
}

// maxwell_flux_w at two face nodes of one face (same normal and weights),
// each value a pair (node 0, node 1).
__device__ __forceinline__ void maxwell_flux_w2(float4 nf, const float2 *qm, const float2 *qp, float4 w,
                                                float alpha, float2 *out) {
  const float2 nx = f2(nf.x), ny = f2(nf.y), nz = f2(nf.z);
  const float2 mnx = f2(-nf.x), mny = f2(-nf.y), mnz = f2(-nf.z);
  const float2 dEx = f2sub(qp[0], qm[0]), dEy = f2sub(qp[1], qm[1]), dEz = f2sub(qp[2], qm[2]);
  const float2 dHx = f2sub(qp[3], qm[3]), dHy = f2sub(qp[4], qm[4]), dHz = f2sub(qp[5], qm[5]);
  const float2 cEx = f2fma(ny, dEz, f2mul(mnz, dEy)), cEy = f2fma(nz, dEx, f2mul(mnx, dEz)),
               cEz = f2fma(nx, dEy, f2mul(mny, dEx));
  const float2 cHx = f2fma(ny, dHz, f2mul(mnz, dHy)), cHy = f2fma(nz, dHx, f2mul(mnx, dHz)),
               cHz = f2fma(nx, dHy, f2mul(mny, dHx));
  const float2 ma = f2(-alpha), pa = f2(alpha), wz = f2(w.z), ww = f2(w.w), wx = f2(w.x), wy = f2(w.y);
  float2 vx = f2fma(wz, dHx, f2mul(ma, cEx)), vy = f2fma(wz, dHy, f2mul(ma, cEy)), vz = f2fma(wz, dHz, f2mul(ma, cEz));
  out[0] = f2mul(wx, f2fma(ny, vz, f2mul(mnz, vy)));
  out[1] = f2mul(wx, f2fma(nz, vx, f2mul(mnx, vz)));
  out[2] = f2mul(wx, f2fma(nx, vy, f2mul(mny, vx)));
  vx = f2fma(ww, dEx, f2mul(pa, cHx));
  vy = f2fma(ww, dEy, f2mul(pa, cHy));
  vz = f2fma(ww, dEz, f2mul(pa, cHz));
  out[3] = f2mul(wy, f2fma(ny, vz, f2mul(mnz, vy)));
  out[4] = f2mul(wy, f2fma(nz, vx, f2mul(mnx, vz)));
  out[5] = f2mul(wy, f2fma(nx, vy, f2mul(mny, vx)));
}

} // namespace dgmx
