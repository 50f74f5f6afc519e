// Shared pieces of the adjoint's reverse-stage kernels (CUDA-core form in
// adjoint.cu, tensor-core form in adjoint_tc.cu): the launch arguments and the
// per-face-node device arithmetic of the transposed flux and of the eps
// gradient's impedance-weight terms.
#pragma once
#include "common.cuh"

namespace dgmx {

struct AdjArgs {
  const float *lr_in;  // lambda_r (read)
  float *lr_out;       // k_adj_lift: lr_scale lr + b lu (may alias lr_in, may be null); k_adj_vol: a * lr (may be
                       // null), or with the next lift fused in a * lr + b_next * lu_out (may alias lr_in)
  float lr_scale;      // k_adj_lift: the factor a of the stage reversed before, still to be applied to lr
  const float *lu_in;  // lambda_u (read; null = 0)
  float *lu_out;       // k_adj_vol: lu + dt A^T lr
  float *g;            // face data [6][K][NFF]
  float *g_next;       // k_adj_vol with the next lift fused in: that lift's face data (not g)
  float b_next;        // ... and the b of the stage it belongs to
  const float *u_s;    // stage state (eps gradient; null = no gradient)
  const float *rhs_s;  // A u_s at that stage
  double *grad;        // K, FP64 accumulation of dt <lr, dA/deps u_s>
  const float *geo;
  const float4 *fgeo;
  const int2 *fconn;
  const float *Dn;     // [3][Np][Npad] D_d[i][j]
  const float *LF;     // [Np][NFF] LIFT
  const uint8_t *fmask, *nbrtab, *nbrface;
  const float4 *fcon;  // tensor-core form: [K][4][4] per-face constants of the transposed flux (launch_adj_face_consts)
  int64_t K;
  float alpha, a, b, dt;
};

namespace adj {

// s[e] += v summed over the lanes of the warp that share e: a warp's lanes
// hold a few consecutive element indices, so for each distinct e the warp sums
// its lanes' values (shuffle tree) and one lane adds the sum to shared memory
// (instead of up to 32 lanes adding to one address). Every lane of the warp
// must call it.
__device__ __forceinline__ void add_by_element(float *s, int e, float v) {
  const int lane = threadIdx.x & 31;
  unsigned rest = 0xffffffffu;
  while (rest) {
    const int src = __ffs(rest) - 1;
    const int e0 = __shfl_sync(0xffffffffu, e, src);
    const bool mine = e == e0;
    rest &= ~__ballot_sync(0xffffffffu, mine);
    float sum = mine ? v : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == src && sum != 0.f) atomicAdd(s + e0, sum);
  }
}

__device__ __forceinline__ void cross3(const float *a, const float *b, float *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Transposed flux Jacobians of one face node for the face owner with normal n
// and weights (Zm, Zp, Ym, Yp), applied to its face data g = (gE, gH):
// contributions to the owner's interior trace (em, hm) and to the exterior
// trace (ep, hp). With flux_E = (Zp/Zs) n x dH - (alpha/Zs) n x n x dE and
// flux_H = -(Yp/Ys) n x dE - (alpha/Ys) n x n x dH, dq = q+ - q-, and
// (n x .)^T = -(n x .), (n x n x .)^T = n x n x .
// The face's zs = 1/(Zm+Zp) and ys = 1/(Ym+Yp) are given (they depend only on
// the face, so they are formed once per face, not per face node).
__device__ __forceinline__ void flux_transpose_w(const float *n, const float *g, float Zp, float Yp, float zs,
                                                 float ys, float alpha, float *ep, float *hp) {
  float nE[3], nH[3], nnE[3], nnH[3];
  cross3(n, g, nE);
  cross3(n, g + 3, nH);
  cross3(n, nE, nnE);
  cross3(n, nH, nnH);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    hp[c] = -(Zp * zs) * nE[c] - (alpha * ys) * nnH[c];
    ep[c] = -(alpha * zs) * nnE[c] + (Yp * ys) * nH[c];
  }
}

// <g, d flux / d(weights)>: the contractions of the face data g with the
// partial derivatives in Zm, Zp, Ym, Yp of the (unscaled) flux at one face
// node, with the face's zs = 1/(Zm+Zp), ys = 1/(Ym+Yp) given: the flux
// (weights zs and -ys) and n x dE, n x dH are formed once and shared.
__device__ __forceinline__ void flux_weight_partials_w(const float *n, const float *qm, const float *qp, float Zp,
                                                       float Yp, float zs, float ys, float alpha, const float *g,
                                                       float &sZm, float &sZp, float &sYm, float &sYp) {
  float dE[3], dH[3], nxdE[3], nxdH[3], v[3], f[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dE[c] = qp[c] - qm[c];
    dH[c] = qp[c + 3] - qm[c + 3];
  }
  cross3(n, dE, nxdE);
  cross3(n, dH, nxdH);
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = Zp * dH[c] - alpha * nxdE[c];
  cross3(n, v, f);
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = Yp * dE[c] + alpha * nxdH[c];
  cross3(n, v, f + 3);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f[c] *= zs;
    f[c + 3] *= -ys;
  }
  sZm = sZp = sYm = sYp = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sZm += g[c] * (-f[c] * zs);
    sZp += g[c] * ((nxdH[c] - f[c]) * zs);
    sYm += g[c + 3] * (-f[c + 3] * ys);
    sYp += g[c + 3] * ((-nxdE[c] - f[c + 3]) * ys);
  }
}

} // namespace adj

// Tensor-core form of the reverse volume stage (adjoint_tc.cu, N <= 5): the
// transposed curl and lift on tcgen05 in the FP16x3 split. Returns
// cudaErrorNotSupported where it does not apply (order, device).
bool adj_tc_supported(const dg_ctx *ctx);
cudaError_t launch_adj_tc(dg_ctx *ctx, const AdjArgs &a, cudaStream_t s);
// The per-face constants the tensor-core form reads (they depend on eps
// through the impedances; computed once per adjoint call): out is [K][4][4]
// float4 {n, 1/(Z-+Z+)}, {Z-, Z+, Y-, Y+}, {1/(Y-+Y+), dZ-/deps, dY-/deps,
// connection kind}, {neighbour element, wall}.
cudaError_t launch_adj_face_consts(const dg_ctx *ctx, float4 *out, cudaStream_t s);
void adj_tc_free(dg_ctx *ctx);

} // namespace dgmx
