// Hand-written discrete adjoint of the LSERK4-stepped DG operator (FP32 CUDA
// cores, FP64 gradient reductions).
//
// The forward map is u_{n+1} = Step(u_n), each step five stages
// r_s = a_s r_{s-1} + dt A u_{s-1}, u_s = u_{s-1} + b_s r_s, with A = A(eps) the
// semi-discrete operator of eq. (semidiscrete-dg). Its exact transpose is
// swept backwards, stage by stage:
//     lr <- lr + b_s lu;   lu <- lu + dt A^T lr;   g_eps += dt <lr, dA/deps u_s>;   lr <- a_s lr
// and the receiver misfit J = sum_n |P u_n - E_ref,n|^2 adds 2 P^T (P u_n - E_ref,n)
// to lu at the end of each step n.
//
// A^T in gather form (no atomics on global memory): with W = diag(1/eps, 1/mu),
//   1. face data g = Fscale * LIFT^T (W lr), element-local (k_adj_lift);
//   2. per element: the transposed curl with D^T and the chain rule, plus the
//      transposed flux Jacobians applied to the element's own g (interior
//      side) and to the neighbour's g at the matching face node (exterior
//      side), with the PEC mirror folded in on walls (k_adj_vol).
// eps enters A through 1/eps on the E rows and through the impedance weights
// Z = sqrt(mu/eps), Y = 1/Z of every face flux in which the element takes
// part (as interior or exterior side); k_adj_vol gathers all of these for its
// own element, so each element's gradient is written by one block only.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dgmx.h"
#include "common.cuh"
#include "adj_common.cuh"
#include "flux.cuh"
#include "tc_api.h"

namespace dgmx {

namespace {

template <int N>
struct AdjCfg {
  using D = Dims<N>;
  static constexpr int MQ = D::NFF / 4;                       // face-node quads
  static constexpr int EB1 = 240 / MQ > 0 ? 240 / MQ : 1;     // elements per lift block
  static constexpr int NT1 = (EB1 * MQ + 31) / 32 * 32;
  static constexpr int EB2 = 80 / D::NQ > 0 ? 80 / D::NQ : 1; // elements per volume block (measured best)
  static constexpr int NT2 = (EB2 * D::NQ + 31) / 32 * 32;
  static constexpr size_t SMEM1 = size_t(6) * EB1 * D::NPP * 4;
  static constexpr size_t SMEM2 = size_t(EB2) * 4 * 64 + (size_t(6) * EB2 * D::NPP * 2 + EB2) * 4 +
                                  ((200 * D::NFP + 15) / 16) * 16;
};

using namespace adj;

// ---- 1. lr <- s lr + b lu (own element; s = the previous stage's a, applied
// here instead of as a separate pass) and g = Fscale * LIFT^T (W lr)
template <int N>
__global__ void __launch_bounds__(AdjCfg<N>::NT1) k_adj_lift(AdjArgs a) {
  using D = Dims<N>;
  using C = AdjCfg<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NQ = D::NQ, NFF = D::NFF, NFP = D::NFP, MQ = C::MQ, EB = C::EB1;
  extern __shared__ float4 smem4[];
  float *s_v = reinterpret_cast<float *>(smem4); // [6][EB][NPP]
  const int tid = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * EB;
  const int64_t KN = a.K * NPP;
  pdl_launch_next_and_wait(); // reverse stage after reverse stage
  for (int idx = tid; idx < 6 * EB * NQ; idx += C::NT1) {
    const int c = idx / (EB * NQ), rem = idx - c * (EB * NQ);
    const int e = rem / NQ, q = rem - e * NQ;
    const int64_t k = k0 + e;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < a.K) {
      const int64_t off = c * KN + k * NPP + 4 * q;
      v = *reinterpret_cast<const float4 *>(a.lr_in + off);
      v.x *= a.lr_scale, v.y *= a.lr_scale, v.z *= a.lr_scale, v.w *= a.lr_scale;
      if (a.lu_in) {
        const float4 lu = *reinterpret_cast<const float4 *>(a.lu_in + off);
        v.x = fmaf(a.b, lu.x, v.x), v.y = fmaf(a.b, lu.y, v.y), v.z = fmaf(a.b, lu.z, v.z), v.w = fmaf(a.b, lu.w, v.w);
      }
      if (4 * q + 3 >= NP) {
        if (4 * q + 0 >= NP) v.x = 0.f;
        if (4 * q + 1 >= NP) v.y = 0.f;
        if (4 * q + 2 >= NP) v.z = 0.f;
        if (4 * q + 3 >= NP) v.w = 0.f;
      }
      if (a.lr_out) *reinterpret_cast<float4 *>(a.lr_out + off) = v;
      const float w = __ldg(a.geo + k * G_STRIDE + (c < 3 ? G_IEPS : G_IMU));
      v.x *= w, v.y *= w, v.z *= w, v.w *= w;
    }
    reinterpret_cast<float4 *>(s_v)[(c * EB + e) * NQ + q] = v;
  }
  __syncthreads();
  const int e = tid / MQ, mq = tid - (tid / MQ) * MQ;
  const int64_t k = k0 + e;
  if (tid >= EB * MQ || k >= a.K) return;
  float acc[6][4];
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int n = 0; n < 4; ++n) acc[c][n] = 0.f;
#pragma unroll 4
  for (int i = 0; i < NP; ++i) {
    const float4 L = ldg4(a.LF + i * NFF + 4 * mq);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float v = s_v[(c * EB + e) * NPP + i];
      acc[c][0] = fmaf(L.x, v, acc[c][0]);
      acc[c][1] = fmaf(L.y, v, acc[c][1]);
      acc[c][2] = fmaf(L.z, v, acc[c][2]);
      acc[c][3] = fmaf(L.w, v, acc[c][3]);
    }
  }
  float fs[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) fs[n] = __ldg(a.fgeo + k * 4 + (4 * mq + n) / NFP).w;
#pragma unroll
  for (int c = 0; c < 6; ++c)
    *reinterpret_cast<float4 *>(a.g + (c * a.K + k) * NFF + 4 * mq) =
        make_float4(fs[0] * acc[c][0], fs[1] * acc[c][1], fs[2] * acc[c][2], fs[3] * acc[c][3]);
}

// ---- 2. lu <- lu + dt A^T lr; lr <- a lr; grad += dt <lr, dA/deps u_s>
// FUSE: the lift of the stage reversed next runs here too (it is element-local:
// lr <- a lr + b_next lu and g_next = Fscale * LIFT^T (W lr) need only this
// element's new lu), which saves the separate pass over lr and lu.
template <int N, bool GRAD, bool FUSE>
__global__ void __launch_bounds__(AdjCfg<N>::NT2) k_adj_vol(AdjArgs a) {
  using D = Dims<N>;
  using C = AdjCfg<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NQ = D::NQ, NFF = D::NFF, NFP = D::NFP, EB = C::EB2, NT = C::NT2;
  constexpr int MQ = C::MQ;
  extern __shared__ float4 smem4[];
  // per face of the block's elements: {n, 1/(Z-+Z+)}, {Z-, Z+, Y-, Y+},
  // {1/(Y-+Y+), dZ-/deps, dY-/deps, connection kind}, {neighbour element, wall}
  float4 *s_face = smem4;                                 // [EB * 4][4]
  float *s_v = reinterpret_cast<float *>(smem4 + EB * 16); // W lr   [6][EB][NPP]
  float *s_w = s_v + 6 * EB * NPP;               // surface contributions [6][EB][NPP]
  float *s_gr = s_w + 6 * EB * NPP;              // gradient partial per element [EB]
  uint8_t *s_fm = reinterpret_cast<uint8_t *>(s_gr + EB);
  uint8_t *s_nb = s_fm + NFF, *s_nf = s_nb + kConnKinds * NFP;
  const int tid = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * EB;
  const int64_t KN = a.K * NPP;

  for (int i = tid; i < NFF + 2 * kConnKinds * NFP; i += NT)
    s_fm[i] = i < NFF ? a.fmask[i] : i < NFF + kConnKinds * NFP ? a.nbrtab[i - NFF] : a.nbrface[i - NFF - kConnKinds * NFP];
  for (int i = tid; i < EB; i += NT) s_gr[i] = 0.f;
  for (int t = tid; t < EB * 4; t += NT) {
    const int e = t >> 2, f = t & 3;
    const int64_t k = k0 + e;
    if (k >= a.K) continue;
    const int2 cn = __ldg(a.fconn + k * 4 + f);
    const float4 nf = __ldg(a.fgeo + k * 4 + f);
    const float Zk = __ldg(a.geo + k * G_STRIDE + G_Z), Yk = __ldg(a.geo + k * G_STRIDE + G_Y);
    const bool wall = cn.y == kBoundaryConn;
    const int64_t k2 = wall ? k : cn.x;
    const float Z2 = wall ? Zk : __ldg(a.geo + k2 * G_STRIDE + G_Z), Y2 = wall ? Yk : __ldg(a.geo + k2 * G_STRIDE + G_Y);
    const float ek = 1.f / __ldg(a.geo + k * G_STRIDE + G_IEPS);
    s_face[t * 4 + 0] = make_float4(nf.x, nf.y, nf.z, 1.f / (Zk + Z2));
    s_face[t * 4 + 1] = make_float4(Zk, Z2, Yk, Y2);
    s_face[t * 4 + 2] = make_float4(1.f / (Yk + Y2), -Zk / (2.f * ek), Yk / (2.f * ek), __int_as_float(cn.y));
    s_face[t * 4 + 3] = make_float4(__int_as_float(int(k2)), __int_as_float(wall ? 1 : 0), 0.f, 0.f);
  }
  // the tables and face constants above are static: the previous kernel's
  // results (lambda, face data, gradient) are read from here on
  pdl_launch_next_and_wait();
  for (int idx = tid; idx < 6 * EB * NQ; idx += NT) {
    const int c = idx / (EB * NQ), rem = idx - c * (EB * NQ);
    const int e = rem / NQ, q = rem - e * NQ;
    const int64_t k = k0 + e;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < a.K) {
      v = *reinterpret_cast<const float4 *>(a.lr_in + c * KN + k * NPP + 4 * q);
      const float w = __ldg(a.geo + k * G_STRIDE + (c < 3 ? G_IEPS : G_IMU));
      v.x *= w, v.y *= w, v.z *= w, v.w *= w;
      if (4 * q + 3 >= NP) {
        if (4 * q + 0 >= NP) v.x = 0.f;
        if (4 * q + 1 >= NP) v.y = 0.f;
        if (4 * q + 2 >= NP) v.z = 0.f;
        if (4 * q + 3 >= NP) v.w = 0.f;
      }
    }
    reinterpret_cast<float4 *>(s_v)[(c * EB + e) * NQ + q] = v;
    reinterpret_cast<float4 *>(s_w)[(c * EB + e) * NQ + q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();

  // -- eps gradient, term of the 1/eps factor: -(1/eps) <lr_E, rhs_E> = -<W lr_E, rhs_E>
  if (GRAD) {
    for (int i0 = 0; i0 < 3 * EB * NQ; i0 += NT) { // whole rounds: every lane takes part in the sums
      const int idx = i0 + tid;
      const int rem = idx % (EB * NQ);
      const int e = rem / NQ, q = rem - e * NQ;
      const int c = idx / (EB * NQ);
      float part = 0.f;
      if (idx < 3 * EB * NQ && k0 + e < a.K) {
        const float4 r = *reinterpret_cast<const float4 *>(a.rhs_s + c * KN + (k0 + e) * NPP + 4 * q);
        const float4 v = reinterpret_cast<const float4 *>(s_v)[(c * EB + e) * NQ + q];
        part = -(v.x * r.x + v.y * r.y + v.z * r.z + v.w * r.w);
      }
      add_by_element(s_gr, e, part);
    }
  }

  // -- transposed flux Jacobians (interior side with own g, exterior side with
  //    the neighbour's g at the matching face node) and the weight terms of the
  //    eps gradient, one face node per item
  for (int it0 = 0; it0 < EB * NFF; it0 += NT) { // whole rounds: every lane takes part in the sums
    const int it = it0 + tid;
    const int e = (it < EB * NFF ? it : EB * NFF - 1) / NFF, fm = it - e * NFF, f = fm / NFP, m = fm - f * NFP;
    const int64_t k = k0 + e;
    float contrib = 0.f;
    if (it < EB * NFF && k < a.K) {
    const float4 *fr = s_face + (e * 4 + f) * 4;
    const float4 r0 = fr[0], r1 = fr[1], r2 = fr[2], r3 = fr[3];
    const float n[3] = {r0.x, r0.y, r0.z};
    const float zs = r0.w, Zk = r1.x, Z2 = r1.y, Yk = r1.z, Y2 = r1.w, ys = r2.x;
    const int cny = __float_as_int(r2.w);
    const int64_t k2 = __float_as_int(r3.x);
    const bool wall = __float_as_int(r3.y) != 0;
    float gk[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) gk[c] = a.g[(c * a.K + k) * NFF + fm];
    float ep[3], hp[3], acc[6];
    flux_transpose_w(n, gk, Z2, Y2, zs, ys, a.alpha, ep, hp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] = -ep[c];      // interior side: the E and H Jacobians are the negatives of the exterior ones
      acc[c + 3] = -hp[c];
    }
    const int fm2 = wall ? 0 : s_nf[cny * NFP + m] + (cny / 6 % 4) * NFP;
    float g2[6];
    if (wall) {
      // exterior state E+ = -E-, H+ = H- folds back onto the interior node
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[c] -= ep[c];
        acc[c + 3] += hp[c];
      }
    } else {
      // the neighbour's flux sees this element as its exterior side
#pragma unroll
      for (int c = 0; c < 6; ++c) g2[c] = a.g[(c * a.K + k2) * NFF + fm2];
      const float n2[3] = {-n[0], -n[1], -n[2]};
      float ep2[3], hp2[3];
      flux_transpose_w(n2, g2, Zk, Yk, zs, ys, a.alpha, ep2, hp2);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[c] += ep2[c];
        acc[c + 3] += hp2[c];
      }
    }
    const int vm = s_fm[fm];
#pragma unroll
    for (int c = 0; c < 6; ++c) atomicAdd(&s_w[(c * EB + e) * NPP + vm], acc[c]);
    if (GRAD) {
      const float dZ = r2.y, dY = r2.z;
      float qm[6], qp[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) qm[c] = __ldg(a.u_s + c * KN + k * NPP + vm);
      if (wall) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          qp[c] = -qm[c];
          qp[c + 3] = qm[c + 3];
        }
      } else {
        const int vn = s_nb[cny * NFP + m];
#pragma unroll
        for (int c = 0; c < 6; ++c) qp[c] = __ldg(a.u_s + c * KN + k2 * NPP + vn);
      }
      float sZm, sZp, sYm, sYp;
      flux_weight_partials_w(n, qm, qp, Z2, Y2, zs, ys, a.alpha, gk, sZm, sZp, sYm, sYp);
      contrib = sZm * dZ + sYm * dY;
      if (wall) {
        contrib += sZp * dZ + sYp * dY; // the mirrored exterior carries the same weights
      } else {
        const float n2[3] = {-n[0], -n[1], -n[2]};
        float tZm, tZp, tYm, tYp;
        flux_weight_partials_w(n2, qp, qm, Zk, Yk, zs, ys, a.alpha, g2, tZm, tZp, tYm, tYp);
        contrib += tZp * dZ + tYp * dY;
      }
    }
    }
    if (GRAD) add_by_element(s_gr, e, contrib);
  }
  __syncthreads();

  // -- transposed volume term: w_T[j] = sum_d sum_i D_d[i][j] q_{T,d}[i] with
  //    the contravariant combinations q_{T,d} = sum_l (dr_d/dx_l) (+-W lr) of
  //    the transposed curl formed per node from the element's metric terms:
  //    H_c <- d_{c+2}^T (W lr)_{E_{c+1}} - d_{c+1}^T (W lr)_{E_{c+2}}
  //    E_c <- -d_{c+2}^T (W lr)_{H_{c+1}} + d_{c+1}^T (W lr)_{H_{c+2}}
  const int e = tid / NQ, q = tid - (tid / NQ) * NQ;
  const int64_t k = k0 + e;
  const bool active = tid < EB * NQ && k < a.K;
  float wl[6][4]; // FUSE: W lr of this lane's nodes after the update, for the fused lift
  if (active) {
    float G[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) G[t] = __ldg(a.geo + k * G_STRIDE + t);
    float acc[6][4];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) acc[c][n] = 0.f;
#pragma unroll 2
    for (int i = 0; i < NP; ++i) {
      float v[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] = s_v[(c * EB + e) * NPP + i];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float4 Dv = ldg4(a.Dn + (d * NP + i) * NPP + 4 * q);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
          const float g1 = G[3 * d + c1], g2 = G[3 * d + c2];
          const float qH = g2 * v[c1] - g1 * v[c2];         // into H_c
          const float qE = -g2 * v[3 + c1] + g1 * v[3 + c2]; // into E_c
          acc[3 + c][0] = fmaf(Dv.x, qH, acc[3 + c][0]);
          acc[3 + c][1] = fmaf(Dv.y, qH, acc[3 + c][1]);
          acc[3 + c][2] = fmaf(Dv.z, qH, acc[3 + c][2]);
          acc[3 + c][3] = fmaf(Dv.w, qH, acc[3 + c][3]);
          acc[c][0] = fmaf(Dv.x, qE, acc[c][0]);
          acc[c][1] = fmaf(Dv.y, qE, acc[c][1]);
          acc[c][2] = fmaf(Dv.z, qE, acc[c][2]);
          acc[c][3] = fmaf(Dv.w, qE, acc[c][3]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int64_t off = c * KN + k * NPP + 4 * q;
      const float4 sw = reinterpret_cast<const float4 *>(s_w)[(c * EB + e) * NQ + q];
      float4 lu = a.lu_in ? *reinterpret_cast<const float4 *>(a.lu_in + off) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float wv[4] = {acc[c][0] + sw.x, acc[c][1] + sw.y, acc[c][2] + sw.z, acc[c][3] + sw.w};
      float o[4] = {lu.x, lu.y, lu.z, lu.w};
#pragma unroll
      for (int n = 0; n < 4; ++n) o[n] = (4 * q + n < NP) ? fmaf(a.dt, wv[n], o[n]) : 0.f;
      *reinterpret_cast<float4 *>(a.lu_out + off) = make_float4(o[0], o[1], o[2], o[3]);
      if (FUSE) {
        // the next lift's first half, in the separate lift's order of operations
        const float4 lr = *reinterpret_cast<const float4 *>(a.lr_in + off);
        const float lv[4] = {lr.x, lr.y, lr.z, lr.w};
        float p[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) p[n] = (4 * q + n < NP) ? fmaf(a.b_next, o[n], lv[n] * a.a) : 0.f;
        *reinterpret_cast<float4 *>(a.lr_out + off) = make_float4(p[0], p[1], p[2], p[3]);
        const float w = __ldg(a.geo + k * G_STRIDE + (c < 3 ? G_IEPS : G_IMU));
#pragma unroll
        for (int n = 0; n < 4; ++n) wl[c][n] = p[n] * w;
      } else if (a.lr_out) {
        const float4 lr = *reinterpret_cast<const float4 *>(a.lr_in + off);
        *reinterpret_cast<float4 *>(a.lr_out + off) = make_float4(a.a * lr.x, a.a * lr.y, a.a * lr.z, a.a * lr.w);
      }
    }
  }
  if (GRAD && tid < EB && k0 + tid < a.K) a.grad[k0 + tid] += double(a.dt) * double(s_gr[tid]);
  if constexpr (FUSE) {
    // the next lift's second half: g_next = Fscale * LIFT^T (W lr), one
    // (element, face-node quad) per item, from the new W lr in shared memory
    __syncthreads(); // every lane has finished reading s_v in the transposed volume term
    if (tid < EB * NQ)
#pragma unroll
      for (int c = 0; c < 6; ++c)
        reinterpret_cast<float4 *>(s_v)[(c * EB + e) * NQ + q] =
            active ? make_float4(wl[c][0], wl[c][1], wl[c][2], wl[c][3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int t = tid; t < EB * MQ; t += NT) {
      const int el = t / MQ, mq = t - (t / MQ) * MQ;
      const int64_t kl = k0 + el;
      if (kl >= a.K) continue;
      float acc[6][4];
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[c][n] = 0.f;
#pragma unroll 4
      for (int i = 0; i < NP; ++i) {
        const float4 L = ldg4(a.LF + i * NFF + 4 * mq);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float v = s_v[(c * EB + el) * NPP + i];
          acc[c][0] = fmaf(L.x, v, acc[c][0]);
          acc[c][1] = fmaf(L.y, v, acc[c][1]);
          acc[c][2] = fmaf(L.z, v, acc[c][2]);
          acc[c][3] = fmaf(L.w, v, acc[c][3]);
        }
      }
      float fs[4];
#pragma unroll
      for (int n = 0; n < 4; ++n) fs[n] = __ldg(a.fgeo + kl * 4 + (4 * mq + n) / NFP).w;
#pragma unroll
      for (int c = 0; c < 6; ++c)
        *reinterpret_cast<float4 *>(a.g_next + (c * a.K + kl) * NFF + 4 * mq) =
            make_float4(fs[0] * acc[c][0], fs[1] * acc[c][1], fs[2] * acc[c][2], fs[3] * acc[c][3]);
    }
  }
}

template <int N>
cudaError_t launch_adj_order(int which, const AdjArgs &a, cudaStream_t s) {
  using C = AdjCfg<N>;
  // the shared-memory opt-in is a per-device function attribute: set it on every launch
  cudaError_t e;
  if (which == 0) {
    e = cudaFuncSetAttribute(k_adj_lift<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM1));
    if (e != cudaSuccess) return e;
    return launch_pdl(k_adj_lift<N>, dim3(unsigned((a.K + C::EB1 - 1) / C::EB1)), dim3(C::NT1), C::SMEM1, s, a);
  } else {
    const unsigned blocks = unsigned((a.K + C::EB2 - 1) / C::EB2);
    auto go = [&](auto kern) {
      cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM2));
      return r != cudaSuccess ? r : launch_pdl(kern, dim3(blocks), dim3(C::NT2), C::SMEM2, s, a);
    };
    if (a.g_next) return a.u_s ? go(k_adj_vol<N, true, true>) : go(k_adj_vol<N, false, true>);
    return a.u_s ? go(k_adj_vol<N, true, false>) : go(k_adj_vol<N, false, false>);
  }
}

cudaError_t launch_adj(int N, int which, const AdjArgs &a, cudaStream_t s) {
  switch (N) {
  case 1: return launch_adj_order<1>(which, a, s);
  case 2: return launch_adj_order<2>(which, a, s);
  case 3: return launch_adj_order<3>(which, a, s);
  case 4: return launch_adj_order<4>(which, a, s);
  case 5: return launch_adj_order<5>(which, a, s);
  case 6: return launch_adj_order<6>(which, a, s);
  case 7: return launch_adj_order<7>(which, a, s);
  case 8: return launch_adj_order<8>(which, a, s);
  case 9: return launch_adj_order<9>(which, a, s);
  default: return cudaErrorInvalidValue;
  }
}

// Receiver residual of one step: res_n = E(u)[recv] - Eref_n (FP32, stored) and
// J += |res_n|^2 (FP64).
__global__ void k_recv_residual(const float *u, int64_t K, int Np, int Npad, const int64_t *recv, int64_t R,
                                const float *Eref, float *resid, double *J) {
  double local = 0.0;
  for (int64_t t = threadIdx.x + int64_t(blockIdx.x) * blockDim.x; t < 3 * R; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / R);
    const int64_t r = t - c * R, node = recv[r];
    const int64_t k = node / Np, i = node - k * Np;
    const float v = u[(c * K + k) * Npad + i] - (Eref ? Eref[t] : 0.f);
    if (resid) resid[t] = v;
    local += double(v) * double(v);
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && J) atomicAdd(J, local);
}

// Adjoint source of one step: lu[E at recv] += 2 res_n (receivers are distinct).
__global__ void k_recv_source(float *lu, int64_t K, int Np, int Npad, const int64_t *recv, int64_t R,
                              const float *resid) {
  for (int64_t t = threadIdx.x + int64_t(blockIdx.x) * blockDim.x; t < 3 * R; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / R);
    const int64_t r = t - c * R, node = recv[r];
    const int64_t k = node / Np, i = node - k * Np;
    lu[(c * K + k) * Npad + i] += 2.f * resid[t];
  }
}

__global__ void k_recv_gather(const float *u, int64_t K, int Np, int Npad, const int64_t *recv, int64_t R, float *out) {
  for (int64_t t = threadIdx.x + int64_t(blockIdx.x) * blockDim.x; t < 3 * R; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / R);
    const int64_t r = t - c * R, node = recv[r];
    const int64_t k = node / Np, i = node - k * Np;
    out[t] = u[(c * K + k) * Npad + i];
  }
}

__global__ void k_check_recv(const int64_t *recv, int64_t R, int64_t nodes, int *bad) {
  for (int64_t t = threadIdx.x + int64_t(blockIdx.x) * blockDim.x; t < R; t += int64_t(gridDim.x) * blockDim.x)
    if (recv[t] < 0 || recv[t] >= nodes) atomicExch(bad, 1);
}

int fail(dg_ctx *ctx, int code, const std::string &msg) {
  ctx->err = msg;
  return code;
}

// Device work buffers of the adjoint and receiver-trace calls, kept in the
// context between calls (an optimisation loop calls them many times) and grown
// on demand; released with the mesh.
struct AdjWorkspace {
  static constexpr int kSlots = 20;
  void *p[kSlots] = {};
  size_t cap[kSlots] = {};
  // a second stream for recomputing one checkpoint segment while the reverse
  // sweep of the next runs, and the events that order the two
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fwd = nullptr, ev_rec[2] = {}, ev_rev[2] = {};
  bool streams_ready() {
    if (s2) return true;
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s2 = nullptr;
      return false;
    }
    bool ok = cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 2; ++i) {
      ok = ok && cudaEventCreateWithFlags(&ev_rec[i], cudaEventDisableTiming) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&ev_rev[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      release_streams();
    }
    return ok;
  }
  void release_streams() {
    if (s2) cudaStreamSynchronize(s2);
    for (cudaEvent_t *ev : {&ev_fwd, &ev_rec[0], &ev_rec[1], &ev_rev[0], &ev_rev[1]}) {
      if (*ev) cudaEventDestroy(*ev);
      *ev = nullptr;
    }
    if (s2) cudaStreamDestroy(s2);
    s2 = nullptr;
  }
  template <class T>
  T *get(int slot, size_t count) {
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    if (cap[slot] < bytes) {
      if (p[slot]) cudaFree(p[slot]);
      p[slot] = nullptr;
      cap[slot] = 0;
      if (cudaMalloc(&p[slot], bytes) != cudaSuccess) {
        cudaGetLastError();
        p[slot] = nullptr;
        return nullptr;
      }
      cap[slot] = bytes;
    }
    return static_cast<T *>(p[slot]);
  }
  ~AdjWorkspace() {
    release_streams();
    for (void *q : p)
      if (q) cudaFree(q);
  }
};

AdjWorkspace &workspace(dg_ctx *c) {
  if (!c->adj) c->adj = new AdjWorkspace();
  return *static_cast<AdjWorkspace *>(c->adj);
}

AdjArgs adj_base(const dg_ctx *c, float alpha) {
  AdjArgs a{};
  a.geo = c->d_geo;
  a.fgeo = c->d_fgeo;
  a.fconn = c->d_fconn;
  a.Dn = c->d_Dn;
  a.LF = c->d_LF;
  a.fmask = c->d_tab;
  a.nbrtab = c->d_tab + 4 * c->ops.Nfp;
  a.nbrface = c->d_tab + 4 * c->ops.Nfp + kConnKinds * c->ops.Nfp;
  a.K = c->K;
  a.alpha = alpha;
  a.lr_scale = 1.f;
  return a;
}

StageArgs stage_base(const dg_ctx *c, float alpha, double dt) {
  StageArgs a{};
  a.geo = c->d_geo;
  a.fgeo = c->d_fgeo;
  a.fconn = c->d_fconn;
  a.fmat = c->d_fmat;
  a.wait_limit = c->wait_limit;
  a.DT = c->d_DT;
  a.LT = c->d_LT;
  a.fmask = c->d_tab;
  a.nbrtab = c->d_tab + 4 * c->ops.Nfp;
  a.K = c->K;
  a.alpha = alpha;
  a.dt = float(dt);
  return a;
}

// One forward LSERK stage of the adjoint's sweeps in the context's precision:
// the tensor-core stage (with its store form) in split-precision contexts at
// N <= 5, else the FP32 CUDA-core stage.
cudaError_t forward_stage(dg_ctx *c, int mode, const StageArgs &a, cudaStream_t s) {
  if (c->precision != DG_FP32 && c->tc && c->N <= 5) return launch_stage_tc(c, mode, a, s);
  return launch_stage_simt(c->N, mode, a, s);
}

int check_common(dg_ctx *ctx, const float *u0, double dt, int nsteps, float alpha, const int64_t *recv, int64_t R,
                 const char *who) {
  if (!ctx) return DG_ERR_ARG;
  if (ctx->K <= 0) return fail(ctx, DG_ERR_ARG, std::string(who) + ": no mesh uploaded");
  if (!u0 || (reinterpret_cast<uintptr_t>(u0) & 15u)) return fail(ctx, DG_ERR_ARG, std::string(who) + ": bad u0");
  if (nsteps < 1 || !std::isfinite(dt) || !std::isfinite(alpha))
    return fail(ctx, DG_ERR_ARG, std::string(who) + ": bad dt/nsteps/alpha");
  if (R < 1 || !recv) return fail(ctx, DG_ERR_ARG, std::string(who) + ": need at least one receiver");
  int *bad = ctx->d_flag + 2, hbad = 0;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) {
    k_check_recv<<<unsigned((R + 255) / 256), 256, 0, ctx->stream>>>(recv, R, ctx->K * ctx->ops.Np, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
  if (hbad) return fail(ctx, DG_ERR_ARG, std::string(who) + ": receiver index outside [0, K*Np)");
  return DG_OK;
}

} // namespace

void adjoint_free(dg_ctx *c) {
  delete static_cast<AdjWorkspace *>(c->adj);
  c->adj = nullptr;
}

} // namespace dgmx

using namespace dgmx;

extern "C" {

int dg_adjoint_segment_steps(const dg_ctx *ctx) { return ctx ? ctx->adj_segment : 0; }

int dg_rhs_transpose(dg_ctx *ctx, const float *v, float *w, float alpha) {
  dgmx::NvtxRange nvtx_range("dg_rhs_transpose");
  if (!ctx) return DG_ERR_ARG;
  if (ctx->K <= 0) return fail(ctx, DG_ERR_ARG, "dg_rhs_transpose: no mesh uploaded");
  if (!v || !w || ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(w)) & 15u))
    return fail(ctx, DG_ERR_ARG, "dg_rhs_transpose: null or misaligned field");
  const size_t bytes = size_t(6) * ctx->K * ctx->ops.Npad * sizeof(float);
  const uintptr_t pv = reinterpret_cast<uintptr_t>(v), pw = reinterpret_cast<uintptr_t>(w);
  if (pv < pw + bytes && pw < pv + bytes) return fail(ctx, DG_ERR_ARG, "dg_rhs_transpose: v and w overlap");
  float *g = workspace(ctx).get<float>(5, size_t(6) * ctx->K * 4 * ctx->ops.Nfp);
  if (!g) return fail(ctx, DG_ERR_OOM, "dg_rhs_transpose: device allocation failed");
  AdjArgs a = adj_base(ctx, alpha);
  a.lr_in = v;
  a.g = g;
  a.dt = 1.f;
  a.lu_out = w;
  cudaError_t e = launch_adj(ctx->N, 0, a, ctx->stream);
  if (e == cudaSuccess) e = launch_adj(ctx->N, 1, a, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_rhs_transpose: ") + cudaGetErrorString(e));
  return DG_OK;
}

int dg_receiver_traces(dg_ctx *ctx, const float *u0, const float *eps, double dt, int nsteps, float alpha,
                       const int64_t *recv, int64_t R, float *out) {
  dgmx::NvtxRange nvtx_range("dg_receiver_traces");
  int rc = check_common(ctx, u0, dt, nsteps, alpha, recv, R, "dg_receiver_traces");
  if (rc) return rc;
  if (!out) return fail(ctx, DG_ERR_ARG, "dg_receiver_traces: null output");
  if (eps && (rc = dg_set_eps(ctx, eps))) return rc;
  const size_t fl = size_t(6) * ctx->K * ctx->ops.Npad;
  AdjWorkspace &ws = workspace(ctx);
  float *u = ws.get<float>(0, fl), *nxt = ws.get<float>(1, fl), *res = ws.get<float>(2, fl);
  if (!u || !nxt || !res) return fail(ctx, DG_ERR_OOM, "dg_receiver_traces: device allocation failed");
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(u, u0, fl * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(res, 0, fl * 4, s);
  StageArgs a = stage_base(ctx, alpha, dt);
  a.res = res;
  const unsigned rb = unsigned((3 * R + 255) / 256);
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
      a.u = u;
      a.u_out = nxt;
      a.rk_a = float(kLserkA[st]);
      a.rk_b = float(kLserkB[st]);
      e = forward_stage(ctx, MODE_LSERK, a, s);
      std::swap(u, nxt);
    }
    if (e == cudaSuccess) {
      k_recv_gather<<<rb, 256, 0, s>>>(u, ctx->K, ctx->ops.Np, ctx->ops.Npad, recv, R, out + int64_t(n) * 3 * R);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_receiver_traces: ") + cudaGetErrorString(e));
  return DG_OK;
}

int dg_adjoint_step(dg_ctx *ctx, const float *u0, const float *eps, double dt, int nsteps, int ckpt_every,
                    float alpha, const int64_t *recv, int64_t R, const float *Eref, double *J, double *dJ_deps,
                    float *dJ_du0) {
  dgmx::NvtxRange nvtx_range("dg_adjoint_step");
  int rc = check_common(ctx, u0, dt, nsteps, alpha, recv, R, "dg_adjoint_step");
  if (rc) return rc;
  if (!Eref) return fail(ctx, DG_ERR_ARG, "dg_adjoint_step: null Eref");
  if (ckpt_every < 0) return fail(ctx, DG_ERR_ARG, "dg_adjoint_step: ckpt_every must be >= 0");
  if (dJ_du0 && (reinterpret_cast<uintptr_t>(dJ_du0) & 15u))
    return fail(ctx, DG_ERR_ARG, "dg_adjoint_step: dJ_du0 must be 16-byte aligned");
  if (eps && (rc = dg_set_eps(ctx, eps))) return rc;
  const size_t fl = size_t(6) * ctx->K * ctx->ops.Npad;
  const size_t gfl = size_t(6) * ctx->K * 4 * ctx->ops.Nfp;
  const size_t hfl = fl / 2; // three of the six fields
  cudaStream_t s = ctx->stream;
  AdjWorkspace &ws = workspace(ctx);

  if (!dJ_deps && !dJ_du0) {
    // misfit only: the forward run and the receiver residuals, no checkpoints
    // and no reverse sweep
    float *u = ws.get<float>(0, fl), *nxt = ws.get<float>(1, fl), *res = ws.get<float>(2, fl);
    float *resid = ws.get<float>(6, size_t(nsteps) * 3 * R);
    double *Jd = ws.get<double>(7, 1);
    if (!u || !nxt || !res || !resid || !Jd) return fail(ctx, DG_ERR_OOM, "dg_adjoint_step: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(u, u0, fl * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(res, 0, fl * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(Jd, 0, sizeof(double), s);
    StageArgs sa = stage_base(ctx, alpha, dt);
    sa.res = res;
    const unsigned rb = unsigned((3 * R + 255) / 256);
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
      for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
        sa.u = u;
        sa.u_out = nxt;
        sa.rk_a = float(kLserkA[st]);
        sa.rk_b = float(kLserkB[st]);
        e = forward_stage(ctx, MODE_LSERK, sa, s);
        std::swap(u, nxt);
      }
      if (e == cudaSuccess) {
        k_recv_residual<<<rb, 256, 0, s>>>(u, ctx->K, ctx->ops.Np, ctx->ops.Npad, recv, R,
                                           Eref + int64_t(n) * 3 * R, resid + int64_t(n) * 3 * R, Jd);
        e = cudaGetLastError();
      }
    }
    double Jh = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&Jh, Jd, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_adjoint_step: ") + cudaGetErrorString(e));
    ctx->adj_segment = 0;
    if (J) *J = Jh;
    if (!std::isfinite(Jh)) return fail(ctx, DG_ERR_NONFINITE, "dg_adjoint_step: misfit is not finite");
    return DG_OK;
  }

  // steps per segment: given, or (0) as many as half of the device memory
  // that is free or already held for segment storage can take
  int C = ckpt_every;
  if (C == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(ctx, DG_ERR_CUDA, "dg_adjoint_step: cudaMemGetInfo");
    const size_t per_step = size_t(5) * (fl + hfl) * sizeof(float);
    const size_t fit = (fr + ws.cap[10] + ws.cap[11]) / 2 / per_step;
    C = fit < size_t(nsteps) ? int(fit) : nsteps;
    if (C < 1) C = 1;
  }
  if (C > nsteps) C = nsteps;
  // with checkpoint segments, two segment buffers: one is recomputed (second
  // stream) while the reverse sweep reads the other; the automatic size
  // halves C so that both fit where one would
  if (ckpt_every == 0 && C < nsteps && C > 1) C /= 2;
  // segments are aligned to the end of the run: all but the first have C
  // steps; the last one is stored during the forward sweep, the others are
  // recomputed from their checkpoints
  const int nseg = (nsteps + C - 1) / C;
  const int first_len = nsteps - (nseg - 1) * C;
  auto seg_start = [&](int sg) { return sg == 0 ? 0 : first_len + (sg - 1) * C; };
  ctx->adj_segment = C;
  float *u = ws.get<float>(0, fl), *nxt = ws.get<float>(1, fl), *res = ws.get<float>(2, fl);
  float *lu = ws.get<float>(3, fl), *lr = ws.get<float>(4, fl), *g = ws.get<float>(5, gfl);
  float *resid = ws.get<float>(6, size_t(nsteps) * 3 * R);
  double *Jd = ws.get<double>(7, 1), *grad = ws.get<double>(8, ctx->K);
  float *ck = ws.get<float>(9, fl * nseg);
  float *g2 = ws.get<float>(16, gfl); // the face data of the lift fused into the volume kernel (two in turn)
  // the reverse volume stage: its contractions on the tensor cores (FP16x3)
  // where supported unless the CUDA-core form was asked for; that form reads
  // per-face constants computed once per call
  const bool tc_reverse = ctx->adj_form != 0 && adj_tc_supported(ctx);
  float4 *fcon = tc_reverse ? ws.get<float4>(17, size_t(16) * ctx->K) : nullptr;
  if (tc_reverse && !fcon) return fail(ctx, DG_ERR_OOM, "dg_adjoint_step: device allocation failed (face constants)");
  // stage states u_s and the E components of the stage right-hand sides A u_s of one segment
  float *US = ws.get<float>(10, fl * 5 * C), *RS = ws.get<float>(11, hfl * 5 * C);
  if (!u || !nxt || !res || !lu || !lr || !g || !g2 || !resid || !Jd || !grad || !ck || !US || !RS)
    return fail(ctx, DG_ERR_OOM, "dg_adjoint_step: device allocation failed (checkpoints and one segment of stage "
                                 "states are kept in device memory)");
  // the second segment buffer and the recompute stream's scratch; without
  // them (no memory, no stream) the segments are recomputed in turn on the
  // caller's stream
  float *USb[2] = {US, nullptr}, *RSb[2] = {RS, nullptr}, *res2 = nullptr, *nxt2 = nullptr;
  bool overlap = nseg > 1 && ws.streams_ready();
  if (overlap) {
    USb[1] = ws.get<float>(12, fl * 5 * C);
    RSb[1] = ws.get<float>(13, hfl * 5 * C);
    res2 = ws.get<float>(14, fl);
    nxt2 = ws.get<float>(15, fl);
    overlap = USb[1] && RSb[1] && res2 && nxt2;
  }
  if (!overlap) USb[1] = US, RSb[1] = RS, res2 = res, nxt2 = nxt;
  cudaError_t e = cudaMemcpyAsync(u, u0, fl * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(res, 0, fl * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Jd, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, ctx->K * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(lu, 0, fl * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(lr, 0, fl * 4, s);
  StageArgs sa = stage_base(ctx, alpha, dt);
  const unsigned rb = unsigned((3 * R + 255) / 256);

  // one step of the stored form on stream `st_`: every stage state and the E
  // components of its right-hand side go to segment buffer b (state j of the
  // segment that starts at checkpoint sg); returns the state after the step
  auto stored_step = [&](int n, int n0, int sg, int b, cudaStream_t st_, float *res_, float *nxt_) -> const float * {
    StageArgs q = sa;
    q.res = res_;
    for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
      const size_t j = size_t(n - n0) * 5 + st;
      q.u = j == 0 ? ck + fl * sg : USb[b] + fl * j;
      q.u_out = (j + 1 < size_t(5) * C) ? USb[b] + fl * (j + 1) : nxt_;
      q.rhs = RSb[b] + hfl * j;
      q.rk_a = float(kLserkA[st]);
      q.rk_b = float(kLserkB[st]);
      e = forward_stage(ctx, MODE_LSERK_STORE, q, st_);
    }
    const size_t jn = size_t(n - n0 + 1) * 5;
    return jn < size_t(5) * C ? USb[b] + fl * jn : nxt_;
  };

  // ---- forward sweep: checkpoints at the segment starts, the last segment
  // stored (the last two when both segment buffers exist), and the receiver
  // residuals
  const int n0_stored = seg_start(overlap && nseg >= 2 ? nseg - 2 : nseg - 1);
  for (int n = 0, sg = 0; n < nsteps && e == cudaSuccess; ++n) {
    if (n == seg_start(sg)) {
      e = cudaMemcpyAsync(ck + fl * sg, u, fl * 4, cudaMemcpyDeviceToDevice, s);
      ++sg;
    }
    const float *after = u;
    if (n >= n0_stored) {
      // step n belongs to segment sg - 1, which starts from its checkpoint copy
      after = stored_step(n, seg_start(sg - 1), sg - 1, (sg - 1) % 2, s, res, nxt);
      if (sg < nseg && n + 1 == seg_start(sg)) {
        // the state after the segment is the next checkpoint's source
        if (e == cudaSuccess && after != u) e = cudaMemcpyAsync(u, after, fl * 4, cudaMemcpyDeviceToDevice, s);
      }
    } else {
      sa.res = res;
      for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
        sa.u = u;
        sa.u_out = nxt;
        sa.rk_a = float(kLserkA[st]);
        sa.rk_b = float(kLserkB[st]);
        e = forward_stage(ctx, MODE_LSERK, sa, s);
        std::swap(u, nxt);
      }
      after = u;
    }
    if (e == cudaSuccess) {
      k_recv_residual<<<rb, 256, 0, s>>>(after, ctx->K, ctx->ops.Np, ctx->ops.Npad, recv, R, Eref + int64_t(n) * 3 * R,
                                         resid + int64_t(n) * 3 * R, Jd);
      e = cudaGetLastError();
    }
  }

  // ---- reverse sweep, segment by segment
  AdjArgs aa = adj_base(ctx, alpha);
  aa.grad = grad;
  aa.dt = float(dt);
  if (tc_reverse && e == cudaSuccess) {
    aa.fcon = fcon;
    e = launch_adj_face_consts(ctx, fcon, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), s);
  }
  auto reverse_stage = [&](const AdjArgs &x) {
    return tc_reverse ? launch_adj_tc(ctx, x, s) : launch_adj(ctx->N, 1, x, s);
  };
  bool lifted = false; // the lift of the step's last stage already ran in the previous volume kernel
  float *gcur = g, *gnext = g2;
  // with two segment buffers, segment seg lives in buffer seg % 2, and the
  // segment before it is recomputed on the second stream while seg is reversed
  if (overlap && e == cudaSuccess) e = cudaEventRecord(ws.ev_fwd, s);
  if (overlap && e == cudaSuccess) e = cudaStreamWaitEvent(ws.s2, ws.ev_fwd, 0);
  for (int seg = nseg - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int n0 = seg_start(seg), n1 = seg + 1 < nseg ? seg_start(seg + 1) : nsteps;
    const int b = seg % 2;
    if (overlap) {
      // segment seg - 1 into the buffer that the reverse sweep of seg + 1 has released
      if (seg >= 1) {
        if (seg + 1 < nseg) e = cudaStreamWaitEvent(ws.s2, ws.ev_rev[(seg + 1) % 2], 0);
        const int p0 = seg_start(seg - 1);
        // (the segment before the last one was stored by the forward sweep)
        if (p0 < n0_stored)
          for (int n = p0; n < n0 && e == cudaSuccess; ++n) stored_step(n, p0, seg - 1, (seg - 1) % 2, ws.s2, res2, nxt2);
        if (e == cudaSuccess) e = cudaEventRecord(ws.ev_rec[(seg - 1) % 2], ws.s2);
      }
      if (seg < nseg - 1 && e == cudaSuccess) e = cudaStreamWaitEvent(s, ws.ev_rec[b], 0);
    } else if (seg < nseg - 1) {
      // recompute the segment from its checkpoint (the last one is already stored)
      for (int n = n0; n < n1 && e == cudaSuccess; ++n) stored_step(n, n0, seg, b, s, res, nxt);
    }
    for (int n = n1 - 1; n >= n0 && e == cudaSuccess; --n) {
      if (!lifted) {
        // the run's last step: its receiver source, then its last stage's lift on its own
        k_recv_source<<<rb, 256, 0, s>>>(lu, ctx->K, ctx->ops.Np, ctx->ops.Npad, recv, R, resid + int64_t(n) * 3 * R);
        e = cudaGetLastError();
        aa.lr_in = lr;
        aa.lu_in = lu;
        aa.lr_out = lr;
        aa.b = float(kLserkB[4]);
        aa.lr_scale = 1.f; // lr is still zero
        aa.g = gcur;
        aa.g_next = nullptr;
        if (e == cudaSuccess) e = launch_adj(ctx->N, 0, aa, s); // lr = pending lr + b lu; g = Fscale LIFT^T W lr
      }
      for (int st = 4; st >= 0 && e == cudaSuccess; --st) {
        const size_t j = size_t(n - n0) * 5 + st;
        aa.lr_in = lr;
        aa.lu_in = lu;
        aa.lu_out = lu;
        aa.g = gcur;
        aa.u_s = j == 0 ? ck + fl * seg : USb[b] + fl * j;
        aa.rhs_s = RSb[b] + hfl * j;
        if (st > 0 || n > 0) {
          // lu += dt A^T lr; grad; then the lift of the stage reversed next,
          // lr = a_st lr + b_next lu and g_next: stage st - 1, or the last stage
          // of step n - 1. That step's receiver source goes into lu first: it
          // and this stage's update both only add to lu
          if (st == 0) {
            k_recv_source<<<rb, 256, 0, s>>>(lu, ctx->K, ctx->ops.Np, ctx->ops.Npad, recv, R,
                                             resid + int64_t(n - 1) * 3 * R);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
          }
          aa.lr_out = lr;
          aa.a = float(kLserkA[st]);
          aa.b_next = float(kLserkB[st > 0 ? st - 1 : 4]);
          aa.g_next = gnext;
          e = reverse_stage(aa);
          std::swap(gcur, gnext);
          lifted = st == 0;
        } else {
          // the run's first stage: nothing to lift after it
          aa.lr_out = nullptr;
          aa.g_next = nullptr;
          e = reverse_stage(aa); // lu += dt A^T lr; grad
        }
      }
    }
    if (overlap && e == cudaSuccess) e = cudaEventRecord(ws.ev_rev[b], s);
  }
  // the second stream's work is all ordered before the last reverse sweep;
  // after an error it may still run, so it is drained before returning
  if (overlap) {
    const cudaError_t e2 = cudaStreamSynchronize(ws.s2);
    if (e == cudaSuccess) e = e2;
  }
  double Jh = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&Jh, Jd, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && dJ_deps) e = cudaMemcpyAsync(dJ_deps, grad, ctx->K * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && dJ_du0) e = cudaMemcpyAsync(dJ_du0, lu, fl * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_adjoint_step: ") + cudaGetErrorString(e));
  if (tc_reverse) {
    // a bounded device wait of the tensor-core reverse stage that ran out
    int flag = 0, zero = 0;
    e = cudaMemcpy(&flag, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemcpy(ctx->d_flag + 1, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_adjoint_step: ") + cudaGetErrorString(e));
    if (flag) return fail(ctx, DG_ERR_TIMEOUT, "dg_adjoint_step: a device wait of the reverse sweep timed out");
  }
  if (J) *J = Jh;
  if (!std::isfinite(Jh)) return fail(ctx, DG_ERR_NONFINITE, "dg_adjoint_step: misfit is not finite");
  return DG_OK;
}

int dg_set_adjoint_form(dg_ctx *ctx, int form) {
  if (!ctx) return DG_ERR_ARG;
  if (form != 0 && form != 1) return fail(ctx, DG_ERR_ARG, "dg_set_adjoint_form: form must be 0 or 1");
  if (form == 1 && !adj_tc_supported(ctx))
    return fail(ctx, DG_ERR_UNSUPPORTED, "dg_set_adjoint_form: the tensor-core form needs N <= 5 and a GB300");
  ctx->adj_form = form;
  return DG_OK;
}

int dg_adjoint_form(const dg_ctx *ctx) {
  if (!ctx) return -1;
  return ctx->adj_form != 0 && adj_tc_supported(ctx) ? 1 : 0;
}

} // extern "C"
