// Tensor-core form of the adjoint's reverse volume stage (sm_103a, N <= 5).
//
// One reverse stage adds dt A^T lambda_r to lambda_u (A = A(eps), the
// semi-discrete operator of eq. semidiscrete-dg), accumulates the eps
// gradient, and runs the lift of the stage reversed next (see adjoint.cu for
// the recursion). Its two dense contractions are the transposes of the
// forward stage's (Section 2, Fig. el-local-ops: the element-local operators
// applied to many elements at once as matrix-matrix products), and run here
// on the tensor cores in the FP16x3 split of the forward kernels (hi*hi +
// hi*lo + lo*hi, FP32 accumulation in tensor memory, one power-of-two scale
// per operand row):
//   GEMM-D  T[(e,f), (d,j)] = sum_i (W lr)[(e,f), i] D_d[i, j]     (d = r, s, t)
//   GEMM-L  G[(e,f), m]     = sum_i (W lr')[(e,f), i] LIFT[i, m]
// with W = diag(1/eps, 1/mu) and the rows (element, field) of a tile of 20
// elements (5 per 32-lane TMEM quarter, as in the forward kernels). The
// transposed curl then has the form of the forward curl applied to T: the
// physical combinations sum_d (dr_d/dx_l) T_d of the rows of an element are
// exchanged between its six field lanes with warp shuffles, E rows taking
// P_{c+1}(H_{c+2}) - P_{c+2}(H_{c+1}) and H rows the negative of the same
// with the E rows (the transpose of the curl is the curl with the derivative
// operators transposed). The transposed flux and the impedance-weight terms
// of the eps gradient stay on the CUDA cores (gathers of the neighbours' face
// data and stage traces), as in the CUDA-core form, whose device arithmetic
// (adj_common.cuh) they share.
//
// Per tile (up to 20 elements: 19 at N = 3, 4 and 18 at N = 5, so that the
// face loop takes whole rounds of the block's threads): the tile's lambda_r,
// lambda_u, the E rows of the stage's right-hand side, its face data and
// per-face constants arrive by bulk copies (requested during the previous
// tile); W lr is split into the A operand of GEMM-D in tensor memory; while
// GEMM-D runs, the face loop scatters the transposed flux into a shared-memory
// buffer; the epilogue forms lambda_u + dt (curl^T + flux^T), the next stage's
// lambda_r = a lambda_r + b_next lambda_u and its split W lr' (over the
// columns of T, which have been read); GEMM-L lifts it, and the face data
// g_next = Fscale G go to global memory. Two blocks per SM at N <= 4 overlap
// each other's phases. Waits are bounded; a wait that runs out sets the
// context's device flag and the block leaves.
#include <cuda_fp16.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/dgmx.h"
#include "adj_common.cuh"
#include "flux.cuh"
#include "tc_common.cuh"
#include "umma.cuh"

namespace dgmx {

namespace {

using namespace tcc;
using namespace adj;

constexpr int kAdjTile = 20; // 4 TMEM lane quarters x 5 elements

template <int N>
struct AT {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NPP = D::NPP, NFP = D::NFP, NFF = D::NFF;
  static constexpr int K1 = rup(NP, 16); // reduction length of both products (volume nodes i)
  static constexpr int NB = K1;          // T columns per derivative direction
  static constexpr int N1 = 3 * NB;      // GEMM-D output columns
  static constexpr int NL = rup(NFF, 16); // GEMM-L output columns (face nodes m)
  // tensor memory: T in [0, N1), G in [N1, N1 + NL); GEMM-D's A operand (W lr,
  // hi then lo, K1 columns) sits in G's columns, which GEMM-L writes only after
  // GEMM-D has completed; GEMM-L's A operand (W lr') sits in T's columns, which
  // the epilogue has read by then
  static constexpr int CT = 0, CG = N1, CAD = CG, CAL = CT;
  static constexpr int TCOLS = tmem_cols(N1 + NL);
  static_assert(K1 <= NL && K1 <= N1, "an A operand must fit in the columns it borrows");
  static_assert(N1 <= 256 && NL <= 256, "one N chunk per product");
  static_assert(N1 + NL <= 512, "accumulators exceed tensor memory");
  // threads per operand row: each takes 16 K values of the split (at least 2)
  static constexpr int PARTS = K1 / 16 > 2 ? K1 / 16 : 2;
  static constexpr int NT = 128 * PARTS;
  static constexpr int MINB = (N <= 4 && TCOLS <= 256) ? 2 : 1; // blocks per SM aimed at
  static constexpr int NCH = (NP + 7) / 8;                      // 8-node chunks of a row
  static constexpr int CPP = (NCH + PARTS - 1) / PARTS;        // chunks per part
  static constexpr int GCH = NL / 8;                            // 8-column chunks of G
  static constexpr int GPP = (GCH + PARTS - 1) / PARTS;
  // elements per tile: at most the 20 rows' worth, fewer where that makes the
  // face loop (4 Nfp items per element over NT threads) one round shorter
  static constexpr int R20 = (kAdjTile * NFF + NT - 1) / NT;
  static constexpr int TE_FIT = R20 > 1 ? (R20 - 1) * NT / NFF : kAdjTile;
  static constexpr int TE = TE_FIT >= 17 && TE_FIT < kAdjTile ? TE_FIT : kAdjTile;
  static constexpr int FS = kAdjTile * NPP + 4; // padded field-block stride of the staged tiles
  static constexpr int B1B = N1 * K1 * 2, B2B = NL * K1 * 2;
  static constexpr int OPS = 2 * B1B + 2 * B2B; // D^T blocks hi, lo, then LIFT^T blocks hi, lo
  static constexpr int OFF_B1H = 0, OFF_B1L = B1B, OFF_B2H = 2 * B1B, OFF_B2L = 2 * B1B + B2B;
  static constexpr int TB = rup(6 * FS * 4, 128);
  static constexpr int OFF_LR = rup(OPS, 128); // fp32 [6][FS] lambda_r of the tile
  static constexpr int OFF_LU = OFF_LR + TB;   // fp32 [6][FS] lambda_u of the tile
  static constexpr int OFF_W = OFF_LU + TB;    // fp32 [6][FS] transposed-flux contributions
  static constexpr int OFF_RS = OFF_W + TB;    // fp32 [3][FS] E rows of the stage's right-hand side
  static constexpr int OFF_FACE = OFF_RS + rup(3 * FS * 4, 128); // float4 [80][4] per-face constants
  static constexpr int OFF_FG = OFF_FACE + kAdjTile * 4 * 64; // float4 [80] {n, Fscale}
  static constexpr int OFF_GEO = OFF_FG + kAdjTile * 4 * 16;  // float [20][G_STRIDE]
  static constexpr int OFF_TAB = OFF_GEO + kAdjTile * G_STRIDE * 4;
  // u32 [128] row maxima, float [128] inverse row scales, float [20] gradient partials
  static constexpr int OFF_MX = OFF_TAB + rup(NFF + 2 * kConnKinds * NFP, 16);
  static constexpr int OFF_BAR = OFF_MX + 2 * 128 * 4 + rup(kAdjTile, 4) * 4; // barS, barF, barD, barL; TMEM slot
  static constexpr int SMEM = OFF_BAR + 48;
  static_assert(SMEM <= 232448, "the reverse tile does not fit in shared memory");
};

// Optional phase timestamps (build with -DDGMX_STAGE_TIMING; off in the
// library): thread 0's SM clock in cycles since the block passed its setup, at
// the phase boundaries of each tile (slots 0-9), per block and tile, of the
// last launch with a fused lift, read back with dgmx_adj_trace()
// (stage_timing.py prints the breakdown).
constexpr int kAdjTraceTiles = 16, kAdjTraceBlocks = 320, kAdjEvents = 12;
#ifdef DGMX_STAGE_TIMING
__device__ uint32_t g_adj_trace[kAdjTraceBlocks * kAdjTraceTiles * kAdjEvents];
#define AT_MARK(ev)                                                                                                 \
  do {                                                                                                              \
    if (fuse && tid == 0 && itn < kAdjTraceTiles && blockIdx.x < kAdjTraceBlocks)                                   \
      g_adj_trace[(blockIdx.x * kAdjTraceTiles + itn) * kAdjEvents + (ev)] = uint32_t(clock64() - at_t0);           \
  } while (0)
#else
#define AT_MARK(ev) \
  do {              \
  } while (0)
#endif

template <int N>
__global__ void __launch_bounds__(AT<N>::NT, AT<N>::MINB)
    k_adj_tc(AdjArgs a, const uint4 *__restrict__ ops, int ntiles, long long wait_limit, int *err_flag) {
  using T = AT<N>;
  constexpr int NP = T::NP, NPP = T::NPP, NFP = T::NFP, NFF = T::NFF, FS = T::FS, NT = T::NT, NB = T::NB;
  constexpr int K1 = T::K1, CPP = T::CPP, NCH = T::NCH, GPP = T::GPP, GCH = T::GCH;
  extern __shared__ __align__(1024) uint8_t smem[];
  float *s_lr = reinterpret_cast<float *>(smem + T::OFF_LR);
  float *s_lu = reinterpret_cast<float *>(smem + T::OFF_LU);
  float *s_w = reinterpret_cast<float *>(smem + T::OFF_W);
  float *s_rs = reinterpret_cast<float *>(smem + T::OFF_RS);
  float4 *s_face = reinterpret_cast<float4 *>(smem + T::OFF_FACE);
  const float4 *s_fg = reinterpret_cast<const float4 *>(smem + T::OFF_FG);
  const float *s_geo = reinterpret_cast<const float *>(smem + T::OFF_GEO);
  uint8_t *s_fm = smem + T::OFF_TAB;
  uint8_t *s_nb = s_fm + NFF, *s_nf = s_nb + kConnKinds * NFP;
  uint32_t *s_rmx = reinterpret_cast<uint32_t *>(smem + T::OFF_MX); // row maxima (float bits)
  float *s_inv = reinterpret_cast<float *>(s_rmx + 128);            // inverse row scales (compact rows)
  float *s_gr = s_inv + 128;                                         // eps-gradient partial per element
  uint64_t *barS = reinterpret_cast<uint64_t *>(smem + T::OFF_BAR);  // the tile's lambda rows staged
  uint64_t *barF = barS + 1;                                         // its face and element data staged
  uint64_t *barD = barS + 2, *barL = barS + 3;                       // GEMM-D, GEMM-L done
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + T::OFF_BAR + 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = tid == NT - 32;
  const int64_t KN = a.K * NPP;
  const uint32_t sbase = umma::smem_u32(smem);
  const long long wlim = umma::wait_cycles(wait_limit);
  const bool fuse = a.g_next != nullptr, grad = a.u_s != nullptr;

  // ---- one-time setup: operators, node tables, barriers, tensor memory
  for (int i = tid; i < T::OPS / 16; i += NT) reinterpret_cast<uint4 *>(smem)[i] = __ldg(ops + i);
  for (int i = tid; i < NFF + 2 * kConnKinds * NFP; i += NT)
    s_fm[i] = i < NFF ? a.fmask[i] : i < NFF + kConnKinds * NFP ? a.nbrtab[i - NFF] : a.nbrface[i - NFF - kConnKinds * NFP];
  for (int i = tid; i < 6 * FS; i += NT) s_w[i] = 0.f;
  for (int i = tid; i < 128; i += NT) s_rmx[i] = 0u, s_inv[i] = 1.f;
  for (int i = tid; i < kAdjTile; i += NT) s_gr[i] = 0.f;
  if (tid == 0) {
    umma::mbar_init(barS, 1);
    umma::mbar_init(barF, 1);
    umma::mbar_init(barD, 1);
    umma::mbar_init(barL, 1);
    umma::fence_mbar_init();
  }
  if (warp == 0) umma::tmem_alloc(tslot, T::TCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  pdl_wait(); // lambda and the face data of the previous reverse stage from here on

  // operand row of this thread (= TMEM lane of its warp's quarter) and the
  // 16 K values it splits; the epilogue's view of the same row
  const int q4 = warp & 3, part = warp >> 2;
  const int r = 32 * q4 + lane;
  const bool lane_used = lane < 30;
  const int ep = lane_used ? lane / 6 : 4;
  const int fld = lane_used ? lane % 6 : 5;
  const int comp = fld % 3;
  const bool isE = fld < 3;
  const float sgn = isE ? 1.f : -1.f;
  const int src1 = ep * 6 + (isE ? 3 : 0) + (comp + 2) % 3;
  const int src2 = ep * 6 + (isE ? 3 : 0) + (comp + 1) % 3;
  const int dl1 = (comp + 2) % 3, dl2 = (comp + 1) % 3;
  const int e_loc = q4 * 5 + ep;
  const int ridx = e_loc * 6 + fld; // compact row (lanes 30, 31 alias a real row and write nothing)
  const int soff = fld * FS + e_loc * NPP;
  const int kb = 16 * part;
  const bool apart = kb < K1;
  const uint32_t lane_taddr = tmem + (uint32_t(q4 * 32) << 16);
  const int ch0 = part * CPP, ch1 = (part + 1) * CPP < NCH ? (part + 1) * CPP : NCH;
  const int gc0 = part * GPP, gc1 = (part + 1) * GPP < GCH ? (part + 1) * GPP : GCH;

  // the bulk copies of tile t (one thread): lambda_r and lambda_u rows on
  // barS, face and element data on barF; the next tile's rows are requested as
  // soon as the epilogue has read this tile's, its face data at the tile's end
  auto stage_rows = [&](int t) {
    const int64_t kb = int64_t(t) * T::TE;
    const uint32_t nb = uint32_t(a.K - kb < T::TE ? a.K - kb : T::TE), bytes = nb * NPP * 4u;
    umma::mbar_arrive_expect_tx(barS, (grad ? 15u : 12u) * bytes);
    for (int f = 0; f < 6; ++f) {
      umma::bulk_g2s(s_lr + f * FS, a.lr_in + f * KN + kb * NPP, bytes, barS);
      umma::bulk_g2s(s_lu + f * FS, a.lu_in + f * KN + kb * NPP, bytes, barS);
    }
    if (grad)
      for (int f = 0; f < 3; ++f) umma::bulk_g2s(s_rs + f * FS, a.rhs_s + f * KN + kb * NPP, bytes, barS);
  };
  auto stage_faces = [&](int t) {
    const int64_t kb = int64_t(t) * T::TE;
    const uint32_t nb = uint32_t(a.K - kb < T::TE ? a.K - kb : T::TE);
    umma::mbar_arrive_expect_tx(barF, nb * (64u + G_STRIDE * 4u + 256u));
    umma::bulk_g2s(smem + T::OFF_FG, a.fgeo + kb * 4, nb * 64u, barF);
    umma::bulk_g2s(smem + T::OFF_GEO, a.geo + kb * G_STRIDE, nb * G_STRIDE * 4u, barF);
    umma::bulk_g2s(s_face, a.fcon + kb * 16, nb * 256u, barF);
  };
  if (tid == 0 && int(blockIdx.x) < ntiles) {
    stage_rows(blockIdx.x);
    stage_faces(blockIdx.x);
  }

  uint32_t phase = 0;
  bool failed = false;
#ifdef DGMX_STAGE_TIMING
  const long long at_t0 = clock64();
#endif
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#ifdef DGMX_STAGE_TIMING
    const int itn = (tile - int(blockIdx.x)) / int(gridDim.x);
#endif
    AT_MARK(0);
    if (tile + int(gridDim.x) >= ntiles) pdl_launch_next(); // this block's last tile
    const int64_t k0 = int64_t(tile) * T::TE;
    const int ne = int(a.K - k0 < T::TE ? a.K - k0 : T::TE);
    const bool live = lane_used && e_loc < ne;

    const bool more = tile + int(gridDim.x) < ntiles;
    // ---- A. the tile's lambda_r, lambda_u, face and element data (bulk copies
    // requested during the previous tile)
    const bool okS = umma::mbar_wait_bounded(barS, phase, wlim) && umma::mbar_wait_bounded(barF, phase, wlim);
    if (__syncthreads_or(!okS)) {
      if (tid == 0) {
        atomicExch(err_flag, 1);
        // the copies in flight land before the block leaves
        umma::mbar_wait_bounded(barS, phase);
        umma::mbar_wait_bounded(barF, phase);
      }
      failed = true;
      break;
    }
    AT_MARK(1);

    // ---- B. W lr split into GEMM-D's A operand; the 1/eps term of the
    // gradient, -<W lr_E, rhs_E>
    float vv[16];
    {
      const float w = live ? s_geo[e_loc * G_STRIDE + (isE ? G_IEPS : G_IMU)] : 0.f;
      float mx = 0.f, gpart = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = kb + j;
        vv[j] = (apart && live && k < NP) ? s_lr[soff + k] * w : 0.f;
        mx = fmaxf(mx, fabsf(vv[j]));
      }
      if (apart && live) {
        atomicMax(s_rmx + r, __float_as_uint(mx));
        if (grad && isE) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            if (kb + j < NPP) {
              const float4 rs = *reinterpret_cast<const float4 *>(s_rs + soff + kb + j);
              gpart -= vv[j] * rs.x + vv[j + 1] * rs.y + vv[j + 2] * rs.z + vv[j + 3] * rs.w;
            }
          }
          if (gpart != 0.f) atomicAdd(s_gr + e_loc, gpart);
        }
      }
    }
    __syncthreads();
    if (apart) {
      float sc = 1.f, inv = 1.f;
      if (lane_used) row_scale(__uint_as_float(s_rmx[r]), sc, inv);
      if (part == 0 && lane_used) s_inv[ridx] = inv;
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 x = f2mul(make_float2(vv[2 * j], vv[2 * j + 1]), f2(sc));
        split2<false>(x.x, x.y, hi[j], lo[j]);
      }
      umma::tmem_st8(lane_taddr + uint32_t(T::CAD + 8 * part), hi);
      umma::tmem_st8(lane_taddr + uint32_t(T::CAD + K1 / 2 + 8 * part), lo);
      umma::tmem_wait_st();
    }
    umma::fence_before_sync();
    __syncthreads();
    if (tid < 128) s_rmx[tid] = 0u; // read above; the epilogue's maxima come after the face loop's barrier
    AT_MARK(2);

    // ---- C. GEMM-D on the tensor cores (asynchronous, overlapping the face loop)
    if (issuer) {
      umma::fence_after_sync();
      issue_split_gemm_ta<false, K1, T::N1>(tmem + uint32_t(T::CT), tmem + uint32_t(T::CAD),
                                            tmem + uint32_t(T::CAD + K1 / 2), sbase + T::OFF_B1H, sbase + T::OFF_B1L);
      umma::commit(barD);
    }

    // ---- D. transposed flux Jacobians (interior side with the element's own
    // g, exterior side with the neighbour's g at the matching face node) into
    // s_w, and the impedance-weight terms of the gradient; one face node per
    // item, whole rounds (every lane takes part in the per-element sums)
    for (int it0 = 0; it0 < ne * NFF; it0 += NT) {
      const int it = it0 + tid;
      const int e = (it < ne * NFF ? it : ne * NFF - 1) / NFF, fm = it - e * NFF, f = fm / NFP, m = fm - f * NFP;
      const int64_t k = k0 + e;
      float contrib = 0.f;
      if (it < ne * NFF) {
        const float4 *fr = s_face + (e * 4 + f) * 4;
        const float4 r0 = fr[0], r1 = fr[1], r2 = fr[2], r3 = fr[3];
        const float n[3] = {r0.x, r0.y, r0.z};
        const float zs = r0.w, Zk = r1.x, Z2 = r1.y, Yk = r1.z, Y2 = r1.w, ys = r2.x;
        const int cny = __float_as_int(r2.w);
        const int64_t k2 = __float_as_int(r3.x);
        const bool wall = __float_as_int(r3.y) != 0;
        const int vm = s_fm[fm];
        const int fm2 = wall ? 0 : s_nf[cny * NFP + m] + (cny / 6 % 4) * NFP;
        const int vn = wall ? 0 : s_nb[cny * NFP + m];
        // every global load of the item first, all in flight together: the
        // own and the neighbour's face data, the stage's own and exterior traces
        float gk[6], g2[6], qm[6], qp[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) gk[c] = a.g[(c * a.K + k) * NFF + fm];
#pragma unroll
        for (int c = 0; c < 6; ++c) g2[c] = wall ? 0.f : a.g[(c * a.K + k2) * NFF + fm2];
        if (grad) {
#pragma unroll
          for (int c = 0; c < 6; ++c) qm[c] = __ldg(a.u_s + c * KN + k * NPP + vm);
#pragma unroll
          for (int c = 0; c < 6; ++c) qp[c] = wall ? 0.f : __ldg(a.u_s + c * KN + k2 * NPP + vn);
        }
        float ep3[3], hp3[3], acc[6];
        flux_transpose_w(n, gk, Z2, Y2, zs, ys, a.alpha, ep3, hp3);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          acc[c] = -ep3[c];
          acc[c + 3] = -hp3[c];
        }
        if (wall) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[c] -= ep3[c];
            acc[c + 3] += hp3[c];
          }
        } else {
          const float n2[3] = {-n[0], -n[1], -n[2]};
          float ep2[3], hp2[3];
          flux_transpose_w(n2, g2, Zk, Yk, zs, ys, a.alpha, ep2, hp2);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[c] += ep2[c];
            acc[c + 3] += hp2[c];
          }
        }
        if (grad) {
          const float dZ = r2.y, dY = r2.z;
          if (wall) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              qp[c] = -qm[c];
              qp[c + 3] = qm[c + 3];
            }
          }
          float sZm, sZp, sYm, sYp;
          flux_weight_partials_w(n, qm, qp, Z2, Y2, zs, ys, a.alpha, gk, sZm, sZp, sYm, sYp);
          contrib = sZm * dZ + sYm * dY;
          if (wall) {
            contrib += sZp * dZ + sYp * dY;
          } else {
            const float n2[3] = {-n[0], -n[1], -n[2]};
            float tZm, tZp, tYm, tYp;
            flux_weight_partials_w(n2, qp, qm, Zk, Yk, zs, ys, a.alpha, g2, tZm, tZp, tYm, tYp);
            contrib += tZp * dZ + tYp * dY;
          }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) atomicAdd(&s_w[c * FS + e * NPP + vm], acc[c]);
      }
      if (grad) add_by_element(s_gr, e, contrib);
    }
    __syncthreads();
    AT_MARK(3);

    // ---- E. epilogue: transposed curl from T (the row's FP16 scale undone
    // through the metric factors), plus the transposed flux; lambda_u updated;
    // with the next lift fused in, lambda_r = a lambda_r + b_next lambda_u and
    // W lambda_r kept for its split
    float g1r = 0.f, g1s = 0.f, g1t = 0.f, g2r = 0.f, g2s = 0.f, g2t = 0.f, wrow = 0.f;
    {
      const float *ge = s_geo + (live ? e_loc : 0) * G_STRIDE;
      const float inv = s_inv[lane_used ? ridx : 0];
      g1r = ge[G_RX + dl1] * inv, g1s = ge[G_SX + dl1] * inv, g1t = ge[G_TX + dl1] * inv;
      g2r = ge[G_RX + dl2] * inv, g2s = ge[G_SX + dl2] * inv, g2t = ge[G_TX + dl2] * inv;
      wrow = ge[isE ? G_IEPS : G_IMU];
    }
    const bool okD = umma::mbar_wait_bounded(barD, phase, wlim);
    if (__syncthreads_or(!okD)) {
      if (tid == 0) {
        atomicExch(err_flag, 1);
        umma::mbar_wait_bounded(barD, phase); // the products in flight end before tensor memory is released
      }
      failed = true;
      break;
    }
    AT_MARK(4);
    umma::fence_after_sync();
    float wl[CPP][8];
    float mx2 = 0.f;
#pragma unroll
    for (int c = 0; c < CPP; ++c) {
      const int ch = ch0 + c;
#pragma unroll
      for (int n = 0; n < 8; ++n) wl[c][n] = 0.f;
      if (ch >= ch1) break;
      const int i0 = ch * 8;
      float tr[8], ts[8], tt[8];
      umma::tmem_ld8(lane_taddr + uint32_t(T::CT + i0), tr);
      umma::tmem_ld8(lane_taddr + uint32_t(T::CT + NB + i0), ts);
      umma::tmem_ld8(lane_taddr + uint32_t(T::CT + 2 * NB + i0), tt);
      umma::tmem_wait_ld();
      umma::reg_fence8(tr);
      umma::reg_fence8(ts);
      umma::reg_fence8(tt);
      float vol[8];
#pragma unroll
      for (int n = 0; n < 8; n += 2) {
        const float2 r2 = make_float2(tr[n], tr[n + 1]), s2 = make_float2(ts[n], ts[n + 1]),
                     t2 = make_float2(tt[n], tt[n + 1]);
        const float2 p1 = f2fma(f2(g1t), t2, f2fma(f2(g1s), s2, f2mul(f2(g1r), r2)));
        const float2 p2 = f2fma(f2(g2t), t2, f2fma(f2(g2s), s2, f2mul(f2(g2r), r2)));
        const float2 v1 = make_float2(__shfl_sync(0xffffffffu, p1.x, src1), __shfl_sync(0xffffffffu, p1.y, src1));
        const float2 v2 = make_float2(__shfl_sync(0xffffffffu, p2.x, src2), __shfl_sync(0xffffffffu, p2.y, src2));
        const float2 d = f2sub(v1, v2);
        vol[n] = d.x;
        vol[n + 1] = d.y;
      }
      if (live) {
        const int64_t goff = fld * KN + (k0 + e_loc) * NPP;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = i0 + 4 * h;
          if (i < NPP) {
            const float4 sw4 = *reinterpret_cast<const float4 *>(s_w + soff + i);
            // read once: cleared here for the next tile (entries no live row reads are never written)
            *reinterpret_cast<float4 *>(s_w + soff + i) = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 lu4 = *reinterpret_cast<const float4 *>(s_lu + soff + i);
            const float4 lr4 = *reinterpret_cast<const float4 *>(s_lr + soff + i);
            const float swv[4] = {sw4.x, sw4.y, sw4.z, sw4.w}, luv[4] = {lu4.x, lu4.y, lu4.z, lu4.w},
                        lrv[4] = {lr4.x, lr4.y, lr4.z, lr4.w};
            float o[4], p[4];
#pragma unroll
            for (int n = 0; n < 4; ++n) {
              const int j = 4 * h + n;
              const float wv = fmaf(sgn, vol[j], swv[n]);
              o[n] = (i + n < NP) ? fmaf(a.dt, wv, luv[n]) : 0.f;
              p[n] = (i + n < NP) ? fmaf(a.b_next, o[n], lrv[n] * a.a) : 0.f;
              wl[c][j] = p[n] * wrow;
              mx2 = fmaxf(mx2, fabsf(wl[c][j]));
            }
            *reinterpret_cast<float4 *>(a.lu_out + goff + i) = make_float4(o[0], o[1], o[2], o[3]);
            if (fuse) *reinterpret_cast<float4 *>(a.lr_out + goff + i) = make_float4(p[0], p[1], p[2], p[3]);
          }
        }
      }
    }
    if (fuse && live) atomicMax(s_rmx + r, __float_as_uint(mx2));
    umma::fence_proxy_async(); // the lambda rows were read: the next tile's copies may overwrite them
    umma::fence_before_sync();
    __syncthreads(); // T has been read; the row maxima of W lambda_r are complete
    AT_MARK(5);
    if (tid == 0 && more) stage_rows(tile + gridDim.x);

    // ---- F. the fused lift: W lambda_r split over T's columns, GEMM-L, and
    // g_next = Fscale * G
    if (fuse) {
      float sc = 1.f, inv = 1.f;
      if (lane_used) row_scale(__uint_as_float(s_rmx[r]), sc, inv);
      if (part == 0 && lane_used) s_inv[ridx] = inv;
#pragma unroll
      for (int c = 0; c < CPP; ++c) {
        const int ch = ch0 + c;
        if (ch >= ch1) break;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 x = f2mul(make_float2(wl[c][2 * j], wl[c][2 * j + 1]), f2(sc));
          split2<false>(x.x, x.y, hi[j], lo[j]);
        }
        umma::tmem_st4(lane_taddr + uint32_t(T::CAL + 4 * ch), hi);
        umma::tmem_st4(lane_taddr + uint32_t(T::CAL + K1 / 2 + 4 * ch), lo);
      }
      if (part == T::PARTS - 1) {
        // K columns past the last node chunk: zeros (T's old values must not enter the products)
        const uint32_t z[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int ch = NCH; ch < K1 / 8; ++ch) {
          umma::tmem_st4(lane_taddr + uint32_t(T::CAL + 4 * ch), z);
          umma::tmem_st4(lane_taddr + uint32_t(T::CAL + K1 / 2 + 4 * ch), z);
        }
      }
      umma::tmem_wait_st();
      umma::fence_before_sync();
      __syncthreads();
      AT_MARK(6);
      if (issuer) {
        umma::fence_after_sync();
        issue_split_gemm_ta<false, K1, T::NL>(tmem + uint32_t(T::CG), tmem + uint32_t(T::CAL),
                                              tmem + uint32_t(T::CAL + K1 / 2), sbase + T::OFF_B2H,
                                              sbase + T::OFF_B2L);
        umma::commit(barL);
      }
      const bool okL = umma::mbar_wait_bounded(barL, phase, wlim);
      if (__syncthreads_or(!okL)) {
        if (tid == 0) {
          atomicExch(err_flag, 1);
          umma::mbar_wait_bounded(barL, phase);
          if (more) umma::mbar_wait_bounded(barS, phase ^ 1u); // the next tile's rows in flight
        }
        failed = true;
        break;
      }
      AT_MARK(7);
      umma::fence_after_sync();
      for (int gc = gc0; gc < gc1; ++gc) { // warp-uniform bounds
        float gv[8];
        umma::tmem_ld8(lane_taddr + uint32_t(T::CG + 8 * gc), gv);
        umma::tmem_wait_ld();
        umma::reg_fence8(gv);
        if (live) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m0 = 8 * gc + 4 * h;
            if (m0 < NFF) {
              float o[4];
#pragma unroll
              for (int n = 0; n < 4; ++n) o[n] = gv[4 * h + n] * inv * s_fg[e_loc * 4 + (m0 + n) / NFP].w;
              *reinterpret_cast<float4 *>(a.g_next + (fld * a.K + k0 + e_loc) * NFF + m0) =
                  make_float4(o[0], o[1], o[2], o[3]);
            }
          }
        }
      }
    }

    AT_MARK(8);
    // ---- G. the tile's gradient partials; buffers cleared for the next tile;
    // the next tile's face data requested (this tile's have been read)
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0 && more) stage_faces(tile + gridDim.x);
    if (tid < kAdjTile) {
      const float gsum = s_gr[tid];
      s_gr[tid] = 0.f;
      // one block per element and launch: the sum is that of a plain update,
      // issued without waiting for the old value
      if (grad && tid < ne) atomicAdd(a.grad + k0 + tid, double(a.dt) * double(gsum));
    }
    if (tid < 128) s_rmx[tid] = 0u;
    __syncthreads();
    AT_MARK(9);
    phase ^= 1u;
  }
  (void)failed;
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, T::TCOLS);
}

// Per-face constants of the transposed flux, one thread per face (see
// launch_adj_face_consts).
__global__ void k_adj_face_consts(int64_t K, const float *__restrict__ geo, const float4 *__restrict__ fgeo,
                                  const int2 *__restrict__ fconn, float4 *__restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 4 * K) return;
  const int64_t k = t >> 2;
  const int2 cn = fconn[t];
  const float4 nf = fgeo[t];
  const float Zk = geo[k * G_STRIDE + G_Z], Yk = geo[k * G_STRIDE + G_Y];
  const bool wall = cn.y == kBoundaryConn;
  const int64_t k2 = wall ? k : cn.x;
  const float Z2 = wall ? Zk : geo[k2 * G_STRIDE + G_Z], Y2 = wall ? Yk : geo[k2 * G_STRIDE + G_Y];
  const float ek = 1.f / geo[k * G_STRIDE + G_IEPS];
  out[t * 4 + 0] = make_float4(nf.x, nf.y, nf.z, 1.f / (Zk + Z2));
  out[t * 4 + 1] = make_float4(Zk, Z2, Yk, Y2);
  out[t * 4 + 2] = make_float4(1.f / (Yk + Y2), -Zk / (2.f * ek), Yk / (2.f * ek), __int_as_float(cn.y));
  out[t * 4 + 3] = make_float4(__int_as_float(int(k2)), __int_as_float(wall ? 1 : 0), 0.f, 0.f);
}

// Host: D^T and LIFT^T in the canonical K-major operand layout (FP16 hi, then
// lo): B1[(d, j), i] = D_d[i, j] and B2[m, i] = LIFT[i, m].
template <int N>
std::vector<uint8_t> build_adjoint_operands(const RefOps &o) {
  using T = AT<N>;
  std::vector<uint8_t> blk(T::OPS, 0);
  auto put = [&](int base_hi, int base_lo, int row, int col, double v) {
    const __half h = __float2half_rn(float(v));
    const __half l = __float2half_rn(float(v - double(__half2float(h))));
    uint16_t hb, lb;
    std::memcpy(&hb, &h, 2);
    std::memcpy(&lb, &l, 2);
    const uint32_t off = umma::kmajor_offset(uint32_t(row), uint32_t(col), uint32_t(T::K1));
    std::memcpy(&blk[base_hi + off], &hb, 2);
    std::memcpy(&blk[base_lo + off], &lb, 2);
  };
  const std::vector<double> *Ds[3] = {&o.Dr, &o.Ds, &o.Dt};
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < T::NP; ++i)
      for (int j = 0; j < T::NP; ++j) put(T::OFF_B1H, T::OFF_B1L, d * T::NB + j, i, (*Ds[d])[i * T::NP + j]);
  for (int i = 0; i < T::NP; ++i)
    for (int m = 0; m < T::NFF; ++m) put(T::OFF_B2H, T::OFF_B2L, m, i, o.LIFT[i * T::NFF + m]);
  return blk;
}

struct AdjTcState {
  void *d_ops = nullptr;
  int sms = 0;
};

template <int N>
cudaError_t launch_adj_tc_order(const AdjArgs &a, const AdjTcState &st, long long wait_limit, int *flag,
                                cudaStream_t s) {
  using T = AT<N>;
  auto kern = k_adj_tc<N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  // the largest shared-memory carveout, so that MINB blocks fit side by side
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T::NT, T::SMEM);
  if (e != cudaSuccess) return e;
  // persistent grid of MINB blocks per SM (registers and shared memory are
  // sized for it: launch bounds, 2 x (SMEM + 1 KB reserved) <= 228 KB), also
  // bounded by tensor memory (a block that cannot allocate would wait for
  // another block of the SM to finish)
  static_assert(T::MINB * (T::SMEM + 1024) <= 233472, "MINB blocks per SM do not fit in shared memory");
  if (per_sm < T::MINB) per_sm = T::MINB;
  const int tmem_fit = 512 / T::TCOLS;
  if (per_sm > tmem_fit) per_sm = tmem_fit;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = int((a.K + T::TE - 1) / T::TE);
  const int cap = per_sm * st.sms;
  const int grid = ntiles < cap ? ntiles : cap;
  return launch_pdl(kern, dim3(unsigned(grid)), dim3(T::NT), size_t(T::SMEM), s, a,
                    reinterpret_cast<const uint4 *>(st.d_ops), ntiles, wait_limit, flag);
}

} // namespace

#ifdef DGMX_STAGE_TIMING
extern "C" int dgmx_adj_trace(uint32_t *host) {
  return int(cudaMemcpyFromSymbol(host, g_adj_trace, sizeof(g_adj_trace)));
}
#endif

bool adj_tc_supported(const dg_ctx *ctx) {
  if (!ctx || ctx->N < 1 || ctx->N > 5) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3;
}

cudaError_t launch_adj_tc(dg_ctx *ctx, const AdjArgs &a, cudaStream_t s) {
  if (!adj_tc_supported(ctx)) return cudaErrorNotSupported;
  AdjTcState *st = static_cast<AdjTcState *>(ctx->adj_tc);
  if (!st) {
    std::vector<uint8_t> blk;
    switch (ctx->N) {
    case 1: blk = build_adjoint_operands<1>(ctx->ops); break;
    case 2: blk = build_adjoint_operands<2>(ctx->ops); break;
    case 3: blk = build_adjoint_operands<3>(ctx->ops); break;
    case 4: blk = build_adjoint_operands<4>(ctx->ops); break;
    default: blk = build_adjoint_operands<5>(ctx->ops); break;
    }
    st = new AdjTcState();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&st->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&st->d_ops, blk.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->d_ops, blk.data(), blk.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s); // blk is a host temporary
    if (e != cudaSuccess) {
      if (st->d_ops) cudaFree(st->d_ops);
      delete st;
      return e;
    }
    ctx->adj_tc = st;
  }
  int *flag = ctx->d_flag + 1;
  switch (ctx->N) {
  case 1: return launch_adj_tc_order<1>(a, *st, ctx->wait_limit, flag, s);
  case 2: return launch_adj_tc_order<2>(a, *st, ctx->wait_limit, flag, s);
  case 3: return launch_adj_tc_order<3>(a, *st, ctx->wait_limit, flag, s);
  case 4: return launch_adj_tc_order<4>(a, *st, ctx->wait_limit, flag, s);
  default: return launch_adj_tc_order<5>(a, *st, ctx->wait_limit, flag, s);
  }
}

cudaError_t launch_adj_face_consts(const dg_ctx *ctx, float4 *out, cudaStream_t s) {
  const int64_t n = 4 * ctx->K;
  k_adj_face_consts<<<unsigned((n + 255) / 256), 256, 0, s>>>(ctx->K, ctx->d_geo, ctx->d_fgeo, ctx->d_fconn, out);
  return cudaGetLastError();
}

void adj_tc_free(dg_ctx *ctx) {
  AdjTcState *st = static_cast<AdjTcState *>(ctx->adj_tc);
  if (st) {
    if (st->d_ops) cudaFree(st->d_ops);
    delete st;
  }
  ctx->adj_tc = nullptr;
}

} // namespace dgmx
