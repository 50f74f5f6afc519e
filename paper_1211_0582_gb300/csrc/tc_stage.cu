// Tensor-core form of the fused right-hand side / LSERK stage (sm_103a).
//
// The two dense contractions of the DG operator run on the fifth-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), in split
// precision: every operand x is stored as a 16-bit pair hi = rn(x),
// lo = rn(x - hi), and each product is formed as hi*hi + hi*lo + lo*hi with
// FP32 accumulation (BF16, or FP16 with power-of-two scales: per row for the
// fields, per field type (E, H) of a tile for the fluxes).
//
// Section 2, Fig. (el-local-ops): the field data of many elements is treated
// as one matrix so that local differentiation and lifting become
// matrix-matrix products. Here the rows are (element, field) pairs of a tile
// of 20 elements (5 per 32-lane TMEM quarter, 30 of 32 lanes used):
//   GEMM1  V[(e,f), (d,i)] = sum_j u[(e,f), j] D_d[i, j]        (d = r, s, t)
//   GEMM2  S[(e,f), i]     = sum_m flux[(e,f), m] LIFT[i, m]
// (the face-node columns m of GEMM2 are padded to an even count per face).
// GEMM1's A operand (the split fields) is written to tensor memory with
// tcgen05.st and read from there; GEMM2's (the split fluxes) goes through
// shared memory.
// The operators (B operands) stay resident in shared memory for the whole
// persistent kernel ("store the matrices, stream the vector data", Section 3).
// The epilogue reads V and S from TMEM with one thread per row, applies the
// chain rule (eq. dg-reference-matrices), exchanges the two needed physical
// derivatives between the six field lanes of an element with warp shuffles to
// form curl H and -curl E, adds the lifted flux, scales by 1/eps, 1/mu and
// either stores the right-hand side or applies the LSERK update.
//
// Orders N = 1..5 (the operators of N = 6, 7 do not fit in shared memory next
// to a tile; those orders stream them, see tc_stage_streamed.cu).
//
// The same kernel also runs many LSERK stages in one cooperative launch
// (ensembles of meshes): a grid barrier separates the stages, since a stage
// reads the neighbours' states that the previous stage wrote.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include "../../include/dgmx.h"
#include "flux.cuh"
#include "grid_sync.cuh"
#include "tc_api.h"
#include "tc_common.cuh"
#include "umma.cuh"

namespace dgmx {

namespace {

using namespace tcc;

constexpr int kThreads = 512;
constexpr int kTileElems = 20; // 4 TMEM lane quarters x 5 elements

// Element ranges of the tiles: whole rounds of full tiles (kTileElems elements,
// `grid` tiles per round), then the remaining elements in tiles of `small`
// elements, sized so that the last round spreads over the whole grid instead
// of leaving most CTAs idle behind a few full tiles.
struct TileMap {
  int nfull, small, ntiles;
  __host__ __device__ int64_t start(int t) const {
    return t < nfull ? int64_t(t) * kTileElems : int64_t(nfull) * kTileElems + int64_t(t - nfull) * small;
  }
  __host__ __device__ int size(int t, int64_t K) const {
    const int64_t k0 = start(t), n = t < nfull ? kTileElems : small;
    return int(K - k0 < n ? K - k0 : n);
  }
};

TileMap make_tiles(int64_t K, int grid) {
  const int64_t nfull = K / kTileElems / grid * grid;
  const int64_t rest = K - nfull * kTileElems;
  int64_t small = (rest + grid - 1) / grid;
  if (small < 1) small = 1;
  if (small > kTileElems) small = kTileElems;
  const int64_t nsmall = (rest + small - 1) / small;
  return TileMap{int(nfull), int(small), int(nfull + nsmall)};
}
constexpr int kMaxTcOrder = 7; // N <= 5 here, N = 6, 7 in tc_stage_streamed.cu

template <int N>
struct TC {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NFP = D::NFP, NPP = D::NPP, NFF = D::NFF;
  static constexpr int K1 = rup(NP, 16);  // GEMM1 reduction length (input nodes)
  static constexpr int NB = rup(NP, 16);  // output columns per derivative direction
  static constexpr int N1 = 3 * NB;       // GEMM1 output columns
  static constexpr int NFPE = (NFP + 1) / 2 * 2; // A2 columns per face (even: column pairs stay in one face)
  static constexpr int K2 = rup(4 * NFPE, 16);   // GEMM2 reduction length (face-node columns)
  static constexpr int N2 = NB;           // GEMM2 output columns
  static constexpr int CA = rup(N1 + N2, 32);  // TMEM column of the A1 operand (hi, then lo): after V and S
  static constexpr int TCOLS = tmem_cols(CA + K1);
  static_assert(CA + K1 <= 512, "accumulators and the A1 operand exceed tensor memory");
  static_assert(K1 <= 16 * (kThreads / 128), "the field split covers 16 K values per warp, four warps per quarter");
  static constexpr int FS = kTileElems * NPP + 4; // padded field-block stride of the staged tiles
  // A2 in the K-major core-matrix layout with padded strides: 144 bytes
  // between the core matrices of a row group along K (not 128) and a row-group
  // stride that is a multiple of 128 bytes. The flux split's 32-bit stores put
  // lanes kp and kp + 4 into two core matrices of one row; 128 bytes apart they
  // would share a bank, 144 bytes apart they do not.
  static constexpr int A2LBO = 144;
  static constexpr int A2SBO = rup(K2 / 8 * A2LBO, 128);
  static constexpr int A2B = 16 * A2SBO, B1B = N1 * K1 * 2, B2B = N2 * K2 * 2;
  static __device__ __forceinline__ uint32_t a2_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * uint32_t(A2SBO) + (k >> 3) * uint32_t(A2LBO) + (row & 7u) * 16u + (k & 7u) * 2u;
  }
  // fp32 [6][FS]: the next tile's fields, staged by bulk copies (the split
  // fields, GEMM1's A operand, live in tensor memory from column CA on)
  static constexpr int STB = rup(6 * FS * 4, 128);
  static constexpr int OFF_STAGE = 0;
  // A2 hi/lo; between the lifting GEMM of one tile and the flux split of the
  // next, the same bytes hold the tile's results [2][6][FS] for the bulk stores
  static constexpr int OUTB = 12 * FS * 4;
  static constexpr int A2R = 2 * A2B > OUTB ? 2 * A2B : OUTB;
  static constexpr int OFF_A2H = OFF_STAGE + STB, OFF_A2L = OFF_A2H + A2B;
  static constexpr int OFF_B1H = OFF_A2H + A2R, OFF_B1L = OFF_B1H + B1B;
  static constexpr int OFF_B2H = OFF_B1L + B1B, OFF_B2L = OFF_B2H + B2B;
  static constexpr int OPS_BYTES = 2 * B1B + 2 * B2B; // contiguous from OFF_B1H
  static constexpr int OFF_U = OFF_B2L + B2B;          // fp32 [6][FS]: fields of the tile
  static constexpr int OFF_RES = OFF_U + 6 * FS * 4;   // fp32 [6][FS]: residual of the tile
  // face and element data of a tile, two slots (current tile, next tile):
  // float4 fgeo[80] {n, Fscale}, float4 fmat[80] flux weights,
  // float geo[20][G_STRIDE], int2 fconn[80]
  static constexpr int FGEO = 0, FMAT = kTileElems * 4 * 16, FELEM = 2 * kTileElems * 4 * 16;
  static constexpr int FCONN = FELEM + kTileElems * G_STRIDE * 4, FSLOT = FCONN + kTileElems * 4 * 8;
  static constexpr int OFF_FACE = OFF_RES + 6 * FS * 4;
  static constexpr int OFF_TAB = OFF_FACE + 2 * FSLOT;
  // [128] A1 row inverse scales, [8] A2 field-type maxima, [128] A1 row maxima
  static constexpr int OFF_MX = OFF_TAB + rup(NFF + kConnKinds * NFP, 16);
  static constexpr int OFF_BAR = OFF_MX + 128 * 4 + 32 + 128 * 4; // mbarriers: GEMM1, GEMM2, residual, next tile; TMEM slot
  static constexpr int SMEM = OFF_BAR + 48;
};

// Three split products per K step: hi*hi, hi*lo, lo*hi, FP32 accumulation.
// Fully unrolled; the operand descriptors are formed once and advanced along K
// by adding to their start-address field (two core matrices per K step: 256
// bytes = 16 in units of 16 bytes for B, 2 ALBO bytes for A; shared-memory
// addresses stay below 2^18, so the field never carries out). B is packed
// (128-byte core-matrix stride along K); A has the strides ALBO, ASBO.
template <bool BF16, int KP, int NR, int ALBO, int ASBO>
__device__ __forceinline__ void issue_split_gemm(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                                 uint32_t b_lo) {
  constexpr uint32_t sbo = uint32_t(KP) * 16u;
  static_assert(ALBO % 16 == 0 && ASBO % 16 == 0, "descriptor strides are in units of 16 bytes");
  const uint64_t dah = umma::make_desc(a_hi, ALBO, ASBO), dal = umma::make_desc(a_lo, ALBO, ASBO);
#pragma unroll
  for (int n0 = 0; n0 < NR; n0 += 256) {
    const uint32_t idesc = umma::make_idesc(BF16, 128, uint32_t(NR - n0 < 256 ? NR - n0 : 256));
    const uint32_t boff = uint32_t(n0 / 8) * sbo;
    const uint64_t dbh = umma::make_desc(b_hi + boff, 128, sbo), dbl = umma::make_desc(b_lo + boff, 128, sbo);
#pragma unroll
    for (int kk = 0; kk < KP / 16; ++kk) {
      const uint64_t ko = uint64_t(kk) * 16u, ka = uint64_t(kk) * uint64_t(2 * ALBO / 16);
      umma::mma_f16(d_tmem + uint32_t(n0), dah + ka, dbh + ko, idesc, kk > 0 ? 1u : 0u);
      umma::mma_f16(d_tmem + uint32_t(n0), dah + ka, dbl + ko, idesc, 1u);
      umma::mma_f16(d_tmem + uint32_t(n0), dal + ka, dbh + ko, idesc, 1u);
    }
  }
}

// The same products with the A operand (hi and lo) in tensor memory: one N
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

// Multi-step persistent form (ensembles): stage coefficients, the two state
// buffers the stages alternate between, the step count and the grid barrier.
struct EnsLaunch {
  StageCoeffs rk;
  float *ua, *ub;
  int nsteps;
  GridBarrier *gb;
};

// ENS = false: one stage (MODE_RHS or MODE_LSERK) over all tiles. ENS = true:
// 5 * nsteps LSERK stages in one cooperative launch, a grid barrier after each
// stage (a stage reads the neighbours' states the previous one wrote), field
// gathers through L2 (another SM's L1 may hold a copy from two stages ago).
template <int N, int MODE, bool BF16, bool ENS>
__global__ void __launch_bounds__(kThreads, 1)
    k_stage_tc(StageArgs a, const uint4 *__restrict__ ops, TileMap tm, int *err_flag, EnsLaunch ens) {
  using T = TC<N>;
  constexpr int NP = T::NP, NFP = T::NFP, NPP = T::NPP, NFF = T::NFF, FS = T::FS;
  extern __shared__ __align__(1024) uint8_t smem[];
  float *s_u = reinterpret_cast<float *>(smem + T::OFF_U);       // [6][FS]: fields of the tile
  float *s_res = reinterpret_cast<float *>(smem + T::OFF_RES);   // [6][FS]: residual of the tile
  float *s_stage = reinterpret_cast<float *>(smem + T::OFF_STAGE); // [6][FS]: next tile's fields
  float *s_out = reinterpret_cast<float *>(smem + T::OFF_A2H);   // [2][6][FS]: results (in A2)
  uint8_t *s_fm = smem + T::OFF_TAB;
  uint8_t *s_nb = s_fm + NFF;
  float *s_inv1 = reinterpret_cast<float *>(smem + T::OFF_MX);  // A1 row inverse scales (compact rows)
  uint32_t *s_mx2 = reinterpret_cast<uint32_t *>(s_inv1 + 128); // A2 maxima of the E and H fluxes (float bits)
  uint32_t *s_rowmx = s_mx2 + 8; // A1 row maxima (float bits), FP16
  uint64_t *bar1 = reinterpret_cast<uint64_t *>(smem + T::OFF_BAR); // GEMM1 done
  uint64_t *bar2 = bar1 + 1;                                        // GEMM2 (and all earlier MMAs) done
  uint64_t *barR = bar1 + 2;                                        // residual tile landed
  uint64_t *barU = bar1 + 3;                                        // fields and face data of a tile landed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + T::OFF_BAR + 32);
  volatile int *s_staged = reinterpret_cast<volatile int *>(smem + T::OFF_BAR + 36); // next tile's copies issued

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // single-thread roles sit in the last four warps, which have the least flux
  // and epilogue work (issuing a tcgen05.mma or a bulk copy stalls the thread):
  // MMA issue, staging of the next tile, residual load, bulk stores
  const bool issuer = tid == kThreads - 32;
  const bool stager = tid == kThreads - 64;
  const bool rloader = tid == kThreads - 96;
  const bool storer = tid == kThreads - 128;
  const int64_t KN = a.K * NPP;
  const uint32_t sbase = umma::smem_u32(smem);
  const long long wlim = umma::wait_cycles(a.wait_limit); // main waits; drains use the default
  // the first LSERK4 stage has a = 0: the residual it overwrites is not read
  bool read_res = MODE == MODE_LSERK && a.rk_a != 0.f;

  // fields of tile t into the staging buffer, its face and element data into
  // a slot (one thread; completes on barU)
  auto stage_tile = [&](int t, int slot) {
    const int64_t kb = tm.start(t);
    const uint32_t nb = uint32_t(tm.size(t, a.K));
    const uint32_t rb = nb * NPP * 4;
    uint8_t *fs = smem + T::OFF_FACE + slot * T::FSLOT;
    umma::mbar_arrive_expect_tx(barU, 6u * rb + nb * (64u + 64u + G_STRIDE * 4u + 32u));
    for (int f = 0; f < 6; ++f) umma::bulk_g2s(s_stage + f * FS, a.u + f * KN + kb * NPP, rb, barU);
    umma::bulk_g2s(fs + T::FGEO, a.fgeo + kb * 4, nb * 64u, barU);
    umma::bulk_g2s(fs + T::FMAT, a.fmat + kb * 4, nb * 64u, barU);
    umma::bulk_g2s(fs + T::FELEM, a.geo + kb * G_STRIDE, nb * G_STRIDE * 4u, barU);
    umma::bulk_g2s(fs + T::FCONN, a.fconn + kb * 4, nb * 32u, barU);
  };

  // ---- one-time setup
  for (int i = tid; i < (T::STB + T::A2R) / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < T::OPS_BYTES / 16; i += kThreads)
    reinterpret_cast<uint4 *>(smem + T::OFF_B1H)[i] = __ldg(ops + i);
  for (int i = tid; i < NFF + kConnKinds * NFP; i += kThreads)
    s_fm[i] = i < NFF ? a.fmask[i] : a.nbrtab[i - NFF];
  for (int i = tid; i < 264; i += kThreads) s_inv1[i] = i < 128 ? 1.f : 0.f;
  if (tid == 0) {
    umma::mbar_init(bar1, 1);
    umma::mbar_init(bar2, 1);
    umma::mbar_init(barR, 1);
    umma::mbar_init(barU, 1);
    umma::fence_mbar_init();
  }
  if (warp == 0) umma::tmem_alloc(tslot, T::TCOLS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  // stage after stage: the setup above may overlap the end of the previous
  // stage, nothing it wrote is read before this point
  if constexpr (!ENS) pdl_wait();

  // field split: warp w writes the TMEM lanes of its quarter w % 4 (lane =
  // operand row) and K values 16 (w / 4) .. +15 of A1 (warps past K1 idle); an
  // FP16 row maximum is combined over the row's warps in shared memory; the
  // padding columns are written as zeros
  const int q1 = warp & 3, p1 = warp >> 2;
  const int r1 = 32 * q1 + lane;            // operand row = TMEM lane of this warp's quarter
  const int cr1 = compact_row(r1);
  const int e1 = cr1 >= 0 ? cr1 / 6 : 0, f1 = cr1 >= 0 ? cr1 % 6 : 0;
  const int kb1 = 16 * p1;                  // this thread's 16 K values
  const bool a1_part = kb1 < T::K1;         // warp-uniform
  const uint32_t a1_hi = tmem + uint32_t(T::CA), a1_lo = a1_hi + uint32_t(T::K1 / 2);
  const uint32_t a1_st = (uint32_t(q1 * 32) << 16) + uint32_t(8 * p1);
  // flux: blocks of 4 elements x 16 columns of A2 (padding columns included,
  // written as zeros), lane -> (element, pair of adjacent columns); column
  // f * NFPE + m holds face node m of face f, so a pair never straddles two
  // faces; block b goes to warp b % 16, so the last warps get the fewest
  constexpr int NFPE = T::NFPE;
  constexpr int KGF = T::K2 / 16;
  constexpr int NBLK = (kTileElems / 4) * KGF;
  constexpr int R2 = (NBLK + 15) / 16;
  const int eo = lane >> 3, kp = lane & 7;

  // epilogue: one thread per (element, field) row of the accumulators
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
  const int soff = fld * FS + e_loc * NPP; // this lane's row in the staged tiles
  const uint32_t lane_taddr = tmem + (uint32_t(quarter * 32) << 16);
  constexpr int NCH = (NP + 7) / 8;
  constexpr int CPP = (NCH + 3) / 4;
  const int ch0 = part * CPP;
  const int ch1 = (part + 1) * CPP < NCH ? (part + 1) * CPP : NCH;

  uint32_t phase = 0;
  // the residual barrier completes only for tiles of stages that read the
  // residual, so its parity is counted separately from the tile parity
  uint32_t rphase = 0;
  bool failed = false;
  const int nstages = ENS ? 5 * ens.nsteps : 1;
  for (int sg = 0; sg < nstages && !failed; ++sg) {
    if constexpr (ENS) {
      const bool flip = (sg & 1) != 0;
      a.u = flip ? ens.ub : ens.ua;
      a.u_out = flip ? ens.ua : ens.ub;
      a.rk_a = ens.rk.a[sg % 5];
      a.rk_b = ens.rk.b[sg % 5];
      read_res = a.rk_a != 0.f;
    }
    // the stage's first tile (the following ones are staged one tile ahead)
    if (stager && int(blockIdx.x) < tm.ntiles) {
      if (ENS) umma::fence_proxy_async_global();
      stage_tile(blockIdx.x, int(phase));
    }
    for (int tile = blockIdx.x; tile < tm.ntiles; tile += gridDim.x) {
      if (!ENS && tile + int(gridDim.x) >= tm.ntiles) pdl_launch_next(); // this block's last tile
      const int64_t k0 = tm.start(tile);
      const int ne = tm.size(tile, a.K);
      const uint32_t rowbytes = uint32_t(ne * NPP * 4);
      const int slot = int(phase);
      const uint8_t *fslot = smem + T::OFF_FACE + slot * T::FSLOT;
      const float4 *s_fgeo = reinterpret_cast<const float4 *>(fslot + T::FGEO);
      const float4 *s_fmat = reinterpret_cast<const float4 *>(fslot + T::FMAT);
      const float *s_geo = reinterpret_cast<const float *>(fslot + T::FELEM);
      const int2 *s_fconn = reinterpret_cast<const int2 *>(fslot + T::FCONN);

      // ---- 1. the staged fields into registers; once the previous tile's bulk
      // stores have read shared memory, the residual copy starts
      const bool okU = umma::mbar_wait_bounded(barU, phase, wlim);
      float4 v[4];
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = kb1 + 4 * j;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a1_part && cr1 >= 0 && k < NPP && e1 < ne) {
          v[j] = *reinterpret_cast<const float4 *>(s_stage + f1 * FS + e1 * NPP + k);
          if (k + 3 >= NP) {
            if (k + 0 >= NP) v[j].x = 0.f;
            if (k + 1 >= NP) v[j].y = 0.f;
            if (k + 2 >= NP) v[j].z = 0.f;
            if (k + 3 >= NP) v[j].w = 0.f;
          }
        }
        if constexpr (!BF16) mx = absmax4(mx, v[j]);
      }
      if (!BF16 && a1_part && cr1 >= 0) atomicMax(s_rowmx + r1, __float_as_uint(mx));
      if (__syncthreads_or(!okU)) {
        if (tid == 0) {
          atomicExch(err_flag, 1);
          umma::mbar_wait_bounded(barU, phase);
        }
        failed = true;
        break;
      }
      if (read_res && rloader) {
        umma::mbar_arrive_expect_tx(barR, 6u * rowbytes);
        for (int f = 0; f < 6; ++f) umma::bulk_g2s(s_res + f * FS, a.res + f * KN + k0 * NPP, rowbytes, barR);
      }
      // ---- 2. the fields to the tile buffer and, split, to the A1 operand in
      // tensor memory
      if (a1_part) {
        float sc1 = 1.f, inv1r = 1.f;
        if constexpr (!BF16) {
          if (cr1 >= 0) row_scale(__uint_as_float(s_rowmx[r1]), sc1, inv1r);
          if (p1 == 0 && cr1 >= 0) s_inv1[cr1] = inv1r;
        }
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = kb1 + 4 * j;
          if (cr1 >= 0 && k < NPP) *reinterpret_cast<float4 *>(s_u + f1 * FS + e1 * NPP + k) = v[j];
          float4 w = v[j];
          if constexpr (!BF16) w.x *= sc1, w.y *= sc1, w.z *= sc1, w.w *= sc1;
          split2<BF16>(w.x, w.y, hi[2 * j], lo[2 * j]);
          split2<BF16>(w.z, w.w, hi[2 * j + 1], lo[2 * j + 1]);
        }
        umma::tmem_st8(a1_hi + a1_st, hi);
        umma::tmem_st8(a1_lo + a1_st, lo);
        umma::tmem_wait_st();
      }
      umma::fence_before_sync();
      __syncthreads();
      if (!BF16 && tid < 128) s_rowmx[tid] = 0u;

      // ---- 3. local differentiation on the tensor cores (asynchronous)
      if (issuer) {
        umma::fence_after_sync();
        issue_split_gemm_ta<BF16, T::K1, T::N1>(tmem, a1_hi, a1_lo, sbase + T::OFF_B1H, sbase + T::OFF_B1L);
        umma::commit(bar1);
      }
      bool ok = true;

      // ---- 4. upwind flux (overlaps GEMM1), in registers: the neighbour traces
      // outside the tile are requested from L2 first (all of a lane's loads in
      // flight together); neighbours inside the tile are read from the staged
      // fields
      float qp[R2][2][6];
      int lidx[R2][2];
#pragma unroll
      for (int s = 0; s < R2; ++s) {
        const int blk = warp + 16 * s;
        const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
        const int f = fm / NFPE, mm = fm - f * NFPE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          lidx[s][h] = -1;
#pragma unroll
          for (int c = 0; c < 6; ++c) qp[s][h][c] = 0.f;
        }
        if (blk < NBLK && f < 4 && e < ne) {
          const int2 cn = s_fconn[e * 4 + f];
          if (cn.y != kBoundaryConn) {
            const int el = cn.x - int(k0);
            const bool local = el >= 0 && el < ne;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (mm + h < NFP) {
                const int node = s_nb[cn.y * NFP + mm + h];
                if (local) {
                  lidx[s][h] = el * NPP + node;
                } else {
                  const float *up = a.u + int64_t(cn.x) * NPP + node;
#pragma unroll
                  for (int c = 0; c < 6; ++c) qp[s][h][c] = ENS ? __ldcg(up + c * KN) : __ldg(up + c * KN);
                }
              }
            }
          }
        }
      }
      float fl[R2][2][6];
      uint32_t fmx[6] = {0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
      for (int s = 0; s < R2; ++s) {
        const int blk = warp + 16 * s;
        const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
        const int f = fm / NFPE, mm = fm - f * NFPE;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 6; ++c) fl[s][h][c] = 0.f;
        if (blk < NBLK && f < 4 && e < ne) {
          const float4 g0 = s_fgeo[e * 4 + f], w1 = s_fmat[e * 4 + f];
          const bool wall = s_fconn[e * 4 + f].y == kBoundaryConn;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (mm + h < NFP) {
              const int vm = s_fm[f * NFP + mm + h];
              float qm[6], q[6];
#pragma unroll
              for (int c = 0; c < 6; ++c) qm[c] = s_u[c * FS + e * NPP + vm];
#pragma unroll
              for (int c = 0; c < 6; ++c) q[c] = lidx[s][h] >= 0 ? s_u[c * FS + lidx[s][h]] : qp[s][h][c];
              if (wall) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  q[c] = -qm[c];
                  q[c + 3] = qm[c + 3];
                }
              }
              maxwell_flux_w(g0, qm, q, w1, a.alpha, fl[s][h]);
            }
          }
        }
        if constexpr (!BF16) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 6; ++c) fmx[c] = max(fmx[c], __float_as_uint(fabsf(fl[s][h][c])));
        }
      }
      // the next tile's fields and face data are staged (issued here rather
      // than right after step 1: earlier, the copies compete with GEMM1 and the
      // flux phase for shared memory, which measured slower)
      if (stager) {
        const bool more = tile + int(gridDim.x) < tm.ntiles;
        if (more) stage_tile(tile + gridDim.x, slot ^ 1);
        *s_staged = more ? 1 : 0;
      }
      if constexpr (!BF16) {
        // one FP16 scale per field type (E, H) of the tile: |x| as float
        // bits orders like |x|
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const uint32_t m = __reduce_max_sync(0xffffffffu, max(fmx[3 * g], max(fmx[3 * g + 1], fmx[3 * g + 2])));
          if (lane == 0) atomicMax(s_mx2 + g, m);
        }
      }
      // the previous tile's bulk stores must have read the A2 bytes
      if (storer) umma::bulk_wait_read_all();
      __syncthreads();

      // ---- 5. split the face fluxes into the A2 operand
      {
        float sc2[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          sc2[c] = 1.f;
          if constexpr (!BF16) {
            float inv;
            row_scale(__uint_as_float(s_mx2[c / 3]), sc2[c], inv);
          }
        }
#pragma unroll
        for (int s = 0; s < R2; ++s) {
          const int blk = warp + 16 * s;
          const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
          if (blk < NBLK) {
            // the six rows of element e lie in one TMEM lane quarter; a column
            // pair is one 32-bit word of a core-matrix row
            const uint32_t r0 = uint32_t(32 * (e / 5) + 6 * (e % 5));
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              uint32_t hi, lo;
              split2<BF16>(fl[s][0][c] * sc2[c], fl[s][1][c] * sc2[c], hi, lo);
              const uint32_t o = T::a2_offset(r0 + uint32_t(c), uint32_t(fm));
              *reinterpret_cast<uint32_t *>(smem + T::OFF_A2H + o) = hi;
              *reinterpret_cast<uint32_t *>(smem + T::OFF_A2L + o) = lo;
            }
          }
        }
      }
      umma::fence_proxy_async();
      __syncthreads();

      // ---- 6. flux lifting on the tensor cores; meanwhile the volume terms
      // from GEMM1: chain rule (eq. dg-reference-matrices) and curls
      if (issuer) {
        umma::fence_after_sync();
        issue_split_gemm<BF16, T::K2, T::N2, T::A2LBO, T::A2SBO>(tmem + uint32_t(T::N1), sbase + T::OFF_A2H,
                                                                 sbase + T::OFF_A2L, sbase + T::OFF_B2H,
                                                                 sbase + T::OFF_B2L);
        umma::commit(bar2);
      }
      const bool live = lane_used && e_loc < ne;
      float g1r = 0.f, g1s = 0.f, g1t = 0.f, g2r = 0.f, g2s = 0.f, g2t = 0.f, w = 0.f, dtk = a.dt;
      if (live) {
        const float *g = s_geo + e_loc * G_STRIDE;
        if (a.dt_geo) dtk = g[G_DT];
        g1r = g[G_RX + dl1], g1s = g[G_SX + dl1], g1t = g[G_TX + dl1];
        g2r = g[G_RX + dl2], g2s = g[G_SX + dl2], g2t = g[G_TX + dl2];
        w = g[isE ? G_IEPS : G_IMU];
      }
      float inv2 = 1.f;
      if constexpr (!BF16) {
        // the row's FP16 scale is undone through the metric factors of the chain rule
        float sc;
        const float inv1 = s_inv1[lane_used ? ridx : 0];
        g1r *= inv1, g1s *= inv1, g1t *= inv1, g2r *= inv1, g2s *= inv1, g2t *= inv1;
        row_scale(__uint_as_float(s_mx2[fld / 3]), sc, inv2);
      }
      ok = umma::mbar_wait_bounded(bar1, phase, wlim) && ok;
      umma::fence_after_sync();
      float vol[CPP][8];
#pragma unroll
      for (int c = 0; c < CPP; ++c) {
        const int ch = ch0 + c;
        if (ch >= ch1) break;
        const int i0 = ch * 8;
        float ur[8], us[8], ut[8];
        umma::tmem_ld8(lane_taddr + uint32_t(i0), ur);
        umma::tmem_ld8(lane_taddr + uint32_t(T::NB + i0), us);
        umma::tmem_ld8(lane_taddr + uint32_t(2 * T::NB + i0), ut);
        umma::tmem_wait_ld();
        umma::reg_fence8(ur);
        umma::reg_fence8(us);
        umma::reg_fence8(ut);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
          const float p1 = g1r * ur[n] + g1s * us[n] + g1t * ut[n];
          const float p2 = g2r * ur[n] + g2s * us[n] + g2t * ut[n];
          const float v1 = __shfl_sync(0xffffffffu, p1, src1);
          const float v2 = __shfl_sync(0xffffffffu, p2, src2);
          vol[c][n] = isE ? (v1 - v2) : (v2 - v1);
        }
      }
      ok = umma::mbar_wait_bounded(bar2, phase, wlim) && ok;
      if (read_res) ok = umma::mbar_wait_bounded(barR, rphase, wlim) && ok;
      // this slot's face and element data are rewritten by the staging after next
      umma::fence_proxy_async();
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(err_flag, 1);
          // give the products and the copies in flight one more bounded wait
          // before tensor and shared memory are released
          umma::mbar_wait_bounded(bar2, phase);
          if (read_res) umma::mbar_wait_bounded(barR, rphase);
          if (*s_staged) umma::mbar_wait_bounded(barU, phase ^ 1u);
        }
        failed = true;
        break;
      }
      umma::fence_after_sync();

      // ---- 7. epilogue: lifted flux, material scale, update; results go to the
      // A2 bytes
#pragma unroll
      for (int c = 0; c < CPP; ++c) {
        const int ch = ch0 + c;
        if (ch >= ch1) break;
        const int i0 = ch * 8;
        float lf[8];
        umma::tmem_ld8(lane_taddr + uint32_t(T::N1 + i0), lf);
        umma::tmem_wait_ld();
        umma::reg_fence8(lf);
        if (live) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = i0 + 4 * h;
            if (i < NPP) {
              float r4[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) r4[q] = (i + q < NP) ? (vol[c][4 * h + q] + lf[4 * h + q] * inv2) * w : 0.f;
              float4 *op = reinterpret_cast<float4 *>(s_out + soff + i);
              if (MODE == MODE_RHS) {
                *op = make_float4(r4[0], r4[1], r4[2], r4[3]);
              } else {
                const float4 rs = read_res ? *reinterpret_cast<const float4 *>(s_res + soff + i)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 uo = *reinterpret_cast<const float4 *>(s_u + soff + i);
                const float rsv[4] = {rs.x, rs.y, rs.z, rs.w}, uov[4] = {uo.x, uo.y, uo.z, uo.w};
                float nr[4], nu[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const bool pad = i + q >= NP;
                  nr[q] = pad ? 0.f : fmaf(a.rk_a, rsv[q], dtk * r4[q]);
                  nu[q] = pad ? 0.f : fmaf(a.rk_b, nr[q], uov[q]);
                }
                op[0] = make_float4(nr[0], nr[1], nr[2], nr[3]);
                op[6 * FS / 4] = make_float4(nu[0], nu[1], nu[2], nu[3]);
              }
            }
          }
        }
      }
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      // ---- 8. write the tile back with asynchronous bulk stores; clear the
      // flux maxima for the next tile
      if (storer) {
        for (int f = 0; f < 6; ++f) {
          if (MODE == MODE_RHS) {
            umma::bulk_s2g(a.rhs + f * KN + k0 * NPP, s_out + f * FS, rowbytes);
          } else {
            umma::bulk_s2g(a.res + f * KN + k0 * NPP, s_out + f * FS, rowbytes);
            umma::bulk_s2g(a.u_out + f * KN + k0 * NPP, s_out + (6 + f) * FS, rowbytes);
          }
        }
        umma::bulk_commit();
      }
      if (!BF16 && tid < 8) s_mx2[tid] = 0u;
      phase ^= 1u;
      if (read_res) rphase ^= 1u;
    }
    if constexpr (ENS) {
      if (!failed) {
        // the stage's results are in global memory before any block reads them
        if (storer) {
          umma::bulk_wait_all();
          umma::fence_proxy_async_global();
        }
        if (!grid_barrier(ens.gb, wlim)) {
          if (tid == 0) atomicExch(err_flag, 1);
          failed = true;
        }
      }
    }
  }
  if (storer) umma::bulk_wait_all();
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
    for (int m = 0; m < T::NFF; ++m)
      put(b2h, b2l, i, (m / T::NFP) * T::NFPE + m % T::NFP, T::K2, o.LIFT[i * T::NFF + m]);
  return blk;
}

template <int N, int MODE, bool BF16>
cudaError_t launch_tc_kernel(const StageArgs &a, const TcState &st, int *flag, cudaStream_t s) {
  using T = TC<N>;
  static_assert(T::SMEM <= 232448, "tensor-core tile does not fit in shared memory");
  auto kern = k_stage_tc<N, MODE, BF16, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  const TileMap tm = make_tiles(a.K, st.sms);
  const int grid = tm.ntiles < st.sms ? tm.ntiles : st.sms;
  return launch_pdl(kern, dim3(unsigned(grid)), dim3(kThreads), size_t(T::SMEM), s, a,
                    reinterpret_cast<const uint4 *>(st.d_ops), tm, flag, EnsLaunch{});
}

// Cooperative launch of the multi-step form: one block per SM, all resident.
template <int N, bool BF16>
cudaError_t launch_tc_ens_kernel(const StageArgs &a, const TcState &st, const EnsLaunch &ens, int *flag,
                                 cudaStream_t s) {
  using T = TC<N>;
  auto kern = k_stage_tc<N, MODE_LSERK, BF16, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  const TileMap tm = make_tiles(a.K, st.sms);
  const int grid = tm.ntiles < st.sms ? tm.ntiles : st.sms;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = T::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, reinterpret_cast<const uint4 *>(st.d_ops), tm, flag, ens);
}

template <int N>
cudaError_t launch_tc_ens_order(bool bf16, const StageArgs &a, const TcState &st, const EnsLaunch &ens, int *flag,
                                cudaStream_t s) {
  return bf16 ? launch_tc_ens_kernel<N, true>(a, st, ens, flag, s) : launch_tc_ens_kernel<N, false>(a, st, ens, flag, s);
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
    ctx->err = "tensor-core precisions support N <= 7";
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
  case 5: blk = build_operand_block<5>(ctx->ops, bf16); break;
  default: blk = build_streamed_operators(ctx->N, ctx->ops, bf16); break;
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

bool tc_ensemble_supported(const dg_ctx *ctx) {
  return ctx->tc != nullptr && ctx->N >= 1 && ctx->N <= 5 &&
         (ctx->precision == DG_BF16X3 || ctx->precision == DG_FP16X3);
}

cudaError_t launch_tc_ensemble(dg_ctx *ctx, const StageArgs &a, const StageCoeffs &rk, float *u_a, float *u_b,
                               int nsteps, GridBarrier *gb, cudaStream_t s) {
  const TcState *st = static_cast<const TcState *>(ctx->tc);
  if (!st || !tc_ensemble_supported(ctx)) return cudaErrorNotSupported;
  const bool bf16 = ctx->precision == DG_BF16X3;
  int *flag = ctx->d_flag + 1;
  const EnsLaunch ens{rk, u_a, u_b, nsteps, gb};
  switch (ctx->N) {
  case 1: return launch_tc_ens_order<1>(bf16, a, *st, ens, flag, s);
  case 2: return launch_tc_ens_order<2>(bf16, a, *st, ens, flag, s);
  case 3: return launch_tc_ens_order<3>(bf16, a, *st, ens, flag, s);
  case 4: return launch_tc_ens_order<4>(bf16, a, *st, ens, flag, s);
  default: return launch_tc_ens_order<5>(bf16, a, *st, ens, flag, s);
  }
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
  default: return launch_tc_streamed(ctx->N, mode, bf16, a, *st, flag, ctx->stream);
  }
}

} // namespace dgmx
