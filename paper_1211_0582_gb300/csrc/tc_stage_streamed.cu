// Tensor-core form of the fused right-hand side / LSERK stage for N = 6, 7
// (sm_103a), with the operators streamed from L2.
//
// Same tile (20 elements x 6 fields = 120 accumulator rows) and the same split
// precision as the kernel for N <= 5: hi*hi + hi*lo + lo*hi products with FP32
// accumulation in tensor memory (Section 2, Fig. el-local-ops: local
// differentiation and lifting as matrix-matrix products over many elements).
// At these orders the hi/lo operators (188 KB at N = 6, 264 KB at N = 7) do
// not fit in shared memory beside a tile, so the paper's "keep the matrices
// on chip, stream the field data" (Section 3) is turned around for them: the
// host stores the operators as a sequence of 24 KB-class slices in the
// canonical operand layout (hi, then lo): for GEMM1 one 16-wide K step of
// [Dr; Ds; Dt], for GEMM2 three K steps of LIFT. A dedicated warp copies the
// slices from L2 (where the few hundred KB stay resident) into a three-slot
// shared-memory ring, two slices ahead of the MMAs that read them
// (full/empty mbarriers; the MMA completion itself releases a slot). The same
// warp issues all MMAs. Fewer, larger slices keep the single issuing thread's
// per-slice overhead (barrier waits, commit, copy issue) small.
//
// Per tile: GEMM1 takes K1/16 slices ([Dr; Ds; Dt] hi, then lo), each feeding
// the three split products as two MMAs: Dr and Ds together (N = 2 NB) and Dt
// (N = NB); GEMM2 takes ceil(K2/48) slices. TMEM holds [ur | us | ut | lifted flux] = 4 NB columns (all 512 at
// N = 7). A1 and A2 share one shared-memory region: A2 is written once GEMM1
// has completed, and after GEMM2 the same bytes take the new residual (or the
// right-hand side) while the new fields overwrite the staged ones; both go out
// as bulk stores whose drain overlaps the next tile's loads. The residual is
// read straight from global memory (warmed in L2 one tile ahead).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>
#include <vector>

#include "../../include/dgmx.h"
#include "flux.cuh"
#include "tc_common.cuh"
#include "umma.cuh"

namespace dgmx {

namespace {

using namespace tcc;

constexpr int kThreadsS = 512;
constexpr int kMmaWarp = 15;   // MMA issue and operator stream (after the field split)
constexpr int kFluxWarps = 15; // warps 0..14
constexpr int kTileS = 20;     // 4 TMEM lane quarters x 5 elements
constexpr int kSlots = 3;      // operator ring depth

template <int N>
struct TS {
  using D = Dims<N>;
  static constexpr int NP = D::NP, NFP = D::NFP, NPP = D::NPP, NFF = D::NFF;
  static constexpr int K1 = rup(NP, 16), NB = K1, K2 = rup(NFF, 16);
  static constexpr int KS1 = K1 / 16, KS2 = K2 / 16;  // K steps of GEMM1, GEMM2
  static constexpr int G2 = 3;                         // GEMM2 K steps per slice
  static constexpr int NS2 = (KS2 + G2 - 1) / G2;      // GEMM2 slices
  static constexpr int PER = KS1 + NS2;                // operator slices per tile
  static constexpr int SUB = 2 * NB * 32;              // GEMM2: NB rows x 16 K, hi then lo
  static constexpr int SL = 3 * SUB;                   // one slice: GEMM1 [Dr;Ds;Dt] hi, lo; GEMM2 three SUB
  static constexpr int STREAM = PER * SL;
  static constexpr int TCOLS = tmem_cols(4 * NB);
  static constexpr int FS = kTileS * NPP + 4; // padded field-block stride of the staged fields
  // A2 with padded core-matrix strides (144 bytes along K, a multiple of 128
  // bytes between row groups), so that the flux split's stores of lanes kp
  // and kp + 4 (two core matrices of one row) fall into different banks
  static constexpr int A2LBO = 144;
  static constexpr int A2SBO = rup(K2 / 8 * A2LBO, 128);
  static constexpr int A1B = 128 * K1 * 2, A2B = 16 * A2SBO;
  static __device__ __forceinline__ uint32_t a2_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * uint32_t(A2SBO) + (k >> 3) * uint32_t(A2LBO) + (row & 7u) * 16u + (k & 7u) * 2u;
  }
  static constexpr int AREG = 2 * (A1B > A2B ? A1B : A2B); // A1 hi/lo, later A2 hi/lo
  static constexpr int OFF_RING = AREG;
  static constexpr int OFF_U = OFF_RING + kSlots * SL;           // fp32 [6][FS]
  static constexpr int OFF_FACE = OFF_U + 6 * FS * 4;            // float4 [80][3]
  static constexpr int OFF_TAB = OFF_FACE + kTileS * 4 * 48;
  // [128] A1 inverse scales, [2 * kTileS] A2 largest exponents per element and field type (E, H)
  static constexpr int OFF_MX = OFF_TAB + rup(NFF + kConnKinds * NFP, 16);
  static constexpr int NBAR = 2 + 2 * kSlots;          // GEMM1, GEMM2, full[kSlots], empty[kSlots]
  static constexpr int OFF_BAR = OFF_MX + 128 * 4 + 2 * kTileS * 4;
  static constexpr int OFF_TSLOT = OFF_BAR + NBAR * 8;  // TMEM base address
  static constexpr int SMEM = OFF_TSLOT + 16;
  static_assert(4 * NB <= 512, "accumulators exceed tensor memory");
  static_assert(SMEM <= 232448, "tile does not fit in shared memory");
};

// Optional phase timestamps (build with -DDGMX_STAGE_TIMING; off in the
// library): thread 0's SM clock (the MMA thread's for slot 13: all of GEMM1
// issued; slot 14: all of GEMM2 issued), in cycles since the block passed its
// setup, per block and tile, read back with dgmx_tcs_trace().
constexpr int kTsTraceTiles = 32, kTsTraceBlocks = 160, kTsEvents = 16;
#ifdef DGMX_STAGE_TIMING
__device__ uint32_t g_tcs_trace[kTsTraceBlocks * kTsTraceTiles * kTsEvents];
#define TS_MARK(who, ev)                                                                                            \
  do {                                                                                                              \
    if ((who) && itn < kTsTraceTiles && blockIdx.x < kTsTraceBlocks)                                                \
      g_tcs_trace[(blockIdx.x * kTsTraceTiles + itn) * kTsEvents + (ev)] = uint32_t(clock64() - ts_t0);             \
  } while (0)
#else
#define TS_MARK(who, ev) \
  do {                   \
  } while (0)
#endif

// Byte offset of stream step st (0 .. PER-1) in the operator stream.
template <int N>
__host__ __device__ constexpr uint32_t slice_offset(int st) {
  return uint32_t(st) * uint32_t(TS<N>::SL);
}

template <int N, int MODE, bool BF16>
__global__ void __launch_bounds__(kThreadsS, 1)
    k_stage_tc_streamed(StageArgs a, const uint8_t *__restrict__ stream, int ntiles, int *err_flag) {
  using T = TS<N>;
  constexpr int NP = T::NP, NFP = T::NFP, NPP = T::NPP, NFF = T::NFF, FS = T::FS, NB = T::NB;
  extern __shared__ __align__(1024) uint8_t smem[];
  float *s_u = reinterpret_cast<float *>(smem + T::OFF_U);  // fields; the new fields after the epilogue
  float *s_out = reinterpret_cast<float *>(smem);           // [6][FS] new residual / rhs (A region)
  float4 *s_face = reinterpret_cast<float4 *>(smem + T::OFF_FACE); // {n, Fs}, {wE, wH, Z+, Y+}, {k2, conn}
  uint8_t *s_fm = smem + T::OFF_TAB;
  uint8_t *s_nb = s_fm + NFF;
  float *s_inv1 = reinterpret_cast<float *>(smem + T::OFF_MX);
  uint32_t *s_ex2 = reinterpret_cast<uint32_t *>(s_inv1 + 128);
  uint64_t *bar1 = reinterpret_cast<uint64_t *>(smem + T::OFF_BAR); // GEMM1 done
  uint64_t *bar2 = bar1 + 1;                                        // GEMM2 done
  uint64_t *full = bar1 + 2;                                        // ring slot filled
  uint64_t *empty = bar1 + 2 + kSlots;                              // ring slot read by its MMAs
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + T::OFF_TSLOT);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp != kMmaWarp;
  const bool issuer = warp == kMmaWarp && lane == 0;
  const int64_t KN = a.K * NPP;
  const uint32_t sbase = umma::smem_u32(smem);
  const long long wlim = umma::wait_cycles(a.wait_limit); // main waits; drains use the default

  // ---- one-time setup
  for (int i = tid; i < T::AREG / 16; i += kThreadsS) reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < NFF + kConnKinds * NFP; i += kThreadsS) s_fm[i] = i < NFF ? a.fmask[i] : a.nbrtab[i - NFF];
  for (int i = tid; i < 128 + 2 * kTileS; i += kThreadsS) s_inv1[i] = i < 128 ? 1.f : 0.f;
  if (tid == 0) {
    umma::mbar_init(bar1, 1);
    umma::mbar_init(bar2, 1);
    for (int s = 0; s < kSlots; ++s) {
      umma::mbar_init(full + s, 1);
      umma::mbar_init(empty + s, 1);
    }
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
  pdl_wait();
#ifdef DGMX_STAGE_TIMING
  const long long ts_t0 = clock64();
#endif

  // operator stream (issuer only): step j of the periodic slice sequence
  // goes to slot j % kSlots
  uint32_t jstep = 0; // next step to consume
  uint32_t jprod = 0; // next step to produce (steps are produced in order)
  auto produce = [&](uint32_t j) {
    const int st = int(j % uint32_t(T::PER)), slot = int(j % uint32_t(kSlots));
    umma::mbar_arrive_expect_tx(full + slot, uint32_t(T::SL));
    umma::bulk_g2s(smem + T::OFF_RING + slot * T::SL, stream + slice_offset<N>(st), uint32_t(T::SL), full + slot);
    jprod = j + 1u;
  };
  // wait for step jstep's slice, issue its MMAs, release the slot when they
  // complete, and refill the previous step's slot with the step kSlots ahead;
  // after a timed-out wait nothing more is waited for or issued (the slices
  // still in flight are waited for before the kernel exits)
  bool stream_ok = true;
  auto consume = [&](auto &&issue) -> bool {
    if (!stream_ok) return false;
    const int slot = int(jstep % uint32_t(kSlots));
    if (!umma::mbar_wait_bounded(full + slot, (jstep / uint32_t(kSlots)) & 1u, wlim)) {
      stream_ok = false;
      return false;
    }
    umma::fence_after_sync();
    issue(sbase + uint32_t(T::OFF_RING + slot * T::SL));
    umma::commit(empty + slot);
    if (jstep >= 1u) {
      const uint32_t pj = jstep - 1u;
      if (umma::mbar_wait_bounded(empty + pj % uint32_t(kSlots), (pj / uint32_t(kSlots)) & 1u, wlim))
        produce(pj + uint32_t(kSlots));
      else
        stream_ok = false;
    }
    ++jstep;
    return stream_ok;
  };
  if (issuer && int(blockIdx.x) < ntiles)
    for (int j = 0; j < kSlots; ++j) produce(uint32_t(j));

  // field split (all 16 warps): warp w owns operand rows 8w..8w+7 (lane ->
  // row, half of a K group of 8; padding columns written as zeros)
  constexpr int KG1 = T::K1 / 8;
  constexpr int R1 = (KG1 + 1) / 2;
  const int r1 = warp * 8 + (lane & 7);
  const int cr1 = compact_row(r1);
  const int e1 = cr1 >= 0 ? cr1 / 6 : 0, f1 = cr1 >= 0 ? cr1 % 6 : 0;
  const int kq1 = 4 * ((lane >> 3) & 1) + 8 * (lane >> 4);
  // flux: blocks of 4 elements x 16 face-node columns of A2, lane -> (element,
  // pair of adjacent columns); Nfp is even at N = 6, 7, so a pair never
  // straddles two faces
  static_assert(NFP % 2 == 0, "column pairs need an even number of nodes per face");
  constexpr int KGF = T::K2 / 16;
  constexpr int NBLK = (kTileS / 4) * KGF;
  constexpr int R2 = (NBLK + kFluxWarps - 1) / kFluxWarps;
  constexpr int BATCH = 1; // blocks whose neighbour gathers are in flight together
  const int eo = lane >> 3, kp = lane & 7;
  // epilogue: one thread per (element, field) row of the accumulators; a
  // warp reads the TMEM lane quarter warp % 4, quarter 3 without the MMA warp
  // has three warps
  const int quarter = warp & 3, part = warp >> 2;
  const int nparts = quarter == 3 ? 3 : 4;
  const bool lane_used = worker && lane < 30;
  const int ep = lane < 30 ? lane / 6 : 4;
  const int fld = lane < 30 ? lane % 6 : 5;
  const int comp = fld % 3;
  const bool isE = fld < 3;
  const float sgn = isE ? 1.f : -1.f;
  const int src1 = ep * 6 + (isE ? 3 : 0) + (comp + 2) % 3;
  const int src2 = ep * 6 + (isE ? 3 : 0) + (comp + 1) % 3;
  const int dl1 = (comp + 2) % 3, dl2 = (comp + 1) % 3;
  const int e_loc = quarter * 5 + ep;
  const int ridx = e_loc * 6 + fld;
  const int soff = fld * FS + e_loc * NPP;
  const uint32_t lane_taddr = tmem + (uint32_t(quarter * 32) << 16);
  constexpr int NCH = (NP + 7) / 8;
  constexpr int CPP = (NCH + 2) / 3; // chunks of a warp of quarter 3 (the most)
  const int cpp = (NCH + nparts - 1) / nparts;
  const int ch0 = part * cpp;
  const int ch1 = !worker ? ch0 : ch0 + cpp < NCH ? ch0 + cpp : NCH;

  // warm L2 with the fields of the CTA's next tile and the residual of this one
  auto prefetch = [&](int tu, int tr) {
    if (tu < ntiles) {
      const int64_t kb = int64_t(tu) * kTileS, nb = a.K - kb < kTileS ? a.K - kb : kTileS;
      for (int f = 0; f < 6; ++f) umma::prefetch_l2(a.u + f * KN + kb * NPP, uint32_t(nb * NPP * 4));
      umma::prefetch_l2(a.fconn + kb * 4, uint32_t(nb * 32));
      umma::prefetch_l2(a.fgeo + kb * 4, uint32_t(nb * 64));
      umma::prefetch_l2(a.fmat + kb * 4, uint32_t(nb * 64));
    }
    if (MODE == MODE_LSERK && a.rk_a != 0.f && tr < ntiles) {
      const int64_t kb = int64_t(tr) * kTileS, nb = a.K - kb < kTileS ? a.K - kb : kTileS;
      for (int f = 0; f < 6; ++f) umma::prefetch_l2(a.res + f * KN + kb * NPP, uint32_t(nb * NPP * 4));
    }
  };
  if (tid == 32 && int(blockIdx.x) < ntiles) prefetch(blockIdx.x, -1);

  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#ifdef DGMX_STAGE_TIMING
    const int itn = (tile - int(blockIdx.x)) / int(gridDim.x);
#endif
    TS_MARK(tid == 0, 0);
    if (tile + int(gridDim.x) >= ntiles) pdl_launch_next(); // this block's last tile
    const int64_t k0 = int64_t(tile) * kTileS;
    const int ne = int(a.K - k0 < kTileS ? a.K - k0 : kTileS);
    bool ok = true;
    if (tid == 32) prefetch(tile + int(gridDim.x), tile);

    // ---- 1. fields and face table of the tile into registers; once the
    // previous tile's bulk stores have read shared memory, the staging and A1
    // the face table first, so that its loads are in flight with the fields'
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = make_float4(0.f, 0.f, 1.f, 1.f);
    int2 cn = make_int2(0, kBoundaryConn);
    if (tid < kTileS * 4 && (tid >> 2) < ne) {
      const int64_t q = (k0 + (tid >> 2)) * 4 + (tid & 3);
      cn = __ldg(a.fconn + q);
      g0 = __ldg(a.fgeo + q);
      g1 = __ldg(a.fmat + q);
    }
    float4 v[R1];
    float mx = 0.f;
#pragma unroll
    for (int s = 0; s < R1; ++s) {
      const int k = kq1 + 16 * s;
      v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cr1 >= 0 && k < NPP && e1 < ne) {
        v[s] = ldg4(a.u + f1 * KN + (k0 + e1) * NPP + k);
        if (k + 3 >= NP) {
          if (k + 0 >= NP) v[s].x = 0.f;
          if (k + 1 >= NP) v[s].y = 0.f;
          if (k + 2 >= NP) v[s].z = 0.f;
          if (k + 3 >= NP) v[s].w = 0.f;
        }
      }
      if constexpr (!BF16) mx = absmax4(mx, v[s]);
    }
#ifdef DGMX_STAGE_TIMING
    if (tid == 0 && mx >= 0.f) TS_MARK(true, 10); // after thread 0's field loads have landed (FP16)
#endif
    if (tid < kTileS * 4) {
      s_face[tid * 3 + 0] = g0;
      s_face[tid * 3 + 1] = g1;
      s_face[tid * 3 + 2] = make_float4(__int_as_float(cn.x), __int_as_float(cn.y), 0.f, 0.f);
    }
    TS_MARK(tid == 0, 12);
    if (issuer) umma::bulk_wait_read_all();
    TS_MARK(issuer, 11);
    __syncthreads();
    TS_MARK(tid == 0, 1);
    {
      float sc1 = 1.f, inv1r = 1.f;
      if constexpr (!BF16) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        row_scale(mx, sc1, inv1r);
        if (cr1 >= 0 && lane < 8) s_inv1[cr1] = inv1r;
      }
#pragma unroll
      for (int s = 0; s < R1; ++s) {
        const int k = kq1 + 16 * s;
        if (cr1 >= 0 && k < T::K1) {
          if (k < NPP) *reinterpret_cast<float4 *>(s_u + f1 * FS + e1 * NPP + k) = v[s];
          float4 w = v[s];
          if constexpr (!BF16) {
            const float2 a01 = f2mul(make_float2(w.x, w.y), f2(sc1)), a23 = f2mul(make_float2(w.z, w.w), f2(sc1));
            w = make_float4(a01.x, a01.y, a23.x, a23.y);
          }
          uint2 hi, lo;
          split2<BF16>(w.x, w.y, hi.x, lo.x);
          split2<BF16>(w.z, w.w, hi.y, lo.y);
          const uint32_t off = umma::kmajor_offset(uint32_t(r1), uint32_t(k), uint32_t(T::K1));
          *reinterpret_cast<uint2 *>(smem + off) = hi;
          *reinterpret_cast<uint2 *>(smem + T::A1B + off) = lo;
        }
      }
    }
    umma::fence_proxy_async();
    __syncthreads();
    TS_MARK(tid == 0, 2);

    // ---- 3. local differentiation, streamed operator slices
    if (issuer) {
      umma::fence_after_sync();
      // Dr, Ds: rows 0 .. 2NB-1 of a half slice (N = 2NB); Dt: rows 2NB .. 3NB-1
      const uint32_t idesc2 = umma::make_idesc(BF16, 128, uint32_t(2 * NB));
      const uint32_t idesc1 = umma::make_idesc(BF16, 128, uint32_t(NB));
      const uint64_t ah0 = umma::make_desc(sbase, 128, T::K1 * 16), al0 = umma::make_desc(sbase + T::A1B, 128, T::K1 * 16);
      for (int kk = 0; kk < T::KS1; ++kk) {
        ok = consume([&](uint32_t b) {
          const uint64_t ko = uint64_t(kk) * 16u;
          const uint32_t lo = b + uint32_t(3 * NB * 32), dt3 = uint32_t(2 * NB * 32);
          const uint64_t bh = umma::make_desc(b, 128, 256), bl = umma::make_desc(lo, 128, 256);
          const uint64_t th = umma::make_desc(b + dt3, 128, 256), tl = umma::make_desc(lo + dt3, 128, 256);
          const uint32_t acc = kk > 0 ? 1u : 0u;
          umma::mma_f16(tmem, ah0 + ko, bh, idesc2, acc);
          umma::mma_f16(tmem, ah0 + ko, bl, idesc2, 1u);
          umma::mma_f16(tmem, al0 + ko, bh, idesc2, 1u);
          umma::mma_f16(tmem + uint32_t(2 * NB), ah0 + ko, th, idesc1, acc);
          umma::mma_f16(tmem + uint32_t(2 * NB), ah0 + ko, tl, idesc1, 1u);
          umma::mma_f16(tmem + uint32_t(2 * NB), al0 + ko, th, idesc1, 1u);
        }) && ok;
      }
      umma::commit(bar1);
      TS_MARK(true, 13);
    }

    // ---- 4. neighbour traces and upwind flux (overlaps GEMM1), in registers
    float fl[R2][2][6];
    if (warp < kFluxWarps) {
#pragma unroll
      for (int s0 = 0; s0 < R2; s0 += BATCH) {
        float qp[BATCH][2][6];
        int lidx[BATCH][2];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
          const int s = s0 + b;
          const int blk = warp + kFluxWarps * s;
          const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            lidx[b][h] = -1;
#pragma unroll
            for (int c = 0; c < 6; ++c) qp[b][h][c] = 0.f;
          }
          if (s < R2 && blk < NBLK && fm < NFF && e < ne) {
            const int f = fm / NFP, mm = fm - f * NFP;
            const float4 r2 = s_face[(e * 4 + f) * 3 + 2];
            const int conn = __float_as_int(r2.y);
            if (conn != kBoundaryConn) {
              const int k2 = __float_as_int(r2.x);
              const int64_t el = int64_t(k2) - k0;
              const bool local = el >= 0 && el < ne;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int node = s_nb[conn * NFP + mm + h];
                if (local) {
                  lidx[b][h] = int(el) * NPP + node;
                } else {
                  const float *up = a.u + int64_t(k2) * NPP + node;
#pragma unroll
                  for (int c = 0; c < 6; ++c) qp[b][h][c] = __ldg(up + c * KN);
                }
              }
            }
          }
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
          const int s = s0 + b;
          if (s >= R2) break;
          const int blk = warp + kFluxWarps * s;
          const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 6; ++c) fl[s][h][c] = 0.f;
          if (blk < NBLK && fm < NFF && e < ne) {
            const int f = fm / NFP;
            const float4 g0 = s_face[(e * 4 + f) * 3 + 0], w1 = s_face[(e * 4 + f) * 3 + 1];
            const bool wall = __float_as_int(s_face[(e * 4 + f) * 3 + 2].y) == kBoundaryConn;
            {
              // both nodes of the pair at once (Nfp is even: both are face nodes)
              const int vm0 = s_fm[fm], vm1 = s_fm[fm + 1];
              float2 qm[6], q[6], o[6];
#pragma unroll
              for (int c = 0; c < 6; ++c) qm[c] = make_float2(s_u[c * FS + e * NPP + vm0], s_u[c * FS + e * NPP + vm1]);
#pragma unroll
              for (int c = 0; c < 6; ++c)
                q[c] = make_float2(lidx[b][0] >= 0 ? s_u[c * FS + lidx[b][0]] : qp[b][0][c],
                                   lidx[b][1] >= 0 ? s_u[c * FS + lidx[b][1]] : qp[b][1][c]);
              if (wall) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  q[c] = make_float2(-qm[c].x, -qm[c].y);
                  q[c + 3] = qm[c + 3];
                }
              }
              maxwell_flux_w2(g0, qm, q, w1, a.alpha, o);
#pragma unroll
              for (int c = 0; c < 6; ++c) {
                fl[s][0][c] = o[c].x;
                fl[s][1][c] = o[c].y;
              }
            }
          }
          if constexpr (!BF16) {
            // FP16: one scale per element and field type (E, H), from the
            // largest exponent over the element's fluxes of that type (packed
            // exponents, bytewise maximum over the element's 8 lanes)
            if (blk < NBLK) { // warp-uniform
              uint32_t mE = 0u, mH = 0u;
#pragma unroll
              for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  mE = max(mE, __float_as_uint(fabsf(fl[s][h][c])));
                  mH = max(mH, __float_as_uint(fabsf(fl[s][h][c + 3])));
                }
              uint32_t wx = ((mE >> 23) & 0xFFu) | (((mH >> 23) & 0xFFu) << 8);
#pragma unroll
              for (int o = 1; o < 8; o <<= 1) wx = __vmaxu4(wx, __shfl_xor_sync(0xffffffffu, wx, o));
              if (kp == 0) {
                atomicMax(s_ex2 + 2 * e, wx & 0xFFu);
                atomicMax(s_ex2 + 2 * e + 1, (wx >> 8) & 0xFFu);
              }
            }
          }
        }
      }
    }
    TS_MARK(tid == 0, 3);
    // A2 overwrites A1: GEMM1 must have completed
    ok = umma::mbar_wait_bounded(bar1, phase, wlim) && ok;
    __syncthreads();
    TS_MARK(tid == 0, 4);

    // ---- 5. split the face fluxes into the A2 operand
    if (warp < kFluxWarps) {
#pragma unroll
      for (int s = 0; s < R2; ++s) {
        const int blk = warp + kFluxWarps * s;
        const int e = 4 * (blk / KGF) + eo, fm = 16 * (blk % KGF) + 2 * kp;
        if (blk < NBLK) {
          float sc2[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) sc2[c] = 1.f;
          if constexpr (!BF16) {
            float inv;
            row_scale(__uint_as_float(s_ex2[2 * e] << 23), sc2[0], inv);
            row_scale(__uint_as_float(s_ex2[2 * e + 1] << 23), sc2[3], inv);
            sc2[1] = sc2[2] = sc2[0];
            sc2[4] = sc2[5] = sc2[3];
          }
          // the element's six rows share a quarter; a column pair is one
          // 32-bit word of a core-matrix row
          const uint32_t r0 = uint32_t(32 * (e / 5) + 6 * (e % 5));
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            uint32_t hi, lo;
            const float2 x = f2mul(make_float2(fl[s][0][c], fl[s][1][c]), f2(sc2[c]));
            split2<BF16>(x.x, x.y, hi, lo);
            const uint32_t o = T::a2_offset(r0 + uint32_t(c), uint32_t(fm));
            *reinterpret_cast<uint32_t *>(smem + o) = hi;
            *reinterpret_cast<uint32_t *>(smem + T::A2B + o) = lo;
          }
        }
      }
    }
    umma::fence_proxy_async();
    __syncthreads();
    TS_MARK(tid == 0, 5);

    // ---- 6. flux lifting (streamed slices); meanwhile the residual rows are read
    if (issuer) {
      umma::fence_after_sync();
      const uint32_t idesc = umma::make_idesc(BF16, 128, uint32_t(NB));
      const uint64_t ah0 = umma::make_desc(sbase, T::A2LBO, T::A2SBO);
      const uint64_t al0 = umma::make_desc(sbase + T::A2B, T::A2LBO, T::A2SBO);
      const uint32_t dt = tmem + uint32_t(3 * NB);
      for (int g = 0; g < T::NS2; ++g) {
        ok = consume([&](uint32_t b) {
#pragma unroll
          for (int j = 0; j < T::G2; ++j) {
            const int kk = g * T::G2 + j;
            if (kk >= T::KS2) break;
            const uint64_t ko = uint64_t(kk) * uint64_t(2 * T::A2LBO / 16); // two core matrices of A2
            const uint32_t sb = b + uint32_t(j * T::SUB);
            const uint64_t bh = umma::make_desc(sb, 128, 256), bl = umma::make_desc(sb + uint32_t(NB * 32), 128, 256);
            umma::mma_f16(dt, ah0 + ko, bh, idesc, kk > 0 ? 1u : 0u);
            umma::mma_f16(dt, ah0 + ko, bl, idesc, 1u);
            umma::mma_f16(dt, al0 + ko, bh, idesc, 1u);
          }
        }) && ok;
      }
      umma::commit(bar2);
      TS_MARK(true, 14);
    }
    const bool live = lane_used && e_loc < ne;
    const int64_t k = k0 + e_loc;
    float g1r = 0.f, g1s = 0.f, g1t = 0.f, g2r = 0.f, g2s = 0.f, g2t = 0.f, w = 0.f;
    if (live) {
      const float *g = a.geo + k * G_STRIDE;
      g1r = __ldg(g + G_RX + dl1), g1s = __ldg(g + G_SX + dl1), g1t = __ldg(g + G_TX + dl1);
      g2r = __ldg(g + G_RX + dl2), g2s = __ldg(g + G_SX + dl2), g2t = __ldg(g + G_TX + dl2);
      w = __ldg(g + (isE ? G_IEPS : G_IMU));
    }
    float inv2 = 1.f;
    if constexpr (!BF16) {
      // the row's FP16 scale is undone through the metric factors of the chain rule
      float sc;
      const float inv1 = s_inv1[lane_used ? ridx : 0];
      g1r *= inv1, g1s *= inv1, g1t *= inv1, g2r *= inv1, g2s *= inv1, g2t *= inv1;
      row_scale(__uint_as_float(s_ex2[lane_used ? 2 * e_loc + fld / 3 : 0] << 23), sc, inv2);
    }
    // residual of one 8-node chunk of this lane's row (loaded one chunk ahead)
    auto load_res = [&](int ch, float4 &r0, float4 &r1) {
      r0 = r1 = make_float4(0.f, 0.f, 0.f, 0.f);
      // (the first LSERK4 stage has a = 0: the residual it overwrites is not read)
      if (MODE != MODE_LSERK || a.rk_a == 0.f || !live || ch >= ch1) return;
      const float *rp = a.res + fld * KN + k * NPP + ch * 8;
      r0 = ldg4(rp);
      if (ch * 8 + 4 < NPP) r1 = ldg4(rp + 4);
    };
    float4 rn0, rn1;
    load_res(ch0, rn0, rn1);
    TS_MARK(tid == 0, 6);
    ok = umma::mbar_wait_bounded(bar2, phase, wlim) && ok;
    TS_MARK(tid == 0, 7);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err_flag, 1);
      // the matrix operations issued for this tile complete before tensor
      // memory is released (bar2 is committed after them in every case)
      if (issuer) umma::mbar_wait_bounded(bar2, phase);
      break;
    }
    TS_MARK(tid == 0, 8);
    umma::fence_after_sync();

    // ---- 7. epilogue: chain rule (eq. dg-reference-matrices), curls, lifted
    // flux, material scale, update; results to shared memory
#pragma unroll
    for (int c = 0; c < CPP; ++c) {
      const int ch = ch0 + c;
      if (ch >= ch1) break;
      const int i0 = ch * 8;
      const float rsv[8] = {rn0.x, rn0.y, rn0.z, rn0.w, rn1.x, rn1.y, rn1.z, rn1.w};
      load_res(ch + 1, rn0, rn1);
      float ur[8], us[8], ut[8], lf[8], vol[8];
      umma::tmem_ld8(lane_taddr + uint32_t(i0), ur);
      umma::tmem_ld8(lane_taddr + uint32_t(NB + i0), us);
      umma::tmem_ld8(lane_taddr + uint32_t(2 * NB + i0), ut);
      umma::tmem_ld8(lane_taddr + uint32_t(3 * NB + i0), lf);
      umma::tmem_wait_ld();
      umma::reg_fence8(ur);
      umma::reg_fence8(us);
      umma::reg_fence8(ut);
      umma::reg_fence8(lf);
      // two nodes at a time in packed FP32 pairs; vol = sign (v1 - v2), with
      // sign +1 on E rows and -1 on H rows
#pragma unroll
      for (int n = 0; n < 8; n += 2) {
        const float2 r2 = make_float2(ur[n], ur[n + 1]), s2 = make_float2(us[n], us[n + 1]),
                     t2 = make_float2(ut[n], ut[n + 1]);
        const float2 p1 = f2fma(f2(g1t), t2, f2fma(f2(g1s), s2, f2mul(f2(g1r), r2)));
        const float2 p2 = f2fma(f2(g2t), t2, f2fma(f2(g2s), s2, f2mul(f2(g2r), r2)));
        const float2 v1 = make_float2(__shfl_sync(0xffffffffu, p1.x, src1), __shfl_sync(0xffffffffu, p1.y, src1));
        const float2 v2 = make_float2(__shfl_sync(0xffffffffu, p2.x, src2), __shfl_sync(0xffffffffu, p2.y, src2));
        const float2 d = f2mul(f2(sgn), f2sub(v1, v2));
        vol[n] = d.x;
        vol[n + 1] = d.y;
      }
      if (live) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = i0 + 4 * h;
          if (i < NPP) {
            // packed FP32 pairs: r = (vol + lift inv2) w, then the update
            float2 r2[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int j = 4 * h + 2 * q;
              r2[q] = f2mul(f2fma(make_float2(lf[j], lf[j + 1]), f2(inv2), make_float2(vol[j], vol[j + 1])), f2(w));
              if (i + 2 * q >= NP) r2[q].x = 0.f;
              if (i + 2 * q + 1 >= NP) r2[q].y = 0.f;
            }
            if (MODE == MODE_RHS) {
              *reinterpret_cast<float4 *>(s_out + soff + i) = make_float4(r2[0].x, r2[0].y, r2[1].x, r2[1].y);
            } else {
              float4 *up = reinterpret_cast<float4 *>(s_u + soff + i);
              const float4 uo = *up;
              const float2 uov[2] = {make_float2(uo.x, uo.y), make_float2(uo.z, uo.w)};
              float2 nr[2], nu[2];
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int j = 4 * h + 2 * q;
                nr[q] = f2fma(f2(a.rk_a), make_float2(rsv[j], rsv[j + 1]), f2mul(f2(a.dt), r2[q]));
                nu[q] = f2fma(f2(a.rk_b), nr[q], uov[q]);
                if (i + 2 * q >= NP) nr[q].x = nu[q].x = 0.f;
                if (i + 2 * q + 1 >= NP) nr[q].y = nu[q].y = 0.f;
              }
              *reinterpret_cast<float4 *>(s_out + soff + i) = make_float4(nr[0].x, nr[0].y, nr[1].x, nr[1].y);
              *up = make_float4(nu[0].x, nu[0].y, nu[1].x, nu[1].y);
            }
          }
        }
      }
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    TS_MARK(tid == 0, 9);
    if (issuer) {
      const uint32_t rowbytes = uint32_t(ne * NPP * 4);
      for (int f = 0; f < 6; ++f) {
        if (MODE == MODE_RHS) {
          umma::bulk_s2g(a.rhs + f * KN + k0 * NPP, s_out + f * FS, rowbytes);
        } else {
          umma::bulk_s2g(a.res + f * KN + k0 * NPP, s_out + f * FS, rowbytes);
          umma::bulk_s2g(a.u_out + f * KN + k0 * NPP, s_u + f * FS, rowbytes);
        }
      }
      umma::bulk_commit();
    }
    if (!BF16 && tid < 2 * kTileS) s_ex2[tid] = 0u;
    phase ^= 1u;
  }
  if (issuer) umma::bulk_wait_all();
  // the slices produced but not consumed must land before exit
  if (issuer)
    for (uint32_t j = jstep; j < jprod; ++j)
      umma::mbar_wait_bounded(full + j % uint32_t(kSlots), (j / uint32_t(kSlots)) & 1u);
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, T::TCOLS);
}

template <int N>
std::vector<uint8_t> build_stream(const RefOps &o, bool bf16) {
  using T = TS<N>;
  std::vector<uint8_t> blk(T::STREAM, 0);
  auto put = [&](size_t base_hi, size_t base_lo, int row, int k, double v) {
    uint16_t hb, lb;
    if (bf16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(float(v));
      const __nv_bfloat16 l = __float2bfloat16_rn(float(v - double(__bfloat162float(h))));
      std::memcpy(&hb, &h, 2);
      std::memcpy(&lb, &l, 2);
    } else {
      const __half h = __float2half_rn(float(v));
      const __half l = __float2half_rn(float(v - double(__half2float(h))));
      std::memcpy(&hb, &h, 2);
      std::memcpy(&lb, &l, 2);
    }
    const uint32_t off = umma::kmajor_offset(uint32_t(row), uint32_t(k), 16u); // one 16-wide K slice
    std::memcpy(&blk[base_hi + off], &hb, 2);
    std::memcpy(&blk[base_lo + off], &lb, 2);
  };
  const std::vector<double> *Ds[3] = {&o.Dr, &o.Ds, &o.Dt};
  for (int kk = 0; kk < T::KS1; ++kk) {
    const size_t hi = slice_offset<N>(kk), lo = hi + size_t(3) * T::NB * 32;
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < T::NP; ++i)
        for (int k = 0; k < 16 && 16 * kk + k < T::NP; ++k)
          put(hi, lo, d * T::NB + i, k, (*Ds[d])[size_t(i) * T::NP + 16 * kk + k]);
  }
  for (int kk = 0; kk < T::KS2; ++kk) {
    const size_t hi = slice_offset<N>(T::KS1 + kk / T::G2) + size_t(kk % T::G2) * T::SUB, lo = hi + size_t(T::NB) * 32;
    for (int i = 0; i < T::NP; ++i)
      for (int k = 0; k < 16 && 16 * kk + k < T::NFF; ++k)
        put(hi, lo, i, k, o.LIFT[size_t(i) * T::NFF + 16 * kk + k]);
  }
  return blk;
}

template <int N, int MODE, bool BF16>
cudaError_t launch_streamed_kernel(const StageArgs &a, const TcState &st, int *flag, cudaStream_t s) {
  using T = TS<N>;
  auto kern = k_stage_tc_streamed<N, MODE, BF16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
  if (e != cudaSuccess) return e;
  const int ntiles = int((a.K + kTileS - 1) / kTileS);
  const int grid = ntiles < st.sms ? ntiles : st.sms;
  return launch_pdl(kern, dim3(unsigned(grid)), dim3(kThreadsS), size_t(T::SMEM), s, a,
                    static_cast<const uint8_t *>(st.d_ops), ntiles, flag);
}

template <int N>
cudaError_t launch_streamed_order(int mode, bool bf16, const StageArgs &a, const TcState &st, int *flag,
                                  cudaStream_t s) {
  if (mode == MODE_RHS)
    return bf16 ? launch_streamed_kernel<N, MODE_RHS, true>(a, st, flag, s)
                : launch_streamed_kernel<N, MODE_RHS, false>(a, st, flag, s);
  return bf16 ? launch_streamed_kernel<N, MODE_LSERK, true>(a, st, flag, s)
              : launch_streamed_kernel<N, MODE_LSERK, false>(a, st, flag, s);
}

} // namespace

namespace tcc {

std::vector<uint8_t> build_streamed_operators(int N, const RefOps &o, bool bf16) {
  return N == 6 ? build_stream<6>(o, bf16) : build_stream<7>(o, bf16);
}

cudaError_t launch_tc_streamed(int N, int mode, bool bf16, const StageArgs &a, const TcState &st, int *flag,
                               cudaStream_t s) {
  switch (N) {
  case 6: return launch_streamed_order<6>(mode, bf16, a, st, flag, s);
  case 7: return launch_streamed_order<7>(mode, bf16, a, st, flag, s);
  default: return cudaErrorNotSupported;
  }
}

} // namespace tcc

#ifdef DGMX_STAGE_TIMING
extern "C" int dgmx_tcs_trace(uint32_t *host) {
  return int(cudaMemcpyFromSymbol(host, g_tcs_trace, sizeof(g_tcs_trace)));
}
#endif
} // namespace dgmx
