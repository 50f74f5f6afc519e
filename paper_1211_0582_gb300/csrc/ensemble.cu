// Ensembles of independent meshes: upload as one disjoint union, advance all
// of them in one persistent cooperative launch per call, replayed from a
// captured CUDA graph, with the elements-per-block of the launch chosen by a
// small autotuner (timed trial runs of every candidate, result cached in a
// text file keyed by GPU name, order and ensemble size).
//
// Section 3 (work decomposition, Fig. el-local-workgroup) and Section 5
// (Fig. tuning-study): the number of elements a work group processes is a
// tuning parameter whose best value no simple model predicts, so it is
// measured.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/dgmx.h"
#include "common.cuh"
#include "ensemble.cuh"
#include "tc_api.h"

namespace dgmx {

int ensemble_candidate_eb_n1(int);
int ensemble_candidate_eb_n2(int);
int ensemble_candidate_eb_n3(int);
int ensemble_candidate_eb_n4(int);
int ensemble_candidate_eb_n5(int);
int ensemble_candidate_eb_n6(int);
int ensemble_candidate_eb_n7(int);
int ensemble_candidate_eb_n8(int);
int ensemble_candidate_eb_n9(int);

extern template cudaError_t launch_ensemble_order<1>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<2>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<3>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<4>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<5>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<6>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<7>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<8>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);
extern template cudaError_t launch_ensemble_order<9>(int, const StageArgs &, const StageCoeffs &, float *, float *, int, GridBarrier *, int *, cudaStream_t, int, int *);

namespace {

constexpr int kEbCandidates = 4;                   // elements per block
constexpr int kCandidates = 2 * kEbCandidates;     // x occupancy levels (all resident blocks, half)
constexpr int kTcTileElems = 20; // elements per tile of the tensor-core form

int candidate_eb(int N, int cand) {
  const int i = cand % kEbCandidates;
  switch (N) {
  case 1: return ensemble_candidate_eb_n1(i);
  case 2: return ensemble_candidate_eb_n2(i);
  case 3: return ensemble_candidate_eb_n3(i);
  case 4: return ensemble_candidate_eb_n4(i);
  case 5: return ensemble_candidate_eb_n5(i);
  case 6: return ensemble_candidate_eb_n6(i);
  case 7: return ensemble_candidate_eb_n7(i);
  case 8: return ensemble_candidate_eb_n8(i);
  default: return ensemble_candidate_eb_n9(i);
  }
}

cudaError_t launch_ensemble(int N, int cand, const StageArgs &a, const StageCoeffs &rk, float *ua, float *ub,
                            int nsteps, GridBarrier *gb, int *flag, cudaStream_t s, int sms, int *used) {
  switch (N) {
  case 1: return launch_ensemble_order<1>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 2: return launch_ensemble_order<2>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 3: return launch_ensemble_order<3>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 4: return launch_ensemble_order<4>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 5: return launch_ensemble_order<5>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 6: return launch_ensemble_order<6>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 7: return launch_ensemble_order<7>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  case 8: return launch_ensemble_order<8>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  default: return launch_ensemble_order<9>(cand, a, rk, ua, ub, nsteps, gb, flag, s, sms, used);
  }
}

struct EnsembleState {
  int M = 0;
  std::vector<int64_t> offsets; // M + 1 element offsets
  GridBarrier *gb = nullptr;
  int sms = 0;
  int best = -1;                // chosen candidate
  float ms[kCandidates] = {};
  int bps[kCandidates] = {}; // blocks per SM each candidate launched with
  std::string gpu;
  // captured graph of one call (rebuilt when its arguments change)
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  float *g_u = nullptr, *g_res = nullptr;
  int g_steps = -1;
  float g_alpha = 0.f;
  bool graph_ok = true;
};

EnsembleState *state(dg_ctx *c) { return static_cast<EnsembleState *>(c->ens); }

int fail(dg_ctx *ctx, int code, const std::string &msg) {
  ctx->err = msg;
  return code;
}

std::string cache_path() {
  const char *p = std::getenv("DGMX_TUNE_CACHE");
  if (p && *p) return p;
  const char *home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/dgmx_ensemble_tune.txt";
}

std::string cache_key(const EnsembleState &st, int N, int precision, int64_t K) {
  std::ostringstream os;
  os << st.gpu << "|N=" << N << "|P=" << precision << "|K=" << K;
  return os.str();
}

// One line per entry: "<key>\t<candidate>".
int cache_lookup(const std::string &key) {
  std::ifstream in(cache_path());
  std::string line;
  int found = -1;
  while (std::getline(in, line)) {
    const size_t tab = line.rfind('\t');
    if (tab != std::string::npos && line.substr(0, tab) == key) found = std::atoi(line.c_str() + tab + 1);
  }
  return found;
}

void cache_store(const std::string &key, int cand) {
  std::ofstream out(cache_path(), std::ios::app);
  if (out) out << key << '\t' << cand << '\n';
}

StageArgs ens_args(const dg_ctx *c, float alpha) {
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
  a.dt_geo = 1;
  return a;
}

StageCoeffs coeffs() {
  StageCoeffs rk{};
  for (int s = 0; s < 5; ++s) {
    rk.a[s] = float(kLserkA[s]);
    rk.b[s] = float(kLserkB[s]);
  }
  return rk;
}

// Enqueue one call: persistent launch for nsteps (the tensor-core form in
// split-precision contexts at N <= 5, whose tile is fixed by the 128-row
// matrix operation; the FP32 form with candidate `cand` otherwise), then the
// copy back when the stage count is odd (the result then sits in the scratch
// buffer).
cudaError_t enqueue(dg_ctx *c, EnsembleState &st, int cand, float *u, float *res, int nsteps, float alpha,
                    cudaStream_t s) {
  StageArgs a = ens_args(c, alpha);
  a.res = res;
  cudaError_t e = tc_ensemble_supported(c)
                      ? launch_tc_ensemble(c, a, coeffs(), u, c->d_scratch, nsteps, st.gb, s)
                      : launch_ensemble(c->N, cand, a, coeffs(), u, c->d_scratch, nsteps, st.gb, c->d_flag + 1, s,
                                        st.sms, &st.bps[cand]);
  if (e == cudaSuccess && (5 * nsteps) % 2 == 1)
    e = cudaMemcpyAsync(u, c->d_scratch, size_t(6) * c->K * c->ops.Npad * sizeof(float), cudaMemcpyDeviceToDevice, s);
  return e;
}

void free_graph(EnsembleState &st) {
  if (st.exec) cudaGraphExecDestroy(st.exec);
  st.exec = nullptr;
  st.g_steps = -1;
}

} // namespace

cudaError_t ensemble_reset_barrier(dg_ctx *c) {
  EnsembleState *st = state(c);
  if (!st || !st->gb) return cudaSuccess;
  return cudaMemsetAsync(st->gb, 0, sizeof(GridBarrier), c->stream);
}

void ensemble_drop_graph(dg_ctx *c) {
  EnsembleState *st = state(c);
  if (st) free_graph(*st);
}

void ensemble_free(dg_ctx *c) {
  EnsembleState *st = state(c);
  if (!st) return;
  free_graph(*st);
  if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
  if (st->gb) cudaFree(st->gb);
  delete st;
  c->ens = nullptr;
}

} // namespace dgmx

using namespace dgmx;

extern "C" {

int dg_ensemble_upload(dg_ctx *ctx, int M, const int64_t *Nv, const double *VX, const double *VY, const double *VZ,
                       const int64_t *K, const int32_t *EToV, const float *eps, const double *dt) {
  if (!ctx) return DG_ERR_ARG;
  if (M < 1 || !Nv || !K || !VX || !VY || !VZ || !EToV || !dt)
    return fail(ctx, DG_ERR_ARG, "dg_ensemble_upload: bad arguments");
  int64_t nv_tot = 0, k_tot = 0;
  for (int i = 0; i < M; ++i) {
    if (Nv[i] < 4 || K[i] < 1 || !(dt[i] > 0.0) || !std::isfinite(dt[i]))
      return fail(ctx, DG_ERR_ARG, "dg_ensemble_upload: mesh " + std::to_string(i) + " has bad sizes or time step");
    nv_tot += Nv[i];
    k_tot += K[i];
  }
  // disjoint union: shift each mesh's vertex indices by the vertices before it
  std::vector<int32_t> etov(size_t(k_tot) * 4);
  std::vector<float> dte(k_tot);
  std::vector<int64_t> offs(M + 1, 0);
  int64_t vbase = 0, kbase = 0;
  for (int i = 0; i < M; ++i) {
    for (int64_t q = 0; q < K[i] * 4; ++q) {
      const int32_t v = EToV[kbase * 4 + q];
      if (v < 0 || v >= Nv[i]) return fail(ctx, DG_ERR_MESH, "dg_ensemble_upload: vertex index out of range in mesh " + std::to_string(i));
      etov[kbase * 4 + q] = int32_t(vbase + v);
    }
    for (int64_t k = 0; k < K[i]; ++k) dte[kbase + k] = float(dt[i]);
    vbase += Nv[i];
    kbase += K[i];
    offs[i + 1] = kbase;
  }
  if (vbase > 0x7fffffff) return fail(ctx, DG_ERR_ARG, "dg_ensemble_upload: too many vertices");
  ensemble_free(ctx);
  int rc = dg_mesh_upload(ctx, nv_tot, VX, VY, VZ, k_tot, etov.data(), eps, nullptr, nullptr);
  if (rc) return rc;
  EnsembleState *st = new EnsembleState();
  st->M = M;
  st->offsets = offs;
  cudaError_t e = cudaMalloc(&st->gb, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMemsetAsync(st->gb, 0, sizeof(GridBarrier), ctx->stream);
  // per-element time step into the spare slot of the geometry record
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(ctx->d_geo + G_DT, G_STRIDE * sizeof(float), dte.data(), sizeof(float), sizeof(float),
                          size_t(k_tot), cudaMemcpyHostToDevice, ctx->stream);
  int dev = 0;
  cudaDeviceProp prop{};
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  ctx->ens = st;
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_ensemble_upload: ") + cudaGetErrorString(e));
  st->sms = prop.multiProcessorCount;
  st->gpu = prop.name;
  return DG_OK;
}

int dg_ensemble_layout(const dg_ctx *ctx, int *M, int64_t *offsets) {
  if (!ctx || !ctx->ens) return DG_ERR_ARG;
  const EnsembleState *st = static_cast<const EnsembleState *>(ctx->ens);
  if (M) *M = st->M;
  if (offsets)
    for (int i = 0; i <= st->M; ++i) offsets[i] = st->offsets[i];
  return DG_OK;
}

int dg_ensemble_tune(dg_ctx *ctx, int force) {
  dgmx::NvtxRange nvtx_range("dg_ensemble_tune");
  if (!ctx || !ctx->ens) return DG_ERR_ARG;
  EnsembleState &st = *state(ctx);
  const std::string key = cache_key(st, ctx->N, ctx->precision, ctx->K);
  if (!force) {
    const int c = cache_lookup(key);
    if (c >= 0 && c < kCandidates) {
      st.best = c;
      return DG_OK;
    }
  }
  const size_t fl = size_t(6) * ctx->K * ctx->ops.Npad;
  float *u = nullptr, *r = nullptr;
  if (cudaMalloc(&u, fl * 4) != cudaSuccess || cudaMalloc(&r, fl * 4) != cudaSuccess) {
    cudaGetLastError();
    if (u) cudaFree(u);
    return fail(ctx, DG_ERR_OOM, "dg_ensemble_tune: device allocation failed");
  }
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaMemsetAsync(u, 0, fl * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(r, 0, fl * 4, s);
  float best_ms = 1e30f;
  int best = -1;
  const bool tc = tc_ensemble_supported(ctx); // one configuration: nothing to choose
  for (int cand = 0; cand < kCandidates && e == cudaSuccess; ++cand) {
    st.ms[cand] = 0.f;
    if (tc && cand > 0) continue;
    const int i = cand % kEbCandidates;
    if (i > 0 && candidate_eb(ctx->N, cand) == candidate_eb(ctx->N, cand - 1)) continue;
    // the second occupancy level only where it launches fewer blocks than the first
    if (cand >= kEbCandidates && (st.ms[i] == 0.f || st.bps[i] <= 1)) continue;
    float t_min = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = enqueue(ctx, st, cand, u, r, 2, 1.f, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      t_min = std::min(t_min, ms);
    }
    st.ms[cand] = t_min / 2.f; // per step
    if (t_min < best_ms) {
      best_ms = t_min;
      best = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(u);
  cudaFree(r);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_ensemble_tune: ") + cudaGetErrorString(e));
  st.best = best;
  cache_store(key, best);
  free_graph(st);
  return DG_OK;
}

int dg_ensemble_tuning(const dg_ctx *ctx, int *best_eb, int *eb, float *ms_per_step) {
  if (!ctx || !ctx->ens) return DG_ERR_ARG;
  const EnsembleState *st = static_cast<const EnsembleState *>(ctx->ens);
  const bool tc = tc_ensemble_supported(ctx);
  auto eb_of = [&](int i) { return tc ? (i == 0 ? kTcTileElems : 0) : candidate_eb(ctx->N, i); };
  if (best_eb) *best_eb = st->best >= 0 ? eb_of(st->best % kEbCandidates) : 0;
  for (int i = 0; i < kEbCandidates; ++i) {
    if (eb) eb[i] = eb_of(i);
    // the better of the elements-per-block candidate's occupancy levels
    const float a = st->ms[i], b = st->ms[i + kEbCandidates];
    if (ms_per_step) ms_per_step[i] = (b > 0.f && (a == 0.f || b < a)) ? b : a;
  }
  return DG_OK;
}

int dg_ensemble_tuning_grid(const dg_ctx *ctx, int *best, int *eb, int *blocks_per_sm, float *ms_per_step) {
  if (!ctx || !ctx->ens) return DG_ERR_ARG;
  const EnsembleState *st = static_cast<const EnsembleState *>(ctx->ens);
  const bool tc = tc_ensemble_supported(ctx);
  if (best) *best = st->best;
  for (int c = 0; c < kCandidates; ++c) {
    if (eb) eb[c] = tc ? (c == 0 ? kTcTileElems : 0) : candidate_eb(ctx->N, c);
    if (blocks_per_sm) blocks_per_sm[c] = st->ms[c] > 0.f ? (tc ? 1 : st->bps[c]) : 0;
    if (ms_per_step) ms_per_step[c] = st->ms[c];
  }
  return DG_OK;
}

int dg_ensemble_step(dg_ctx *ctx, float *u, float *res, int nsteps, float alpha) {
  dgmx::NvtxRange nvtx_range("dg_ensemble_step");
  if (!ctx) return DG_ERR_ARG;
  if (!ctx->ens) return fail(ctx, DG_ERR_ARG, "dg_ensemble_step: no ensemble uploaded");
  if (!u || !res || ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(res)) & 15u))
    return fail(ctx, DG_ERR_ARG, "dg_ensemble_step: null or misaligned field");
  if (nsteps < 1 || !std::isfinite(alpha)) return fail(ctx, DG_ERR_ARG, "dg_ensemble_step: bad nsteps/alpha");
  EnsembleState &st = *state(ctx);
  if (st.best < 0) {
    int rc = dg_ensemble_tune(ctx, 0);
    if (rc) return rc;
  }
  cudaError_t e = cudaSuccess;
  if (st.graph_ok && (!st.exec || st.g_u != u || st.g_res != res || st.g_steps != nsteps || st.g_alpha != alpha)) {
    free_graph(st);
    if (!st.cap_stream) e = cudaStreamCreateWithFlags(&st.cap_stream, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e_launch = enqueue(ctx, st, st.best, u, res, nsteps, alpha, st.cap_stream);
      e = cudaStreamEndCapture(st.cap_stream, &graph);
      if (e == cudaSuccess) e = e_launch;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&st.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      // capture of cooperative launches unavailable: launch directly from now on
      cudaGetLastError();
      st.graph_ok = false;
      free_graph(st);
      e = cudaSuccess;
    } else {
      st.g_u = u;
      st.g_res = res;
      st.g_steps = nsteps;
      st.g_alpha = alpha;
    }
  }
  if (st.graph_ok && st.exec)
    e = cudaGraphLaunch(st.exec, ctx->stream);
  else
    e = enqueue(ctx, st, st.best, u, res, nsteps, alpha, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, DG_ERR_CUDA, std::string("dg_ensemble_step: ") + cudaGetErrorString(e));
  return DG_OK;
}

int dg_ensemble_graph_used(const dg_ctx *ctx) {
  if (!ctx || !ctx->ens) return 0;
  const EnsembleState *st = static_cast<const EnsembleState *>(ctx->ens);
  return st->graph_ok && st->exec ? 1 : 0;
}

} // extern "C"
