// C ABI of libdgmx: context, mesh upload, right-hand side, LSERK4 step,
// energy. Declarations and contracts are in include/dgmx.h.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dgmx.h"
#include "adj_common.cuh"
#include "common.cuh"
#include "tc_api.h"

namespace dgmx {

// Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme.
const double kLserkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                           -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLserkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                           1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                           2277821191437.0 / 14882151754819.0};
const double kLserkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                           2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

} // namespace dgmx

using namespace dgmx;

namespace {

thread_local std::string g_create_error;

int set_err(dg_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_err(dg_ctx *ctx, cudaError_t e, const char *where) {
  return set_err(ctx, DG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_mesh(dg_ctx *c) {
  dfree(c->d_geo);
  dfree(c->d_fgeo);
  dfree(c->d_fmat);
  dfree(c->d_fconn);
  dfree(c->d_DT);
  dfree(c->d_LT);
  dfree(c->d_tab);
  dfree(c->d_Dn);
  dfree(c->d_LF);
  dfree(c->d_M);
  dfree(c->d_scratch);
  dfree(c->d_red);
  dfree(c->d_flag);
  tc_free(c);
  ensemble_free(c);
  adjoint_free(c);
  adj_tc_free(c);
  c->K = 0;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_ready(dg_ctx *ctx) {
  if (!ctx) return DG_ERR_ARG;
  if (ctx->K <= 0) return set_err(ctx, DG_ERR_ARG, "no mesh uploaded");
  return DG_OK;
}

bool overlap(const void *a, const void *b, size_t bytes) {
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

size_t field_bytes(const dg_ctx *c) { return size_t(6) * c->K * c->ops.Npad * sizeof(float); }

StageArgs base_args(const dg_ctx *c) {
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
  return a;
}

cudaError_t launch_stage(dg_ctx *c, int mode, const StageArgs &a) {
  if (c->precision == DG_FP32) return launch_stage_simt(c->N, mode, a, c->stream);
  return launch_stage_tc(c, mode, a);
}

} // namespace

extern "C" {

int dg_create(dg_ctx **out, int N, int precision, void *cuda_stream) {
  if (!out) return set_err(nullptr, DG_ERR_ARG, "dg_create: out is NULL");
  *out = nullptr;
  if (N < 1 || N > kMaxOrder) return set_err(nullptr, DG_ERR_ARG, "dg_create: N must be in 1..9");
  if (precision != DG_FP32 && precision != DG_BF16X3 && precision != DG_FP16X3 && precision != DG_FP32_TC)
    return set_err(nullptr, DG_ERR_ARG, "dg_create: unknown precision");
  if (precision == DG_FP32_TC) precision = DG_FP16X3; // the split that reaches FP32 error
  dg_ctx *c = new (std::nothrow) dg_ctx();
  if (!c) return set_err(nullptr, DG_ERR_OOM, "dg_create: out of host memory");
  c->N = N;
  c->precision = precision;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  std::string err;
  if (!build_refops(N, c->ops, err)) {
    delete c;
    return set_err(nullptr, DG_ERR_ARG, "dg_create: " + err);
  }
  *out = c;
  return DG_OK;
}

int dg_set_node_alpha(dg_ctx *ctx, double alpha) {
  if (!ctx) return DG_ERR_ARG;
  ctx->err.clear();
  if (ctx->K > 0) return set_err(ctx, DG_ERR_ARG, "dg_set_node_alpha: the context already holds a mesh");
  RefOps o;
  std::string err;
  if (!build_refops(ctx->N, o, err, alpha)) return set_err(ctx, DG_ERR_ARG, "dg_set_node_alpha: " + err);
  ctx->ops = std::move(o);
  return DG_OK;
}

double dg_optimised_node_alpha(int N) { return optimised_alpha(N); }

int dg_destroy(dg_ctx *ctx) {
  if (!ctx) return DG_OK;
  free_mesh(ctx);
  delete ctx;
  return DG_OK;
}

const char *dg_last_error(const dg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int dg_layout(const dg_ctx *ctx, int *Np, int *Np_pad, int64_t *K) {
  if (!ctx) return DG_ERR_ARG;
  if (Np) *Np = ctx->ops.Np;
  if (Np_pad) *Np_pad = ctx->ops.Npad;
  if (K) *K = ctx->K;
  return DG_OK;
}

int dg_operators(const dg_ctx *ctx, double *r, double *s, double *t, double *Dr, double *Ds, double *Dt, double *M,
                 double *LIFT, int32_t *Fmask) {
  if (!ctx) return DG_ERR_ARG;
  const RefOps &o = ctx->ops;
  auto cp = [](double *dst, const std::vector<double> &v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  cp(r, o.r);
  cp(s, o.s);
  cp(t, o.t);
  cp(Dr, o.Dr);
  cp(Ds, o.Ds);
  cp(Dt, o.Dt);
  cp(M, o.M);
  cp(LIFT, o.LIFT);
  if (Fmask)
    for (size_t i = 0; i < o.Fmask.size(); ++i) Fmask[i] = o.Fmask[i];
  return DG_OK;
}

int dg_mesh_upload(dg_ctx *ctx, int64_t Nv, const double *VX, const double *VY, const double *VZ, int64_t K,
                   const int32_t *EToV, const float *eps, const float *mu, const int32_t *bc) {
  dgmx::NvtxRange nvtx_range("dg_mesh_upload");
  if (!ctx) return DG_ERR_ARG;
  ctx->err.clear();
  if (!VX || !VY || !VZ || !EToV) return set_err(ctx, DG_ERR_ARG, "dg_mesh_upload: null input array");
  if (Nv < 4 || K < 1) return set_err(ctx, DG_ERR_ARG, "dg_mesh_upload: need Nv >= 4 and K >= 1");
  if (K > (int64_t(1) << 30) / 6) return set_err(ctx, DG_ERR_ARG, "dg_mesh_upload: K too large");
  for (int64_t k = 0; k < K; ++k) {
    if (eps && !(eps[k] > 0.f && std::isfinite(eps[k])))
      return set_err(ctx, DG_ERR_ARG, "dg_mesh_upload: eps must be positive and finite");
    if (mu && !(mu[k] > 0.f && std::isfinite(mu[k])))
      return set_err(ctx, DG_ERR_ARG, "dg_mesh_upload: mu must be positive and finite");
  }
  Connectivity con;
  std::string err;
  if (!build_connectivity(K, Nv, EToV, con, err)) return set_err(ctx, DG_ERR_MESH, "dg_mesh_upload: " + err);
  if (bc)
    for (int64_t q = 0; q < K * 4; ++q)
      if (con.conn[q] == kBoundaryConn && bc[q] != 1)
        return set_err(ctx, DG_ERR_UNSUPPORTED, "dg_mesh_upload: only perfect-conductor boundaries (tag 1)");
  free_mesh(ctx);
  const RefOps &o = ctx->ops;
  const int Np = o.Np, Nfp = o.Nfp, Npad = o.Npad;
  cudaStream_t s = ctx->stream;

  // host-side operator layouts for the CUDA-core kernels
  std::vector<float> DT(size_t(3) * Np * Npad, 0.f), LT(size_t(4) * Nfp * Npad, 0.f);
  const std::vector<double> *Ds[3] = {&o.Dr, &o.Ds, &o.Dt};
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < Np; ++i) DT[(size_t(d) * Np + j) * Npad + i] = float((*Ds[d])[i * Np + j]);
  for (int m = 0; m < 4 * Nfp; ++m)
    for (int i = 0; i < Np; ++i) LT[size_t(m) * Npad + i] = float(o.LIFT[i * 4 * Nfp + m]);
  std::vector<uint8_t> tab(4 * Nfp + 2 * kConnKinds * Nfp);
  for (int q = 0; q < 4 * Nfp; ++q) tab[q] = uint8_t(o.Fmask[q]);
  std::memcpy(tab.data() + 4 * Nfp, o.nbr_node.data(), o.nbr_node.size());
  std::memcpy(tab.data() + 4 * Nfp + kConnKinds * Nfp, o.nbr_fnode.data(), o.nbr_fnode.size());
  std::vector<float> Dn(size_t(3) * Np * Npad, 0.f), LF(size_t(Np) * 4 * Nfp, 0.f);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j) Dn[(size_t(d) * Np + i) * Npad + j] = float((*Ds[d])[i * Np + j]);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < 4 * Nfp; ++m) LF[size_t(i) * 4 * Nfp + m] = float(o.LIFT[i * 4 * Nfp + m]);
  std::vector<int2> fconn(K * 4);
  for (int64_t q = 0; q < K * 4; ++q) fconn[q] = make_int2(con.nbr_elem[q], con.conn[q]);

  double *d_vert = nullptr;
  int32_t *d_EToV = nullptr;
  float *d_eps = nullptr, *d_mu = nullptr;
  auto cleanup = [&]() {
    dfree(d_vert);
    dfree(d_EToV);
    dfree(d_eps);
    dfree(d_mu);
  };
  auto alloc = [&](void **p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
  bool ok = alloc((void **)&ctx->d_geo, size_t(K) * G_STRIDE * sizeof(float)) &&
            alloc((void **)&ctx->d_fgeo, size_t(K) * 4 * sizeof(float4)) &&
            alloc((void **)&ctx->d_fmat, size_t(K) * 4 * sizeof(float4)) &&
            alloc((void **)&ctx->d_fconn, size_t(K) * 4 * sizeof(int2)) &&
            alloc((void **)&ctx->d_DT, DT.size() * sizeof(float)) &&
            alloc((void **)&ctx->d_LT, LT.size() * sizeof(float)) && alloc((void **)&ctx->d_tab, tab.size()) &&
            alloc((void **)&ctx->d_Dn, Dn.size() * sizeof(float)) && alloc((void **)&ctx->d_LF, LF.size() * sizeof(float)) &&
            alloc((void **)&ctx->d_M, size_t(Np) * Np * sizeof(double)) &&
            alloc((void **)&ctx->d_scratch, size_t(6) * K * Npad * sizeof(float)) &&
            alloc((void **)&ctx->d_red, 16 * sizeof(double)) && alloc((void **)&ctx->d_flag, 16 * sizeof(int)) &&
            alloc((void **)&d_vert, size_t(3) * Nv * sizeof(double)) &&
            alloc((void **)&d_EToV, size_t(K) * 4 * sizeof(int32_t)) &&
            (!eps || alloc((void **)&d_eps, size_t(K) * sizeof(float))) &&
            (!mu || alloc((void **)&d_mu, size_t(K) * sizeof(float)));
  if (!ok) {
    cudaGetLastError();
    cleanup();
    free_mesh(ctx);
    return set_err(ctx, DG_ERR_OOM, "dg_mesh_upload: device allocation failed");
  }
  ctx->K = K;
  ctx->Nv = Nv;
  cudaError_t e = cudaSuccess;
  auto h2d = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  h2d(ctx->d_DT, DT.data(), DT.size() * sizeof(float));
  h2d(ctx->d_LT, LT.data(), LT.size() * sizeof(float));
  h2d(ctx->d_tab, tab.data(), tab.size());
  h2d(ctx->d_Dn, Dn.data(), Dn.size() * sizeof(float));
  h2d(ctx->d_LF, LF.data(), LF.size() * sizeof(float));
  h2d(ctx->d_M, o.M.data(), o.M.size() * sizeof(double));
  h2d(ctx->d_fconn, fconn.data(), fconn.size() * sizeof(int2));
  h2d(d_vert, VX, Nv * sizeof(double));
  h2d(d_vert + Nv, VY, Nv * sizeof(double));
  h2d(d_vert + 2 * Nv, VZ, Nv * sizeof(double));
  h2d(d_EToV, EToV, size_t(K) * 4 * sizeof(int32_t));
  if (eps) h2d(d_eps, eps, K * sizeof(float));
  if (mu) h2d(d_mu, mu, K * sizeof(float));
  int bad_init = int(K < 0x7fffffff ? K : 0x7fffffff);
  h2d(ctx->d_flag, &bad_init, sizeof(int));
  if (e == cudaSuccess) {
    GeometryArgs g{K, d_vert, d_vert + Nv, d_vert + 2 * Nv, d_EToV, d_eps, d_mu, ctx->d_geo, ctx->d_fgeo,
                   ctx->d_flag};
    e = launch_geometry(g, s);
    if (e == cudaSuccess) e = launch_face_weights(K, ctx->d_geo, ctx->d_fgeo, ctx->d_fconn, ctx->d_fmat, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_scratch, 0, field_bytes(ctx), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag + 1, 0, 15 * sizeof(int), s);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) {
    free_mesh(ctx);
    return cuda_err(ctx, e, "dg_mesh_upload");
  }
  if (bad != bad_init) {
    free_mesh(ctx);
    return set_err(ctx, DG_ERR_MESH, "dg_mesh_upload: element " + std::to_string(bad) + " has J <= 0");
  }
  ctx->host_vert.assign(VX, VX + Nv);
  ctx->host_vert.insert(ctx->host_vert.end(), VY, VY + Nv);
  ctx->host_vert.insert(ctx->host_vert.end(), VZ, VZ + Nv);
  ctx->host_EToV.assign(EToV, EToV + K * 4);
  if (ctx->precision != DG_FP32) {
    int rc = tc_prepare(ctx);
    if (rc != DG_OK) {
      free_mesh(ctx);
      return rc;
    }
  }
  return DG_OK;
}

int dg_node_coords(dg_ctx *ctx, double *xyz) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!xyz) return set_err(ctx, DG_ERR_ARG, "dg_node_coords: null output");
  const RefOps &o = ctx->ops;
  const int64_t K = ctx->K, Nv = ctx->Nv;
  const int Np = o.Np;
  for (int64_t k = 0; k < K; ++k) {
    const int32_t *v = &ctx->host_EToV[k * 4];
    for (int i = 0; i < Np; ++i) {
      double w[4] = {-(1.0 + o.r[i] + o.s[i] + o.t[i]) / 2.0, (1.0 + o.r[i]) / 2.0, (1.0 + o.s[i]) / 2.0,
                     (1.0 + o.t[i]) / 2.0};
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int q = 0; q < 4; ++q) acc += w[q] * ctx->host_vert[c * Nv + v[q]];
        xyz[(c * K + k) * Np + i] = acc;
      }
    }
  }
  return DG_OK;
}

int dg_set_eps(dg_ctx *ctx, const float *eps_dev) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!eps_dev) return set_err(ctx, DG_ERR_ARG, "dg_set_eps: null pointer");
  int bad_init = int(ctx->K < 0x7fffffff ? ctx->K : 0x7fffffff), bad = 0;
  cudaError_t e = cudaMemcpyAsync(ctx->d_flag, &bad_init, sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_set_eps(ctx->K, eps_dev, ctx->d_geo, ctx->d_flag, ctx->stream);
  if (e == cudaSuccess)
    e = launch_face_weights(ctx->K, ctx->d_geo, ctx->d_fgeo, ctx->d_fconn, ctx->d_fmat, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dg_set_eps");
  if (bad != bad_init) return set_err(ctx, DG_ERR_ARG, "dg_set_eps: eps must be positive");
  return DG_OK;
}

int dg_rhs(dg_ctx *ctx, const float *u, float *rhs, float alpha) {
  dgmx::NvtxRange nvtx_range("dg_rhs");
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!u || !rhs) return set_err(ctx, DG_ERR_ARG, "dg_rhs: null field pointer");
  if (!aligned16(u) || !aligned16(rhs)) return set_err(ctx, DG_ERR_ARG, "dg_rhs: fields must be 16-byte aligned");
  if (overlap(u, rhs, field_bytes(ctx))) return set_err(ctx, DG_ERR_ARG, "dg_rhs: u and rhs overlap");
  if (!std::isfinite(alpha)) return set_err(ctx, DG_ERR_ARG, "dg_rhs: alpha must be finite");
  StageArgs a = base_args(ctx);
  a.u = u;
  a.rhs = rhs;
  a.alpha = alpha;
  cudaError_t e = launch_stage(ctx, MODE_RHS, a);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dg_rhs");
  return DG_OK;
}

int dg_step(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha) {
  dgmx::NvtxRange nvtx_range("dg_step");
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!u || !res) return set_err(ctx, DG_ERR_ARG, "dg_step: null field pointer");
  if (!aligned16(u) || !aligned16(res)) return set_err(ctx, DG_ERR_ARG, "dg_step: fields must be 16-byte aligned");
  if (overlap(u, res, field_bytes(ctx))) return set_err(ctx, DG_ERR_ARG, "dg_step: u and res overlap");
  if (nsteps < 0 || !std::isfinite(dt) || !std::isfinite(alpha)) return set_err(ctx, DG_ERR_ARG, "dg_step: bad dt/nsteps/alpha");
  return lserk_drive(ctx, u, res, dt, nsteps, alpha, ctx->d_scratch, "dg_step");
}

int dg_set_nonfinite_check(dg_ctx *ctx, int enabled) {
  if (!ctx) return DG_ERR_ARG;
  ctx->check_nonfinite = enabled ? 1 : 0;
  return DG_OK;
}

int dg_sync(dg_ctx *ctx) {
  if (!ctx) return DG_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dg_sync");
  if (ctx->K <= 0) return DG_OK;
  int flag = 0, zero = 0;
  e = cudaMemcpy(&flag, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemcpy(ctx->d_flag + 1, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dg_sync");
  if (flag) {
    // blocks of a persistent launch that gave up leave its grid barrier half-counted
    e = ensemble_reset_barrier(ctx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "dg_sync");
    return set_err(ctx, DG_ERR_TIMEOUT,
                   "a device wait timed out (tensor-core MMA / copy barrier or ensemble grid barrier)");
  }
  return DG_OK;
}

int dg_set_wait_limit(dg_ctx *ctx, long long cycles) {
  if (!ctx) return DG_ERR_ARG;
  if (cycles < 0) return set_err(ctx, DG_ERR_ARG, "dg_set_wait_limit: negative limit");
  ctx->wait_limit = cycles;
  ensemble_drop_graph(ctx); // a captured ensemble launch carries the old limit
  return DG_OK;
}

int dg_energy(dg_ctx *ctx, const float *u, double *E_out) {
  dgmx::NvtxRange nvtx_range("dg_energy");
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (!u || !E_out) return set_err(ctx, DG_ERR_ARG, "dg_energy: null pointer");
  cudaError_t e = launch_energy(ctx->N, ctx->K, ctx->ops.Npad, u, ctx->d_geo, ctx->d_M, ctx->d_red, ctx->stream);
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, ctx->d_red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dg_energy");
  *E_out = v;
  if (!std::isfinite(v)) return set_err(ctx, DG_ERR_NONFINITE, "dg_energy: energy is not finite");
  return DG_OK;
}

} // extern "C"

namespace dgmx {

int lserk_drive(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha, float *pingpong,
                const char *who) {
  StageArgs a = base_args(ctx);
  a.alpha = alpha;
  a.dt = float(dt);
  a.res = res;
  const float *cur = u;
  float *nxt = pingpong;
  for (int step = 0; step < nsteps; ++step)
    for (int st = 0; st < 5; ++st) {
      a.u = cur;
      a.u_out = nxt;
      a.rk_a = float(kLserkA[st]);
      a.rk_b = float(kLserkB[st]);
      cudaError_t e = launch_stage(ctx, MODE_LSERK, a);
      if (e != cudaSuccess) return cuda_err(ctx, e, who);
      float *prev = const_cast<float *>(cur);
      cur = nxt;
      nxt = prev;
    }
  if (cur != u) {
    cudaError_t e = cudaMemcpyAsync(u, cur, field_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, who);
  }
  if (ctx->check_nonfinite && nsteps > 0) {
    int *flag = ctx->d_flag + 3;
    int bad = 0;
    const int64_t n = int64_t(field_bytes(ctx) / sizeof(float));
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_nonfinite_check(u, n, flag, ctx->stream);
    if (e == cudaSuccess) e = launch_nonfinite_check(res, n, flag, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, who);
    if (bad)
      return set_err(ctx, DG_ERR_NONFINITE,
                     std::string(who) + ": the state or the residual holds a NaN or an infinity after the last stage");
  }
  return DG_OK;
}

cudaError_t launch_stage_simt(int N, int mode, const StageArgs &a, cudaStream_t s) {
  switch (N) {
  case 1: return launch_simt_order<1>(mode, a, s);
  case 2: return launch_simt_order<2>(mode, a, s);
  case 3: return launch_simt_order<3>(mode, a, s);
  case 4: return launch_simt_order<4>(mode, a, s);
  case 5: return launch_simt_order<5>(mode, a, s);
  case 6: return launch_simt_order<6>(mode, a, s);
  case 7: return launch_simt_order<7>(mode, a, s);
  case 8: return launch_simt_order<8>(mode, a, s);
  case 9: return launch_simt_order<9>(mode, a, s);
  default: return cudaErrorInvalidValue;
  }
}

} // namespace dgmx
