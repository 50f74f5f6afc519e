// Geometric factors of affine tetrahedra, computed in FP64 on the device.
//
// Section 2, eq. (dg-reference-matrices): every straight-sided element is the
// image of the reference tetrahedron under an affine map Psi_k, so the
// Jacobian J_k and the metric terms dr/dx are constant per element. The outward
// face normals follow from the metric terms (n = -grad t, -grad s,
// grad(r+s+t), -grad r on the faces t=-1, s=-1, r+s+t=-1, r=-1); the face
// Jacobian is sJ = J |grad ...|, so Fscale = sJ / J = |grad ...|.
// Results are stored in FP32 for the right-hand-side kernels; the energy norm
// uses the FP32-stored J as well.
#include <cmath>

#include "common.cuh"

namespace dgmx {

namespace {

__global__ void k_geometry(GeometryArgs a) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  double P[4][3];
  for (int v = 0; v < 4; ++v) {
    int32_t id = a.EToV[k * 4 + v];
    P[v][0] = a.VX[id];
    P[v][1] = a.VY[id];
    P[v][2] = a.VZ[id];
  }
  // x = 1/2 (-(1+r+s+t) Pa + (1+r) Pb + (1+s) Pc + (1+t) Pd): columns x_r, x_s, x_t
  double xr[3], xs[3], xt[3];
  for (int c = 0; c < 3; ++c) {
    xr[c] = 0.5 * (P[1][c] - P[0][c]);
    xs[c] = 0.5 * (P[2][c] - P[0][c]);
    xt[c] = 0.5 * (P[3][c] - P[0][c]);
  }
  auto crossv = [](const double *u, const double *v, double *w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  double gr[3], gs[3], gt[3];
  crossv(xs, xt, gr); // J grad r = x_s x x_t
  crossv(xt, xr, gs); // J grad s = x_t x x_r
  crossv(xr, xs, gt); // J grad t = x_r x x_s
  double J = xr[0] * gr[0] + xr[1] * gr[1] + xr[2] * gr[2];
  if (!(J > 0.0)) {
    atomicMin(a.bad, int(k < 0x7fffffff ? k : 0x7fffffff));
    J = 1.0;
  }
  for (int c = 0; c < 3; ++c) {
    gr[c] /= J;
    gs[c] /= J;
    gt[c] /= J;
  }
  double eps = a.eps ? double(a.eps[k]) : 1.0;
  double mu = a.mu ? double(a.mu[k]) : 1.0;
  float *g = a.geo + k * G_STRIDE;
  g[G_RX] = float(gr[0]); g[G_RY] = float(gr[1]); g[G_RZ] = float(gr[2]);
  g[G_SX] = float(gs[0]); g[G_SY] = float(gs[1]); g[G_SZ] = float(gs[2]);
  g[G_TX] = float(gt[0]); g[G_TY] = float(gt[1]); g[G_TZ] = float(gt[2]);
  g[G_IEPS] = float(1.0 / eps);
  g[G_IMU] = float(1.0 / mu);
  double Z = sqrt(mu / eps);
  g[G_Z] = float(Z);
  g[G_Y] = float(1.0 / Z);
  g[G_J] = float(J);
  g[14] = 0.f;
  g[15] = 0.f;
  for (int f = 0; f < 4; ++f) {
    double n[3];
    for (int c = 0; c < 3; ++c)
      n[c] = f == 0 ? -gt[c] : f == 1 ? -gs[c] : f == 2 ? gr[c] + gs[c] + gt[c] : -gr[c];
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    a.fgeo[k * 4 + f] = make_float4(float(n[0] / len), float(n[1] / len), float(n[2] / len), float(len));
  }
}

__global__ void k_set_eps(int64_t K, const float *eps, float *geo, int *bad) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double e = eps[k];
  if (!(e > 0.0)) {
    atomicMin(bad, int(k < 0x7fffffff ? k : 0x7fffffff));
    return;
  }
  float *g = geo + k * G_STRIDE;
  double mu = 1.0 / double(g[G_IMU]);
  double Z = sqrt(mu / e);
  g[G_IEPS] = float(1.0 / e);
  g[G_Z] = float(Z);
  g[G_Y] = float(1.0 / Z);
}

__global__ void k_face_weights(int64_t K, const float *geo, const float4 *fgeo, const int2 *fconn, float4 *fmat) {
  int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= K * 4) return;
  const int64_t k = q >> 2;
  const int2 cn = fconn[q];
  const float zm = geo[k * G_STRIDE + G_Z], ym = geo[k * G_STRIDE + G_Y];
  float zp = zm, yp = ym;
  if (cn.y != kBoundaryConn) {
    zp = geo[int64_t(cn.x) * G_STRIDE + G_Z];
    yp = geo[int64_t(cn.x) * G_STRIDE + G_Y];
  }
  const float fs = fgeo[q].w;
  fmat[q] = make_float4(fs / (zm + zp), -fs / (ym + yp), zp, yp);
}

} // namespace

cudaError_t launch_face_weights(int64_t K, const float *geo, const float4 *fgeo, const int2 *fconn, float4 *fmat,
                                cudaStream_t s) {
  k_face_weights<<<unsigned((K * 4 + 255) / 256), 256, 0, s>>>(K, geo, fgeo, fconn, fmat);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const GeometryArgs &a, cudaStream_t s) {
  unsigned blocks = unsigned((a.K + 127) / 128);
  k_geometry<<<blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_set_eps(int64_t K, const float *eps, float *geo, int *bad, cudaStream_t s) {
  unsigned blocks = unsigned((K + 127) / 128);
  k_set_eps<<<blocks, 128, 0, s>>>(K, eps, geo, bad);
  return cudaGetLastError();
}

} // namespace dgmx
