// Reference-element operators of the nodal DG method, host side in FP64.
//
// Section 2 of the paper: a nodal Lagrange basis on Np = dim P_N interpolation
// nodes (the warp & blend nodes of [warburton_explicit_2006]; blend parameter 0
// by default since the paper names none, or the value of least Lebesgue
// constant per order, kOptimisedAlpha below), the mass, differentiation and face mass
// matrices of eq. (dg-global-matrices) on the reference element, and the
// lifting matrix of Fig. (lifting-matrix). Operators are built from the
// orthonormal Proriol-Koornwinder-Dubiner basis: V_ij = psi_j(x_i),
// D_r = V_r V^-1, M^-1 = V V^T, LIFT = V V^T E with E the face mass matrices
// embedded at the face nodes.
#include "refops.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

namespace dgmx {

const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

namespace {

// ---------------------------------------------------------------- linear algebra
// LU factorisation with partial pivoting of an n x n row-major matrix.
struct LU {
  int n = 0;
  std::vector<double> a;
  std::vector<int> piv;
  bool factor(int n_, const std::vector<double> &A) {
    n = n_;
    a = A;
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
      int p = k;
      for (int i = k + 1; i < n; ++i)
        if (std::fabs(a[i * n + k]) > std::fabs(a[p * n + k])) p = i;
      if (std::fabs(a[p * n + k]) < 1e-300) return false;
      piv[k] = p;
      if (p != k)
        for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
      for (int i = k + 1; i < n; ++i) {
        double l = a[i * n + k] / a[k * n + k];
        a[i * n + k] = l;
        for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
      }
    }
    return true;
  }
  // Solves A x = b in place.
  void solve(double *b) const {
    for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
    for (int i = 1; i < n; ++i)
      for (int j = 0; j < i; ++j) b[i] -= a[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) b[i] -= a[i * n + j] * b[j];
      b[i] /= a[i * n + i];
    }
  }
};

// Eigenvalues of a small dense symmetric matrix by cyclic Jacobi rotations.
std::vector<double> sym_eigenvalues(int n, std::vector<double> A) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-32) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) { // columns p, q
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { // rows p, q
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
  std::sort(ev.begin(), ev.end());
  return ev;
}

// ---------------------------------------------------------------- Jacobi polynomials
// Orthonormal Jacobi polynomials for the weight (1-x)^al (1+x)^be on [-1,1],
// from the symmetric three-term recurrence x p_n = a_{n+1} p_{n+1} + b_n p_n + a_n p_{n-1}.
double rec_a(int n, double al, double be) {
  double s = 2.0 * n + al + be;
  if (n == 1) return 2.0 / (2.0 + al + be) * std::sqrt((1.0 + al) * (1.0 + be) / (3.0 + al + be));
  return 2.0 / s * std::sqrt(n * (n + al + be) * (n + al) * (n + be) / ((s - 1.0) * (s + 1.0)));
}
double rec_b(int n, double al, double be) {
  if (n == 0) return (be - al) / (al + be + 2.0);
  double s = 2.0 * n + al + be;
  return (be * be - al * al) / (s * (s + 2.0));
}
double ojacobi(int n, double al, double be, double x) {
  double g0 = std::exp((al + be + 1.0) * std::log(2.0) + std::lgamma(al + 1.0) + std::lgamma(be + 1.0) -
                       std::lgamma(al + be + 2.0));
  double pm = 0.0, p = 1.0 / std::sqrt(g0);
  for (int k = 0; k < n; ++k) {
    double pn = ((x - rec_b(k, al, be)) * p - (k > 0 ? rec_a(k, al, be) * pm : 0.0)) / rec_a(k + 1, al, be);
    pm = p;
    p = pn;
  }
  return p;
}
// d/dx p_n^(al,be) = sqrt(n (n+al+be+1)) p_{n-1}^(al+1,be+1)
double dojacobi(int n, double al, double be, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + al + be + 1.0)) * ojacobi(n - 1, al + 1.0, be + 1.0, x);
}

// x^e for e >= 0; the callers only form negative powers where the factor they
// multiply is exactly zero, so 0 is returned there.
double pw(double x, int e) { return e < 0 ? 0.0 : std::pow(x, e); }

// ---------------------------------------------------------------- 1D nodes
// Gauss-Lobatto-Legendre points: +-1 plus the Gauss-Jacobi(1,1) points, which
// are the eigenvalues of the symmetric Jacobi matrix (Golub-Welsch).
std::vector<double> lgl_points(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  int n = N - 1;
  if (n > 0) {
    std::vector<double> T(n * n, 0.0);
    for (int i = 0; i < n; ++i) T[i * n + i] = rec_b(i, 1.0, 1.0);
    for (int i = 0; i + 1 < n; ++i) T[i * n + i + 1] = T[(i + 1) * n + i] = rec_a(i + 1, 1.0, 1.0);
    std::vector<double> ev = sym_eigenvalues(n, T);
    for (int i = 0; i < n; ++i) x[i + 1] = ev[i];
  }
  return x;
}

// Warp & blend displacement along one edge: the interpolant (on equidistant
// points, barycentric Lagrange form) of the LGL-minus-equidistant offsets,
// divided by 1 - r^2 so that multiplying by the edge blend 4 l_P l_Q restores it.
struct EdgeWarp {
  int N;
  std::vector<double> req, off, w;
  explicit EdgeWarp(int N_) : N(N_), req(N_ + 1), off(N_ + 1), w(N_ + 1) {
    std::vector<double> xl = lgl_points(N);
    double binom = 1.0;
    for (int i = 0; i <= N; ++i) {
      req[i] = -1.0 + 2.0 * i / N;
      off[i] = xl[i] - req[i];
      w[i] = ((i % 2) ? -1.0 : 1.0) * binom;
      binom = binom * (N - i) / (i + 1);
    }
  }
  double operator()(double r) const {
    if (std::fabs(r) >= 1.0 - 1e-10) return 0.0;
    double num = 0.0, den = 0.0;
    for (int i = 0; i <= N; ++i) {
      double d = r - req[i];
      if (d == 0.0) return off[i] / (1.0 - r * r);
      num += w[i] / d * off[i];
      den += w[i] / d;
    }
    return num / den / (1.0 - r * r);
  }
};

// Warp & blend nodes in barycentric coordinates (l_a, l_b, l_c, l_d) of the
// vertices a=(-1,-1,-1), b=(1,-1,-1), c=(-1,1,-1), d=(-1,-1,1). Every face
// displaces its nodes along each of its edges (P,Q) by 4 l_P l_Q w(l_Q - l_P),
// in barycentric units (e_Q - e_P)/2; a face's displacement is blended into the
// volume by l_P l_Q l_R / prod(l_X + l_O/2) (O the opposite vertex); nodes on an
// edge of the surface take the unblended face displacement. With blend
// parameter alpha, the edge (P, Q) term is scaled by 1 + (alpha l_R)^2, R the
// face's third vertex.
void warp_blend_nodes(int N, double alpha, std::vector<double> &r, std::vector<double> &s, std::vector<double> &t) {
  EdgeWarp warp(N);
  const int faces[4][4] = {{3, 0, 1, 2}, {2, 0, 1, 3}, {0, 1, 2, 3}, {1, 0, 2, 3}}; // opposite, then face
  const double tol = 1e-10;
  r.clear(), s.clear(), t.clear();
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - k - j; ++i) {
        std::array<double, 4> l = {double(N - i - j - k) / N, double(i) / N, double(j) / N, double(k) / N};
        std::array<double, 4> d = {0, 0, 0, 0};
        for (const auto &F : faces) {
          int o = F[0];
          std::array<double, 4> fd = {0, 0, 0, 0};
          for (int e = 0; e < 3; ++e) {
            int P = F[1 + e], Q = F[1 + (e + 1) % 3], R = F[1 + (e + 2) % 3];
            const double ar = alpha * l[R];
            double mag = 4.0 * l[P] * l[Q] * warp(l[Q] - l[P]) * 0.5 * (1.0 + ar * ar);
            fd[Q] += mag;
            fd[P] -= mag;
          }
          double lp = l[F[1]], lq = l[F[2]], lr = l[F[3]];
          double blend = lp * lq * lr;
          double den = (lp + 0.5 * l[o]) * (lq + 0.5 * l[o]) * (lr + 0.5 * l[o]);
          if (den > tol) blend /= den;
          bool surface_edge = l[o] < tol && ((lp > tol) + (lq > tol) + (lr > tol)) < 3;
          for (int v = 0; v < 4; ++v) d[v] = surface_edge ? fd[v] : d[v] + blend * fd[v];
        }
        r.push_back(2.0 * (l[1] + d[1]) - 1.0);
        s.push_back(2.0 * (l[2] + d[2]) - 1.0);
        t.push_back(2.0 * (l[3] + d[3]) - 1.0);
      }
}

// ---------------------------------------------------------------- orthonormal bases
struct Grad {
  double v, dr, ds, dt;
};

// psi_ijk = 2 sqrt(2) p_i(a) p_j^(2i+1,0)(b) (1-b)^i p_k^(2i+2j+2,0)(c) (1-c)^(i+j),
// a = 2(1+r)/(-s-t) - 1, b = 2(1+s)/(1-t) - 1, c = t; gradient through the
// collapsed coordinates with the singular 1/(1-b), 1/(1-c) folded into the powers.
Grad pkd(int i, int j, int k, double r, double s, double t) {
  double a = (std::fabs(s + t) > 1e-12) ? 2.0 * (1.0 + r) / (-s - t) - 1.0 : -1.0;
  double b = (std::fabs(1.0 - t) > 1e-12) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  double c = t;
  const double al2 = 2.0 * i + 1.0, al3 = 2.0 * i + 2.0 * j + 2.0;
  double A = ojacobi(i, 0, 0, a), dA = dojacobi(i, 0, 0, a);
  double B = ojacobi(j, al2, 0, b), dB = dojacobi(j, al2, 0, b);
  double C = ojacobi(k, al3, 0, c), dC = dojacobi(k, al3, 0, c);
  const int p = i, q = i + j;
  const double k8 = 2.0 * std::sqrt(2.0);
  double ob = 1.0 - b, oc = 1.0 - c;
  Grad g;
  g.v = k8 * A * B * pw(ob, p) * C * pw(oc, q);
  // dpsi/da * da/dr with da/dr = 4 / ((1-b)(1-c))
  double Ar = k8 * dA * B * pw(ob, p - 1) * C * pw(oc, q - 1);
  // (1-b)^p B(b) differentiated in b
  double Bb = dB * pw(ob, p) - p * B * pw(ob, p - 1);
  // (1-c)^q C(c) differentiated in c
  double Cc = dC * pw(oc, q) - q * C * pw(oc, q - 1);
  g.dr = 4.0 * Ar;
  double a_part = 2.0 * (1.0 + a) * Ar; // da/ds = da/dt = 2(1+a)/((1-b)(1-c))
  double bs = k8 * A * Bb * C * pw(oc, q - 1);
  g.ds = a_part + 2.0 * bs;                             // db/ds = 2/(1-c)
  g.dt = a_part + (1.0 + b) * bs + k8 * A * B * pw(ob, p) * Cc; // db/dt = (1+b)/(1-c), dc/dt = 1
  return g;
}

// Orthonormal triangle basis phi_ij = sqrt(2) p_i(a) p_j^(2i+1,0)(y) (1-y)^i, a = 2(1+x)/(1-y) - 1.
double dubiner(int i, int j, double x, double y) {
  double a = (std::fabs(1.0 - y) > 1e-12) ? 2.0 * (1.0 + x) / (1.0 - y) - 1.0 : -1.0;
  return std::sqrt(2.0) * ojacobi(i, 0, 0, a) * ojacobi(j, 2.0 * i + 1.0, 0, y) * pw(1.0 - y, i);
}

} // namespace

// Blend parameters of least Lebesgue constant, N = 1..9: the result of a search
// over alpha in [0, 3] (grid of step 0.05 on the order-30 equidistant lattice of
// the tetrahedron, then a golden-section search on the order-60 lattice); N <= 4
// gained nothing over alpha = 0. The constant drops 0.7% (N = 5) to 9% (N = 8).
double optimised_alpha(int N) {
  static const double table[kMaxOrder] = {0.0, 0.0, 0.0, 0.0, 1.150, 1.719, 1.419, 1.338, 1.162};
  return N >= 1 && N <= kMaxOrder ? table[N - 1] : -1.0;
}

bool build_refops(int N, RefOps &o, std::string &err, double alpha) {
  if (N < 1 || N > kMaxOrder) {
    err = "polynomial order out of range";
    return false;
  }
  if (!(alpha >= 0.0 && alpha <= 10.0)) {
    err = "blend parameter outside [0, 10]";
    return false;
  }
  o.N = N;
  o.alpha = alpha;
  o.Np = num_nodes(N);
  o.Nfp = num_face_nodes(N);
  o.Npad = padded_nodes(N);
  const int Np = o.Np, Nfp = o.Nfp;
  warp_blend_nodes(N, alpha, o.r, o.s, o.t);

  // Vandermonde and its gradient, column m = mode (i, j, k).
  std::vector<double> V(Np * Np), Vr(Np * Np), Vs(Np * Np), Vt(Np * Np);
  int m = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k, ++m)
        for (int n = 0; n < Np; ++n) {
          Grad g = pkd(i, j, k, o.r[n], o.s[n], o.t[n]);
          V[n * Np + m] = g.v;
          Vr[n * Np + m] = g.dr;
          Vs[n * Np + m] = g.ds;
          Vt[n * Np + m] = g.dt;
        }
  // D V = V_r  <=>  V^T D^T = V_r^T: solve column by column with LU of V^T.
  std::vector<double> VT(Np * Np);
  for (int a = 0; a < Np; ++a)
    for (int b = 0; b < Np; ++b) VT[a * Np + b] = V[b * Np + a];
  LU lu;
  if (!lu.factor(Np, VT)) {
    err = "singular Vandermonde matrix";
    return false;
  }
  auto diff = [&](const std::vector<double> &Vd, std::vector<double> &D) {
    D.assign(Np * Np, 0.0);
    std::vector<double> col(Np);
    for (int row = 0; row < Np; ++row) { // row of D = row of Vd times V^-1
      for (int q = 0; q < Np; ++q) col[q] = Vd[row * Np + q];
      lu.solve(col.data());
      for (int q = 0; q < Np; ++q) D[row * Np + q] = col[q];
    }
  };
  diff(Vr, o.Dr);
  diff(Vs, o.Ds);
  diff(Vt, o.Dt);

  // M^-1 = V V^T; M = V^-T V^-1.
  std::vector<double> Minv(Np * Np, 0.0);
  for (int a = 0; a < Np; ++a)
    for (int b = 0; b < Np; ++b) {
      double acc = 0.0;
      for (int q = 0; q < Np; ++q) acc += V[a * Np + q] * V[b * Np + q];
      Minv[a * Np + b] = acc;
    }
  {
    LU lm;
    if (!lm.factor(Np, Minv)) {
      err = "singular mass matrix";
      return false;
    }
    o.M.assign(Np * Np, 0.0);
    std::vector<double> col(Np);
    for (int c = 0; c < Np; ++c) {
      std::fill(col.begin(), col.end(), 0.0);
      col[c] = 1.0;
      lm.solve(col.data());
      for (int a = 0; a < Np; ++a) o.M[a * Np + c] = col[a];
    }
  }

  // Face nodes: faces t=-1, s=-1, r+s+t=-1, r=-1 (in node order).
  o.Fmask.assign(4 * Nfp, -1);
  for (int f = 0; f < 4; ++f) {
    int cnt = 0;
    for (int n = 0; n < Np; ++n) {
      double dist = f == 0 ? 1.0 + o.t[n] : f == 1 ? 1.0 + o.s[n] : f == 2 ? 1.0 + o.r[n] + o.s[n] + o.t[n] : 1.0 + o.r[n];
      if (std::fabs(dist) < 1e-10) {
        if (cnt == Nfp) {
          err = "face node count mismatch";
          return false;
        }
        o.Fmask[f * Nfp + cnt++] = n;
      }
    }
    if (cnt != Nfp) {
      err = "face node count mismatch";
      return false;
    }
  }

  // Face mass matrices (V2 V2^T)^-1 in the face's two free reference coordinates,
  // embedded into E (Np x 4Nfp); LIFT = M^-1 E.
  std::vector<double> E(Np * 4 * Nfp, 0.0);
  for (int f = 0; f < 4; ++f) {
    std::vector<double> V2(Nfp * Nfp);
    for (int a = 0; a < Nfp; ++a) {
      int n = o.Fmask[f * Nfp + a];
      double x = f == 0 || f == 1 ? o.r[n] : o.s[n];
      double y = f == 0 ? o.s[n] : o.t[n];
      int q = 0;
      for (int i = 0; i <= N; ++i)
        for (int j = 0; j <= N - i; ++j, ++q) V2[a * Nfp + q] = dubiner(i, j, x, y);
    }
    std::vector<double> G(Nfp * Nfp, 0.0);
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) {
        double acc = 0.0;
        for (int q = 0; q < Nfp; ++q) acc += V2[a * Nfp + q] * V2[b * Nfp + q];
        G[a * Nfp + b] = acc;
      }
    LU lf;
    if (!lf.factor(Nfp, G)) {
      err = "singular face mass matrix";
      return false;
    }
    std::vector<double> col(Nfp);
    for (int b = 0; b < Nfp; ++b) {
      std::fill(col.begin(), col.end(), 0.0);
      col[b] = 1.0;
      lf.solve(col.data()); // column b of the face mass matrix
      for (int a = 0; a < Nfp; ++a) E[o.Fmask[f * Nfp + a] * 4 * Nfp + f * Nfp + b] += col[a];
    }
  }
  o.LIFT.assign(Np * 4 * Nfp, 0.0);
  for (int a = 0; a < Np; ++a)
    for (int q = 0; q < 4 * Nfp; ++q) {
      double acc = 0.0;
      for (int b = 0; b < Np; ++b) acc += Minv[a * Np + b] * E[b * 4 * Nfp + q];
      o.LIFT[a * 4 * Nfp + q] = acc;
    }

  // Neighbour node tables. Face node m of face f has barycentric weights on the
  // face's three local vertices; for neighbour face f2 whose local vertices
  // hold global vertices in permutation perm of ours (ours[v] = theirs[perm[v]]),
  // the same point has the weight of our vertex v on their vertex perm[v].
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  auto bary = [&](int n) {
    return std::array<double, 4>{-(1.0 + o.r[n] + o.s[n] + o.t[n]) / 2.0, (1.0 + o.r[n]) / 2.0, (1.0 + o.s[n]) / 2.0,
                                 (1.0 + o.t[n]) / 2.0};
  };
  o.nbr_node.assign(kConnKinds * Nfp, 0);
  o.nbr_fnode.assign(kConnKinds * Nfp, 0);
  for (int f = 0; f < 4; ++f)
    for (int f2 = 0; f2 < 4; ++f2)
      for (int p = 0; p < 6; ++p)
        for (int a = 0; a < Nfp; ++a) {
          auto l = bary(o.Fmask[f * Nfp + a]);
          double want[3];
          for (int v = 0; v < 3; ++v) want[perms[p][v]] = l[kFaceVerts[f][v]];
          int found = -1, found_b = -1;
          for (int b = 0; b < Nfp && found < 0; ++b) {
            auto l2 = bary(o.Fmask[f2 * Nfp + b]);
            double d = 0.0;
            for (int v = 0; v < 3; ++v) d += std::fabs(l2[kFaceVerts[f2][v]] - want[v]);
            if (d < 1e-9) {
              found = o.Fmask[f2 * Nfp + b];
              found_b = b;
            }
          }
          if (found < 0) {
            err = "face nodes are not symmetric under vertex permutations";
            return false;
          }
          o.nbr_node[((f * 4 + f2) * 6 + p) * Nfp + a] = static_cast<uint8_t>(found);
          o.nbr_fnode[((f * 4 + f2) * 6 + p) * Nfp + a] = static_cast<uint8_t>(found_b);
        }
  return true;
}

bool build_connectivity(int64_t K, int64_t Nv, const int32_t *EToV, Connectivity &out, std::string &err) {
  struct Face {
    std::array<int32_t, 3> key;
    int32_t k;
    int8_t f;
  };
  std::vector<Face> faces(static_cast<size_t>(K) * 4);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      Face &F = faces[k * 4 + f];
      for (int v = 0; v < 3; ++v) {
        int32_t id = EToV[k * 4 + kFaceVerts[f][v]];
        if (id < 0 || id >= Nv) {
          err = "EToV vertex index out of range at element " + std::to_string(k);
          return false;
        }
        F.key[v] = id;
      }
      std::sort(F.key.begin(), F.key.end());
      if (F.key[0] == F.key[1] || F.key[1] == F.key[2]) {
        err = "degenerate element " + std::to_string(k) + " (repeated vertex)";
        return false;
      }
      F.k = static_cast<int32_t>(k);
      F.f = static_cast<int8_t>(f);
    }
  std::sort(faces.begin(), faces.end(), [](const Face &a, const Face &b) { return a.key < b.key; });
  out.nbr_elem.assign(K * 4, 0);
  out.conn.assign(K * 4, kBoundaryConn);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) out.nbr_elem[k * 4 + f] = static_cast<int32_t>(k);
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  auto link = [&](const Face &A, const Face &B) {
    int32_t ga[3], gb[3];
    for (int v = 0; v < 3; ++v) {
      ga[v] = EToV[int64_t(A.k) * 4 + kFaceVerts[A.f][v]];
      gb[v] = EToV[int64_t(B.k) * 4 + kFaceVerts[B.f][v]];
    }
    for (int p = 0; p < 6; ++p)
      if (ga[0] == gb[perms[p][0]] && ga[1] == gb[perms[p][1]] && ga[2] == gb[perms[p][2]]) {
        out.nbr_elem[int64_t(A.k) * 4 + A.f] = B.k;
        out.conn[int64_t(A.k) * 4 + A.f] = (A.f * 4 + B.f) * 6 + p;
        return;
      }
  };
  for (size_t q = 0; q < faces.size();) {
    size_t e = q + 1;
    while (e < faces.size() && faces[e].key == faces[q].key) ++e;
    if (e - q > 2) {
      err = "non-conforming mesh: a face is shared by more than two elements";
      return false;
    }
    if (e - q == 2) {
      if (faces[q].k == faces[q + 1].k) {
        err = "element " + std::to_string(faces[q].k) + " has two identical faces";
        return false;
      }
      link(faces[q], faces[q + 1]);
      link(faces[q + 1], faces[q]);
    }
    q = e;
  }
  return true;
}

} // namespace dgmx
