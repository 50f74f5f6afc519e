/*
 * FP64 single-threaded CPU oracle of the nodal discontinuous Galerkin operator
 * for the 3D Maxwell equations on straight-sided tetrahedra, following
 * Kloeckner, Warburton & Hesthaven, "High-Order Discontinuous Galerkin Methods
 * by GPU Metaprogramming" (arXiv 1211.0582).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; the product library never touches it.
 *
 * Plain loops, no blocking or reordering beyond what the definitions state.
 * Sections of the paper followed:
 *  - Section 2, eq. (semidiscrete-dg): du/dt = -sum_nu D^nu F(u) + L [n.F - (n.F)*].
 *  - Section 2, eq. (dg-global-matrices): M, S, D = M^-1 S, face mass M^A.
 *  - Section 2, Fig. (lifting-matrix): L = M^-1 [M^A1 ... M^A4] embedded at face nodes.
 *  - Section 2, eq. (dg-reference-matrices): affine elements, per-element
 *    constant Jacobian J_k and metric terms dr/dx.
 *  - Section 2, eq. (num-flux) and Section 5, Fig. (flux-code) a: the Maxwell
 *    flux n.(F - F*)_E = 1/2 n x ([H] - alpha n x [E]); the H part and the
 *    material weights are the dual reading (see the project design notes).
 *  - Section 2: interpolation nodes of [warburton_explicit_2006] (warp & blend,
 *    blend parameter 0 since the paper names none).
 *  - Section 5: RK4 time stepping, here Carpenter & Kennedy's five-stage
 *    fourth-order low-storage scheme.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static char g_err[512] = "";
const char *or_error(void) { return g_err; }
static int fail(const char *msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return -1;
}

int or_np(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
int or_nfp(int N) { return (N + 1) * (N + 2) / 2; }

/* ------------------------------------------------------------------ */
/* Dense matrix helpers (row-major, n x n).                            */
/* ------------------------------------------------------------------ */

/* Gauss-Jordan inverse with partial pivoting; returns -1 if singular. */
static int mat_inverse(int n, const double *A, double *Ainv) {
  double *W = (double *)malloc(sizeof(double) * n * 2 * n);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) W[i * 2 * n + j] = A[i * n + j];
    for (int j = 0; j < n; ++j) W[i * 2 * n + n + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(W[i * 2 * n + c]) > fabs(W[p * 2 * n + c])) p = i;
    if (fabs(W[p * 2 * n + c]) < 1e-300) {
      free(W);
      return -1;
    }
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) {
        double tmp = W[c * 2 * n + j];
        W[c * 2 * n + j] = W[p * 2 * n + j];
        W[p * 2 * n + j] = tmp;
      }
    double piv = W[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) W[c * 2 * n + j] /= piv;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      double f = W[i * 2 * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) W[i * 2 * n + j] -= f * W[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * 2 * n + n + j];
  free(W);
  return 0;
}

/* C (n x m) = A (n x p) * B (p x m) */
static void mat_mul(int n, int p, int m, const double *A, const double *B, double *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int q = 0; q < p; ++q) acc += A[i * p + q] * B[q * m + j];
      C[i * m + j] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Jacobi polynomials P_n^(a,b): Abramowitz & Stegun 22.7.1 recurrence,  */
/* normalised by the closed-form weighted L2 norm (A&S 22.2.1).          */
/* ------------------------------------------------------------------ */

static double jacobi_raw(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int k = 2; k <= n; ++k) {
    double c1 = 2.0 * k * (k + a + b) * (2.0 * k + a + b - 2.0);
    double c2 = (2.0 * k + a + b - 1.0) * ((2.0 * k + a + b) * (2.0 * k + a + b - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * (2.0 * k + a + b);
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double jacobi_norm(int n, double a, double b) {
  double lg = (a + b + 1.0) * log(2.0) - log(2.0 * n + a + b + 1.0) + lgamma(n + a + 1.0) +
              lgamma(n + b + 1.0) - lgamma(n + a + b + 1.0) - lgamma(n + 1.0);
  return sqrt(exp(lg));
}

/* orthonormal value and derivative (d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)) */
static double jnorm(int n, double a, double b, double x) { return jacobi_raw(n, a, b, x) / jacobi_norm(n, a, b); }
static double djnorm(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi_raw(n - 1, a + 1.0, b + 1.0, x) / jacobi_norm(n, a, b);
}

/* ------------------------------------------------------------------ */
/* 1D nodes                                                            */
/* ------------------------------------------------------------------ */

/* LGL nodes: endpoints plus the roots of P_N' (proportional to P_{N-1}^(1,1)),
 * found by Newton's method from Chebyshev-Gauss-Lobatto starting points. */
int or_lgl(int N, double *x) {
  if (N < 1) return fail("or_lgl: N must be >= 1");
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double xi = -cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double f = jacobi_raw(N - 1, 1.0, 1.0, xi);
      double df = 0.5 * (N + 2.0) * jacobi_raw(N - 2, 2.0, 2.0, xi);
      double dx = f / df;
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  return 0;
}

/* Warp function: the 1D displacement mapping equidistant to LGL nodes,
 * interpolated on the equidistant nodes, divided by the edge blend 1 - r^2. */
static double warp_factor(int N, const double *xlgl, double r) {
  if (fabs(r) >= 1.0 - 1e-10) return 0.0;
  double w = 0.0;
  for (int i = 0; i <= N; ++i) {
    double ri = -1.0 + 2.0 * i / N;
    double li = 1.0;
    for (int j = 0; j <= N; ++j) {
      if (j == i) continue;
      double rj = -1.0 + 2.0 * j / N;
      li *= (r - rj) / (ri - rj);
    }
    w += (xlgl[i] - ri) * li;
  }
  return w / (1.0 - r * r);
}

/* ------------------------------------------------------------------ */
/* Warp & blend nodes on the tetrahedron (blend parameter alpha; 0 = plain), */
/* built in the equilateral tetrahedron and mapped back.               */
/* ------------------------------------------------------------------ */

/* 2D face shift in the equilateral-triangle frame: edges bottom (left->right),
 * right (right->top), left (top->left), each warped by the 1D warp along the
 * edge and blended by 4 * (product of the edge's two barycentrics) times
 * (1 + (alpha * barycentric of the vertex opposite the edge)^2), the blend
 * parameter of the warp & blend construction (Section 2's node reference). */
static void face_shift(int N, const double *xlgl, double alpha, double Lleft, double Lright, double Ltop,
                       double *dx, double *dy) {
  double wb = 4.0 * Lleft * Lright * warp_factor(N, xlgl, Lright - Lleft) * (1.0 + (alpha * Ltop) * (alpha * Ltop));
  double wr = 4.0 * Lright * Ltop * warp_factor(N, xlgl, Ltop - Lright) * (1.0 + (alpha * Lleft) * (alpha * Lleft));
  double wl = 4.0 * Ltop * Lleft * warp_factor(N, xlgl, Lleft - Ltop) * (1.0 + (alpha * Lright) * (alpha * Lright));
  *dx = wb + cos(2.0 * M_PI / 3.0) * wr + cos(4.0 * M_PI / 3.0) * wl;
  *dy = sin(2.0 * M_PI / 3.0) * wr + sin(4.0 * M_PI / 3.0) * wl;
}

int or_nodes_alpha(int N, double alpha, double *r, double *s, double *t) {
  if (N < 1 || N > 12) return fail("or_nodes: N out of range");
  if (!(alpha >= 0.0 && alpha <= 10.0)) return fail("or_nodes: blend parameter outside [0, 10]");
  double xlgl[16];
  or_lgl(N, xlgl);
  /* equilateral vertices for reference vertices a=(-1,-1,-1), b=(1,-1,-1), c=(-1,1,-1), d=(-1,-1,1) */
  const double V[4][3] = {{-1.0, -1.0 / sqrt(3.0), -1.0 / sqrt(6.0)},
                          {1.0, -1.0 / sqrt(3.0), -1.0 / sqrt(6.0)},
                          {0.0, 2.0 / sqrt(3.0), -1.0 / sqrt(6.0)},
                          {0.0, 0.0, 3.0 / sqrt(6.0)}};
  /* faces: opposite vertex, then (left, right, top) */
  const int F[4][4] = {{3, 0, 1, 2}, {2, 0, 1, 3}, {0, 1, 2, 3}, {1, 0, 2, 3}};
  const double tol = 1e-10;
  int idx = 0;
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - k - j; ++i) {
        double req = -1.0 + 2.0 * i / N, seq = -1.0 + 2.0 * j / N, teq = -1.0 + 2.0 * k / N;
        double L[4] = {-(1.0 + req + seq + teq) / 2.0, (1.0 + req) / 2.0, (1.0 + seq) / 2.0, (1.0 + teq) / 2.0};
        double X[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v)
          for (int c = 0; c < 3; ++c) X[c] += L[v] * V[v][c];
        double shift[3] = {0, 0, 0};
        for (int f = 0; f < 4; ++f) {
          int o = F[f][0], pl = F[f][1], pr = F[f][2], pt = F[f][3];
          double t1[3], t2[3], n1 = 0, n2 = 0;
          for (int c = 0; c < 3; ++c) {
            t1[c] = V[pr][c] - V[pl][c];
            t2[c] = V[pt][c] - 0.5 * (V[pl][c] + V[pr][c]);
            n1 += t1[c] * t1[c];
            n2 += t2[c] * t2[c];
          }
          for (int c = 0; c < 3; ++c) {
            t1[c] /= sqrt(n1);
            t2[c] /= sqrt(n2);
          }
          double dx, dy;
          face_shift(N, xlgl, alpha, L[pl], L[pr], L[pt], &dx, &dy);
          double blend = L[pl] * L[pr] * L[pt];
          double denom = (L[pl] + 0.5 * L[o]) * (L[pr] + 0.5 * L[o]) * (L[pt] + 0.5 * L[o]);
          if (denom > tol) blend = blend / denom;
          for (int c = 0; c < 3; ++c) shift[c] += blend * (dx * t1[c] + dy * t2[c]);
          int on_face = L[o] < tol;
          int npos = (L[pl] > tol) + (L[pr] > tol) + (L[pt] > tol);
          if (on_face && npos < 3)
            for (int c = 0; c < 3; ++c) shift[c] = dx * t1[c] + dy * t2[c];
        }
        for (int c = 0; c < 3; ++c) X[c] += shift[c];
        /* barycentrics of X: solve X - Va = lb (Vb-Va) + lc (Vc-Va) + ld (Vd-Va) by Cramer */
        double A[3][3], rhs[3];
        for (int c = 0; c < 3; ++c) {
          A[c][0] = V[1][c] - V[0][c];
          A[c][1] = V[2][c] - V[0][c];
          A[c][2] = V[3][c] - V[0][c];
          rhs[c] = X[c] - V[0][c];
        }
        double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        double sol[3];
        for (int q = 0; q < 3; ++q) {
          double B[3][3];
          memcpy(B, A, sizeof B);
          for (int c = 0; c < 3; ++c) B[c][q] = rhs[c];
          sol[q] = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                    B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                    B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0])) / det;
        }
        r[idx] = 2.0 * sol[0] - 1.0;
        s[idx] = 2.0 * sol[1] - 1.0;
        t[idx] = 2.0 * sol[2] - 1.0;
        ++idx;
      }
  return 0;
}

int or_nodes(int N, double *r, double *s, double *t) { return or_nodes_alpha(N, 0.0, r, s, t); }

/* ------------------------------------------------------------------ */
/* Orthonormal bases                                                   */
/* ------------------------------------------------------------------ */

/* Modes of P_N on the tetrahedron, ordered i outer, j middle, k inner. */
static void mode_ijk(int N, int m, int *pi, int *pj, int *pk) {
  int c = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k) {
        if (c == m) {
          *pi = i;
          *pj = j;
          *pk = k;
          return;
        }
        ++c;
      }
}

/* PKD basis psi_ijk = sqrt(8) P_i(a) P_j^(2i+1,0)(b) (1-b)^i P_k^(2i+2j+2,0)(c) (1-c)^(i+j)
 * in collapsed coordinates a = 2(1+r)/(-s-t) - 1, b = 2(1+s)/(1-t) - 1, c = t, with
 * its gradient by the chain rule through (a, b, c); the removable singular
 * factors 1/(1-b), 1/(1-c) are absorbed into the powers (1-b)^i, (1-c)^(i+j). */
int or_basis(int N, int m, double r, double s, double t, double *val, double *dr, double *ds,
             double *dt) {
  int i, j, k;
  mode_ijk(N, m, &i, &j, &k);
  double a = (fabs(s + t) > 1e-12) ? 2.0 * (1.0 + r) / (-s - t) - 1.0 : -1.0;
  double b = (fabs(t - 1.0) > 1e-12) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  double c = t;
  double fa = jnorm(i, 0, 0, a), dfa = djnorm(i, 0, 0, a);
  double gb = jnorm(j, 2.0 * i + 1.0, 0, b), dgb = djnorm(j, 2.0 * i + 1.0, 0, b);
  double hc = jnorm(k, 2.0 * i + 2.0 * j + 2.0, 0, c), dhc = djnorm(k, 2.0 * i + 2.0 * j + 2.0, 0, c);
  double s8 = sqrt(8.0);
  if (val) *val = s8 * fa * gb * pow(1.0 - b, i) * hc * pow(1.0 - c, i + j);
  /* d/dr: only through a, da/dr = 4 / ((1-b)(1-c)) */
  double vr = 0.0;
  if (i > 0) vr = s8 * dfa * gb * pow(1.0 - b, i - 1) * 4.0 * hc * pow(1.0 - c, i + j - 1);
  /* a-term shared by d/ds and d/dt: da/ds = da/dt = 2(1+a)/((1-b)(1-c)) */
  double va = 0.0;
  if (i > 0) va = s8 * dfa * (1.0 + a) * gb * pow(1.0 - b, i - 1) * 2.0 * hc * pow(1.0 - c, i + j - 1);
  /* d/db of g(b) = P_j(b) (1-b)^i */
  double dg = dgb * pow(1.0 - b, i) - ((i > 0) ? i * gb * pow(1.0 - b, i - 1) : 0.0);
  double vbs = 0.0, vbt = 0.0;
  if (i + j > 0) {
    /* db/ds = 2/(1-c), db/dt = (1+b)/(1-c) */
    vbs = s8 * fa * dg * 2.0 * hc * pow(1.0 - c, i + j - 1);
    vbt = s8 * fa * dg * (1.0 + b) * hc * pow(1.0 - c, i + j - 1);
  }
  /* d/dc of h(c) = P_k(c) (1-c)^(i+j) */
  double dh = dhc * pow(1.0 - c, i + j) - ((i + j > 0) ? (i + j) * hc * pow(1.0 - c, i + j - 1) : 0.0);
  double vc = s8 * fa * gb * pow(1.0 - b, i) * dh;
  if (dr) *dr = vr;
  if (ds) *ds = va + vbs;
  if (dt) *dt = va + vbt + vc;
  return 0;
}

/* Orthonormal Dubiner basis on the triangle (-1,-1),(1,-1),(-1,1):
 * phi_ij = sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i, a = 2(1+x)/(1-y) - 1, b = y. */
static double basis2d(int N, int m, double x, double y) {
  int c = 0, ii = 0, jj = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j) {
      if (c == m) {
        ii = i;
        jj = j;
      }
      ++c;
    }
  double a = (fabs(y - 1.0) > 1e-12) ? 2.0 * (1.0 + x) / (1.0 - y) - 1.0 : -1.0;
  return sqrt(2.0) * jnorm(ii, 0, 0, a) * jnorm(jj, 2.0 * ii + 1.0, 0, y) * pow(1.0 - y, ii);
}

/* ------------------------------------------------------------------ */
/* Reference operators                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
  int N, Np, Nfp;
  double *r, *s, *t;
  double *V, *Dr, *Ds, *Dt, *M, *Minv, *LIFT, *Mf; /* Mf: 4 x Nfp x Nfp */
  int *Fmask;                                      /* 4 x Nfp */
} ref_ops;

static void ops_free(ref_ops *o) {
  free(o->r); free(o->s); free(o->t); free(o->V); free(o->Dr); free(o->Ds); free(o->Dt);
  free(o->M); free(o->Minv); free(o->LIFT); free(o->Mf); free(o->Fmask);
}

static int ops_build(int N, double alpha, ref_ops *o) {
  memset(o, 0, sizeof *o);
  int Np = or_np(N), Nfp = or_nfp(N);
  o->N = N; o->Np = Np; o->Nfp = Nfp;
  o->r = malloc(sizeof(double) * Np); o->s = malloc(sizeof(double) * Np); o->t = malloc(sizeof(double) * Np);
  if (or_nodes_alpha(N, alpha, o->r, o->s, o->t)) return -1;
  size_t nn = (size_t)Np * Np;
  o->V = malloc(sizeof(double) * nn);
  double *Vr = malloc(sizeof(double) * nn), *Vs = malloc(sizeof(double) * nn), *Vt = malloc(sizeof(double) * nn);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < Np; ++m)
      or_basis(N, m, o->r[i], o->s[i], o->t[i], &o->V[i * Np + m], &Vr[i * Np + m], &Vs[i * Np + m], &Vt[i * Np + m]);
  double *Vinv = malloc(sizeof(double) * nn);
  if (mat_inverse(Np, o->V, Vinv)) return fail("singular Vandermonde");
  o->Dr = malloc(sizeof(double) * nn); o->Ds = malloc(sizeof(double) * nn); o->Dt = malloc(sizeof(double) * nn);
  mat_mul(Np, Np, Np, Vr, Vinv, o->Dr);
  mat_mul(Np, Np, Np, Vs, Vinv, o->Ds);
  mat_mul(Np, Np, Np, Vt, Vinv, o->Dt);
  /* M^-1 = V V^T (orthonormal basis), M = (V V^T)^-1 */
  o->Minv = malloc(sizeof(double) * nn);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += o->V[i * Np + m] * o->V[j * Np + m];
      o->Minv[i * Np + j] = acc;
    }
  o->M = malloc(sizeof(double) * nn);
  if (mat_inverse(Np, o->Minv, o->M)) return fail("singular mass matrix");
  /* face masks: t=-1, s=-1, r+s+t=-1, r=-1 */
  o->Fmask = malloc(sizeof(int) * 4 * Nfp);
  int cnt[4] = {0, 0, 0, 0};
  for (int i = 0; i < Np; ++i) {
    double on[4] = {fabs(1.0 + o->t[i]), fabs(1.0 + o->s[i]), fabs(1.0 + o->r[i] + o->s[i] + o->t[i]), fabs(1.0 + o->r[i])};
    for (int f = 0; f < 4; ++f)
      if (on[f] < 1e-10) {
        if (cnt[f] >= Nfp) return fail("too many face nodes");
        o->Fmask[f * Nfp + cnt[f]++] = i;
      }
  }
  for (int f = 0; f < 4; ++f)
    if (cnt[f] != Nfp) return fail("face node count mismatch");
  /* face mass matrices on the reference triangle in the face's own two coordinates */
  o->Mf = malloc(sizeof(double) * 4 * Nfp * Nfp);
  double *V2 = malloc(sizeof(double) * Nfp * Nfp), *MfInv = malloc(sizeof(double) * Nfp * Nfp);
  for (int f = 0; f < 4; ++f) {
    for (int m = 0; m < Nfp; ++m) {
      int i = o->Fmask[f * Nfp + m];
      double x2, y2;
      if (f == 0) { x2 = o->r[i]; y2 = o->s[i]; }
      else if (f == 1) { x2 = o->r[i]; y2 = o->t[i]; }
      else { x2 = o->s[i]; y2 = o->t[i]; }
      for (int q = 0; q < Nfp; ++q) V2[m * Nfp + q] = basis2d(N, q, x2, y2);
    }
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) {
        double acc = 0.0;
        for (int q = 0; q < Nfp; ++q) acc += V2[a * Nfp + q] * V2[b * Nfp + q];
        MfInv[a * Nfp + b] = acc;
      }
    if (mat_inverse(Nfp, MfInv, o->Mf + (size_t)f * Nfp * Nfp)) return fail("singular face mass");
  }
  /* LIFT = M^-1 E, E embeds the face mass matrices at the face nodes */
  double *E = calloc((size_t)Np * 4 * Nfp, sizeof(double));
  for (int f = 0; f < 4; ++f)
    for (int m = 0; m < Nfp; ++m)
      for (int n = 0; n < Nfp; ++n)
        E[o->Fmask[f * Nfp + m] * 4 * Nfp + f * Nfp + n] += o->Mf[(size_t)f * Nfp * Nfp + m * Nfp + n];
  o->LIFT = malloc(sizeof(double) * Np * 4 * Nfp);
  mat_mul(Np, Np, 4 * Nfp, o->Minv, E, o->LIFT);
  free(E); free(V2); free(MfInv); free(Vinv); free(Vr); free(Vs); free(Vt);
  return 0;
}

int or_operators_alpha(int N, double alpha, double *V, double *Dr, double *Ds, double *Dt, double *M,
                       int32_t *Fmask, double *Mf, double *LIFT) {
  ref_ops o;
  if (N < 1 || N > 10) return fail("or_operators: N out of range");
  if (ops_build(N, alpha, &o)) { ops_free(&o); return -1; }
  size_t nn = (size_t)o.Np * o.Np;
  if (V) memcpy(V, o.V, sizeof(double) * nn);
  if (Dr) memcpy(Dr, o.Dr, sizeof(double) * nn);
  if (Ds) memcpy(Ds, o.Ds, sizeof(double) * nn);
  if (Dt) memcpy(Dt, o.Dt, sizeof(double) * nn);
  if (M) memcpy(M, o.M, sizeof(double) * nn);
  if (Fmask) for (int q = 0; q < 4 * o.Nfp; ++q) Fmask[q] = o.Fmask[q];
  if (Mf) memcpy(Mf, o.Mf, sizeof(double) * 4 * o.Nfp * o.Nfp);
  if (LIFT) memcpy(LIFT, o.LIFT, sizeof(double) * o.Np * 4 * o.Nfp);
  ops_free(&o);
  return 0;
}

int or_operators(int N, double *V, double *Dr, double *Ds, double *Dt, double *M, int32_t *Fmask, double *Mf,
                 double *LIFT) {
  return or_operators_alpha(N, 0.0, V, Dr, Ds, Dt, M, Fmask, Mf, LIFT);
}

/* Lebesgue constant of the warp & blend nodes with blend parameter alpha,
 * estimated as the largest sum over the nodal basis of |l_i(x)| over the
 * points x of the order-M equidistant lattice of the tetrahedron. l_i(x) =
 * sum_m phi_m(x) (V^-1)_{m i}, with V the orthonormal-basis Vandermonde at the
 * nodes (the definition of the Lagrange basis through the modal one). */
int or_lebesgue(int N, double alpha, int M, double *lambda) {
  if (M < 1 || M > 200) return fail("or_lebesgue: lattice order out of range");
  ref_ops o;
  if (N < 1 || N > 10) return fail("or_lebesgue: N out of range");
  if (ops_build(N, alpha, &o)) { ops_free(&o); return -1; }
  const int Np = o.Np;
  double *Vinv = malloc(sizeof(double) * Np * Np), *phi = malloc(sizeof(double) * Np);
  if (mat_inverse(Np, o.V, Vinv)) { free(Vinv); free(phi); ops_free(&o); return fail("singular Vandermonde"); }
  double best = 0.0;
  for (int k = 0; k <= M; ++k)
    for (int j = 0; j <= M - k; ++j)
      for (int i = 0; i <= M - k - j; ++i) {
        const double r = -1.0 + 2.0 * i / M, s = -1.0 + 2.0 * j / M, t = -1.0 + 2.0 * k / M;
        double d0, d1, d2;
        for (int m = 0; m < Np; ++m) or_basis(N, m, r, s, t, &phi[m], &d0, &d1, &d2);
        double sum = 0.0;
        for (int q = 0; q < Np; ++q) {
          double l = 0.0;
          for (int m = 0; m < Np; ++m) l += phi[m] * Vinv[m * Np + q];
          sum += fabs(l);
        }
        if (sum > best) best = sum;
      }
  *lambda = best;
  free(Vinv); free(phi); ops_free(&o);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Mesh: connectivity, geometry, exterior node map                     */
/* ------------------------------------------------------------------ */

struct or_mesh {
  ref_ops o;
  int64_t K;
  double *x, *y, *z;    /* K x Np */
  double *G;            /* K x 10: rx ry rz sx sy sz tx ty tz J */
  double *F;            /* K x 4 x 5: nx ny nz sJ Fscale */
  int64_t *EToE, *EToF; /* K x 4 */
  int64_t *ext;         /* K x 4 x Nfp */
  double *eps, *mu;     /* K */
};

/* local vertices of each reference face: t=-1 (a,b,c), s=-1 (a,b,d), r+s+t=-1 (b,c,d), r=-1 (a,c,d) */
static const int FACE_V[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

typedef struct {
  int64_t v[3];
  int64_t k;
  int f;
} face_key;

static int cmp_face(const void *pa, const void *pb) {
  const face_key *a = pa, *b = pb;
  for (int q = 0; q < 3; ++q)
    if (a->v[q] != b->v[q]) return a->v[q] < b->v[q] ? -1 : 1;
  return 0;
}

void or_mesh_destroy(or_mesh *m) {
  if (!m) return;
  ops_free(&m->o);
  free(m->x); free(m->y); free(m->z); free(m->G); free(m->F); free(m->EToE); free(m->EToF);
  free(m->ext); free(m->eps); free(m->mu);
  free(m);
}

int64_t or_mesh_K(const or_mesh *m) { return m->K; }

or_mesh *or_mesh_create_alpha(int N, double alpha, int64_t Nv, const double *VX, const double *VY, const double *VZ,
                              int64_t K, const int32_t *EToV, const double *eps, const double *mu) {
  if (K < 1 || Nv < 4) { fail("or_mesh_create: empty mesh"); return NULL; }
  or_mesh *m = calloc(1, sizeof(or_mesh));
  if (ops_build(N, alpha, &m->o)) { or_mesh_destroy(m); return NULL; }
  int Np = m->o.Np, Nfp = m->o.Nfp;
  m->K = K;
  m->x = malloc(sizeof(double) * K * Np); m->y = malloc(sizeof(double) * K * Np); m->z = malloc(sizeof(double) * K * Np);
  m->G = malloc(sizeof(double) * K * 10);
  m->F = malloc(sizeof(double) * K * 20);
  m->EToE = malloc(sizeof(int64_t) * K * 4); m->EToF = malloc(sizeof(int64_t) * K * 4);
  m->ext = malloc(sizeof(int64_t) * K * 4 * Nfp);
  m->eps = malloc(sizeof(double) * K); m->mu = malloc(sizeof(double) * K);
  for (int64_t k = 0; k < K; ++k) {
    m->eps[k] = eps ? eps[k] : 1.0;
    m->mu[k] = mu ? mu[k] : 1.0;
    if (!(m->eps[k] > 0.0) || !(m->mu[k] > 0.0)) { fail("non-positive material"); or_mesh_destroy(m); return NULL; }
  }
  for (int64_t k = 0; k < K; ++k) {
    double P[4][3];
    for (int v = 0; v < 4; ++v) {
      int32_t id = EToV[k * 4 + v];
      if (id < 0 || id >= Nv) { fail("EToV index out of range"); or_mesh_destroy(m); return NULL; }
      P[v][0] = VX[id]; P[v][1] = VY[id]; P[v][2] = VZ[id];
    }
    /* affine map x = 1/2 (-(1+r+s+t) Pa + (1+r) Pb + (1+s) Pc + (1+t) Pd) */
    for (int i = 0; i < Np; ++i) {
      double r = m->o.r[i], s = m->o.s[i], t = m->o.t[i];
      double w[4] = {-(1.0 + r + s + t) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0, (1.0 + t) / 2.0};
      double X = 0, Y = 0, Z = 0;
      for (int v = 0; v < 4; ++v) { X += w[v] * P[v][0]; Y += w[v] * P[v][1]; Z += w[v] * P[v][2]; }
      m->x[k * Np + i] = X; m->y[k * Np + i] = Y; m->z[k * Np + i] = Z;
    }
    /* A = dx/d(r,s,t): columns x_r, x_s, x_t; rows of A^-1 are grad r, grad s, grad t */
    double A[9], Ai[9];
    for (int c = 0; c < 3; ++c) {
      A[c * 3 + 0] = 0.5 * (P[1][c] - P[0][c]);
      A[c * 3 + 1] = 0.5 * (P[2][c] - P[0][c]);
      A[c * 3 + 2] = 0.5 * (P[3][c] - P[0][c]);
    }
    double J = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(J > 0.0)) { fail("element with non-positive Jacobian"); or_mesh_destroy(m); return NULL; }
    if (mat_inverse(3, A, Ai)) { fail("singular element map"); or_mesh_destroy(m); return NULL; }
    for (int q = 0; q < 9; ++q) m->G[k * 10 + q] = Ai[q];
    m->G[k * 10 + 9] = J;
    /* faces: outward unit normal from the cross product of two physical edges,
     * surface Jacobian = physical area / reference-triangle area (2) */
    for (int f = 0; f < 4; ++f) {
      const double *p0 = P[FACE_V[f][0]], *p1 = P[FACE_V[f][1]], *p2 = P[FACE_V[f][2]];
      int opp = 6 - FACE_V[f][0] - FACE_V[f][1] - FACE_V[f][2];
      double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
      double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
      double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double to_opp = (P[opp][0] - p0[0]) * n[0] + (P[opp][1] - p0[1]) * n[1] + (P[opp][2] - p0[2]) * n[2];
      double sgn = to_opp > 0 ? -1.0 : 1.0;
      double area = 0.5 * len;
      double sJ = area / 2.0;
      double *Fk = m->F + (k * 4 + f) * 5;
      Fk[0] = sgn * n[0] / len; Fk[1] = sgn * n[1] / len; Fk[2] = sgn * n[2] / len;
      Fk[3] = sJ;
      Fk[4] = sJ / J;
    }
  }
  /* connectivity: match faces by their sorted global vertex triples */
  face_key *keys = malloc(sizeof(face_key) * K * 4);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t v[3] = {EToV[k * 4 + FACE_V[f][0]], EToV[k * 4 + FACE_V[f][1]], EToV[k * 4 + FACE_V[f][2]]};
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
          if (v[b] < v[a]) { int64_t tmp = v[a]; v[a] = v[b]; v[b] = tmp; }
      face_key *fk = &keys[k * 4 + f];
      fk->v[0] = v[0]; fk->v[1] = v[1]; fk->v[2] = v[2]; fk->k = k; fk->f = f;
      m->EToE[k * 4 + f] = -1;
      m->EToF[k * 4 + f] = -1;
    }
  qsort(keys, (size_t)K * 4, sizeof(face_key), cmp_face);
  for (int64_t q = 0; q < K * 4;) {
    int64_t e = q + 1;
    while (e < K * 4 && cmp_face(&keys[q], &keys[e]) == 0) ++e;
    if (e - q > 2) { free(keys); fail("non-conforming face shared by more than two elements"); or_mesh_destroy(m); return NULL; }
    if (e - q == 2) {
      m->EToE[keys[q].k * 4 + keys[q].f] = keys[q + 1].k;
      m->EToF[keys[q].k * 4 + keys[q].f] = keys[q + 1].f;
      m->EToE[keys[q + 1].k * 4 + keys[q + 1].f] = keys[q].k;
      m->EToF[keys[q + 1].k * 4 + keys[q + 1].f] = keys[q].f;
    }
    q = e;
  }
  free(keys);
  /* exterior nodes: the neighbour's face node at the same physical point */
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t k2 = m->EToE[k * 4 + f];
      int64_t f2 = m->EToF[k * 4 + f];
      for (int a = 0; a < Nfp; ++a) {
        int64_t *out = &m->ext[(k * 4 + f) * Nfp + a];
        if (k2 < 0) { *out = -1; continue; }
        int i = m->o.Fmask[f * Nfp + a];
        double X = m->x[k * Np + i], Y = m->y[k * Np + i], Z = m->z[k * Np + i];
        int best = -1;
        double bestd = 1e300;
        for (int b = 0; b < Nfp; ++b) {
          int i2 = m->o.Fmask[f2 * Nfp + b];
          double dx = X - m->x[k2 * Np + i2], dy = Y - m->y[k2 * Np + i2], dz = Z - m->z[k2 * Np + i2];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d < bestd) { bestd = d; best = i2; }
        }
        if (bestd > 1e-9) { fail("face nodes of neighbouring elements do not coincide"); or_mesh_destroy(m); return NULL; }
        *out = k2 * Np + best;
      }
    }
  return m;
}

or_mesh *or_mesh_create(int N, int64_t Nv, const double *VX, const double *VY, const double *VZ, int64_t K,
                        const int32_t *EToV, const double *eps, const double *mu) {
  return or_mesh_create_alpha(N, 0.0, Nv, VX, VY, VZ, K, EToV, eps, mu);
}

int or_mesh_coords(const or_mesh *m, double *x, double *y, double *z) {
  size_t n = (size_t)m->K * m->o.Np;
  if (x) memcpy(x, m->x, sizeof(double) * n);
  if (y) memcpy(y, m->y, sizeof(double) * n);
  if (z) memcpy(z, m->z, sizeof(double) * n);
  return 0;
}

int or_mesh_geometry(const or_mesh *m, double *G, double *F, int64_t *EToE, int64_t *EToF) {
  if (G) memcpy(G, m->G, sizeof(double) * m->K * 10);
  if (F) memcpy(F, m->F, sizeof(double) * m->K * 20);
  if (EToE) memcpy(EToE, m->EToE, sizeof(int64_t) * m->K * 4);
  if (EToF) memcpy(EToF, m->EToF, sizeof(int64_t) * m->K * 4);
  return 0;
}

int or_mesh_exterior(const or_mesh *m, int64_t *ext) {
  memcpy(ext, m->ext, sizeof(int64_t) * m->K * 4 * m->o.Nfp);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Right-hand side                                                     */
/* ------------------------------------------------------------------ */

static void cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Interior and exterior traces at face node a of face f of element k. PEC
 * walls mirror the interior state: E+ = -E-, H+ = H-, with the interior
 * material on both sides. */
static void traces(const or_mesh *m, const double *u, int64_t k, int f, int a, double qm[6], double qp[6],
                   double *Zm, double *Zp, double *Ym, double *Yp) {
  int Np = m->o.Np, Nfp = m->o.Nfp;
  int64_t KNp = m->K * Np;
  int i = m->o.Fmask[f * Nfp + a];
  for (int c = 0; c < 6; ++c) qm[c] = u[c * KNp + k * Np + i];
  *Zm = sqrt(m->mu[k] / m->eps[k]);
  *Ym = 1.0 / *Zm;
  int64_t g = m->ext[(k * 4 + f) * Nfp + a];
  if (g < 0) {
    for (int c = 0; c < 3; ++c) { qp[c] = -qm[c]; qp[c + 3] = qm[c + 3]; }
    *Zp = *Zm;
    *Yp = *Ym;
  } else {
    int64_t k2 = g / Np;
    for (int c = 0; c < 6; ++c) qp[c] = u[c * KNp + g];
    *Zp = sqrt(m->mu[k2] / m->eps[k2]);
    *Yp = 1.0 / *Zp;
  }
}

/* Maxwell numerical flux difference n.(F - F*) at one face node, with
 * jumps dq = q+ - q- (Fig. flux-code a for Z- = Z+ = 1):
 *   flux_E = n x (Z+ dH - alpha n x dE) / (Z- + Z+)
 *   flux_H = -n x (Y+ dE + alpha n x dH) / (Y- + Y+)              */
static void maxwell_flux(const double n[3], const double qm[6], const double qp[6], double Zm, double Zp,
                         double Ym, double Yp, double alpha, double fE[3], double fH[3]) {
  double dE[3], dH[3], nxdE[3], nxdH[3], tmp[3], v[3];
  for (int c = 0; c < 3; ++c) { dE[c] = qp[c] - qm[c]; dH[c] = qp[c + 3] - qm[c + 3]; }
  cross(n, dE, nxdE);
  cross(n, dH, nxdH);
  for (int c = 0; c < 3; ++c) v[c] = Zp * dH[c] - alpha * nxdE[c];
  cross(n, v, tmp);
  for (int c = 0; c < 3; ++c) fE[c] = tmp[c] / (Zm + Zp);
  for (int c = 0; c < 3; ++c) v[c] = Yp * dE[c] + alpha * nxdH[c];
  cross(n, v, tmp);
  for (int c = 0; c < 3; ++c) fH[c] = -tmp[c] / (Ym + Yp);
}

int or_flux(const double *n, const double *qm, const double *qp, double Zm, double Zp, double alpha, double *fE,
            double *fH) {
  maxwell_flux(n, qm, qp, Zm, Zp, 1.0 / Zm, 1.0 / Zp, alpha, fE, fH);
  return 0;
}

/* rhs for element k into out[6][Np] (stride Np per field). */
static void element_rhs(const or_mesh *m, const double *u, int64_t k, double alpha, double *out) {
  int Np = m->o.Np, Nfp = m->o.Nfp;
  int64_t KNp = m->K * Np;
  const double *G = m->G + k * 10;
  double *d = malloc(sizeof(double) * 6 * 3 * Np); /* d[field][x|y|z][i] */
  double *flux = malloc(sizeof(double) * 6 * 4 * Nfp);
  /* local differentiation: d/dx = rx Dr + sx Ds + tx Dt etc. (eq. dg-reference-matrices) */
  for (int c = 0; c < 6; ++c) {
    const double *q = u + c * KNp + k * Np;
    for (int i = 0; i < Np; ++i) {
      double ur = 0, us = 0, ut = 0;
      for (int j = 0; j < Np; ++j) {
        ur += m->o.Dr[i * Np + j] * q[j];
        us += m->o.Ds[i * Np + j] * q[j];
        ut += m->o.Dt[i * Np + j] * q[j];
      }
      for (int x = 0; x < 3; ++x) d[(c * 3 + x) * Np + i] = G[0 + x] * ur + G[3 + x] * us + G[6 + x] * ut;
    }
  }
  /* flux gather (eq. num-flux), scaled by Fscale = sJ/J */
  for (int f = 0; f < 4; ++f) {
    const double *Fk = m->F + (k * 4 + f) * 5;
    for (int a = 0; a < Nfp; ++a) {
      double qm[6], qp[6], Zm, Zp, Ym, Yp, fE[3], fH[3];
      traces(m, u, k, f, a, qm, qp, &Zm, &Zp, &Ym, &Yp);
      maxwell_flux(Fk, qm, qp, Zm, Zp, Ym, Yp, alpha, fE, fH);
      for (int c = 0; c < 3; ++c) {
        flux[c * 4 * Nfp + f * Nfp + a] = Fk[4] * fE[c];
        flux[(c + 3) * 4 * Nfp + f * Nfp + a] = Fk[4] * fH[c];
      }
    }
  }
  /* eps dE/dt = curl H + L flux_E,  mu dH/dt = -curl E + L flux_H */
  double ie = 1.0 / m->eps[k], im = 1.0 / m->mu[k];
  for (int i = 0; i < Np; ++i) {
    double curlH[3], curlE[3];
    /* d index: field*3 + direction; Ex..Ez = 0..2, Hx..Hz = 3..5 */
#define D(field, dir) d[((field) * 3 + (dir)) * Np + i]
    curlH[0] = D(5, 1) - D(4, 2);
    curlH[1] = D(3, 2) - D(5, 0);
    curlH[2] = D(4, 0) - D(3, 1);
    curlE[0] = D(2, 1) - D(1, 2);
    curlE[1] = D(0, 2) - D(2, 0);
    curlE[2] = D(1, 0) - D(0, 1);
#undef D
    for (int c = 0; c < 6; ++c) {
      double lift = 0.0;
      for (int q = 0; q < 4 * Nfp; ++q) lift += m->o.LIFT[i * 4 * Nfp + q] * flux[c * 4 * Nfp + q];
      if (c < 3) out[c * Np + i] = ie * (curlH[c] + lift);
      else out[c * Np + i] = im * (-curlE[c - 3] + lift);
    }
  }
  free(d);
  free(flux);
}

int or_rhs(const or_mesh *m, const double *u, double *rhs, double alpha) {
  int Np = m->o.Np;
  int64_t KNp = m->K * Np;
  /* Elements are independent. A build of this file with OpenMP (long
   * reference runs only) splits them over threads; the arithmetic of each
   * element is the same as in the default single-threaded build. */
#pragma omp parallel
  {
    double *out = malloc(sizeof(double) * 6 * Np);
#pragma omp for schedule(static)
    for (int64_t k = 0; k < m->K; ++k) {
      element_rhs(m, u, k, alpha, out);
      for (int c = 0; c < 6; ++c)
        for (int i = 0; i < Np; ++i) rhs[c * KNp + k * Np + i] = out[c * Np + i];
    }
    free(out);
  }
  return 0;
}

int or_rhs_subset(const or_mesh *m, const double *u, double *rhs_sub, double alpha, const int64_t *elems, int64_t n) {
  int Np = m->o.Np;
  double *out = malloc(sizeof(double) * 6 * Np);
  for (int64_t q = 0; q < n; ++q) {
    if (elems[q] < 0 || elems[q] >= m->K) { free(out); return fail("element index out of range"); }
    element_rhs(m, u, elems[q], alpha, out);
    for (int c = 0; c < 6; ++c)
      for (int i = 0; i < Np; ++i) rhs_sub[(c * n + q) * Np + i] = out[c * Np + i];
  }
  free(out);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Time stepping                                                       */
/* ------------------------------------------------------------------ */

int or_lserk_coeffs(double *a, double *b, double *c) {
  const double A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                       -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
  const double B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                       1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                       2277821191437.0 / 14882151754819.0};
  const double C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                       2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
  for (int q = 0; q < 5; ++q) {
    if (a) a[q] = A[q];
    if (b) b[q] = B[q];
    if (c) c[q] = C[q];
  }
  return 0;
}

int or_lserk(const or_mesh *m, double *u, double *res, double dt, int nsteps, double alpha) {
  double a[5], b[5];
  or_lserk_coeffs(a, b, NULL);
  int64_t n = 6 * m->K * m->o.Np;
  double *rhs = malloc(sizeof(double) * n);
  for (int step = 0; step < nsteps; ++step)
    for (int s = 0; s < 5; ++s) {
      or_rhs(m, u, rhs, alpha);
      for (int64_t q = 0; q < n; ++q) {
        res[q] = a[s] * res[q] + dt * rhs[q];
        u[q] = u[q] + b[s] * res[q];
      }
    }
  free(rhs);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Energy and the closed-form upwind dissipation                       */
/* ------------------------------------------------------------------ */

double or_energy(const or_mesh *m, const double *u) {
  int Np = m->o.Np;
  int64_t KNp = m->K * Np;
  double total = 0.0;
  for (int64_t k = 0; k < m->K; ++k) {
    double J = m->G[k * 10 + 9];
    for (int c = 0; c < 6; ++c) {
      const double *q = u + c * KNp + k * Np;
      double w = (c < 3) ? m->eps[k] : m->mu[k];
      double acc = 0.0;
      for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) acc += q[i] * m->o.M[i * Np + j] * q[j];
      total += 0.5 * J * w * acc;
    }
  }
  return total;
}

double or_face_dissipation(const or_mesh *m, const double *u, double alpha) {
  int Nfp = m->o.Nfp;
  double total = 0.0;
  double *tE = malloc(sizeof(double) * 3 * Nfp), *tH = malloc(sizeof(double) * 3 * Nfp);
  for (int64_t k = 0; k < m->K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t k2 = m->EToE[k * 4 + f];
      if (k2 >= 0 && k2 < k) continue; /* each interior face once */
      const double *Fk = m->F + (k * 4 + f) * 5;
      double Zm = 0, Zp = 0, Ym = 0, Yp = 0;
      for (int a = 0; a < Nfp; ++a) {
        double qm[6], qp[6], dE[3], dH[3], t1[3], t2[3];
        traces(m, u, k, f, a, qm, qp, &Zm, &Zp, &Ym, &Yp);
        for (int c = 0; c < 3; ++c) { dE[c] = qp[c] - qm[c]; dH[c] = qp[c + 3] - qm[c + 3]; }
        /* tangential jump components: n x dq has the same length as dq_t */
        cross(Fk, dE, t1);
        cross(Fk, dH, t2);
        for (int c = 0; c < 3; ++c) { tE[c * Nfp + a] = t1[c]; tH[c * Nfp + a] = t2[c]; }
      }
      const double *Mf = m->o.Mf + (size_t)f * Nfp * Nfp;
      double sE = 0.0, sH = 0.0;
      for (int c = 0; c < 3; ++c)
        for (int a = 0; a < Nfp; ++a)
          for (int b = 0; b < Nfp; ++b) {
            sE += tE[c * Nfp + a] * Mf[a * Nfp + b] * tE[c * Nfp + b];
            sH += tH[c * Nfp + a] * Mf[a * Nfp + b] * tH[c * Nfp + b];
          }
      if (k2 < 0) {
        /* PEC wall seen from one side only: dE = -2E-, dH = 0, so the rate
         * -(alpha/Z) |E-_t|^2 equals -(alpha/(4Z)) |dE_t|^2 */
        total += Fk[3] * alpha / (4.0 * Zm) * sE;
      } else {
        total += Fk[3] * (alpha / (Zm + Zp) * sE + alpha / (Ym + Yp) * sH);
      }
    }
  free(tE);
  free(tH);
  return total;
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint                                                    */
/* ------------------------------------------------------------------ */

/* w = A^T v for the linear operator u -> or_rhs(u). Each element's rows are
 * rhs_k = W_k (Vol_k u_k + LIFT (Fscale flux(u-, u+))), W_k = diag(1/eps, 1/mu);
 * transposing: scale v by W, apply the transposed curl with D^T, and scatter
 * the transposed flux Jacobians onto the interior and exterior nodes. */
int or_rhs_transpose(const or_mesh *m, const double *v, double *w, double alpha) {
  int Np = m->o.Np, Nfp = m->o.Nfp;
  int64_t KNp = m->K * Np;
  memset(w, 0, sizeof(double) * 6 * KNp);
  double *vt = malloc(sizeof(double) * 6 * Np), *g = malloc(sizeof(double) * 6 * 4 * Nfp);
  for (int64_t k = 0; k < m->K; ++k) {
    const double *G = m->G + k * 10;
    double ie = 1.0 / m->eps[k], im = 1.0 / m->mu[k];
    for (int c = 0; c < 6; ++c)
      for (int i = 0; i < Np; ++i) vt[c * Np + i] = (c < 3 ? ie : im) * v[c * KNp + k * Np + i];
    /* volume: rows E_c receive curl H, rows H_c receive -curl E.
     * curl_c(F) = d_{c+1} F_{c+2} - d_{c+2} F_{c+1}; transposing d_x = rx Dr + sx Ds + tx Dt
     * gives d_x^T = rx Dr^T + sx Ds^T + tx Dt^T. */
    for (int c = 0; c < 3; ++c) {
      int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      for (int j = 0; j < Np; ++j) {
        double tE1 = 0, tE2 = 0, tH1 = 0, tH2 = 0;
        for (int i = 0; i < Np; ++i) {
          double dx1 = G[0 + c1] * m->o.Dr[i * Np + j] + G[3 + c1] * m->o.Ds[i * Np + j] + G[6 + c1] * m->o.Dt[i * Np + j];
          double dx2 = G[0 + c2] * m->o.Dr[i * Np + j] + G[3 + c2] * m->o.Ds[i * Np + j] + G[6 + c2] * m->o.Dt[i * Np + j];
          tE1 += dx1 * vt[c * Np + i];       /* d_{c1}^T vE_c -> H_{c2} */
          tE2 += dx2 * vt[c * Np + i];       /* -d_{c2}^T vE_c -> H_{c1} */
          tH1 += dx1 * vt[(c + 3) * Np + i]; /* -d_{c1}^T vH_c -> E_{c2} */
          tH2 += dx2 * vt[(c + 3) * Np + i]; /* d_{c2}^T vH_c -> E_{c1} */
        }
        w[(3 + c2) * KNp + k * Np + j] += tE1;
        w[(3 + c1) * KNp + k * Np + j] -= tE2;
        w[c2 * KNp + k * Np + j] -= tH1;
        w[c1 * KNp + k * Np + j] += tH2;
      }
    }
    /* surface: g = Fscale * LIFT^T vt, then transposed flux Jacobians */
    for (int c = 0; c < 6; ++c)
      for (int q = 0; q < 4 * Nfp; ++q) {
        double acc = 0.0;
        for (int i = 0; i < Np; ++i) acc += m->o.LIFT[i * 4 * Nfp + q] * vt[c * Np + i];
        g[c * 4 * Nfp + q] = acc * m->F[(k * 4 + q / Nfp) * 5 + 4];
      }
    for (int f = 0; f < 4; ++f) {
      const double *n = m->F + (k * 4 + f) * 5;
      for (int a = 0; a < Nfp; ++a) {
        double qm[6], qp[6], Zm, Zp, Ym, Yp;
        traces(m, v, k, f, a, qm, qp, &Zm, &Zp, &Ym, &Yp); /* only for the materials */
        double gE[3], gH[3], nxgE[3], nxgH[3], nnE[3], nnH[3];
        for (int c = 0; c < 3; ++c) { gE[c] = g[c * 4 * Nfp + f * Nfp + a]; gH[c] = g[(c + 3) * 4 * Nfp + f * Nfp + a]; }
        cross(n, gE, nxgE);
        cross(n, gH, nxgH);
        cross(n, nxgE, nnE);
        cross(n, nxgH, nnH);
        double Zs = Zm + Zp, Ys = Ym + Yp;
        double aEp[3], aEm[3], aHp[3], aHm[3];
        for (int c = 0; c < 3; ++c) {
          /* flux_E = (Z+/Zs) n x (H+ - H-) - (alpha/Zs) n x n x (E+ - E-);
           * flux_H = -(Y+/Ys) n x (E+ - E-) - (alpha/Ys) n x n x (H+ - H-);
           * (n x .)^T = -(n x .), (n x n x .)^T = n x n x . */
          aHp[c] = -(Zp / Zs) * nxgE[c] - (alpha / Ys) * nnH[c];
          aHm[c] = (Zp / Zs) * nxgE[c] + (alpha / Ys) * nnH[c];
          aEp[c] = -(alpha / Zs) * nnE[c] + (Yp / Ys) * nxgH[c];
          aEm[c] = (alpha / Zs) * nnE[c] - (Yp / Ys) * nxgH[c];
        }
        int i = m->o.Fmask[f * Nfp + a];
        int64_t ge = m->ext[(k * 4 + f) * Nfp + a];
        for (int c = 0; c < 3; ++c) {
          w[c * KNp + k * Np + i] += aEm[c];
          w[(c + 3) * KNp + k * Np + i] += aHm[c];
          if (ge < 0) { /* PEC: E+ = -E-, H+ = H- */
            w[c * KNp + k * Np + i] -= aEp[c];
            w[(c + 3) * KNp + k * Np + i] += aHp[c];
          } else {
            w[c * KNp + ge] += aEp[c];
            w[(c + 3) * KNp + ge] += aHp[c];
          }
        }
      }
    }
  }
  free(vt);
  free(g);
  return 0;
}

/* grad[k] += <lam, d(A u)/d eps_k> for all k. eps enters through 1/eps_k on the
 * E rows of element k and through Z = sqrt(mu/eps), Y = 1/Z in the flux weights
 * of the faces of k (as the interior value) and of its neighbours (as the
 * exterior value); dZ/deps = -Z/(2 eps), dY/deps = Y/(2 eps). */
static void eps_sensitivity(const or_mesh *m, const double *u, const double *lam, double alpha, double scale,
                            double *grad) {
  int Np = m->o.Np, Nfp = m->o.Nfp;
  int64_t KNp = m->K * Np;
  double *out = malloc(sizeof(double) * 6 * Np), *la = malloc(sizeof(double) * 6 * 4 * Nfp);
  for (int64_t k = 0; k < m->K; ++k) {
    double ie = 1.0 / m->eps[k], im = 1.0 / m->mu[k];
    /* 1/eps factor: d/deps (1/eps X) = -1/eps * rhs_E */
    element_rhs(m, u, k, alpha, out);
    double acc = 0.0;
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < Np; ++i) acc += lam[c * KNp + k * Np + i] * out[c * Np + i];
    grad[k] += scale * (-ie * acc);
    /* flux weights: la = LIFT^T lam (per face node), times Fscale and 1/eps or 1/mu */
    for (int c = 0; c < 6; ++c)
      for (int q = 0; q < 4 * Nfp; ++q) {
        double s = 0.0;
        for (int i = 0; i < Np; ++i) s += m->o.LIFT[i * 4 * Nfp + q] * lam[c * KNp + k * Np + i];
        la[c * 4 * Nfp + q] = s * m->F[(k * 4 + q / Nfp) * 5 + 4] * (c < 3 ? ie : im);
      }
    for (int f = 0; f < 4; ++f) {
      const double *n = m->F + (k * 4 + f) * 5;
      int64_t k2 = m->EToE[k * 4 + f];
      for (int a = 0; a < Nfp; ++a) {
        double qm[6], qp[6], Zm, Zp, Ym, Yp, fE[3], fH[3], nxdH[3], nxdE[3], dE[3], dH[3];
        traces(m, u, k, f, a, qm, qp, &Zm, &Zp, &Ym, &Yp);
        maxwell_flux(n, qm, qp, Zm, Zp, Ym, Yp, alpha, fE, fH);
        for (int c = 0; c < 3; ++c) { dE[c] = qp[c] - qm[c]; dH[c] = qp[c + 3] - qm[c + 3]; }
        cross(n, dH, nxdH);
        cross(n, dE, nxdE);
        double Zs = Zm + Zp, Ys = Ym + Yp;
        /* partial derivatives of the flux in the four weights */
        double sZm = 0, sZp = 0, sYm = 0, sYp = 0;
        for (int c = 0; c < 3; ++c) {
          double lE = la[c * 4 * Nfp + f * Nfp + a], lH = la[(c + 3) * 4 * Nfp + f * Nfp + a];
          sZm += lE * (-fE[c] / Zs);
          sZp += lE * (nxdH[c] / Zs - fE[c] / Zs);
          sYm += lH * (-fH[c] / Ys);
          sYp += lH * (-nxdE[c] / Ys - fH[c] / Ys);
        }
        int64_t kp = (k2 < 0) ? k : k2;
        double dZm = -Zm / (2.0 * m->eps[k]), dYm = Ym / (2.0 * m->eps[k]);
        double dZp = -Zp / (2.0 * m->eps[kp]), dYp = Yp / (2.0 * m->eps[kp]);
        grad[k] += scale * (sZm * dZm + sYm * dYm);
        grad[kp] += scale * (sZp * dZp + sYp * dYp);
      }
    }
  }
  free(out);
  free(la);
}

static void misfit_residual(const or_mesh *m, const double *u, const int64_t *recv, int64_t R, const double *Eref,
                            double *J, double *lam_add) {
  int64_t KNp = m->K * m->o.Np;
  for (int c = 0; c < 3; ++c)
    for (int64_t q = 0; q < R; ++q) {
      double d = u[c * KNp + recv[q]] - Eref[c * R + q];
      *J += d * d;
      if (lam_add) lam_add[c * KNp + recv[q]] += 2.0 * d;
    }
}

static void set_eps(or_mesh *m, const double *eps) {
  for (int64_t k = 0; k < m->K; ++k) m->eps[k] = eps[k];
}

int or_receiver_traces(const or_mesh *mc, const double *u0, const double *eps, double dt, int nsteps, double alpha,
                       const int64_t *recv, int64_t R, double *out) {
  or_mesh *m = (or_mesh *)mc;
  int64_t n = 6 * m->K * m->o.Np, KNp = m->K * m->o.Np;
  double *save = malloc(sizeof(double) * m->K);
  memcpy(save, m->eps, sizeof(double) * m->K);
  if (eps) set_eps(m, eps);
  double *u = malloc(sizeof(double) * n), *res = calloc(n, sizeof(double));
  memcpy(u, u0, sizeof(double) * n);
  for (int step = 0; step < nsteps; ++step) {
    or_lserk(m, u, res, dt, 1, alpha);
    for (int c = 0; c < 3; ++c)
      for (int64_t q = 0; q < R; ++q) out[((int64_t)step * 3 + c) * R + q] = u[c * KNp + recv[q]];
  }
  set_eps(m, save);
  free(save); free(u); free(res);
  return 0;
}

/* Reverse sweep of the LSERK4 recursion r_s = a_s r_{s-1} + dt A u_{s-1},
 * u_s = u_{s-1} + b_s r_s, with every step's start state stored (plain, no
 * checkpointing): for s = 5..1, lr += b_s lu; lu += dt A^T lr; grad_eps +=
 * dt <lr, dA/deps u_{s-1}>; lr *= a_s. */
int or_misfit_gradient(const or_mesh *mc, const double *u0, const double *eps, double dt, int nsteps, double alpha,
                       const int64_t *recv, int64_t R, const double *Eref, double *J, double *dJ_deps,
                       double *dJ_du0) {
  or_mesh *m = (or_mesh *)mc;
  int64_t n = 6 * m->K * m->o.Np;
  double a[5], b[5];
  or_lserk_coeffs(a, b, NULL);
  double *save = malloc(sizeof(double) * m->K);
  memcpy(save, m->eps, sizeof(double) * m->K);
  if (eps) set_eps(m, eps);
  double *states = malloc(sizeof(double) * n * (size_t)(nsteps + 1));
  double *res = calloc(n, sizeof(double));
  memcpy(states, u0, sizeof(double) * n);
  double Jv = 0.0;
  for (int step = 0; step < nsteps; ++step) {
    double *u = states + (size_t)(step + 1) * n;
    memcpy(u, states + (size_t)step * n, sizeof(double) * n);
    or_lserk(m, u, res, dt, 1, alpha);
    misfit_residual(m, u, recv, R, Eref + (int64_t)step * 3 * R, &Jv, NULL);
  }
  if (J) *J = Jv;
  double *lu = calloc(n, sizeof(double)), *lr = calloc(n, sizeof(double));
  double *stage = malloc(sizeof(double) * n * 5), *rr = malloc(sizeof(double) * n), *tmp = malloc(sizeof(double) * n);
  double *grad = calloc(m->K, sizeof(double));
  for (int step = nsteps - 1; step >= 0; --step) {
    double dummy = 0.0;
    misfit_residual(m, states + (size_t)(step + 1) * n, recv, R, Eref + (int64_t)step * 3 * R, &dummy, lu);
    /* stage inputs u_0..u_4 of this step */
    memcpy(stage, states + (size_t)step * n, sizeof(double) * n);
    memset(rr, 0, sizeof(double) * n);
    for (int s = 0; s < 4; ++s) {
      or_rhs(m, stage + (size_t)s * n, tmp, alpha);
      for (int64_t q = 0; q < n; ++q) {
        rr[q] = a[s] * rr[q] + dt * tmp[q];
        stage[(size_t)(s + 1) * n + q] = stage[(size_t)s * n + q] + b[s] * rr[q];
      }
    }
    for (int s = 4; s >= 0; --s) {
      for (int64_t q = 0; q < n; ++q) lr[q] += b[s] * lu[q];
      or_rhs_transpose(m, lr, tmp, alpha);
      for (int64_t q = 0; q < n; ++q) lu[q] += dt * tmp[q];
      eps_sensitivity(m, stage + (size_t)s * n, lr, alpha, dt, grad);
      for (int64_t q = 0; q < n; ++q) lr[q] *= a[s];
    }
  }
  if (dJ_deps) memcpy(dJ_deps, grad, sizeof(double) * m->K);
  if (dJ_du0) memcpy(dJ_du0, lu, sizeof(double) * n);
  set_eps(m, save);
  free(save); free(states); free(res); free(lu); free(lr); free(stage); free(rr); free(tmp); free(grad);
  return 0;
}
