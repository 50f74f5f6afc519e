/*
 * FP64 single-threaded CPU oracle of the nodal DG Maxwell operator.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use this library; the product path never
 * links, loads or calls it, and it shares no code with the CUDA library.
 *
 * Every array is row-major FP64 unless noted. Field vectors are laid out
 * [6][K][Np] with fields ordered Ex, Ey, Ez, Hx, Hy, Hz. Functions return 0 on
 * success and a negative value on error (see or_error()).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_mesh or_mesh;

const char *or_error(void);

/* Np = (N+1)(N+2)(N+3)/6, Nfp = (N+1)(N+2)/2. */
int or_np(int N);
int or_nfp(int N);

/* 1D Legendre-Gauss-Lobatto nodes x[0..N] (ascending). */
int or_lgl(int N, double *x);

/* Warp-and-blend nodes (blend parameter 0) on the reference tetrahedron
 * (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1); equidistant lattice order
 * (t outer, s middle, r inner). */
int or_nodes(int N, double *r, double *s, double *t);
/* The same with blend parameter alpha in [0, 10]: every edge warp of a face is
 * scaled by (1 + (alpha * barycentric of the face vertex opposite the edge)^2). */
int or_nodes_alpha(int N, double alpha, double *r, double *s, double *t);
/* Lebesgue constant of those nodes, estimated on the order-M equidistant lattice. */
int or_lebesgue(int N, double alpha, int M, double *lambda);

/* Reference operators (Section 2, eq. dg-global-matrices, Fig. lifting-matrix):
 * V (Np x Np), Dr/Ds/Dt (Np x Np), M (Np x Np), Fmask (4 x Nfp, int32),
 * Mf (4 x Nfp x Nfp face mass matrices), LIFT (Np x 4Nfp). Any pointer may be NULL. */
int or_operators(int N, double *V, double *Dr, double *Ds, double *Dt, double *M,
                 int32_t *Fmask, double *Mf, double *LIFT);
/* The same on the nodes of blend parameter alpha. */
int or_operators_alpha(int N, double alpha, double *V, double *Dr, double *Ds, double *Dt, double *M,
                       int32_t *Fmask, double *Mf, double *LIFT);

/* Orthonormal PKD basis function m (i outer, j, k inner ordering) and its
 * gradient at (r,s,t). */
int or_basis(int N, int m, double r, double s, double t, double *val, double *dr,
             double *ds, double *dt);

/* Mesh: vertices VX/VY/VZ (Nv), EToV (K x 4, int32, 0-based), eps/mu per element
 * (NULL = 1). All boundary faces are perfect electric conductors. */
or_mesh *or_mesh_create(int N, int64_t Nv, const double *VX, const double *VY,
                        const double *VZ, int64_t K, const int32_t *EToV,
                        const double *eps, const double *mu);
/* The same on the nodes of blend parameter alpha. */
or_mesh *or_mesh_create_alpha(int N, double alpha, int64_t Nv, const double *VX, const double *VY,
                              const double *VZ, int64_t K, const int32_t *EToV,
                              const double *eps, const double *mu);
void or_mesh_destroy(or_mesh *m);
int64_t or_mesh_K(const or_mesh *m);

/* Node coordinates, each K x Np. */
int or_mesh_coords(const or_mesh *m, double *x, double *y, double *z);
/* Geometric factors: G (K x 10: rx ry rz sx sy sz tx ty tz J),
 * F (K x 4 x 5: nx ny nz sJ Fscale), EToE / EToF (K x 4, int64, -1 = boundary). */
int or_mesh_geometry(const or_mesh *m, double *G, double *F, int64_t *EToE, int64_t *EToF);
/* Exterior node of every face node: K x 4 x Nfp global node index k*Np+i, -1 on boundary. */
int or_mesh_exterior(const or_mesh *m, int64_t *ext);

/* The flux difference n.(F - F*) at one face node for interior/exterior states
 * qm/qp (Ex Ey Ez Hx Hy Hz), impedances Zm/Zp (Y = 1/Z); fE/fH get 3 values each. */
int or_flux(const double *n, const double *qm, const double *qp, double Zm, double Zp, double alpha, double *fE,
            double *fH);

/* Semi-discrete right-hand side (eq. semidiscrete-dg with the Maxwell flux of
 * Fig. flux-code a): rhs = A(eps) u. alpha = 1 upwind, 0 central. */
int or_rhs(const or_mesh *m, const double *u, double *rhs, double alpha);
/* Same, only for the listed elements: rhs_sub is [6][n][Np]. */
int or_rhs_subset(const or_mesh *m, const double *u, double *rhs_sub, double alpha,
                  const int64_t *elems, int64_t n);

/* Carpenter-Kennedy five-stage fourth-order low-storage RK coefficients. */
int or_lserk_coeffs(double *a, double *b, double *c);
/* nsteps LSERK4 steps of size dt applied in place to u; res is the [6][K][Np]
 * low-storage residual, also in place (zero it before the first step). */
int or_lserk(const or_mesh *m, double *u, double *res, double dt, int nsteps, double alpha);

/* Discrete energy 1/2 sum_k J_k (eps_k E^T M E + mu_k H^T M H). */
double or_energy(const or_mesh *m, const double *u);
/* Closed-form upwind dissipation: sum over faces of the face-mass-weighted
 * alpha/(Z-+Z+) |dE_t|^2 + alpha/(Y-+Y+) |dH_t|^2 (each interior face once). */
double or_face_dissipation(const or_mesh *m, const double *u, double alpha);

/* Transpose of the right-hand side operator in the Euclidean inner product:
 * w = A^T v (the hand-built discrete adjoint of or_rhs). */
int or_rhs_transpose(const or_mesh *m, const double *v, double *w, double alpha);

/* Receiver misfit J = sum over steps n=1..nsteps and receivers of |E(t_n) - Eref_n|^2
 * for the run started from u0 with permittivity eps (K), and its exact gradient with
 * respect to eps (dJ_deps, K) and to the initial field (dJ_du0, [6][K][Np]). recv
 * holds R node indices into [K*Np]; Eref is [nsteps][3][R]. Any output may be NULL. */
int or_misfit_gradient(const or_mesh *m, const double *u0, const double *eps, double dt,
                       int nsteps, double alpha, const int64_t *recv, int64_t R,
                       const double *Eref, double *J, double *dJ_deps, double *dJ_du0);
/* Receiver traces of a forward run: out is [nsteps][3][R]. */
int or_receiver_traces(const or_mesh *m, const double *u0, const double *eps, double dt,
                       int nsteps, double alpha, const int64_t *recv, int64_t R, double *out);

#ifdef __cplusplus
}
#endif
#endif
