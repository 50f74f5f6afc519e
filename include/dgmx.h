/*
 * dgmx — nodal discontinuous Galerkin solver for the 3D Maxwell equations on
 * straight-sided tetrahedra, for one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Kloeckner, Warburton & Hesthaven, "High-Order Discontinuous Galerkin
 * Methods by GPU Metaprogramming" (arXiv 1211.0582).
 *   - Section 2, eq. (semidiscrete-dg): du/dt = -sum_nu D^nu F(u) + L [n.F - (n.F)*],
 *     evaluated element by element (local differentiation + flux gather + flux lifting).
 *   - Section 2, eq. (dg-reference-matrices): affine elements, per-element J_k, dr/dx.
 *   - Section 2, Fig. (lifting-matrix): lifting matrix L = M^-1 [M^A1 ... M^A4].
 *   - Section 5, Fig. (flux-code) a: Maxwell flux n.(F - F*)_E = 1/2 n x ([H] - alpha n x [E]).
 *   - Section 5: RK4 time stepping (here the five-stage low-storage scheme of
 *     Carpenter & Kennedy, 2N storage).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Fields: six FP32 fields ordered Ex, Ey, Ez, Hx, Hy, Hz. A field vector is a
 * DEVICE buffer laid out [6][K][Np_pad] (element-major structure of arrays):
 * value of field c at node i of element k is at c*K*Np_pad + k*Np_pad + i.
 * Np = (N+1)(N+2)(N+3)/6 nodes per element, Np_pad = Np rounded up to a
 * multiple of 4 (16-byte rows). Padding entries are ignored on input and
 * written as zero on output. Field buffers must be 16-byte aligned.
 * Node order within an element is the warp & blend lattice order
 * (t outer, s middle, r inner) on the reference tetrahedron
 * (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1); dg_node_coords() returns it.
 *
 * Ownership: the caller owns every field, residual and gradient buffer; the
 * library owns operators, mesh/geometry data and internal scratch, allocated by
 * dg_mesh_upload() and freed by dg_destroy(). All device work is ordered on the
 * CUDA stream given to dg_create() (borrowed, not owned; NULL = legacy default
 * stream). Calls return after enqueueing, except where a host output is written.
 *
 * Errors: every function returns a dg_status; no exception crosses the ABI and
 * nothing aborts the process. dg_last_error() describes the last failure on a
 * context. A context is not thread-safe: use one per host thread.
 */
#ifndef DGMX_H
#define DGMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,         /* invalid argument (null pointer, size, alignment) */
  DG_ERR_MESH = -2,        /* invalid mesh (bad index, inverted element, non-conforming face) */
  DG_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  DG_ERR_NONFINITE = -4,   /* a NaN or Inf was detected in a result */
  DG_ERR_TIMEOUT = -5,     /* a device-side wait exceeded its iteration limit */
  DG_ERR_UNSUPPORTED = -6, /* valid request that this build does not implement */
  DG_ERR_OOM = -7          /* device allocation failed */
} dg_status;

typedef enum {
  DG_FP32 = 0,   /* FP32 arithmetic on the CUDA cores */
  DG_BF16X3 = 1, /* D and LIFT contractions on tensor cores, BF16 hi+lo split, FP32 accumulate */
  DG_FP16X3 = 2, /* same with FP16 hi+lo split, FP32 accumulate; power-of-two scaled per
                    (element, field) row of the field operand and per element and field
                    type (E, H) of the flux operand (FP16 range) */
  DG_FP32_TC = 3  /* FP32-level accuracy on the tensor cores: the split whose error matches
                     the FP32 path (FP16X3; the context then reports and behaves as FP16X3) */
} dg_precision;
/* The FP32 precision covers N = 1..9. The tensor-core precisions cover
 * N = 1..7 (DG_ERR_UNSUPPORTED at mesh upload for N = 8, 9): up to N = 5 the split operators
 * stay in shared memory, at N = 6, 7 they are streamed from L2 slice by slice.
 * They need an sm_103 device (GB300). */

/* Create a context for polynomial order N (1..9) and the given arithmetic.
 * cuda_stream is a cudaStream_t (may be NULL). *out receives the context.
 * Builds the reference operators on the host and makes no CUDA call; the
 * tensor-core precisions are checked against the device at dg_mesh_upload.
 * Errors: DG_ERR_ARG (N out of range, bad precision), DG_ERR_CUDA. */
int dg_create(dg_ctx **out, int N, int precision, void *cuda_stream);

/* Release the context and everything it owns. NULL is accepted. */
int dg_destroy(dg_ctx *ctx);

/* Interpolation nodes (Section 2: the warp & blend nodes of the paper's node
 * reference, which names no blend parameter). dg_create builds the operators
 * on the plain construction (alpha = 0); this rebuilds them, on the host, on
 * the nodes whose face warps along edge (P, Q) are scaled by
 * (1 + (alpha * l_R)^2), l_R the barycentric of the face's third vertex.
 * alpha in [0, 10]. Only before a mesh is uploaded: with a mesh on ctx it
 * fails and changes nothing. Needs no GPU.
 * Errors: DG_ERR_ARG (alpha out of range, a mesh present). */
int dg_set_node_alpha(dg_ctx *ctx, double alpha);

/* Blend parameter of least Lebesgue constant for order N in 1..9, from a
 * built-in table (a search over alpha in [0, 3] on equidistant lattices of the
 * tetrahedron; 0 where no alpha lowers the constant, N <= 4); -1 outside 1..9. */
double dg_optimised_node_alpha(int N);

/* Message of the last failure on ctx ("" if none); valid until the next call.
 * ctx may be NULL (then the last failure of dg_create is reported). */
const char *dg_last_error(const dg_ctx *ctx);

/* Set up operators (Section 2: warp & blend nodes, orthonormal-basis
 * Vandermonde, Dr/Ds/Dt, LIFT, face-node maps) and upload the mesh.
 * All inputs are HOST arrays: VX/VY/VZ (Nv vertex coordinates, FP64), EToV
 * (K x 4 vertex indices, 0-based, int32), eps/mu (K relative permittivity and
 * permeability per element, > 0; NULL means 1), bc (K x 4 face tags or NULL:
 * every boundary face is a perfect electric conductor, the only supported
 * boundary, tag 1; tags of interior faces are ignored). Geometric factors and
 * Jacobian inverses are computed on the device in FP64 and stored in FP32.
 * Replaces any previous mesh. Synchronises the stream before returning.
 * Errors: DG_ERR_ARG, DG_ERR_MESH (index out of range, J_k <= 0, a face shared
 * by more than two elements, neighbouring face nodes that do not coincide),
 * DG_ERR_UNSUPPORTED (a boundary tag other than 1), DG_ERR_OOM, DG_ERR_CUDA. */
int dg_mesh_upload(dg_ctx *ctx, int64_t Nv, const double *VX, const double *VY, const double *VZ,
                   int64_t K, const int32_t *EToV, const float *eps, const float *mu,
                   const int32_t *bc);

/* Sizes of the uploaded layout: Np, Np_pad and K (any pointer may be NULL). */
int dg_layout(const dg_ctx *ctx, int *Np, int *Np_pad, int64_t *K);

/* Reference operators built by dg_create (HOST FP64 copies, row-major; any
 * pointer may be NULL): nodes r, s, t (Np), Dr/Ds/Dt and the mass matrix M
 * (Np x Np), LIFT (Np x 4Nfp, face blocks in the order t=-1, s=-1,
 * r+s+t=-1, r=-1) and Fmask (4 x Nfp volume node of each face node). Needs no
 * GPU and no mesh. */
int dg_operators(const dg_ctx *ctx, double *r, double *s, double *t, double *Dr, double *Ds, double *Dt,
                 double *M, double *LIFT, int32_t *Fmask);

/* Physical node coordinates, HOST output xyz[3][K][Np] (FP64, unpadded). */
int dg_node_coords(dg_ctx *ctx, double *xyz);

/* Replace the per-element permittivity (DEVICE pointer to K FP32 values > 0)
 * without re-uploading the mesh; impedances are recomputed on the device. */
int dg_set_eps(dg_ctx *ctx, const float *eps_dev);

/* Semi-discrete right-hand side rhs = A(eps) u (eq. semidiscrete-dg with the
 * Maxwell flux; alpha = 1 upwind, 0 central): the volume term (local
 * differentiation with the chain rule, giving curl H and -curl E), the flux
 * gather (upwind flux with impedance-weighted material jumps, PEC mirror on
 * boundary faces) and the flux lifting, scaled by 1/eps and 1/mu.
 * u and rhs are DEVICE field vectors ([6][K][Np_pad] FP32) and must not alias.
 * Errors: DG_ERR_ARG (null/misaligned/aliasing), DG_ERR_CUDA. */
int dg_rhs(dg_ctx *ctx, const float *u, float *rhs, float alpha);

/* Advance nsteps LSERK4 steps of size dt: for each of the five stages s,
 * res <- a_s res + dt A u, u <- u + b_s res (one fused kernel per stage).
 * u and res are DEVICE field vectors, updated in place; the entry value of
 * res is not read (a_1 = 0: the first stage overwrites it), on exit res holds
 * the last stage's residual.
 * Uses a library-owned scratch field vector for the stage ping-pong.
 * With the non-finite check enabled (dg_set_nonfinite_check), u and res are
 * scanned for NaN/Inf after the last stage, the stream is synchronised and
 * DG_ERR_NONFINITE is returned if one is found (the fields are left as the
 * stages wrote them).
 * Errors: DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_NONFINITE (check enabled). */
int dg_step(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha);

/* Failure detection on the stepping path: enabled != 0 makes every following
 * dg_step / dg_step_noalloc call with nsteps > 0 check the state u and the
 * residual res for NaN or Inf after its last stage (one extra read of both
 * field vectors, then a stream synchronisation) and return DG_ERR_NONFINITE
 * if one is found; 0 (the default) turns the check off, leaving the calls
 * asynchronous. Needs no mesh. Errors: DG_ERR_ARG (ctx NULL). */
int dg_set_nonfinite_check(dg_ctx *ctx, int enabled);

/* Same as dg_step, but allocates no device memory in any form: the stage
 * ping-pong buffer is a fixed array inside the library's device image instead
 * of the scratch that dg_mesh_upload allocates. For callers that cannot let
 * the library allocate: applications whose device memory is owned up front by
 * their own allocator or arena, and time loops that must not risk a cudaMalloc
 * stall or failure. (The paper has no counterpart; this is a deployment
 * variant of the LSERK4 driver.)
 * Limit: 6 * K * Np_pad <= 4,194,304 floats (16 MiB, e.g. N=5 with K <= 12,483);
 * larger meshes get DG_ERR_ARG. Every GPU that loads the library holds the
 * 16 MiB array until the process exits. Every call looks up the array's
 * device address in the current context (the first lookup on a device may
 * load the library's device code there: make the first call before any
 * stream capture). All calls share the array and it keeps the last
 * call's contents (nothing in it needs to start at zero); calls whose work
 * overlaps on the GPU race on it. u, res, dt, nsteps, alpha, the non-finite
 * check (dg_set_nonfinite_check) and the errors are those of dg_step. */
int dg_step_noalloc(dg_ctx *ctx, float *u, float *res, double dt, int nsteps, float alpha);

/* Ensembles of independent meshes (uneven sizes, own materials, own time
 * steps) advanced together. Upload (HOST arrays): M meshes; Nv[i] and K[i]
 * their vertex and element counts; VX/VY/VZ the vertices of all meshes
 * concatenated; EToV all element tables concatenated with each mesh's own
 * 0-based vertex numbering; eps all elements' permittivities concatenated
 * (NULL = 1); dt[i] the time step of mesh i. The meshes are stored as one
 * disjoint union, so a field vector is [6][sum K][Np_pad] with mesh i owning
 * elements [offsets[i], offsets[i+1]) (dg_ensemble_layout). Replaces any mesh.
 * Errors as dg_mesh_upload. */
int dg_ensemble_upload(dg_ctx *ctx, int M, const int64_t *Nv, const double *VX, const double *VY, const double *VZ,
                       const int64_t *K, const int32_t *EToV, const float *eps, const double *dt);

/* Number of meshes and the M+1 element offsets (HOST outputs, may be NULL). */
int dg_ensemble_layout(const dg_ctx *ctx, int *M, int64_t *offsets);

/* Advance every mesh of the ensemble by nsteps LSERK4 steps of its own dt in
 * ONE persistent cooperative kernel launch (a grid-wide barrier with a bounded
 * wait separates the stages; a wait that runs out sets the flag reported by
 * dg_sync), replayed from a CUDA graph captured on the first call with these
 * arguments. FP32 contexts and N = 6, 7: the FP32 CUDA-core stage, elements
 * per block autotuned on the first call unless dg_ensemble_tune ran.
 * BF16X3/FP16X3 contexts at N <= 5: the tensor-core stage of dg_step (FP32
 * fields, split-precision contractions), one block per SM, tiles of 20
 * elements fixed by the 128-row matrix operation (nothing to tune; FP16X3
 * scales each tile's fluxes, so a tile spanning two meshes couples their
 * roundings, within the split's error). u and res are DEVICE field vectors
 * (in/out; the entry value of res is not read). */
int dg_ensemble_step(dg_ctx *ctx, float *u, float *res, int nsteps, float alpha);

/* Autotuner: time every candidate of the persistent launch on the uploaded
 * ensemble (2 steps, best of 3) and keep the fastest. The candidates form a
 * two-axis grid: 4 elements-per-block values x 2 occupancy levels (as many
 * blocks per SM as fit, or half as many: fewer blocks take part in each grid
 * barrier and each loops over more tiles); the second level is timed only
 * where it launches fewer blocks;
 * the choice is cached in a text file (environment DGMX_TUNE_CACHE, default
 * $HOME/.cache/dgmx_ensemble_tune.txt) keyed by GPU name, N and total element
 * count, and reused unless force is nonzero. Synchronises the stream. */
int dg_ensemble_tune(dg_ctx *ctx, int force);

/* Tuning log: the chosen elements per block, and for each of the 4
 * elements-per-block candidates its value and its measured ms per step at the
 * better of its occupancy levels (0 = not timed; the tensor-core form has one
 * candidate, 20). HOST outputs. */
int dg_ensemble_tuning(const dg_ctx *ctx, int *best_eb, int *eb, float *ms_per_step);

/* The whole tuning grid: *best = the chosen candidate (0..7, -1 before
 * tuning); for each of the 8 candidates (elements-per-block value c % 4,
 * occupancy level c / 4) its elements per block, the blocks per SM it was
 * launched with and its ms per step (0 = not timed). HOST outputs, may be
 * NULL. The tensor-core form has one candidate (20, one block per SM). */
int dg_ensemble_tuning_grid(const dg_ctx *ctx, int *best, int *eb, int *blocks_per_sm, float *ms_per_step);

/* 1 if the last dg_ensemble_step was replayed from a captured CUDA graph. */
int dg_ensemble_graph_used(const dg_ctx *ctx);

/* Wait for all work enqueued on the context's stream and report device-side
 * failures: returns DG_ERR_TIMEOUT (and clears the flag) if a kernel gave up
 * on a device-side wait (a tensor-core kernel on its MMA or copy barriers, the
 * ensemble launch on its grid barrier) after the wait limit, DG_ERR_CUDA if the
 * stream reports an error. After a timeout the work of that launch is
 * incomplete (its outputs are unspecified) but the context stays usable. */
int dg_sync(dg_ctx *ctx);

/* Device-side watchdog: every bounded wait of the stage kernels (tensor-core
 * barriers, the ensemble grid barrier, the tensor-core reverse stage of
 * dg_adjoint_step) gives up after `cycles` SM clock cycles; 0 restores the
 * default of 2^31 cycles (about one second). A limit shorter than the work
 * waited for makes the launch give up and dg_sync (dg_adjoint_step for its
 * reverse stage) return DG_ERR_TIMEOUT: the failure-detection path, exercised
 * without a GPU fault.
 * Waits that only drain copies or matrix operations already in flight before
 * a kernel exits keep the default limit. Drops a captured ensemble graph.
 * Returns DG_ERR_ARG for a negative limit. */
int dg_set_wait_limit(dg_ctx *ctx, long long cycles);

/* Transpose of the right-hand-side operator in the Euclidean inner product,
 * w = A(eps)^T v (DEVICE field vectors, no aliasing), in FP32 on the CUDA
 * cores: face data Fscale * LIFT^T (W v) per element, then the transposed
 * curl with D^T and the transposed flux Jacobians gathered from the element's
 * own and its neighbours' face data. Synchronises the stream. */
int dg_rhs_transpose(dg_ctx *ctx, const float *v, float *w, float alpha);

/* Forward LSERK4 run from u0 (DEVICE, not modified) for nsteps steps with
 * permittivity eps (DEVICE, K values; NULL keeps the current one, otherwise it
 * replaces it as dg_set_eps does), recording E at R receiver nodes after every
 * step: out (DEVICE FP32) is [nsteps][3][R]; recv (DEVICE int64, R entries) holds
 * node indices k*Np + i in [0, K*Np). The context's stage kernel (FP32 CUDA
 * cores; the tensor-core stage in split-precision contexts at N <= 5).
 * Synchronises. */
int dg_receiver_traces(dg_ctx *ctx, const float *u0, const float *eps, double dt, int nsteps, float alpha,
                       const int64_t *recv, int64_t R, float *out);

/* Receiver misfit J = sum_{n=1..nsteps} sum_r |E(recv_r, t_n) - Eref[n-1][.][r]|^2
 * of the run of dg_receiver_traces, and its exact discrete gradient by the
 * hand-written adjoint: the transposed LSERK4 recursion swept backwards stage
 * by stage (lambda_r += b_s lambda_u; lambda_u += dt A^T lambda_r;
 * dJ/deps += dt <lambda_r, dA/deps u_s>; lambda_r *= a_s). The run is cut
 * into segments of ckpt_every steps, aligned to its end (the first segment
 * takes the remainder); every stage state and the E components of every stage
 * right-hand side of one segment are held at a time. The forward sweep saves a
 * checkpoint at each segment start and stores the last segment directly, so
 * only the earlier segments are recomputed (nsteps - ckpt_every forward steps
 * in all). With more than one segment, the recomputation of a segment runs on
 * a second stream owned by the context while the reverse sweep of the next
 * one runs on the context's stream (two segment buffers; events order them),
 * and the forward sweep fills both buffers: the last two segments are stored
 * directly (nsteps - 2 ckpt_every steps recomputed).
 * ckpt_every = 0 picks the longest segment that fits in half of the device
 * memory that is free or already held by these buffers (then halved when
 * more than one segment is needed, for the two buffers; one segment, no
 * recomputation, when the whole run fits); dg_adjoint_segment_steps reports
 * the choice. Inputs (DEVICE): u0 [6][K][Np_pad], eps (K, or NULL = current),
 * recv (R), Eref [nsteps][3][R] FP32. Outputs: *J (HOST double), dJ_deps
 * (DEVICE, K doubles, reduced in FP64; may be NULL), dJ_du0 (DEVICE field
 * vector; may be NULL). With both gradient outputs NULL only the forward run
 * and the misfit are computed (no checkpoints, no reverse sweep; segment
 * length reported as 0). The forward sweeps run the context's stage: the
 * FP32 CUDA-core stage in FP32 contexts (and at N > 5), the tensor-core stage
 * in split-precision contexts (the gradient of that context's forward map).
 * Each reverse stage is one volume
 * kernel that also runs the next stage's lift (one separate lift per step,
 * after the receiver source); for N <= 5 on a GB300 its two contractions (the
 * transposed differentiation and lifting matrices) run on the tensor cores in
 * the FP16x3 split (FP32-level accuracy), unless dg_set_adjoint_form chose
 * the CUDA-core form.
 * Device memory: about (nsteps/ckpt_every + 7.5 ckpt_every + 8)
 * field vectors in one segment, (nsteps/ckpt_every + 15 ckpt_every + 10) with
 * several. Synchronises. Errors: DG_ERR_ARG (also ckpt_every < 0),
 * DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NONFINITE, DG_ERR_TIMEOUT (a bounded device
 * wait of the tensor-core reverse stage ran out; see dg_set_wait_limit). */
int dg_adjoint_step(dg_ctx *ctx, const float *u0, const float *eps, double dt, int nsteps, int ckpt_every,
                    float alpha, const int64_t *recv, int64_t R, const float *Eref, double *J, double *dJ_deps,
                    float *dJ_du0);

/* The form of dg_adjoint_step's reverse volume stage: 0 = FP32 CUDA cores,
 * 1 = tensor cores (FP16x3 split of the transposed differentiation and lifting
 * contractions; N <= 5 and a GB300, else DG_ERR_UNSUPPORTED). The default is
 * the tensor-core form where it is supported. No counterpart in the paper
 * (which has no adjoint); both forms compute the same discrete adjoint. */
int dg_set_adjoint_form(dg_ctx *ctx, int form);

/* The form the next dg_adjoint_step will use (0 or 1; -1 for a NULL ctx). */
int dg_adjoint_form(const dg_ctx *ctx);

/* Steps per segment used by the last dg_adjoint_step call on ctx (0 before
 * the first call, or for ctx == NULL). */
int dg_adjoint_segment_steps(const dg_ctx *ctx);

/* Discrete energy 1/2 sum_k J_k (eps_k E^T M E + mu_k H^T M H), reduced in
 * FP64 on the device; *E_out is a HOST double. Synchronises the stream.
 * Returns DG_ERR_NONFINITE if the energy is NaN or Inf. */
int dg_energy(dg_ctx *ctx, const float *u, double *E_out);

#ifdef __cplusplus
}
#endif
#endif /* DGMX_H */
