/*
 * riesz.h -- C ABI of the GB300 (sm_103a) solver for the high-order Riesz maps
 * of the de Rham complex, after Brubeck, Farrell, Kirby & Parker, "Fast solvers
 * for the high-order FEM simplicial de Rham complex" (arXiv 2506.17406).
 *
 * Problem (Eq. (2.8), pure Neumann, Section 7.1): find u in V with
 * beta (u, v) + alpha (d u, d v) = (f, v) for all v in V (alpha = beta = 1 by
 * default: the Riesz map), V one of
 *   RIESZ_H1     CG_p     (d = grad),  Eq. (2.5), k = 0
 *   RIESZ_HCURL  Ned1_p   (d = curl),  Eq. (2.5), k = 1
 *   RIESZ_HDIV   RT_p     (d = div),   Eq. (2.5), k = 2
 *   RIESZ_HCURL2 NedTwo_p = P_p^3 (d = curl), Eq. (2.6), k = 1
 *   RIESZ_HDIV2  BDM_p    = P_p^3 (d = div),  Eq. (2.6), k = 2
 * on an affine tetrahedral mesh, in the paper's orthogonality-promoting basis
 * (Sections 3-4: the dual basis of the DOFs of Eqs. (3.14), (3.16), (3.18)).
 *
 * Solver: PCG (Section 7.1) preconditioned by the interior/interface splitting
 * of Eq. (6.11), PAFW_0(X_Gamma) + J(X_I), applied additively:
 *   P^{-1} = diag(A_II)^{-1}  (+)  sum_V R_V^T A_V^{-1} R_V,
 * A_V the matrix restricted to the interface DOFs of the star of vertex V,
 * factorised by dense Cholesky (Section 6.4).
 *
 * Global DOF layout (the numbering the paper leaves to the implementation):
 *   [vertex DOFs | edge DOFs (edge-major) | face DOFs (face-major) |
 *    interior DOFs (cell-major)]
 * edges / faces are the sorted vertex pairs / triples of the mesh in
 * lexicographic order; inside an entity Whitney, type I, type II, each in
 * eigen order.  Every interface DOF comes before every interior DOF.
 *
 * Conventions for every call:
 *   - Return value: RIESZ_OK (0) or one of the RIESZ_ERR_* codes below;
 *     riesz_last_error() then returns a message (thread-local, valid until the
 *     next call on the same thread).  No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory pointers on the handle's device,
 *     owned by the caller, FP64, contiguous, right-hand sides stacked as
 *     [nrhs][N].  "host" pointers are ordinary CPU memory owned by the caller.
 *   - stream: a cudaStream_t cast to void*, or NULL for the legacy default
 *     stream.  Device work is enqueued on it; calls that return host values
 *     synchronise it.
 *   - The handle owns its mesh maps, reference tables, factors and workspace
 *     and frees them in riesz_destroy.  A handle is not thread-safe.
 */
#ifndef RIESZ_H
#define RIESZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct riesz_handle riesz_handle;
typedef struct riesz_hodge riesz_hodge;

enum { RIESZ_H1 = 0, RIESZ_HCURL = 1, RIESZ_HDIV = 2 };
/* X^3 = DG_{p-1}, the last space of the complex ending in RT_p: only for
   riesz_ref_tabulate (no Riesz-map handle: its Riesz map is the diagonal
   mass matrix). */
enum { RIESZ_L2 = 3 };
/* The second-kind spaces of Eq. (2.6) (Section 3.4: NedTwo_p's gradient
   moments use the CG_{p+1} eigenbasis; BDM_p's face and curl moments use the
   NedTwo_{p+1} eigenbasis).  Everything that depends only on k (pullbacks,
   geometric factors, patches, W^k) is shared with the first kind; W^k is the
   same Whitney space (Lemma 4.1), so the lowest-order coarse route uses
   Ned1_1 / RT_1.  The Hiptmair-Toselli potentials of NedTwo_p are CG_{p+1}. */
enum { RIESZ_HCURL2 = 4, RIESZ_HDIV2 = 5 };

enum {
  RIESZ_OK = 0,
  RIESZ_ERR_INVALID_ARG = 1,   /* bad pointer, size, space, degree or option */
  RIESZ_ERR_BAD_MESH = 2,      /* vertex index out of range, repeated vertex, |det J| ~ 0 */
  RIESZ_ERR_OOM = 3,           /* device allocation failed */
  RIESZ_ERR_NOT_CONVERGED = 4, /* maxit reached; x holds the last iterate */
  RIESZ_ERR_NONFINITE = 5,     /* NaN/Inf in the right-hand side or the recurrence */
  RIESZ_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  RIESZ_ERR_INTERNAL = 7,      /* e.g. a patch matrix that is not positive definite */
  RIESZ_ERR_NO_DEVICE = 8      /* a device call on a handle without device state */
};

enum { RIESZ_PREC_FP64 = 0, RIESZ_PREC_FP32 = 1, RIESZ_PREC_BF16X3 = 2 };
enum { RIESZ_APPLY_MATRIX_FREE = 0, RIESZ_APPLY_ELEMENT = 1 };
enum { RIESZ_LOOP_HOST = 0, RIESZ_LOOP_GRAPH = 1 };
enum { RIESZ_DECOMP_VERTEX_STAR = 0, RIESZ_DECOMP_HT = 1, RIESZ_DECOMP_EDGE_STAR = 2 };
enum { RIESZ_FORM_ADDITIVE = 0, RIESZ_FORM_HYBRID = 1 };

typedef struct {
  /* Precision of the stored patch Cholesky factors and of the triangular
     sweeps of riesz_precond (the factorisation itself is always FP64).
     With RIESZ_PREC_FP32 riesz_solve uses flexible (Polak-Ribiere) PCG. */
  int precond_precision;
  /* RIESZ_APPLY_MATRIX_FREE: y_T = sum_q g_q(T) R_q x_T with the Q reference
     matrices (7 for H1 and H(div), 12 for H(curl)) and per-cell geometric
     factors of the affine pullbacks (Eq. (2.7)).  RIESZ_APPLY_ELEMENT: the
     same sum formed once per cell at setup and stored (n_ref^2 FP64 per cell),
     so each apply reads it instead of recontracting. */
  int apply_mode;
  double rtol; /* target ||b - A x||_2 / ||b||_2 of riesz_solve (default 1e-8) */
  int maxit;   /* PCG iteration cap (default 1000) */
  int nrhs_max;/* largest nrhs passed to apply / precond / solve (default 1) */
  /* Coefficients of Eq. (2.8): a(u, v) = beta (u, v) + alpha (d u, d v), both
     positive constants (default 1, 1: the Riesz map). */
  double alpha, beta;
  /* Precision of the operator products inside riesz_solve's iterations
     (RIESZ_APPLY_ELEMENT only).  RIESZ_PREC_FP32 keeps an FP32 copy of the
     element matrices for the search-direction products and recovers FP64
     accuracy by replacing the recursive residual with the FP64 true residual
     b - A x whenever a right-hand side gains four digits
     and at convergence (the stopping test is always on the FP64 residual);
     the first residual needs no product when x = 0.  riesz_apply is always
     FP64.  RIESZ_PREC_BF16X3 (any apply_mode, every degree up to 10): the same
     products, and the residual updates of the hybrid sweep, matrix-free on
     the tensor cores (tcgen05): Y_T = sum_q g_q(T) R_q X_T as a GEMM over
     tiles of 128 (cell, right-hand side) rows with every operand split into
     two BF16 parts (hi + lo) and the three leading products accumulated in
     FP32 in tensor memory (relative error ~1e-5 per product); no FP32
     element matrices are stored.  With the hybrid form and FP32 patch
     sweeps, RIESZ_PREC_FP32 also moves the sweep's residual updates to the
     FP32 element matrices.  Default RIESZ_PREC_FP64. */
  int apply_precision;
  /* Who drives the PCG iterations of riesz_solve.  RIESZ_LOOP_GRAPH (default):
     the iterations run as a CUDA graph whose WHILE node repeats the body
     (preconditioner, search-direction update, operator product, x/r update)
     until a one-thread control kernel finds every right-hand side below rtol,
     a reliable update due, a non-finite value or maxit; the host only acts
     between graph launches (true-residual check, residual replacement,
     restart), so there is no host round trip per iteration.  RIESZ_LOOP_HOST:
     the host launches every kernel and reads the scalars each iteration
     (overlapped with the next preconditioner step).  Both run the same
     kernels in the same order and give bitwise equal results.  While the
     profiler records any kind launched inside the loop, riesz_solve uses the
     host-driven loop (CUDA events cannot time the passes of a graph loop). */
  int loop;
  /* 1 (default): riesz_setup_device times the patch Cholesky with one CTA per
     patch and with a 2-CTA cluster per patch, each with 2, 3, 4 and the
     maximum number of resident CTAs per SM, on the handle's own patches, and
     keeps the fastest (see riesz_tuning); done only when the mesh has more
     patches than SMs and at most 24 per SM, where these choices decide how
     evenly the work spreads over the SMs.  The choice is kept per device,
     space, degree and patch structure for the life of the process, so later
     handles of the same shape reuse it without timing.  The factors are
     bitwise the same for every choice.  0: one CTA per patch, maximum
     residency, no timing.
     2: 2-CTA clusters per patch, maximum residency, no timing. */
  int autotune;
  /* 1 (default): add the lowest-order space W^k to the preconditioner (the
     first summand of the PAFW decomposition, Section 6.2; by Lemma 4.1 its
     basis is the first DOF of every vertex (H1), edge (H(curl)) or face
     (H(div))): z += w R_0^T A_0^{-1} R_0 r with A_0 = R_0 A R_0^T, additive
     with weight w = 1/2 (every W^k function also lies in the vertex-star
     spaces, so the unweighted sum over-corrects).  A_0 is assembled densely at
     device setup, factored by a blocked FP64 Cholesky, its inverse
     L^{-T} L^{-1} formed in FP64 (positive definite by construction, exact to
     FP64 rounding) and applied as a dense FP64 product, so it is used only
     when W^k has at most 2048 DOFs (3072 for H1, whose lowest-order route
     below is point-Jacobi PCG; 6144 for the blocks of the Hodge-Laplace
     preconditioner, which MINRES needs linear).  Above that the coarse problem,
     which is the lowest-order Riesz map on the same mesh (Lemma 4.1), is
     held by an internal p = 1 handle and solved approximately by coarse_its
     PCG steps from zero preconditioned by that handle's own vertex-star
     patches (on the lowest-order H(curl)/H(div) problems these are robust
     in h: 3 steps reduce the residual 10x on 8^3 and 16^3 Kuhn meshes), all
     on the device with the main loop's PCG kernels.  Either way the coarse
     solve only perturbs the preconditioner: solves run flexible PCG and stop
     on the FP64 true residual.  riesz_tuning reports the coarse size and
     route.  0: one-level preconditioner.  2: the lowest-order PCG route
     whatever the size. */
  int coarse;
  /* 0 (default): pure Neumann (the paper's benchmarks).  1: homogeneous
     Dirichlet conditions on Gamma_D (X_{p,D} of Eq. (2.8); Gamma_D the whole
     boundary, or the part chosen by dirichlet_vertices): every DOF of a
     vertex, edge or face of Gamma_D is fixed (riesz_dirichlet_map lists
     them).  The system becomes
     [A_ff 0; 0 I]: riesz_apply gives y_f = A_ff x_f, y_d = x_d;
     riesz_precond gives z_d = r_d and leaves the fixed DOFs out of every
     patch and of W^k; riesz_load writes b_d = 0; a solve returns x_d = b_d. */
  int dirichlet;
  /* Space decomposition of the interface preconditioner.
     RIESZ_DECOMP_VERTEX_STAR (default): PAFW vertex stars (Eq. (6.11)).
     RIESZ_DECOMP_HT (H(curl) only, Neumann): the Hiptmair-Toselli splitting
     of Eq. (6.19) with the interface/interior split: exact solves on the
     type-I interface DOFs of every edge star (the edge's Whitney DOF and the
     type-I DOFs of the faces containing it) plus gradients of CG_p interface
     functions on every vertex star, whose potential problems
     (grad u, beta grad v) are factored in a CG_p handle owned by this one
     (Eq. (6.18)); the gradient map is the signed incidence / identity of
     Eq. (5.3).  Interior Jacobi and W^k as for the vertex stars.  The
     patches are much smaller (Ned1_6: 431-DOF potential and 121-DOF edge
     problems instead of 1164-DOF vertex stars), so the FP64 factorisation
     is far cheaper; PCG takes somewhat more iterations.
     RIESZ_DECOMP_EDGE_STAR (H(div) only): PAFW_1 of Eq. (6.24), exact solves
     on the interface DOFs of every edge star (the DOFs of the faces
     containing the edge; with Dirichlet conditions the free ones), interior
     Jacobi and W^k as above.  RT_8: 216-DOF edge problems instead of
     1296-DOF vertex stars. */
  int decomposition;
  /* How the subspace corrections combine.  RIESZ_FORM_ADDITIVE (default):
     the sum above.  RIESZ_FORM_HYBRID: the paper's symmetric multiplicative
     sweep over X_1 = interior DOFs (point-Jacobi), X_2 = interface DOFs (the
     patch solves of the decomposition) and X_3 = W^k (when coarse is on),
     in the order X_1, X_2, X_3, X_2, X_1 with the residual updated by an
     operator product between steps, each correction divided by its weight
     rho_m = (lambda_min + 3 lambda_max) / 4 of the extreme eigenvalues of the
     subspace operator against its solver, estimated at device setup by 10
     Lanczos (CG) steps (Section 7.1, Eqs. (7.2)-(7.3)); riesz_hybrid_weights
     reads or sets them. */
  int form;
  /* PCG steps of the lowest-order coarse route (see coarse; 1..1000,
     default 4). */
  int coarse_its;
  /* With dirichlet = 1: NULL (default) fixes the whole boundary; otherwise
     a host array of one flag per mesh vertex, and Gamma_D of Eq. (2.8) is
     the boundary faces whose three vertices are all flagged (a part of the
     boundary with its closure: those faces, their edges and vertices carry
     the fixed DOFs).  Read during riesz_create only. */
  const uint8_t* dirichlet_vertices;
  /* With inexact inner products (apply_precision FP32 or BF16X3): replace the
     recursive residual by the FP64 true residual whenever a right-hand side's
     residual norm has fallen by this many digits since the last replacement.
     0 (default): 4 with FP32 products, 2 with BF16x3 products; 1..12 sets
     it.  Each replacement costs one FP64 operator product; fewer of them let
     the recursive residual drift further from the true one. */
  int replace_digits;
} riesz_opts;

/* Fill *o with the defaults: FP64 preconditioner, element-matrix apply,
   rtol 1e-8, maxit 1000, nrhs_max 1, alpha = beta = 1, FP64 apply,
   graph-driven loop, autotune on, coarse space on, Neumann boundary,
   vertex-star decomposition. */
void riesz_default_opts(riesz_opts* o);

/* ---- host-only calls (no GPU needed) ---------------------------------- */

/* Build the reference element (Sections 3-4, host FP64, cached per (space,p))
   and the mesh maps (entities, DOF numbering, vertex-star patches) of a mesh.
   space: RIESZ_H1, RIESZ_HCURL, RIESZ_HDIV, RIESZ_HCURL2 or RIESZ_HDIV2.
   verts: host [nverts][3] FP64 coordinates; cells: host [ncells][4] vertex
   indices (any order; each cell's vertices are sorted internally).
   p: 1..10.  opts may be NULL (defaults).  *out receives a new handle. */
int riesz_create(int space, int p, int64_t nverts, const double* verts, int64_t ncells,
                 const int64_t* cells, const riesz_opts* opts, riesz_handle** out);

/* N = total DOFs, n_interior = DOFs of cell interiors (the last n_interior). */
int riesz_num_dofs(const riesz_handle* h, int64_t* n, int64_t* n_interior);

/* info[0..7] = n_ref, interior DOFs per cell, value components, derivative
   components, DOFs per vertex, per edge, per face, per cell interior. */
int riesz_ref_info(const riesz_handle* h, int* info);

/* cell_dofs: host [ncells][n_ref] global DOF of each local reference DOF. */
int riesz_dof_map(const riesz_handle* h, int32_t* cell_dofs);

/* mask: host [N]; 1 for the DOFs fixed by the Dirichlet condition
   (opts.dirichlet), 0 otherwise. */
int riesz_dirichlet_map(const riesz_handle* h, uint8_t* mask);

/* *npatches = the number of stars the patches are taken over: the mesh
   vertices for RIESZ_DECOMP_VERTEX_STAR, the mesh edges (in the order of
   increasing vertex pairs) for RIESZ_DECOMP_HT and RIESZ_DECOMP_EDGE_STAR. */
int riesz_patch_count(const riesz_handle* h, int64_t* npatches);

/* offsets: host [npatches + 1]; dofs: host [offsets[npatches]] (query the
   size by passing dofs == NULL).  Patch of star s (vertex or edge, see
   riesz_patch_count) = dofs[offsets[s] .. offsets[s+1]), increasing global
   DOF indices (without the Dirichlet DOFs when opts.dirichlet is set).  For
   RIESZ_DECOMP_HT these are the edge-star patches of this handle; the
   potential problems live on the CG_p vertex stars. */
int riesz_patch_map(const riesz_handle* h, int64_t* offsets, int32_t* dofs);

/* The gradient map of a RIESZ_DECOMP_HT handle (Eq. (5.3)) as a signed CSR
   list over the Ned1_p (NedTwo_p) interface DOFs: row d lists the CG_p
   (CG_{p+1}) interface DOFs c with the coefficient (+1 or -1) of grad phi^CG_c
   in DOF d.
   ptr: host [n_interface + 1]; idx, sgn: host [ptr[n_interface]] (query the
   size with idx == NULL).  RIESZ_ERR_INVALID_ARG for other handles. */
int riesz_ht_gradient_map(const riesz_handle* h, int64_t* ptr, int32_t* idx, float* sgn);

/* Tabulate the reference basis of (space, p) at npts points of the reference
   tetrahedron (edge length 2, centroid 0, vertices (-1,-1/sqrt3,-1/sqrt6),
   (1,-1/sqrt3,-1/sqrt6), (0,2/sqrt3,-1/sqrt6), (0,0,3/sqrt6)).
   vals: host [npts][n_ref][ncomp]; dvals: host [npts][n_ref][dcomp] (grad,
   curl or div); either may be NULL.  space: any of the five Riesz-map spaces
   (RIESZ_HCURL2 / RIESZ_HDIV2 give NedTwo_p / BDM_p), or RIESZ_L2: DG_{p-1}, n_ref =
   p(p+1)(p+2)/6, ncomp = dcomp = 1, the basis dual to the mean and the
   moments against the divergences of the RT_p interior eigenbasis (values
   1/|T| and div Phi_{C,j}); dvals are zero (d^3 = 0). */
int riesz_ref_tabulate(int space, int p, int64_t npts, const double* pts, double* vals, double* dvals);

/* Reference coupling tables of the Hodge-Laplace problem (k = 1: CG_p -> Ned1_p,
   k = 2: Ned1_p -> RT_p, k = 3: RT_p -> DG_{p-1}): for k = 3, out host
   [1][n_RT][n_DG], entry [j][i] = (div phi^RT_j, psi^DG_i) on the reference
   cell, scaled on a cell by 1 / |det J|; for k = 1, 2, out host
   [6][n_{k-1}][n_k], entry [q][j][i] =
   integral over the reference tetrahedron of (d phi^{k-1}_j)_b (phi^k_i)_a
   (+ the same with a and b exchanged when a != b) for the metric entry
   q = (a, b) in the order 00, 11, 22, 01, 02, 12.  On a cell,
   (d phi^{k-1}_j, phi^k_i) = sum_q G_q R_q[j][i] with G the symmetric metric
   |det J| J^{-1} J^{-T} (k = 1) or J^T J / |det J| (k = 2). */
int riesz_ref_mixed_tables(int k, int p, double* out);

/* ---- device calls ---------------------------------------------------- */

/* Upload the maps and tables to the current CUDA device and run the device
   setup: per-cell geometric factors, interior diagonal, patch assembly and
   batched FP64 Cholesky (Section 6.4).  Synchronises the stream. */
int riesz_setup_device(riesz_handle* h, void* stream);

/* riesz_create followed by riesz_setup_device. */
int riesz_setup(int space, int p, int64_t nverts, const double* verts, int64_t ncells,
                const int64_t* cells, const riesz_opts* opts, void* stream, riesz_handle** out);

/* y = A x (matrix-free operator of Eq. (2.8)); x, y: device [nrhs][N]. */
int riesz_apply(riesz_handle* h, const double* x, double* y, int nrhs, void* stream);

/* y = A x for one right-hand side, like riesz_apply, but without any memory
   the call or the handle allocated for it: the per-cell interface results
   that riesz_apply keeps in a handle-owned buffer go to a fixed device array
   compiled into this library (2^21 doubles = 16 MiB, reserved on every GPU
   that loads the library until the process exits).  It exists for callers
   that must not call cudaMalloc on their hot path: code whose device memory
   is owned by another allocator or a fixed budget (for example a framework
   caching allocator that already holds the free memory), and latency-bound
   loops where an allocation's implicit synchronisation is not acceptable.
   The paper has no counterpart; it is an interface convenience.
   x, y: device [N] on the handle's device, which must be current.
   Limits: n_interface_per_cell * ncells <= 2^21 (RIESZ_ERR_INVALID_ARG
   otherwise, nothing launched).  The first call on a device looks up the
   array's device address (cudaGetSymbolAddress), so make that first call
   before any stream capture.  The address is kept per device ordinal for the
   life of the process: after cudaDeviceReset (or any teardown of the
   device's primary context) the library's module is loaded afresh and the
   kept address no longer names the array, so do not call this entry point
   on a device after resetting it.  All calls share the one array, which keeps the
   last call's contents; calls that overlap on the GPU (other streams, other
   handles on the same device) race on it and must be serialised by the
   caller.  Every scratch entry a call reads is written earlier in the same
   call, so stale contents never reach y. */
int riesz_apply_noalloc(riesz_handle* h, const double* x, double* y, void* stream);

/* z = P^{-1} r (Eq. (6.11), additive); r, z: device [nrhs][N]. */
int riesz_precond(riesz_handle* h, const double* r, double* z, int nrhs, void* stream);

/* PCG for A x = b to ||b - A x|| <= rtol ||b|| (true residual, checked at
   exit).  x: device [nrhs][N], the initial guess on entry, the solution on
   return.  The right-hand sides advance in lockstep (one operator and one
   preconditioner launch per iteration for all of them) until every one has
   converged; iters[k] is that common count.  nrhs <= opts.nrhs_max.
   iters, relres: host [nrhs] (may be NULL).  Synchronises. */
int riesz_solve(riesz_handle* h, const double* b, double* x, int nrhs, void* stream, int* iters,
                double* relres);

/* Solve count independent systems together: the PCG loops of all handles are
   branches of one CUDA graph (each a device-driven loop as with
   RIESZ_LOOP_GRAPH), launched once, so the kernels of different systems run
   concurrently on the GPU and no host round trip separates iterations.
   Handles whose loops stop for a host step (true-residual check, residual
   replacement, restart) continue in further launches.  The systems may differ
   in space, degree, mesh and options.
   hs: host [count] distinct handles with device state on the current device;
   b[i], x[i]: device [nrhs[i]][N_i] (x[i] the initial guess on entry);
   nrhs: host [count] (NULL = 1 each, each <= its handle's nrhs_max);
   iters, relres: host [sum of nrhs] in handle order (may be NULL);
   status: host [count] per-system status (may be NULL).
   Returns RIESZ_OK when every system converged, else the first non-OK status
   in handle order.  Uses the graph-driven loop whatever opts.loop says; with
   the profiler recording a loop kind on any handle it returns
   RIESZ_ERR_INVALID_ARG.  Synchronises the stream. */
int riesz_solve_batch(riesz_handle* const* hs, int count, const double* const* b, double* const* x,
                      const int* nrhs, void* stream, int* iters, double* relres, int* status);

/* riesz_solve with host buffers: b_host, x_host are host [nrhs][N]; the
   copies to and from the device are part of the call. */
int riesz_solve_host(riesz_handle* h, const double* b_host, double* x_host, int nrhs, void* stream,
                     int* iters, double* relres);

/* Number of DOFs of CG_p on the handle's mesh (the space of riesz_load's f). */
int riesz_num_cg_dofs(const riesz_handle* h, int64_t* n_cg);

/* b_i = (f, phi_i) for f whose Cartesian components lie in CG_p of the same
   mesh with global coefficients fcg: device [ncomp][n_cg] (ncomp = 1 for H1,
   3 otherwise).  b: device [N]. */
int riesz_load(riesz_handle* h, const double* fcg, double* b, void* stream);

/* Recompute the device setup (geometric factors, element matrices, interior
   diagonal, patch assembly and Cholesky) for new vertex coordinates of the
   same mesh topology.  verts: device [nverts][3] FP64 (copied).  Use after a
   mesh moves, or to time the device setup from resident data. */
int riesz_update_geometry(riesz_handle* h, const double* verts, void* stream);

/* riesz_update_geometry for count independent systems at once (batched
   device setup): each system's geometry, element matrices and patch assembly
   run on a stream of its own, forked from stream; then the patch
   factorisations of all systems run as one persistent launch over a single
   work list, largest patches first (uneven patch sizes across systems balance
   over the SMs); then each system's FP32 factor copies, joined back into
   stream.  The host checks (factorisation status, hybrid weights) follow once
   all have finished.  Each system gets bitwise the same factors as from
   riesz_update_geometry.  Allocates the work list (a few bytes per patch)
   for the duration of the call.  hs, verts: host
   arrays of count handles (distinct, on the current device) and device
   vertex arrays [nverts_i][3] FP64. */
int riesz_update_geometry_batch(riesz_handle* const* hs, int count, const double* const* verts, void* stream);

/* Kernel kinds reported by the profiler. */
enum {
  RIESZ_K_GEOM = 0,         /* a1 geometric factors                      */
  RIESZ_K_ELEM = 1,         /* element matrices A_T = sum_q g_q R_q      */
  RIESZ_K_DIAG = 2,         /* a6 interior diagonal                      */
  RIESZ_K_ASSEMBLE = 3,     /* a8 patch assembly                         */
  RIESZ_K_CHOLESKY = 4,     /* a8 batched FP64 Cholesky                  */
  RIESZ_K_TO_F32 = 5,       /* FP64 -> FP32 factor copy                  */
  RIESZ_K_APPLY = 6,        /* a3-a4 gather + contraction                */
  RIESZ_K_GATHER = 7,       /* a5 deterministic interface scatter        */
  RIESZ_K_PATCH_SOLVE = 8,  /* a7 patch triangular sweeps                */
  RIESZ_K_PRECOND_GATHER = 9, /* a6 Jacobi + a7 patch-result sum         */
  RIESZ_K_DOT = 10,         /* a9 dot-product partial sums               */
  RIESZ_K_SCALAR = 11,      /* a9 reduction finish + scalar update       */
  RIESZ_K_UPDATE = 12,      /* a9 vector updates                         */
  RIESZ_K_LOAD = 13,        /* right-hand side assembly                  */
  RIESZ_K_APPLY32 = 14,     /* a3-a4 with the FP32 element matrices      */
  RIESZ_K_COARSE = 15,      /* W^k: A_0 assembly and block inversion     */
  RIESZ_K_COARSE_APPLY = 16,/* W^k: coarse correction A_0^{-1} R_0 r     */
  RIESZ_K_HT = 17,          /* HT: gradient map and potential gather     */
  RIESZ_K_APPLY_TC = 18,    /* a3-a4 BF16x3 contraction on tensor cores  */
  RIESZ_NKIND = 19
};

/* Per-kernel timing with CUDA events recorded on the launching stream around
   the kernels of the handle.  enable is a bit mask of kinds (bit k records
   kind k; -1 records all, 0 turns the profiler off); every call clears the
   accumulators.  riesz_profile_read synchronises the recorded events and
   returns the summed milliseconds and launch counts per kind (arrays of
   RIESZ_NKIND entries, either may be NULL). */
int riesz_profile(riesz_handle* h, int enable);
int riesz_profile_read(riesz_handle* h, double* ms, int64_t* counts);

/* Choices made at setup: out[0] = resident k_cholesky CTAs per SM picked by
   the autotuner (0: no limit), out[1] = candidates timed for this shape (by
   this handle or an earlier one; 0 when tuning does not apply), out[2] = DOFs of the W^k coarse space (0 when it is off),
   out[3] = CTAs per patch in the factorisation (1, or 2 for a 2-CTA cluster
   that shares each patch), out[4] = the W^k solve: 0 none, 1 dense inverse,
   2 lowest-order PCG steps.  out: host [5]. */
int riesz_tuning(const riesz_handle* h, int* out);

/* The shape of the FP32 patch sweeps for several right-hand sides over
   patches of 33..256 DOFs (the edge stars of Eqs. (6.19) and (6.24)), picked
   at riesz_setup_device by timing each candidate on the handle's own factors
   (autotune = 1; kept per device and patch structure for the life of the
   process): *shape = 0 one CTA per patch streaming the factor tiles through a
   bulk-copy ring, 4 or 8 one warp per patch with that many warps per block,
   -1 when the choice does not apply (FP64 factors, one right-hand side,
   larger or smaller patches).  *timed (may be NULL) = candidates timed. */
int riesz_sweep_shape(const riesz_handle* h, int* shape, int* timed);

/* Timings (ms) and sizes of the last setup / solve:
   out[0] setup host ms, out[1] setup device ms, out[2] device bytes held,
   out[3] patch factor bytes, out[4] last solve iterations (rhs 0),
   out[5] kernels launched by the handle since riesz_create,
   out[6] flops of one tile-sparse patch Cholesky pass (all patches),
   out[7] bytes one riesz_precond call reads and writes for the patch sweeps
          (stored factor tiles and diagonal inverses twice, patch vectors). */
int riesz_stats(const riesz_handle* h, double* out);

/* Device bytes riesz_setup_device will allocate for this handle (host-only,
   no GPU needed): *bytes = the sum of the handle's device buffers (those of
   its internal potential-problem handle included), equal to riesz_stats'
   out[2] once the setup has run; *nalloc (may be NULL) = the number of
   device allocations, so that a caller can add the allocator's rounding
   (at most one 2 MiB page per allocation).  Lets a scheduler budget HBM
   before a request touches the device. */
int riesz_plan_bytes(const riesz_handle* h, double* bytes, int64_t* nalloc);

/* y = A x with the products of the given precision, as riesz_solve runs them
   inside its iterations: RIESZ_PREC_FP64 (= riesz_apply), RIESZ_PREC_FP32
   (the FP32 element matrices; handles that keep them) or RIESZ_PREC_BF16X3
   (the tensor-core contraction; handles with apply_precision BF16X3).
   x, y: device [nrhs][N], distinct.  RIESZ_ERR_INVALID_ARG when the handle
   does not hold that precision. */
int riesz_apply_prec(riesz_handle* h, const double* x, double* y, int nrhs, int prec, void* stream);

/* Weights rho_1, rho_2, rho_3 of the hybrid form (opts.form =
   RIESZ_FORM_HYBRID; Section 7.1, Eq. (7.3)) for X_1 = interior DOFs,
   X_2 = interface DOFs, X_3 = W^k.  set = 0: rho (host [3]) receives the
   weights estimated at the last device setup (10 Lanczos steps from a fixed
   start vector; rho_3 = 1 for the W^k solve, which is exact or the
   lowest-order PCG steps);
   set = 1: the handle uses rho from now on and keeps them through later
   setups (riesz_update_geometry).  RIESZ_ERR_INVALID_ARG for other handles
   or non-positive weights. */
int riesz_hybrid_weights(riesz_handle* h, double* rho, int set);

/* Measurement helper (no counterpart in the paper): the FP64 fused
   multiply-add rate of the current device, in TFLOP/s, from one timed launch
   (CUDA events on stream) of a kernel with eight independent dependent-FMA
   chains per thread, iters steps each, four CTAs of 256 threads per SM, after
   one shorter warm-up launch.  iters in 1..2^24 (about 2^14 gives tens of
   milliseconds on one GPU).  Synchronises the stream.  Used as the measured
   FP64 peak for the roofline of the FP64 kernels; changes no GPU setting. */
int riesz_probe_fp64(int iters, void* stream, double* tflops);

int riesz_destroy(riesz_handle* h);

const char* riesz_last_error(void);

/* ---- Hodge-Laplace problems (Section 7.2) ----------------------------- */

/* The mixed Hodge-Laplace problem of Eq. (7.5) for k = 1 (sigma in CG_p,
   u in Ned1_p), k = 2 (sigma in Ned1_p, u in RT_p) or k = 3 (sigma in RT_p,
   u in DG_{p-1}: mixed Poisson, d^3 = 0; DG DOFs cell-major, dg_dim(p) =
   p(p+1)(p+2)/6 per cell) on one mesh, pure Neumann (the paper's Fichera
   corner has Gamma_N = the whole boundary):
     -(sigma, tau) + (u, d tau) = 0,   (d sigma, v) + (d u, d v) = (f, v).
   Block vectors are device [sigma (n0) | u (n1)] FP64 (riesz_hodge_sizes),
   each block in the numbering of riesz_dof_map of its space.
   Preconditioner: block diagonal, the weighted Riesz maps of Eq. (7.6),
   (sigma, tau) + gamma (d sigma, d tau) on X^{k-1} and
   gamma^{-1} (u, v) + (d u, d v) on X^k, each replaced by one application
   of its Schwarz preconditioner (interior Jacobi, patches, W^k as
   configured by opts).  opts->decomposition = RIESZ_DECOMP_VERTEX_STAR:
   vertex stars in both blocks; any other value: the paper's choice of
   Section 7.2 (vertex stars for CG_p, Hiptmair-Toselli for Ned1_p, edge
   stars for RT_p).  opts->precond_precision, coarse, autotune, rtol and
   maxit apply; alpha, beta, nrhs_max, loop, apply_mode and apply_precision
   are set internally; dirichlet must be 0.  opts->form = RIESZ_FORM_HYBRID
   makes every Riesz block the paper's multiplicative hybrid (Section 7.1)
   instead of the additive sum (a fixed symmetric positive definite
   operator with FP64 sweeps, as MINRES needs).  gamma > 0.  For k = 3 the DG
   block gamma^{-1} M_DG is diagonal (the DG basis is L2-orthogonal) and is
   inverted exactly.
   Setup builds both blocks' maps on the host and runs the device setup on
   the current device (stream may be NULL); the handle owns all its memory. */
int riesz_hodge_setup(int k, int p, int64_t nverts, const double* verts, int64_t ncells, const int64_t* cells,
                      double gamma, const riesz_opts* opts, void* stream, riesz_hodge** out);
/* *n0 = dim X^{k-1}, *n1 = dim X^k, *ncg (may be NULL) = dim CG_p (the
   source coefficients of riesz_hodge_load). */
int riesz_hodge_sizes(const riesz_hodge* h, int64_t* n0, int64_t* n1, int64_t* ncg);
/* y = A x with A = [-M_{k-1} B^T; B K_k], B_ij = (d phi^{k-1}_j, phi^k_i).
   x, y: device [n0 + n1], distinct. */
int riesz_hodge_apply(riesz_hodge* h, const double* x, double* y, void* stream);
/* z = P^{-1} r, the block-diagonal preconditioner above.  r, z: device [n0 + n1]. */
int riesz_hodge_precond(riesz_hodge* h, const double* r, double* z, void* stream);
/* b = [0 | (f, v)_{v in X^k}] for f with CG_p coefficients per Cartesian
   component (device [3][n_cg], as riesz_load on X^k; for k = 3 a scalar f,
   device [n_cg]).  b: device [n0 + n1]. */
int riesz_hodge_load(riesz_hodge* h, const double* fcg, double* b, void* stream);
/* New vertex coordinates (device [nverts][3], same connectivity): recompute
   every block's element matrices, patch factors and the coupling. */
int riesz_hodge_update_geometry(riesz_hodge* h, const double* verts, void* stream);
/* Preconditioned MINRES (Paige-Saunders) from the initial guess in x
   (device [n0 + n1], overwritten by the iterate).  Stops when the
   P^{-1}-norm of the residual has dropped by rtol; *iters and *relres (host,
   may be NULL) receive the iteration count and the true relative residual
   ||b - A x||_2 / ||b||_2.  RIESZ_ERR_NOT_CONVERGED at maxit (x holds the
   last iterate).  The host synchronises with the stream once per iteration. */
int riesz_hodge_solve(riesz_hodge* h, const double* b, double* x, void* stream, int* iters, double* relres);
/* out (host [6]): kernel launches so far (all blocks), last iteration count,
   last true relative residual, last P^{-1}-norm residual ratio, n0, n1. */
int riesz_hodge_stats(const riesz_hodge* h, double* out);
int riesz_hodge_destroy(riesz_hodge* h);

#ifdef __cplusplus
}
#endif

#endif /* RIESZ_H */
