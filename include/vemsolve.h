/*
 * vemsolve.h -- C-ABI of the GB300 (sm_103a) mixed virtual element solver.
 *
 * The library discretises  -div(K grad p) = f  in mixed form (flux u and
 * pressure p) on polyhedral meshes of a domain with the mixed virtual
 * element method of Dassi & Scacchi (arXiv:1901.02330) and solves the
 * resulting saddle-point system with a block-preconditioned Krylov method:
 *
 *   model problem  ...................... Sec. 3, eq. mod_prob_eq, bilin_form
 *   local velocity space and DOFs ....... Sec. 4.1, eq. vectSpaceDef,
 *                                         facePoly, gradMom, crossMom
 *   pressure space and DOFs ............. Sec. 4.2, eq. presSpace, presMom
 *   local forms, stabilisation .......... Sec. 4.3 (a_{h,P}, b_{h,P}, f_{h,P}, s_P)
 *   discrete problem .................... Sec. 4.3, eq. mod_prob_eqDisc
 *   block preconditioners, Krylov ....... Sec. 5, eq. B_D, block_schur
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All functions return a vem_status; none aborts.  On failure the
 *    handle keeps a message (vem_last_error) and output buffers are left
 *    untouched.  Passing NULL where a pointer is required, or sizes that
 *    disagree with the mesh, gives VEM_ERR_BAD_INPUT.
 *  - Unless stated otherwise pointers are HOST pointers and the library
 *    copies what it needs before returning; the caller keeps ownership.
 *    The library owns all device memory it allocates and frees it in
 *    vem_destroy.
 *  - Work is issued on the CUDA stream given to vem_create (NULL = the
 *    legacy default stream).  Calls that return data to the host
 *    synchronise that stream.
 *  - Global unknown layout (the layout of u_out / p_out):
 *      face DOF (f, beta)       -> nfd * f + beta
 *      interior DOF l of cell c -> nfd * n_faces + nid * c + l
 *      pressure of cell c       -> c
 *    E0:  nfd = 1, nid = 0.  The face DOF is the mean normal flux
 *         (1/|f|) int_f u.n_f along the face's global normal.
 *    K1 (the paper's k = 1): nfd = 3, nid = 3.  Face DOFs are the moments
 *         (1/|f|) int_f (u.n_f) m^f_beta, beta = (0,0), (1,0), (0,1), with
 *         m^f_(1,0) = (x - x_f).t1 / h_f, m^f_(0,1) = (x - x_f).t2 / h_f,
 *         n_f the face's global normal (right-hand rule on its vertex
 *         loop), t1 = (v1 - v0)/|v1 - v0| from its first two vertices and
 *         t2 = n_f x t1.  Interior DOFs are the cross moments
 *         (1/|P|) int_P u.(m_I ^ e_q), q = x, y, z, m_I = (x - x_P)/h_P.
 *    The pressure unknown is the cell mean (the P0 moment of eq. presMom)
 *    with the physical sign.
 */
#ifndef VEMSOLVE_H
#define VEMSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vem_handle vem_handle;   /* opaque */

typedef enum {
  VEM_OK = 0,
  VEM_ERR_BAD_INPUT = 1,        /* NULL pointer, size mismatch, K <= 0, bad option */
  VEM_ERR_DEGENERATE_MESH = 2,  /* zero-area face, zero-volume or non-convex cell */
  VEM_ERR_NOT_CONVERGED = 3,    /* iteration cap reached; outputs hold the last iterate */
  VEM_ERR_BREAKDOWN = 4,        /* Krylov breakdown (non-positive curvature, zero norm) */
  VEM_ERR_NONFINITE = 5,        /* NaN / Inf met in data or in a reduction */
  VEM_ERR_OOM = 6,              /* device allocation failed */
  VEM_ERR_CUDA = 7,             /* any other CUDA runtime error */
  VEM_ERR_UNSUPPORTED = 8       /* option combination not built */
} vem_status;

/* Mesh (Sec. 4: a polyhedral decomposition Omega_h).  Faces are planar
 * polygons given by vertex loops; cells list their faces.  A face belongs
 * to one cell (boundary) or two (interior).  Cells must be convex (every
 * face plane separates the cell's barycentre from the outside).
 * face_bc: 0 interior, 1 Dirichlet pressure (g_D enters the right-hand
 * side as -int_f g_D v.n), 2 prescribed normal flux u.n = u_N (paper Sec. 3,
 * the space V): the face's flux DOFs are fixed to (1/|f|) int_f (u.n_f)
 * m_beta and eliminated (unit rows in the assembled matrix, their coupling
 * moved to the right-hand side, no contribution to S).  When every boundary
 * face has flag 2 the pressure is taken in Q = {int p = 0} (Sec. 3) with the
 * paper's mean-zero Lagrange multiplier: vem_solve returns the mean-zero
 * pressure (sum |P| p_P = 0) and the multiplier in vem_stats.  Prescribed
 * flux faces are not supported by vem_solve_batched and vem_adjoint
 * (VEM_ERR_UNSUPPORTED). */
typedef struct {
  int64_t n_vertices;
  const double *xyz;              /* [n_vertices][3] */
  int64_t n_faces;
  const int64_t *face_vtx_ptr;    /* [n_faces + 1], face_vtx_ptr[0] = 0 */
  const int32_t *face_vtx;        /* [face_vtx_ptr[n_faces]] vertex ids, >= 3 per face */
  int64_t n_cells;
  const int64_t *cell_face_ptr;   /* [n_cells + 1] */
  const int32_t *cell_face;       /* [cell_face_ptr[n_cells]] face ids, >= 4 per cell */
  const int8_t *face_bc;          /* [n_faces] */
} vem_mesh;

/* Elements: E0 (face moments against M_0(f), P0 pressure), K1 (the paper's
 * k = 1: 3 face moments, 3 cross moments, P0 pressure), K2 (the paper's
 * k = 2, Sec. 4.1-4.3: 6 face moments against M_2(f), 3 gradient and 11
 * cross moments, P1 pressure moments: 4 pressure unknowns per cell, cell c's
 * at n_u + 4c .. n_u + 4c + 3).  K2 solves with Dirichlet and prescribed-
 * flux faces (the mean-zero pressure then constrains the constant moments,
 * c = |P| on them) and the block-diagonal and block-triangular
 * preconditioners (Jacobi-PCG, the scalar AMG without the multiplier, or
 * the point-block AMG VEM_INNER_BLOCK_AMG for S), Block-Reg (both reg_cycle
 * forms; B^T W^-1 B sums over the four pressure rows of a cell),
 * vem_solve_batched (Jacobi-PCG inner solver, as for every element) and
 * vem_adjoint (Dirichlet boundaries).  Its cell quadrature points
 * (VEM_QP_CELL) are those of a degree-3 rule on the fan tetrahedra of every
 * cell (27 per tetrahedron), built on first use. */
enum { VEM_ELEMENT_E0 = 0, VEM_ELEMENT_K1 = 1, VEM_ELEMENT_K2 = 2 };
enum { VEM_KRYLOV_MINRES = 0, VEM_KRYLOV_FGMRES = 1 };
/* Block preconditioners of the saddle-point system [M B^T; B 0] (Sec. 5):
 *   BLOCK_DIAG  diag(diag(M), S) with S = B diag(M)^-1 B^T (Block-Schur,
 *               eq. block_schur; the S block solved by the inner solver);
 *   BLOCK_TRI   the block upper-triangular form with the same blocks;
 *   BLOCK_REG   Block-Reg (eq. block_diag): diag(A_reg, W) with W = gamma I,
 *               A_reg = M + B^T W^-1 B applied through one V-cycle of a
 *               smoothed-aggregation AMG of A_reg (two Chebyshev steps of the
 *               Jacobi iteration before and after the coarse correction) and
 *               W^-1 = I / gamma; gamma = vem_options.reg_gamma, or h^2 with
 *               h the mean cell diameter (eq. meshSize, the paper's choice)
 *               when that is 0.  The V-cycle is symmetric positive definite,
 *               so MINRES accepts it; no inner solve (inner, inner_rtol are
 *               unused).  Not supported by vem_solve_batched. */
enum { VEM_PREC_BLOCK_DIAG = 0, VEM_PREC_BLOCK_TRI = 1, VEM_PREC_BLOCK_REG = 2 };
/* Inner solver for S: Jacobi-preconditioned CG, or CG preconditioned by one
 * V(1,1) cycle of a smoothed-aggregation AMG built from S (Vanek, Mandel &
 * Brezina 1996; aggregates from a distance-2 maximal independent set, Bell,
 * Dalton & Olson 2012).  With the AMG the inner CG is always FP64;
 * VEM_PRECISION_MIXED runs the V-cycle (matrix values, vectors and
 * arithmetic of every level) in FP32.  The AMG is single-system:
 * vem_solve_batched gives VEM_ERR_UNSUPPORTED with it. */
/* VEM_INNER_BLOCK_AMG (the paper's k = 2 element only): CG preconditioned
 * by one V-cycle of a point-block smoothed-aggregation AMG of S that keeps
 * the four pressure moments of a cell together: aggregates of the graph of
 * 4 x 4 blocks (strength by Frobenius norms), a tentative prolongator from
 * the pressure DOFs of 1, x, y, z orthonormalised per aggregate (Vanek,
 * Mandel & Brezina 1996), damped block-Jacobi smoothing with the weight
 * from a Lanczos estimate of rho(D^-1 S) (or two block-Chebyshev steps with
 * inner_smoother), FP64 only.  The scalar AMG treats every moment as its own
 * node and loses to plain Jacobi-PCG on this S. */
enum { VEM_INNER_PCG = 0, VEM_INNER_AMG = 1, VEM_INNER_BLOCK_AMG = 2 };
enum { VEM_PRECISION_FP64 = 0, VEM_PRECISION_MIXED = 1 };
enum { VEM_SMOOTH_JACOBI = 0, VEM_SMOOTH_CHEBYSHEV = 1 };
/* Block-Reg's approximate inverse of A_reg (vem_options.reg_cycle):
 *   SCALAR_AMG  one V-cycle of the scalar smoothed-aggregation AMG of A_reg
 *               (two Chebyshev steps of Jacobi); FP64 or FP32 (MIXED);
 *   CONDENSED   the paper's k = 1 and k = 2 elements, FP64: the interior
 *               DOFs of A_reg, which couple only within their cell, are
 *               eliminated exactly (nid x nid blocks A_ii: 3 x 3 at k = 1,
 *               14 x 14 at k = 2), and the face system
 *               S_f = A_ff - A_fi A_ii^-1 A_if gets one V-cycle of the
 *               point-block AMG with the face moments of a face (3 or 6) as
 *               a block, the face DOFs of the three constant fields as
 *               near-null space (n_f[j] times the face means of the face
 *               monomials) and two block-Chebyshev steps; the interior DOFs
 *               are then recovered.  Symmetric positive definite.  At k = 2
 *               the scalar cycle barely reduces the residual; use this one. */
enum { VEM_REG_SCALAR_AMG = 0, VEM_REG_CONDENSED = 1 };

typedef struct {
  int element;        /* VEM_ELEMENT_*                                      */
  int krylov;         /* VEM_KRYLOV_*; MINRES needs BLOCK_DIAG or BLOCK_REG */
  int restart;        /* FGMRES restart length m (1..256)                   */
  double rtol;        /* stop when ||b - A x||_2 <= rtol ||b||_2 (true residual) */
  int maxit;          /* outer iteration cap                                */
  int precond;        /* VEM_PREC_*                                         */
  int inner;          /* VEM_INNER_* : solver for S = B diag(M)^-1 B^T      */
  double inner_rtol;  /* inner relative residual target                     */
  int inner_maxit;    /* inner iteration cap per application                */
  int precision;      /* VEM_PRECISION_*: MIXED runs the Schur solve of the */
                      /* preconditioner in FP32 (values, vectors and        */
                      /* arithmetic); the outer Krylov method, its A-apply, */
                      /* orthogonalisation and restart residuals stay FP64. */
                      /* Needs FGMRES; inner_rtol >= 1e-6 is meaningful.    */
                      /* With BLOCK_REG: the V-cycle of A_reg in FP32.      */
  int device_io;      /* 0: vem_solve's x0/u_out/p_out are host pointers;   */
                      /* 1: device pointers (e.g. torch tensors' data_ptr)  */
  int reuse;          /* 1: cells that are translates of one another (same  */
                      /* vertex offsets from the barycentre, to 2^-40 of    */
                      /* the mesh diagonal, and same face/vertex order)     */
                      /* share one evaluation of their geometry-only local  */
                      /* matrices, scaled by nu_P; 0: every cell evaluated. */
  double reg_gamma;   /* BLOCK_REG: gamma > 0, or 0 for h^2 (default 0)     */
  int inner_smoother; /* VEM_SMOOTH_*: smoother of the AMG V-cycle of S     */
                      /* (inner = AMG): one damped-Jacobi step before and   */
                      /* after the coarse correction (default), or two      */
                      /* Chebyshev steps of the Jacobi iteration on         */
                      /* [rho/10, rho] (rho the Gershgorin bound of         */
                      /* rho(D^-1 S); the Block-Reg cycle's smoother)       */
  int reg_cycle;      /* BLOCK_REG: VEM_REG_* (default SCALAR_AMG)          */
} vem_options;

typedef struct {
  int32_t iterations;        /* outer Krylov iterations                     */
  int32_t inner_iterations;  /* total inner (Schur) iterations              */
  double relres;             /* true final ||b - A x|| / ||b||               */
  double t_assemble_ms;      /* element kernel + scatter + Schur build      */
  double t_solve_ms;         /* Krylov solve                                */
  int64_t n_u, n_p;          /* unknown counts                              */
  int64_t nnz_A, nnz_S;      /* nonzeros of [M B^T; B 0] and of S           */
  double t_element_ms;       /* of t_assemble_ms: the element kernel        */
  double t_scatter_ms;       /* of t_assemble_ms: scatter + Schur build     */
  int64_t n_classes;         /* congruence classes of cells evaluated by the */
                             /* element kernel (= n_cells without reuse)    */
  double t_schur_spmv_ms;    /* of t_solve_ms: the Schur-complement SpMV    */
  int64_t n_schur_spmv;      /* its launches (each timed with CUDA events)  */
  double t_amg_setup_ms;     /* of t_solve_ms: building the AMG hierarchy   */
                             /* (0 when it was reused or not used)          */
  int32_t amg_levels;        /* levels of the AMG hierarchy (0: none)       */
  double t_saddle_spmv_ms;   /* of t_solve_ms: the saddle-matrix SpMV       */
  int64_t n_saddle_spmv;     /* its timed launches (at most 16 per solve)   */
  double multiplier;         /* the mean-zero Lagrange multiplier (flux     */
                             /* data on the whole boundary; 0 otherwise)    */
  int32_t schur_tile;        /* batched solves: systems per tile of the     */
                             /* Schur SpMV chosen by the autotuner          */
  double reg_gamma;          /* BLOCK_REG: the gamma used (0 otherwise)     */
  int64_t nnz_reg;           /* BLOCK_REG: nonzeros of A_reg (0 otherwise)  */
  double t_vc_resid_ms;      /* inner AMG: the finest-level residual launch */
  int64_t n_vc_resid;        /* (r = b - S x) of the first, eagerly launched */
  double t_vc_post_ms;       /* V-cycle of every inner solve, and its post-  */
  int64_t n_vc_post;         /* smoothing launch: summed times (CUDA events) */
                             /* and counts                                  */
} vem_stats;

/* Fill *opt with the defaults: E0, FGMRES(30), block-diagonal, Jacobi-PCG
 * inner solve to 1e-12 (at most 2000 iterations), rtol 1e-12, maxit 2000,
 * FP64, host I/O, reuse on, damped-Jacobi smoothing in the AMG of S. */
vem_status vem_default_options(vem_options *opt);

/* Create a solver for a mesh: copies the mesh to the device, computes the
 * face and cell geometry (Sec. 2: barycentres, diameters, face frames) and
 * the DOF layout.  cuda_stream: a cudaStream_t (may be NULL).  On success
 * *out receives the handle; on failure *out is NULL. */
vem_status vem_create(const vem_mesh *mesh, const vem_options *opt, void *cuda_stream,
                      vem_handle **out);

/* Replace the options (element changes invalidate the assembly). */
vem_status vem_set_options(vem_handle *h, const vem_options *opt);

/* Unknown counts for the current element. */
vem_status vem_sizes(const vem_handle *h, int64_t *n_u, int64_t *n_p);

/* Quadrature points at which the caller evaluates the data (the paper leaves
 * the quadrature of b_h and f_h open, Sec. 4.3 remark):
 *   which = VEM_QP_CELL : E0 / K1: one point per cell, its barycentre x_P;
 *                         the load is F_P = |P| f(x_P)  (n = n_cells).
 *                         K2: for every cell, in cell order, its fan
 *                         tetrahedra (x_P, x_f, v_i, v_{i+1}) face by face,
 *                         each with the 27 points of the collapsed 3-point
 *                         Gauss product rule (degree 3); the load is
 *                         F_P = |P| H_1^-1 (int_P f m_q)_q  (n = 27 * sum
 *                         over cells of their faces' vertex counts);
 *   which = VEM_QP_BFACE: for every face with face_bc 1 or 2, in face
 *                         order, its fan triangles (x_f, v_i, v_{i+1}) each
 *                         with the 6-point degree-4 rule of Dunavant (1985)
 *                         for E0 and K1, Radon's 7-point degree-5 rule for
 *                         K2 (g_D m^f has degree 5 for the cubic pressures
 *                         of the k = 2 patch test) (n = 6 or 7 * sum of
 *                         those faces' vertex counts; an element change
 *                         between K2 and the others rebuilds the points and
 *                         clears the boundary data).
 * vem_quadrature_count gives n; vem_quadrature_points writes [n][3]
 * coordinates to xyz_out, a host buffer or a device buffer of the handle's
 * device (the copy's direction follows the pointer; the k = 2 cell set of a
 * 128^3 mesh holds 1.36e9 points, which are best evaluated where they
 * are).  vem_bface_info writes, for every
 * VEM_QP_BFACE point, the outward unit normal of its face ([n][3]) and the
 * face flag ([n]); either pointer may be NULL. */
enum { VEM_QP_CELL = 0, VEM_QP_BFACE = 1 };
vem_status vem_bface_info(vem_handle *h, double *normals_out, int8_t *flags_out);
vem_status vem_quadrature_count(const vem_handle *h, int which, int64_t *n);
vem_status vem_quadrature_points(vem_handle *h, int which, double *xyz_out);

/* Per-cell permeability K > 0 (nu = 1/K in a_h, eq. bilin_form); host array
 * [n_cells].  Invalidates the assembly. */
vem_status vem_set_coefficient(vem_handle *h, const double *K_cell);

/* Data at the quadrature points: f at VEM_QP_CELL points; at VEM_QP_BFACE
 * points g_D on Dirichlet faces and the outward normal flux u_N = u.n on
 * prescribed-flux faces (host arrays; NULL means zero).  Invalidates the
 * right-hand side (and the assembly when prescribed-flux faces exist). */
vem_status vem_set_source(vem_handle *h, const double *f_qp, const double *gD_qp);

/* Same as vem_set_coefficient / vem_set_source with DEVICE arrays. */
vem_status vem_set_coefficient_device(vem_handle *h, const double *K_cell_dev);

/* The coefficient as theta_P = log K_P per cell (DEVICE array [n_cells]):
 * the parameter of the adjoint gradient (vem_adjoint returns dL/dtheta_P).
 * The library forms nu_P = exp(-theta_P) = 1/K_P (Sec. 3, nu = K^-1) on the
 * device.  VEM_ERR_NONFINITE (the previous coefficient kept) if a theta is
 * not finite or exp(-theta) over- or underflows.  Invalidates the assembly. */
vem_status vem_set_log_coefficient_device(vem_handle *h, const double *logK_cell_dev);
vem_status vem_set_source_device(vem_handle *h, const double *f_qp_dev, const double *gD_qp_dev);

/* Assemble: element-batched local matrices M_P, B_P and loads (Sec. 4.3),
 * scatter into the global CSR matrix [M B^T; B 0], and build the Schur
 * approximation S = B diag(M)^-1 B^T (Sec. 5, eq. block_schur). */
vem_status vem_assemble(vem_handle *h);

/* Solve [M B^T; B 0][u; -p] = [g; F] with the configured Krylov method and
 * block preconditioner, from x0 = (u0, p0) (NULL: zero; layout u then p,
 * physical pressure sign).  Assembles first if needed.  Writes u_out
 * [n_u] and p_out [n_p] (host or device per options.device_io) and, if
 * stats != NULL, the statistics.  Returns VEM_ERR_NOT_CONVERGED (outputs
 * written) if rtol is not reached within maxit. */
vem_status vem_solve(vem_handle *h, const double *x0, double *u_out, double *p_out, vem_stats *stats);

/* Batched solve of nbatch problems on the same mesh (the batched form of the
 * same discretisation: per-system coefficient and data, Sec. 4.3 forms):
 * K [nbatch][n_cells] (> 0), f_qp [nbatch][n_cqp] and gD_qp
 * [nbatch][n_bqp] at the VEM_QP_CELL / VEM_QP_BFACE points (NULL = zero;
 * n_cqp = vem_quadrature_count(VEM_QP_CELL): n_cells for E0 and K1, the
 * fan-tetrahedron points for K2).
 * The systems share the sparsity structure: their saddle matrices and Schur
 * approximations are stored as one structure with per-system values, and
 * every A-apply, Schur product and vector operation is one launch over all
 * systems.  With FGMRES every system runs its own Krylov process: its own
 * Arnoldi coefficients, Givens rotations, restarts and stopping test
 * (||b_b - A_b x_b|| <= rtol ||b_b||), and its own inner Jacobi-PCG on its
 * Schur block (own alpha, beta and convergence test); converged systems are
 * skipped, and a system's result does not depend on the other systems.
 * With MINRES one Krylov process runs on the block-diagonal stacked system,
 * stopped when every system's true relative residual is <= rtol.  Writes u_out [nbatch][n_u], p_out
 * [nbatch][n_p] (host or device per options.device_io) and, if not NULL,
 * relres_out [nbatch] (host).  stats->relres is the worst system's. */
vem_status vem_solve_batched(vem_handle *h, int64_t nbatch, const double *K, const double *f_qp,
                             const double *gD_qp, double *u_out, double *p_out, double *relres_out,
                             vem_stats *stats);

/* Adjoint gradient with respect to per-cell log K (theta_P = log K_P), for
 * a loss L(u, p) of the last vem_solve's solution: solves the adjoint system
 * A lambda = (dL/du, -dL/dp) (A is symmetric; the sign converts to the
 * p~ = -p unknown) with the same Krylov method and preconditioner, then
 * returns dL/dtheta_P = lambda_{u,P}^T M_P u_P for every cell (M_P is
 * proportional to nu_P = exp(-theta_P), so dM_P/dtheta_P = -M_P;
 * Sec. 4.3, a_{h,P}).  dL_du [n_u] and dL_dp [n_p] may be NULL (zero);
 * dL_dlogK receives [n_cells].  Host or device pointers per
 * options.device_io.  VEM_ERR_BAD_INPUT if no solution of the current
 * assembly is held. */
vem_status vem_adjoint(vem_handle *h, const double *dL_du, const double *dL_dp, double *dL_dlogK,
                       vem_stats *stats);

/* ---- inspection entry points (used by the parity tests) ---- */

/* Geometry: face area, barycentre [3], unit normal [3], diameter per face;
 * cell volume, barycentre [3], diameter per cell.  Host buffers, any may be
 * NULL. */
vem_status vem_get_geometry(vem_handle *h, double *face_area, double *face_centroid,
                            double *face_normal, double *face_diam, double *cell_volume,
                            double *cell_centroid, double *cell_diam);

/* Element matrices only (every element), without the scatter into the
 * global matrices: the geometry-only local matrices of every congruence
 * class of cells, on the device; vem_local_time reports the element
 * kernel's time (ms, CUDA events) and the number of classes evaluated. */
vem_status vem_assemble_local(vem_handle *h);
vem_status vem_local_time(const vem_handle *h, double *element_ms, int64_t *n_classes);

/* Local matrices after vem_assemble or vem_assemble_local: for each cell,
 * M_P (n_loc x n_loc, row-major) and B_P (nq x n_loc, row-major; nq = 1, or
 * 4 for K2) in the cell's local DOF order (its faces in cell_face order, nfd
 * moments each, then nid interior DOFs), with n_loc = nfd * n_faces(cell) +
 * nid.  vem_local_size gives the total lengths; M_offsets[n_cells + 1]
 * receives the start of each cell's M_P in M_out (in doubles); B_P of cell
 * c starts at nq * (nfd * cell_face_ptr[c] + nid * c) in B_out.  Host
 * buffers; any may be NULL. */
vem_status vem_local_size(const vem_handle *h, int64_t *m_total, int64_t *b_total);
vem_status vem_get_local(vem_handle *h, double *M_out, int64_t *M_offsets, double *B_out);

/* The assembled system: CSR of [M B^T; B 0] with (n_u + n_p) rows, int64 row
 * pointers, int32 columns, double values; rhs [n_u + n_p] = [g; F]. */
vem_status vem_get_system(vem_handle *h, int64_t *row_ptr, int32_t *col, double *val, double *rhs);

/* The Schur approximation S (n_p x n_p CSR) and diag(M) [n_u]. */
vem_status vem_get_schur(vem_handle *h, int64_t *row_ptr, int32_t *col, double *val, double *diagM);

/* y = [M B^T; B 0] x on the device (x, y device arrays of length n_u + n_p). */
vem_status vem_apply_device(vem_handle *h, const double *x_dev, double *y_dev);

/* Residual norm without any device allocation.  (The paper has no
 * counterpart: this is a service for callers that must not let a library
 * allocate device memory -- frameworks that own all device memory through
 * their own pool or budget, where a foreign cudaMalloc can fail or fragment
 * the pool, and latency-sensitive pipelines where cudaFree's implicit
 * device-wide synchronisation would stall other streams.)
 *
 * For a CSR matrix A (rows rows, int64 row_ptr[rows + 1], int32 col, double
 * val) and vectors x, b, computes out[0] = ||b - A x||_2, out[1] = ||b||_2 and
 * out[2] = out[0] / out[1] (out[0] when b = 0).  Every pointer is a DEVICE
 * pointer owned by the caller; the work is enqueued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * synchronising.  It is the same reduction the solver uses for its true
 * residual, e.g. on vem_get_system's matrix and right-hand side with
 * x = (u, -p).
 *
 * Scratch: a static device array of 1 MiB (one pair of partial sums per
 * 2048-row tile), present on every GPU that loads the library until the
 * process exits.  rows above 134,217,728 (65,536 tiles) give
 * VEM_ERR_BAD_INPUT.  The first call on a device resolves the array's
 * device address with that device current; make that first call before any
 * stream capture.  Each call overwrites every partial it reads, so nothing
 * needs clearing, but all calls share the one array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be ordered by
 * the caller.  The array's address is kept per device for the life of the
 * process: do not call this entry point again on a device after
 * cudaDeviceReset (or any other destruction of its primary context).  A CUDA
 * error already pending when the call starts (from earlier, unrelated work)
 * gives VEM_ERR_CUDA before any launch and is left pending for its owner.
 * The matrix is read one warp per row.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
vem_status vem_residual_norm_noalloc(int64_t rows, const int64_t *row_ptr, const int32_t *col,
                                     const double *val, const double *x, const double *b,
                                     double *out, void *cuda_stream);

/* ---- AMG inspection ----
 * which = VEM_AMG_SCHUR: the hierarchy of S (VEM_INNER_AMG); level 0 is S.
 * which = VEM_AMG_REG: the hierarchy of A_reg (VEM_PREC_BLOCK_REG); level 0
 * is A_reg (n_u rows).  vem_amg_setup builds the hierarchy from the current
 * assembly (vem_solve does this on demand after every vem_assemble), with
 * the handle's precision and, for A_reg, its reg_gamma.
 * vem_amg_levels: *nlev levels (at most 12); rows[l], nnz[l] of each
 * level's operator and nnz_p[l] of its prolongator (0 on the coarsest);
 * arrays of at least 12 entries, any may be NULL.
 * With reg_cycle = VEM_REG_CONDENSED the VEM_AMG_REG hierarchy is that of
 * the face system S_f (level 0 has the 3 n_f face rows; one aggregate per
 * face block) and vem_amg_vcycle_device applies the whole condensed cycle
 * to vectors of n_u entries.
 * vem_amg_get_level: host CSR of level l's operator (row_ptr[rows + 1],
 * col[nnz], val[nnz]), its aggregate of every row (agg[rows], -1 for rows
 * outside the coarse space; with VEM_INNER_BLOCK_AMG one entry per point
 * block, agg[rows / block size]) and its prolongator P (rows x rows of level
 * l + 1; prow_ptr[rows + 1], pcol/pval[nnz_p]); any pointer may be NULL,
 * agg and P are left untouched on the coarsest level.
 * vem_amg_vcycle_device: x = V(b), one cycle, device vectors of the
 * level-0 size (n_p for S, n_u for A_reg).
 * All return VEM_ERR_BAD_INPUT before vem_amg_setup / after vem_assemble. */
enum { VEM_AMG_SCHUR = 0, VEM_AMG_REG = 1 };
vem_status vem_amg_setup(vem_handle *h, int32_t which);
vem_status vem_amg_levels(vem_handle *h, int32_t which, int32_t *nlev, int64_t *rows, int64_t *nnz,
                          int64_t *nnz_p);
vem_status vem_amg_get_level(vem_handle *h, int32_t which, int32_t level, int64_t *row_ptr, int32_t *col,
                             double *val, int32_t *agg, int64_t *prow_ptr, int32_t *pcol, double *pval);
vem_status vem_amg_vcycle_device(vem_handle *h, int32_t which, const double *b_dev, double *x_dev);

/* Number of CUDA kernel launches the library has issued in this process
 * (all handles), for accounting the work of a timed region. */
vem_status vem_launch_count(int64_t *n);

/* Message for the last failing call on this handle ("" if none). */
const char *vem_last_error(const vem_handle *h);

/* Free every device and host resource of the handle (NULL is a no-op).
 * Device memory goes back to the library's stream-ordered pool of the
 * current device (freed in the handle's stream order), which keeps it
 * reserved for the next handle; small pinned host buffers are kept too. */
void vem_destroy(vem_handle *h);

/* Return the unused memory of the current device's pool and the cached
 * pinned host buffers to the system (synchronises the device).  Memory of
 * live handles is unaffected. */
vem_status vem_release_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* VEMSOLVE_H */
