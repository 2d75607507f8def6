// Host-side state of a solver handle and the host helpers shared by the
// translation units of the library.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"

namespace vem {
struct AmgState;   // smoothed-aggregation hierarchy (amg.cu)
}

// The operator a Krylov solve works on: the saddle matrix A, the Schur
// approximation S and the preconditioner's diagonals, with sizes.  nbatch > 1
// stacks nbatch systems that share the mesh as one block-diagonal system with
// the vector layout [u_0 .. u_{nb-1}; p_0 .. p_{nb-1}].
struct VemOp {
  vem::SellMat A, S;
  double *diagM = nullptr, *dinvM = nullptr, *s_dinv = nullptr;  // dinvM = 1 / diagM
  float *S_val32 = nullptr, *s_dinv32 = nullptr;
  int64_t n_u = 0, n_p = 0, n = 0;       // stacked sizes
  int64_t n_u1 = 0, n_p1 = 0;            // sizes of one system
  int nbatch = 1;
};

struct vem_handle {
  vem_options opt{};
  cudaStream_t stream = nullptr;
  std::string last_error;

  // ---- mesh sizes ----
  int64_t nv = 0, nf = 0, nc = 0, n_fv = 0, n_cf = 0;
  int max_nf_cell = 0, max_nv_face = 0;
  int nq = 1;                                    // pressure DOFs per cell (4 for paper k = 2)
  bool local_ready = false;                      // element matrices of the current coefficients
  // paper k = 2: |P| H_1^-1 per class (the load map) and the cell points
  double *hq_inv = nullptr;
  double *pm_hat = nullptr;   // K2: per class, the pressure DOFs of 1 and x_j - x_P,j (4 x 4)
  double *pmodes = nullptr;   // K2: near-null space of S (n_p x 4) for the point-block AMG
  double *fmodes = nullptr;   // face DOFs of the constant fields (nfd n_f x 3), condensed Block-Reg
  int64_t hq_inv_n = 0;
  int64_t *cqp_off = nullptr;                    // [nc + 1] first point of each cell
  double *cqp_x = nullptr, *cqp_w = nullptr;     // [n_cqp][3], [n_cqp]
  int64_t n_cqp = 0;
  bool cqp_valid = false;

  // ---- DOF layout (depends on the element) ----
  int nfd = 1, nid = 0;
  int64_t n_u = 0, n_p = 0, n = 0;

  // ---- host copies of small topology arrays ----

  // ---- device mesh ----
  double *xyz = nullptr;
  int64_t *fv_ptr = nullptr, *cf_ptr = nullptr;
  int32_t *fv = nullptr, *cf = nullptr;
  int8_t *fbc = nullptr;

  // ---- geometry ----
  double *f_area = nullptr, *f_cent = nullptr, *f_norm = nullptr, *f_t1 = nullptr,
         *f_diam = nullptr;
  int32_t *f_cell = nullptr, *f_loc = nullptr;   // [2 nf]; second cell -1 on the boundary
  double *c_vol = nullptr, *c_cent = nullptr, *c_diam = nullptr;
  int8_t *cf_sigma = nullptr;                    // [n_cf] orientation of face in cell
  int *d_err = nullptr;                          // device error flags
  int *h_err = nullptr;                          // pinned mirror

  // ---- data ----
  int64_t n_bqp = 0;
  int64_t *bqp_off = nullptr;                    // [nf + 1] offsets of bface points
  double *bqp_xyz = nullptr;                     // [n_bqp][3]
  double *nu = nullptr;                          // 1/K per cell
  double *f_qp = nullptr, *gD_qp = nullptr;
  bool have_coef = false, assembled = false, rhs_ready = false;

  // ---- local matrices: one per congruence class of cells, computed with
  // nu = 1 (M_P = nu_P Mhat_class, B_P = Bhat_class) ----
  int64_t *m_off = nullptr;                      // [nc + 1] class offsets in Mloc (ncls + 1 used)
  int64_t *b_off = nullptr;                      // [nc + 1] class offsets in Bloc
  int32_t *cls_of = nullptr;                     // [nc] class of every cell
  int32_t *cls_rep = nullptr;                    // [nc] representative cell of every class
  int64_t ncls = 0;
  bool cls_valid = false;                        // classes of the current layout and reuse option
  int cls_nfd = 0, cls_nid = 0, cls_reuse = -1;
  double lref = 1.0;                             // mesh bounding-box diagonal
  void *cls_scratch = nullptr;                   // classification scratch
  size_t cls_scratch_bytes = 0;
  int64_t m_total = 0, b_total = 0;
  double *Mloc = nullptr, *Bloc = nullptr;

  // ---- global system ----
  // [M B^T; B 0] and S in sliced ELL (SELL-32): rows in slices of 32, each
  // slice padded to its longest row and stored column-major, so a warp reads
  // element j of 32 consecutive rows with one coalesced load.
  vem::SellMat A, S;
  double *rhs = nullptr;                         // [n] = [g; F]
  double *bt_face = nullptr;                     // [2 nf] B entries of each face's cells
  int32_t *bface = nullptr;                      // [n_bface] the boundary faces, increasing
  int bq_ppt = 6;                                // boundary-data points per fan triangle (7 at k = 2)
  int64_t n_bface = 0;
  // several pressure DOFs per cell: the B^T entries of every flux row of A
  // (pressure column, value), kBtRow per row in row order, zero-padded
  int32_t *bt_col = nullptr;
  double *bt_val = nullptr;
  int64_t bt_rows_n = 0;
  double *diagM = nullptr;                       // [n_u]
  double *dinvM = nullptr;                       // [n_u] 1 / diagM
  double *s_dinv = nullptr;                      // [n_p] 1 / diag(S)
  float *S_val32 = nullptr;                      // FP32 copy of S's values
  float *s_dinv32 = nullptr;                     // FP32 copy of 1 / diag(S)
  int64_t s32_stored = 0;

  // ---- workspace ----
  double *part = nullptr;                        // kMaxSlots * kMaxBlocks partial sums
  double *scal = nullptr;                        // device scalars
  double *h_scal = nullptr;                      // pinned host mirror
  unsigned int *ctr = nullptr;                   // last-block counters (zeroed)
  double *work = nullptr;                        // Krylov vectors
  double *xsol = nullptr;                        // [n] solution iterate
  double *lam = nullptr;                         // [n] adjoint solution
  double *arhs = nullptr;                        // [n] adjoint right-hand side
  double *grad = nullptr;                        // [n_cells] adjoint gradient
  bool have_solution = false;
  int64_t *cnt_buf = nullptr;                    // [n] row counts for the scans
  int64_t *scan_buf = nullptr;                   // scan block sums
  int64_t *slice_buf = nullptr;                  // per-slice sizes
  int64_t slice_buf_n = 0;
  size_t work_n = 0;

  std::vector<void *> allocations;               // everything cudaMalloc'ed
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  static constexpr int kTimed = 16;              // timed Schur SpMV launches per poll
  cudaEvent_t tev[2 * kTimed] = {};
  double t_schur_spmv_ms = 0.0;                  // accumulated over a solve
  int64_t n_schur_spmv = 0;
  double t_vc_resid_ms = 0.0, t_vc_post_ms = 0.0;  // timed finest-level cycle launches of a solve
  int64_t n_vc_resid = 0, n_vc_post = 0;
  static constexpr int kTimedA = 16;             // timed saddle SpMV launches per solve
  cudaEvent_t aev[2 * kTimedA] = {};
  int n_saddle_pending = 0;
  double t_saddle_spmv_ms = 0.0;
  int64_t n_saddle_spmv = 0;
  double t_assemble_ms = 0.0, t_element_ms = 0.0, t_scatter_ms = 0.0;

  // ---- batched systems ----
  VemOp bop;                                     // stacked operator (values per batch)
  double *b_nu = nullptr, *b_rhs = nullptr, *b_x = nullptr, *b_fqp = nullptr, *b_gqp = nullptr;
  int b_cap = 0;                                 // batches the buffers hold
  int64_t b_ncp = 0;                             // cell quadrature points per system they hold

  // ---- AMG for the inner Schur solve ----
  vem::AmgState *amg = nullptr;

  // ---- Block-Reg: A_reg = M + B^T B / gamma and its AMG ----
  vem::SellMat Areg;                             // n_u rows, the flux pattern of the saddle matrix
  float *Areg_val32 = nullptr;                   // FP32 values (FP32 cycle)
  int64_t areg32_stored = 0;
  bool areg_valid = false;                       // A_reg matches the current assembly
  bool areg_has32 = false;                       // Areg_val32 matches A_reg
  double reg_gamma = 0.0;                        // gamma of the current A_reg
  vem::AmgState *amg_reg = nullptr;

  // ---- prescribed-flux faces and the mean-zero pressure ----
  int64_t n_flux_faces = 0, n_dir_faces = 0;
  bool multiplier = false;                       // flux data on the whole boundary
  double *xfix = nullptr;                        // [n] prescribed values (0 elsewhere)
  double *rhs_corr = nullptr;                    // [n] A x_fix with the full matrix
  double *npart = nullptr;                       // partial sums of the projections
  double *bproj = nullptr;                       // [n_p] mean-free inner right-hand side
  int last_pcg_iters = 0;                        // iterations of the last inner solve
  bool x_zero = false;                           // the solve starts from x = 0
  int schur_tile = 1;                            // systems per tile of the batched Schur SpMV
  // CUDA graph of a chunk of inner CG iterations (captured on cap_stream,
  // launched on stream; rebuilt when any launch argument changes)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pcg_graph = nullptr;          // 4 inner PCG iterations
  cudaGraphExec_t pcg_graph16 = nullptr;        // 16 inner PCG iterations
  // per-system batched solve: scalars, partial sums, the inner PCG's graphs
  double *sys_gs = nullptr, *sys_dd = nullptr, *sys_part = nullptr, *bc_part = nullptr, *bc_sc = nullptr;
  size_t sys_n = 0, sys_dd_n = 0, sys_part_n = 0, bc_part_n = 0, bc_sc_n = 0;
  cudaGraphExec_t bpcg_graph = nullptr, bpcg_graph16 = nullptr;
  std::vector<uintptr_t> bpcg_key;
  int64_t bpcg_kernels = 0, bpcg16_kernels = 0;
  int last_bpcg_iters = 0;
  std::vector<uintptr_t> pcg_graph_key, pcg_graph16_key;
  int64_t pcg_graph_kernels = 0, pcg_graph16_kernels = 0;
  double lambda = 0.0;                           // the mean-zero multiplier
};

namespace vem {

// Record an error on the handle and return its code.
vem_status fail(vem_handle *h, vem_status code, const char *fmt, ...);

// cudaMalloc that records the allocation; returns VEM_ERR_OOM on failure.
vem_status dalloc(vem_handle *h, void **p, size_t bytes);
template <class T>
vem_status dalloc_n(vem_handle *h, T **p, size_t n) {
  return dalloc(h, reinterpret_cast<void **>(p), n * sizeof(T) + 16);
}
void dfree(vem_handle *h, void *p);

// Map a CUDA error to a status.
vem_status cuda_check(vem_handle *h, cudaError_t e, const char *what);

// Read the device error flags (synchronises the stream) and map them.
vem_status check_device_errors(vem_handle *h, const char *what);

int grid_for(int64_t n, int threads, int per_sm = 8);

// ---- entry points implemented in the translation units ----
vem_status geometry_build(vem_handle *h);
vem_status assemble_local(vem_handle *h);
vem_status assemble_rhs(vem_handle *h);
vem_status assemble_rhs_into(vem_handle *h, const double *f_qp, const double *gD_qp, double *g, double *F);
vem_status assemble_global(vem_handle *h);

// BLAS-like launches (blas.cu)
void spmv(cudaStream_t s, const SellMat &A, const double *x, double *y, double *dot_part = nullptr);
// batched: nb systems sharing A's structure, values of system b at
// vals + b * A.stored, vectors in the stacked layout with split `split`
void spmv_batched(cudaStream_t s, const SellMat &A, int nb, int64_t split, const double *vals,
                  const double *x, double *y, double *dot_part = nullptr);
int spmv_nblocks(const SellMat &A, int nbatch = 1);
int one_wave_blocks(const void *kernel);
int nblocks_vec(int64_t n);
void dot_partials(cudaStream_t s, int64_t n, const double *x, const double *y, double *part);
// CSR view of a SELL matrix on the host (row_ptr[rows + 1], col, val)
vem_status sell_to_host_csr(vem_handle *h, const SellMat &A, int64_t *rp, int32_t *col, double *val);

// Krylov solve (krylov.cu)
vem_status krylov_solve(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st);
// the batched systems each with its own FGMRES and inner PCG (krylov.cu)
vem_status run_fgmres_systems(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st,
                              double *relres);
// The single-system operator view of the handle.
VemOp single_op(vem_handle *h);

vem_status assemble_batched_values(vem_handle *h, int nb, const double *nu_b, VemOp &op);
// Congruence classes of cells and the per-class layout of Mloc / Bloc.
vem_status classify_cells(vem_handle *h);
// Adjoint contraction (adjoint.cu): g_c = lam_{u,c}^T M_c u_c per cell.
vem_status adjoint_contract(vem_handle *h, const double *lam, const double *x, double *g);

// Prescribed-flux faces and the mean-zero pressure (neumann.cu, element.cu,
// geometry.cu)
vem_status flux_fixed(vem_handle *h, double *xfix);
vem_status bface_info(vem_handle *h, double *nout, int8_t *flag);
vem_status element_k2(vem_handle *h);       // paper k = 2 local matrices (element_k2.cu)
vem_status cell_points_k2(vem_handle *h);   // paper k = 2 cell quadrature points (lazily)
vem_status assemble_rhs_k2(vem_handle *h, const double *f_qp, const double *gD_qp, double *g, double *F);
vem_status neumann_rhs(vem_handle *h, double *rhs);
vem_status neumann_mean_free(vem_handle *h, int64_t n, const double *b, double *out);
vem_status neumann_shift(vem_handle *h, double *xp);

// Exclusive scan of cnt[n] into out[n + 1] (out[0] = 0); *total = out[n]
// (synchronises the stream).
vem_status scan_counts(vem_handle *h, int64_t n, const int64_t *cnt, int64_t *out, int64_t *total);
// boundary-face points for ppt points per fan triangle (element change)
vem_status rebuild_bface_points(vem_handle *h, int ppt);

// Smoothed-aggregation AMG (amg.cu): h->amg of S, h->amg_reg of A_reg.
// setup builds (or rebuilds) the hierarchy in *slot from the level-0
// operator A0 (kept as a view); A0_val32: its FP32 values in the same SELL
// layout, used by an FP32 cycle (fp32); pin_last: A0 is singular with the
// constants as null space; smoother: kSmooth*.
enum { kSmoothJacobi = 0, kSmoothChebyshev = 1 };
// the smoother of the S hierarchy chosen by the options
inline int schur_smoother(const vem_handle *h) {
  return h->opt.inner_smoother == VEM_SMOOTH_CHEBYSHEV ? kSmoothChebyshev : kSmoothJacobi;
}
vem_status amg_setup(vem_handle *h, AmgState *&slot, const SellMat &A0, const float *A0_val32, bool fp32,
                     bool pin_last, int smoother);
// The point-block hierarchy (FP64) of A0 with bs0 x bs0 blocks and the
// near-null space B0 (device, rows x m, row-major; kept by reference).
vem_status amg_setup_block(vem_handle *h, AmgState *&slot, const SellMat &A0, int bs0, const double *B0, int m,
                           bool pin_last, int smoother);
bool amg_is_block(const AmgState *S);
// Block-Reg's condensed cycle: the interior DOFs of A_reg (rows >= nfr, nid
// per cell) eliminated exactly and the point-block hierarchy of the face
// system (nfd x nfd blocks, near-null space Bf of m columns); amg_vcycle then
// applies the whole condensed cycle to vectors of A_reg's size.
vem_status amg_setup_condensed(vem_handle *h, AmgState *&slot, const SellMat &Areg, int64_t nfr, int nid, int nfd,
                               const double *Bf, int m, int smoother);
bool amg_is_condensed(const AmgState *S);
// the face DOFs of the three constant fields for the paper's k = 1 element
vem_status flux_modes_k1(vem_handle *h, int64_t nf, const double *f_norm, double *B);
// The same for the paper's k = 2 element (six face moments per face).
vem_status flux_modes_k2(vem_handle *h, double *B);
// A_reg and its hierarchy for the options (krylov.cu)
vem_status ensure_reg(vem_handle *h);
// the hierarchy of S for the options' inner solver (krylov.cu)
vem_status schur_amg_setup(vem_handle *h, const SellMat &S, const float *S_val32);
bool amg_valid(const AmgState *S);
bool amg_is_fp32(const AmgState *S);
int64_t amg_generation(const AmgState *S);
void amg_invalidate(AmgState *S);
double amg_setup_ms(const AmgState *S);
int amg_levels(const AmgState *S);
int amg_smoother(const AmgState *S);
// Time the level-0 residual and post-smoothing launches of the next cycle
// with CUDA events (an eager cycle: not one captured into a graph); collect
// adds their durations to h->t_vc_resid_ms / t_vc_post_ms after a sync.
void amg_time_next_cycle(AmgState *S);
void amg_collect_timing(vem_handle *h, AmgState *S);
void amg_free(AmgState *&S);
// x = V(b) on the finest level (device vectors of the level-0 size); sc: the
// PCG scalars whose first entry, when non-zero, turns the launches into
// no-ops (NULL: run)
void amg_vcycle(vem_handle *h, AmgState *S, const double *b, double *x, const double *sc);
vem_status amg_level_info(vem_handle *h, const AmgState *S, int *nlev, int64_t *rows, int64_t *nnz,
                          int64_t *nnz_p);
vem_status amg_level_copy(vem_handle *h, AmgState *S, int l, int64_t *rp, int32_t *col, double *val,
                          int32_t *agg, int64_t *prp, int32_t *pcol, double *pval);
double amg_omega(const AmgState *S, int l);

// Block-Reg (assembly.cu): A_reg = M + B^T B / gamma over the flux DOFs with
// the prescribed-flux DOFs eliminated, gamma from the options or h^2 (the
// mean cell diameter squared); FP32 copy when fp32.
vem_status assemble_reg(vem_handle *h, bool fp32);
// sum of a device vector (fixed-order partial sums; synchronises)
vem_status device_sum(vem_handle *h, int64_t n, const double *a, double *out);

}  // namespace vem

#define VEM_CUDA(h, call)                                                  \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return vem::cuda_check((h), e_, #call);         \
  } while (0)

#define VEM_TRY(call)                        \
  do {                                       \
    vem_status s_ = (call);                  \
    if (s_ != VEM_OK) return s_;             \
  } while (0)
