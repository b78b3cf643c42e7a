// Launchers of the library's CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "efe_internal.h"

#include <algorithm>
#include <atomic>

namespace efe {

// number of kernels launched by this library since it was loaded
extern std::atomic<int64_t> g_launches;

// multiprocessor count of the current device (cached per device ordinal)
int current_sm_count();

// Reference element and mesh geometry passed by value to the set-up kernels.
struct RefElem {
  double z[NP1], w[NP1];
  double M1[NP1 * NP1], K1[NP1 * NP1];
};

struct MeshDev {
  int nc[3];
  int nn[3];
  const double* brk;  // concatenated break points: x (nc0+1), y (nc1+1), z (nc2+1)
};

// ---- set-up / set_potential ----
void launch_potential_analytic(const double* qpts, int64_t nq, const double* axyz, const double* aZ, int na,
                               int nuclear, const double* gA, const double* gs, const double* gc, int nt,
                               double omega, double* V, cudaStream_t st);
void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st);
void launch_gather_sum(int64_t n_out, const double* base, const int64_t* cptr, const int64_t* cidx,
                       const double* blk, double* out, cudaStream_t st);
void launch_permute(int64_t n, const double* src, const int64_t* perm, double* dst, cudaStream_t st);
void launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st);

// ---- hot path (FP64 and FP32 storage) ----
// W_c(cell nodes) += H_e Y_e for the cells of one parity colour
void launch_cell_apply_f64(const double* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                           const double* Y, int64_t ldy, double* W, int64_t ldw, int N, cudaStream_t st);
void launch_cell_apply_f32(const float* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                           const float* Y, int64_t ldy, float* W, int64_t ldw, int N, cudaStream_t st);
// narrow blocks (N <= 8): one warp per row of H_e
void launch_cell_apply_narrow_f64(const double* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                                  const double* Y, int64_t ldy, double* W, int64_t ldw, int N, cudaStream_t st);
void launch_cell_apply_narrow_f32(const float* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                                  const float* Y, int64_t ldy, float* W, int64_t ldw, int N, cudaStream_t st);
// node-major enrichment products with FP32 arithmetic (mixed-precision filter) over
// blocks of coup_block_nodes() pattern nodes: slot_off / slots list the functions of
// every block, tile holds the values as dense (slots x block) FP32 tiles
int coup_block_nodes();
size_t coup_smem(int nE, int N, bool rows);
int coup_resident_ctas(int nE, int N, int n_sm, bool rows);   // CTAs of one product resident at once
// CTA b of the rows / columns products takes the node blocks cta_blk[b] .. cta_blk[b + 1]
void launch_tile_scatter(int64_t nnz, const int64_t* pos, const float* val, float* tile, cudaStream_t st);
template <typename T>
void launch_coup_rows(int64_t n_tn, int ncta, const int64_t* cta_blk, const int32_t* t_nodes,
                      const int64_t* slot_off, const int32_t* slots, const float* tile, const double* scale,
                      const T* X, int64_t ldx, int nE, int N, float* part, cudaStream_t st);
void launch_coup_reduce(int nb, int nE, int N, const float* part, double sgn, const double* base, int64_t ldb,
                        double alpha_base, double* out, int64_t ldo, cudaStream_t st);
template <typename T>
void launch_coup_cols(int64_t n_tn, int ncta, const int64_t* cta_blk, const int32_t* t_nodes,
                      const int64_t* slot_off, const int32_t* slots, const float* tile, float sgn, const double* Xe,
                      int64_t ldxe, int nE, int N, T* W, int64_t ldw, cudaStream_t st);
void launch_cheb_combine_f4(int64_t nrows, int ld, const double* rowscale, const float* X, const float* Yc,
                            const float* Yp, float* Yn, const double* coef, cudaStream_t st);
// mixed coupling for many enrichment functions (FP32 products, FP64 partial sums):
// rows product over function groups (items: first function, functions, node
// positions [j0, j1) of the group's shared row pattern); part: n_items x
// grp_kmax() x N doubles; then a fixed-order reduction per function
int grp_kmax();
void launch_grp_rows(int n_items, const int4* items, const int64_t* ec_ptr, const int32_t* ec_col, const float* coef,
                     const float* Xc, int64_t ldx, double* part, int N, cudaStream_t st);
void launch_grp_reduce(int nE, const int32_t* f_it0, const int32_t* f_it1, const int32_t* f_slot, const double* part,
                       int N, double sgn, const double* base, int64_t ldb, double alpha, double* out, int64_t ldo,
                       cudaStream_t st);
// FP64-grade coupling on the FP32 pipe (double-float sums; coefficients and
// vector values as (hi, lo) float pairs): coefficient pairs (optionally times
// scale[col[q]]), vector rows to pairs, the node-major columns product (adds into
// out) and the grouped rows product (partials per item, reduced by launch_grp_reduce)
void launch_df_coef(int64_t n, const double* v, const double* scale, const int32_t* col, float2* out,
                    cudaStream_t st);
void launch_df_rows(int64_t rows, int N, const double* X, int64_t ldx, float2* out, cudaStream_t st);
void launch_spmm_nodes_df(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                          const float2* val, float sgn, const float2* Xe2, int N, double* out, int64_t ldo,
                          cudaStream_t st);
void launch_grp_rows_df(int n_items, const int4* items, const int64_t* ec_ptr, const int32_t* ec_col,
                        const float2* coef, const double* Xc, int64_t ldx, double* part, int N, cudaStream_t st);
// columns product over the dense tiles' node blocks (X_e rows staged once per block), FP32
void launch_coup_cols_chunk(int64_t n_tn, const int32_t* t_nodes, const int64_t* slot_off, const int32_t* slots,
                            const float* tile, float sgn, const float* Xe, int64_t ldxe, int N, float* W, int64_t ldw,
                            cudaStream_t st);
// the same product with each node's own entries only (t_slot: slot of every
// transposed-pattern entry within its 32-node block; val: FP32 values in that order)
void launch_coup_cols_sparse(int64_t n_tn, const int32_t* t_nodes, const int64_t* t_ptr, const int32_t* t_slot,
                             const float* val, const int64_t* slot_off, const int32_t* slots, float sgn,
                             const float* Xe, int64_t ldxe, int N, float* W, int64_t ldw, cudaStream_t st);
// columns product, node-major, FP32 (Xe: FP32 rows, ldxe)
void launch_spmm_nodes_f32(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                           const float* val, float sgn, const float* Xe, int64_t ldxe, float* out, int64_t ldo, int N,
                           cudaStream_t st);
// out[node_r] += sgn * sum_q val[q] * Xe[col[q]]   (rows = nodes that meet a support)
template <typename T>
void launch_spmm_nodes(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                       const double* val, double sgn, const double* Xe, int64_t ldxe, T* out, int64_t ldo,
                       int N, cudaStream_t st);
// part[seg] = sum_{q in seg} val[q] * scale[col[q]] * Xc[col[q]]  (scale may be NULL)
template <typename T>
void launch_spmm_segments(int64_t nseg, const int64_t* seg_start, const int64_t* seg_end, const int32_t* col,
                          const double* val, const double* scale, const T* Xc, int64_t ldx, double* part,
                          int N, cudaStream_t st);
// out[r] = alpha_base * base[r] + sgn * sum_{segs of r} part[seg]
void launch_seg_reduce(int nrows, const int64_t* row_seg_ptr, const double* part, double sgn,
                       const double* base, int64_t ldb, double alpha_base, double* out, int64_t ldo, int N,
                       cudaStream_t st);
// Chebyshev combine: Ynew = alpha (x - c Ycur) + beta Yprev, x = scale_row * Xsrc, with
// coef = {alpha, c, beta} in device memory
template <typename T>
void launch_cheb_combine(int64_t nrows, const double* rowscale, const T* Xsrc, int64_t ldx, const T* Ycur,
                         int64_t ldc, const T* Yprev, int64_t ldp, T* Ynew, int64_t ldn, const double* coef, int N,
                         cudaStream_t st);
template <typename T>
void launch_row_scale(int64_t nrows, const double* rowscale, const T* X, int64_t ldx, T* Y, int64_t ldy, int N,
                      cudaStream_t st);
void launch_f64_to_f32_rows(int64_t nrows, const double* X, int64_t ldx, float* Y, int64_t ldy, int N,
                            cudaStream_t st);
void launch_f32_to_f64_rows(int64_t nrows, const float* X, int64_t ldx, double* Y, int64_t ldy, int N,
                            cudaStream_t st);
void launch_copy_rows(int64_t nrows, const double* X, int64_t ldx, double* Y, int64_t ldy, int N,
                      cudaStream_t st);
void launch_zero_rows(int64_t nrows, double* X, int64_t ldx, int N, cudaStream_t st);
void launch_zero_rows_f32(int64_t nrows, float* X, int64_t ldx, int N, cudaStream_t st);

// ---- tcgen05 cell products (efe_cell_tc3.cu) ----
int64_t tc3_image_elems(int64_t n_cell);
// FP32 image of every H^cc_e in the MMA's core-matrix layout (split into TF32 parts in the kernel)
void launch_build_aimg(const double* Hcc, int64_t n_cell, float* A, cudaStream_t st);
// tile: column tile width (64, 96 or 160; 0 = default 160)
// stall (tests only): the MMA warp first waits on a barrier nothing completes, so the
// bounded wait runs out and the launch takes its abort path
// mode 0: one TF32 pass; 1: 3-term TF32 split (FP32-grade); 2: BF16 operands (FP32 accumulate)
int launch_cell_tc3(const float* A, const int32_t* cells, int64_t ncells, const MeshDev& m,
                    const float* Y, int64_t ldy, float* W, int64_t ldw, int N, int mode, int n_sm, int* err,
                    cudaStream_t st, int tile = 0, int stall = 0);
const int* tc3_tiles(int* count);

// ---- FP64-grade products on the BF16 tensor cores (efe_oz.cu) ----
// stall (tests only, every launcher below): the MMA warp first waits on a
// barrier nothing completes, so the bounded wait runs out and the launch takes
// its abort path
int64_t oz_hexp_elems(int64_t n_cell);
void launch_oz_hexp(const double* Hcc, int64_t n_cell, int* hexp, cudaStream_t st);
void launch_oz_colexp(const double* Y, int64_t ldy, int64_t rows, int N, int* fexp, cudaStream_t st);
void launch_oz_rowexp(const double* A, int64_t lda, int64_t rows, int K, int* aexp, cudaStream_t st);
// Aimg: pre-sliced digit images of H^cc_e (launch_oz_preslice), or NULL to slice on the fly
int launch_oz_cell(const double* Hcc, const int* hexp, const int32_t* cells, int64_t ncells, const MeshDev& m,
                   const double* Y, int64_t ldy, const int* fexp, double* W, int64_t ldw, int N, int n_sm, int* err,
                   cudaStream_t st, const unsigned char* Aimg = nullptr, int stall = 0);
int64_t oz_cell_image_bytes();
void launch_oz_preslice(const double* Hcc, const int* hexp, int64_t n_cell, unsigned char* img, cudaStream_t st);
int launch_oz_rows(const double* A, int64_t lda, int64_t rows, int K, const int* aexp, const double* B, int64_t ldb,
                   const int* bexp, double* C, int64_t ldc, int N, int n_sm, int* err, cudaStream_t st,
                   const unsigned char* Aimg = nullptr, const unsigned char* Bimg = nullptr, int stall = 0);
// pre-sliced operand images for the ROWS / GRAM products (bytes, builders)
int64_t oz_img_rows_bytes(int64_t rows, int K);
int64_t oz_img_cols_bytes(int64_t nch, int ncols);
void launch_oz_img_rows(const double* A, int64_t lda, int64_t rows, int K, const int* aexp, unsigned char* img,
                        cudaStream_t st);
void launch_oz_img_cols(const double* A, int64_t lda, int64_t Krows, int ncols, const int* cexp, int64_t nch,
                        unsigned char* img, cudaStream_t st);
// C (Na x N) = A^T B (+ C when accumulate), A: K x Na, B: K x N (K large); aexp / bexp per
// column (launch_oz_colexp)
int launch_oz_gram(int64_t K, int Na, int N, const double* A, int64_t lda, const int* aexp, const double* B,
                   int64_t ldb, const int* bexp, double* C, int64_t ldc, bool sym, double* work, int64_t work_elems,
                   int2* pairs_dev, int n_sm, int* err, cudaStream_t st, unsigned char* img_a = nullptr,
                   int64_t img_a_bytes = 0, unsigned char* img_b = nullptr, int64_t img_b_bytes = 0,
                   bool accumulate = false, int stall = 0);
int oz_gram_max_pairs(int Na, int N);

// ---- dense FP64 ----
// C[M x Nc] = alpha * A[M x K] B[K x Nc] + beta * C   (row-major, lda/ldb/ldc)
void launch_gemm_nn(int64_t M, int Nc, int K, double alpha, const double* A, int64_t lda, const double* B,
                    int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t st);
// C_b = A_b B_b for b < batch (members at strides sA, sB, sC elements); grid.y = ceil(Nc / 48) <= 65535
void launch_gemm_nn_batched(int64_t M, int Nc, int K, const double* A, int64_t lda, int64_t sA, const double* B,
                            int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC, int batch,
                            cudaStream_t st);
// C[Na x Nb] = A^T B with A[K x Na], B[K x Nb], K large (split-K, deterministic reduce)
// sym: the product is symmetric in exact arithmetic (A^T A, Q^T H Q, Q^T M Q): only
// tiles on or above the diagonal are formed and the rest mirrored
void launch_gemm_tn(int64_t K, int Na, int Nb, const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, double* work, int64_t work_elems, cudaStream_t st, bool sym = false);
int64_t gemm_tn_work_elems(int64_t K, int Na, int Nb);
void launch_chol(double* A, int n, int lda, int* info, cudaStream_t st, double* min_ratio = nullptr);
void launch_shift_diag(double* A, int n, int lda, double coef, cudaStream_t st);
void launch_trinv_lower(const double* L, int n, int lda, double* Li, int ldi, cudaStream_t st);
void launch_transpose(const double* A, int n, int lda, double* B, int ldb, cudaStream_t st);
void launch_symmetrize(double* A, int n, int lda, cudaStream_t st);
// A[i][j] = A[j][i] for i > j (the strict lower triangle from the upper one)
void launch_mirror_upper(double* A, int n, int lda, cudaStream_t st);

// ---- dense N x N kernels for large N (efe_dense.cu) ----
// blocked Cholesky A = L L^T in place (lower; upper zeroed); info: 0 or j + 1 of the
// first breakdown; min_ratio (optional): min_j L_jj^2 / A_jj; scratch: chol_blocked_scratch(n) doubles
void launch_chol_blocked(double* A, int n, int lda, int* info, double* min_ratio, double* scratch, cudaStream_t st);
int64_t chol_blocked_scratch(int n);
// Li = L^-1 by 2 x 2 block recursion; scratch: n * n / 4 + 64 n doubles
void launch_trinv_blocked(const double* L, int n, int lda, double* Li, int ldi, double* scratch, cudaStream_t st);
// symmetric C = V diag(w) V^T by multi-CTA block Jacobi in precision T (float or double);
// 0: converged (off-diagonal square sum <= tol2 x total), 1: sweeps ran out, -1: CUDA error;
// ratio_out (optional): the last off / total ratio.  scratch: block_jacobi_scratch_bytes(n, sizeof(T))
template <typename T>
int block_jacobi(const double* C, int n, int ldc, T* V, int ldv, T* w, int max_sweeps, double tol2, void* scratch,
                 cudaStream_t st, double* ratio_out);
int64_t block_jacobi_scratch_bytes(int n, int elem);
void launch_jacobi(double* A, int n, int lda, double* V, int ldv, double* w, int max_sweeps, int* info,
                   cudaStream_t st);
// FP32 cyclic Jacobi to a relative off-diagonal size of 1e-6 (pre-diagonalisation)
void launch_jacobi_f32(float* A, int n, int lda, float* V, int ldv, float* w, int max_sweeps, int* info,
                       cudaStream_t st);
void launch_sort_eig(const double* w, const double* V, int n, int ldv, double* ws, double* Vs, int ldvs,
                     cudaStream_t st);
// per-column ||HX - eps MX||^2 partial sums, then sqrt
void launch_resid_norms(int64_t nrows, const double* HX, int64_t ldh, const double* MX, int64_t ldm,
                        const double* eps, int N, double* part, double* out, cudaStream_t st);
void launch_dot(int64_t n, const double* x, const double* y, double* part, double* out, cudaStream_t st);
void launch_axpby3(int64_t n, double* w, const double* v, const double* vp, double a, double b, cudaStream_t st);
void launch_scale(int64_t n, const double* x, double s, double* y, cudaStream_t st);

// ---- self-consistent field (efe_scf.cu) ----
constexpr int ANDERSON_MAX = 8;   // stages of Anderson mixing

struct LeafDev {          // tensor Gauss boxes of the quadrature
  const int64_t* off;     // first point of each leaf
  const int32_t* n;       // points per axis
  const int32_t* cell;    // owning cell
  const double* qpts;     // (x, y, z, w) per point
  int nmax;               // largest n
};

struct EnrDev {           // enrichment values at the points of the enriched cells
  const int32_t* cell_enr;  // cell -> enriched-cell index or -1 (NULL: no enrichment)
  const int32_t* cf_ptr;
  const int32_t* cf_idx;
  const int64_t* qoff;      // first point of each cell
  const int64_t* eq_off;    // per enriched cell: offset of its [point][function] block
  double* Eq;
  int64_t n_nodes;          // row of the first enrichment coefficient
};

struct BandsDev {         // assembled 1-D stiffness / exact mass, 9 entries per row (offsets -4..4)
  const double* K[3];
  const double* M[3];
  int nn[3];
};

struct HistDev {          // Anderson history, oldest first
  const double* rin[ANDERSON_MAX];
  const double* rout[ANDERSON_MAX];
  int n;
};

struct AndersonCoef {
  double t[ANDERSON_MAX];
};

// fp32: orbital values in FP32 arithmetic (mixed mode); rho and its orbital sums stay FP64
int launch_leaf_density(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re, const EnrDev& en,
                        int kmax, const double* X, int64_t ldx, int N, const double* occ, double* rho, bool fp32,
                        cudaStream_t st);
size_t leaf_density_smem(int nm, int kmax);
void launch_leaf_interp(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re, const double* phi,
                        double* out, cudaStream_t st);
void launch_hartree_load(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re,
                         const int64_t* leaf_ptr, const double* rho, const double* mask, int64_t n_nodes,
                         double* lb, double* b, cudaStream_t st);
void launch_enr_values(const EnrDev& en, const int32_t* enr_cells, const int64_t* qoff, const double* qpts,
                       const DevFunc* funcs, int64_t n_enr, cudaStream_t st);
// potential parts of H^cc_e (all cells) and of the enrichment blocks P, Q (enriched cells)
int launch_hcc_sf(const RefElem& re, const MeshDev& m, const LeafDev& lf, const int64_t* leaf_ptr, const double* V,
                  int64_t n_cell, double* Hcc, cudaStream_t st);
int launch_enr_sf(const RefElem& re, const MeshDev& m, const LeafDev& lf, const int64_t* leaf_ptr, const EnrDev& en,
                  const int32_t* enr_cells, int64_t n_enr, const double* V, const int64_t* blkP_off,
                  const int64_t* blkQ_off, double* Pblk, double* Qblk, cudaStream_t st);
int64_t stiff_tiles(const BandsDev& bd);
int reduce_blocks();
// r = mask (b - A phi), partials of |r|^2 per tile
int launch_stiff_resid(const BandsDev& bd, const double* phi, const double* b, const double* mask, double* r64,
                       double* part_rr, cudaStream_t st);
// phi_interior += A_ii^-1 r_interior by fast diagonalisation (U0, U1: interior-sized work arrays)
void launch_fd_solve(const BandsDev& bd, const double* const* V, const double* const* Vt, const double* const* lam,
                     const double* r, double* U0, double* U1, double* phi, cudaStream_t st);
void launch_moments(const double* qpts, const double* rho, int64_t nq, double* part, double* mom, cudaStream_t st);
void launch_finish(const double* part, int nb, int nv, double* out, cudaStream_t st);
void launch_hartree_bc(const MeshDev& m, const double* node_xyz, const double* mask, const double* mom,
                       int64_t n_nodes, double* phi, cudaStream_t st);
void launch_lda(int64_t nq, const double* rho, double* exc, double* vxc, cudaStream_t st);
void launch_veff(int64_t nq, const double* rho, const double* vext, const double* vh, double* vxc, double* veff,
                 cudaStream_t st);
void launch_scf_sums(const double* qpts, int64_t nq, const double* rho_in, const double* rho_out, const double* vh_in,
                     const double* vxc_in, const double* vh_out, double* part, double* out, cudaStream_t st);
int anderson_values(int n);
void launch_anderson_gram(const double* qpts, int64_t nq, const HistDev& hs, double* part, double* out,
                          cudaStream_t st);
void launch_anderson_mix(int64_t nq, const HistDev& hs, const AndersonCoef& th, double beta, double* out,
                         cudaStream_t st);
void launch_scale_to(int64_t n, double* x, const double* num, double target, cudaStream_t st);

// ---- learned initial density (efe_learn.cu) ----
constexpr int DESC_MAX_SPECIES = 4, DESC_MAX_RADIAL = 16, DESC_MAX_ANG = 8;

struct DescDev {
  int n_species, n_radial, n_ang;
  double radial_mu[DESC_MAX_RADIAL];
  double radial_sigma;
  double ang_mu[DESC_MAX_ANG];
  double ang_sigma;
  double r_cut;
  int standardise;
  double offset[DESC_MAX_SPECIES * (DESC_MAX_RADIAL + DESC_MAX_ANG)];
  double scale[DESC_MAX_SPECIES * (DESC_MAX_RADIAL + DESC_MAX_ANG)];
};

struct SadShellDev {      // one atom: up to three Slater shells
  int n_shells;
  int n[3];
  double zeta[3], occ[3], c[3];   // c: radial normalisation constant
};

void launch_sad(const double* qpts, int64_t nq, const double* axyz, int na, const SadShellDev* sh, double* rho,
                cudaStream_t st);
template <typename T>
void launch_descriptors(const double* qpts, int64_t nq, const double* axyz, const int32_t* slot, int na,
                        const DescDev& p, T* D, cudaStream_t st);
int64_t mlp_param_count(const int* dims, int nl);
int64_t mlp_work_elems(const int* dims, int nl, int64_t n);
int64_t mlp_scratch_elems(const int* dims, int nl, int64_t n);
template <typename T>
void mlp_forward(const int* dims, int nl, const T* params, const T* X, int64_t n, T* y, T* work, cudaStream_t st);
template <typename T>
void mlp_backward(const int* dims, int nl, const T* params, const T* X, int64_t n, const T* work, const T* dy,
                  T* grads, T* scratch, cudaStream_t st);
template <typename T>
void launch_wmse(const T* yh, const T* y, const T* c, int64_t n, T* dy, double* part, double* stats, cudaStream_t st);
template <typename T>
void launch_adam(int64_t n, T* p, const T* g, T* m, T* v, double lr, double b1, double b2, double eps, int t,
                 cudaStream_t st);
template <typename T>
void launch_apply_correction(int64_t n, const double* rs, const T* y, double floor, double* rho, cudaStream_t st);
template <typename T>
void launch_log_ratio(int64_t n, const double* rho, const double* rs, double floor, T* y, cudaStream_t st);
// x *= target / sum_q w_q x_q
void launch_scale_count(const double* qpts, int64_t nq, double target, double* x, double* part, cudaStream_t st);
int learn_reduce_blocks();

}  // namespace efe
