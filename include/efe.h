/*
 * efe.h -- C ABI of the GB300 (sm_103a) enriched finite-element ChFSI library.
 *
 * The library discretises the Kohn-Sham eigenproblem in the enriched finite
 * element basis of Kanungo & Gavini (arXiv:1610.02121): degree-4 spectral
 * (GLL) hexahedral elements (Sec. III) augmented by compactly supported,
 * atom-centred enrichment functions (Sec. IV.A-B), with an adaptive quadrature
 * on enriched cells (Sec. IV.C), and solves it by Chebyshev-filtered subspace
 * iteration (Sec. V) using the block-wise overlap inverse (Sec. IV.D).
 *
 * Conventions shared by every call
 * --------------------------------
 * Ownership: the caller owns every buffer passed in; the library owns only the
 *   opaque handle, its operator storage and its workspace (device memory it
 *   allocates with cudaMalloc in efe_create / efe_set_potential* / efe_reserve,
 *   released by efe_destroy).
 * Device: every call runs on the CUDA device that is current when efe_create is
 *   called.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream); all device work of a call is ordered on that stream.  Calls that
 *   return host values (eigenvalues, bounds) synchronise that stream.
 * Block layout ("X layout"): a block of N vectors is a row-major FP64 device
 *   array with n_nodes + n_enrich rows and leading dimension ld >= N
 *   (elements).  Rows 0 .. n_nodes-1 are the classical coefficients at the
 *   nodes of the tensor-product GLL node grid, node index
 *   ix + NX*(iy + NY*iz) (x fastest), boundary nodes included: the box faces
 *   carry homogeneous Dirichlet conditions (Sec. III.A), so boundary rows must
 *   be zero on input and are zero on output.  Rows n_nodes .. n_nodes+n_enrich-1
 *   are the enrichment coefficients psi^E_alpha (Eq. EFEMPsi), in the order of
 *   efe_basis_desc.
 * Errors: every function returns EFE_OK (0) or a positive EFE_ERR_* code and
 *   never aborts, traps or throws; efe_last_error() gives a message for the
 *   last failing call on a handle.  Bounded device waits return
 *   EFE_ERR_TIMEOUT instead of hanging.
 */
#ifndef EFE_H
#define EFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EFE_OK 0
#define EFE_ERR_ARG 1      /* invalid argument or unsupported size */
#define EFE_ERR_CUDA 2     /* a CUDA runtime call failed */
#define EFE_ERR_CHOL 3     /* Cholesky breakdown (Gram matrix, S, or projected overlap) */
#define EFE_ERR_NOCONV 4   /* an iteration did not converge */
#define EFE_ERR_TIMEOUT 5  /* a bounded device wait ran out */
#define EFE_ERR_NAN 6      /* non-finite value in an input or a result */
#define EFE_ERR_ALLOC 7    /* device or host allocation failed */
#define EFE_ERR_STATE 8    /* call out of order (e.g. no potential set) */

/* precision modes of efe_chfsi_step (spec mixed-precision filter) */
#define EFE_PREC_FP64 0    /* every product in FP64 */
#define EFE_PREC_FP32 1    /* classical block in FP32, cell GEMMs FP32 (SIMT FFMA), FP32 accumulate */
#define EFE_PREC_TF32 2    /* classical block in FP32, cell GEMMs on tcgen05 kind::tf32 (one pass), FP32 accumulate */
#define EFE_PREC_BF16 3    /* classical block in FP32 storage, cell GEMMs on tcgen05 kind::f16 with BF16 operands
                              (rounded to nearest in shared memory), FP32 accumulate */
#define EFE_PREC_TF32X3 4  /* classical block in FP32, cell GEMMs on tcgen05 kind::tf32 with the 3-term operand
                              split (a1 b1 + a1 b2 + a2 b1): FP32-grade products, FP32 accumulate */

typedef struct efe_handle efe_handle;

/* Tensor-product mesh of axis-aligned hexahedral cells (Sec. III.A, III.B). */
typedef struct {
  int32_t degree;            /* FE polynomial degree p; this build supports p = 4 only (HEX125SPEC) */
  int32_t n_cells[3];        /* cells per axis, each >= 1 */
  const double* breaks[3];   /* host; n_cells[d] + 1 strictly increasing break points (bohr) */
  int32_t n_gauss;           /* Gauss points per axis in non-enriched cells (1..10) */
} efe_mesh_desc;

/* Nuclei (Eq. vext). */
typedef struct {
  int32_t n_atoms;
  const double* xyz;         /* host, 3 * n_atoms, bohr */
  const double* Z;           /* host, n_atoms nuclear charges */
} efe_atoms_desc;

/* Orbital enrichment functions N_alpha = R_nl(r) h(r~) Y_lm (Eqs. KSOrbitalSplit,
 * EnrichedPsi, Moll1) and the adaptive rule of Sec. IV.C. */
typedef struct {
  int32_t n_funcs;           /* n_E (may be 0: classical basis only) */
  const int32_t* atom;       /* host arrays of length n_funcs */
  const int32_t* n;          /* principal quantum number (1 or 2) */
  const int32_t* l;          /* 0 or 1 */
  const int32_t* m;          /* -l..l; real Y_1m = sqrt(3/4pi) (y, z, x)/r for m = -1, 0, 1 */
  const int32_t* kind;       /* 0: hydrogenic radial of the atom's Z; 1: Slater radial with zeta */
  const double* zeta;        /* Slater exponent (kind 1) */
  const double* r0;          /* cutoff start r0 (bohr) */
  const double* t;           /* cutoff width parameter t; support radius r0 + r0/t */
  double quad_tau;           /* absolute tolerance of the adaptive rule */
  int32_t quad_max_depth;    /* cap on box bisections */
  int32_t quad_n;            /* Gauss points per axis in each adaptive box */
} efe_basis_desc;

/* Analytic local potential V(x) = -sum_I Z_I/|x - R_I| (if nuclear)
 *   + sum_g A_g exp(-|x - c_g|^2 / (2 s_g^2)) + omega^2 |x|^2 / 2. */
typedef struct {
  int32_t nuclear;
  int32_t n_terms;
  const double* A;           /* host, n_terms */
  const double* s;           /* host, n_terms */
  const double* c;           /* host, 3 * n_terms */
  double omega;
} efe_potential_desc;

/* Build the mesh, quadrature (Gauss; adaptive on cells that meet an enrichment
 * support, Sec. IV.C), the diagonal GLL overlap D (Sec. III.B), the overlap
 * blocks M^ec, M^ee and the kinetic parts of H^ec, H^ee (Eqs. Hec, Hee, Mec,
 * Mee), the Schur complement S = M^ee - M^ec D^-1 M^ec^T and S^-1 by Cholesky
 * (Sec. IV.D), and upload them to the current device.  Descriptors are read
 * during the call only.  Returns EFE_ERR_CHOL if S is not positive definite. */
int efe_create(const efe_mesh_desc* mesh, const efe_atoms_desc* atoms,
               const efe_basis_desc* basis, efe_handle** out);

/* Release all device and host memory of the handle (NULL is accepted). */
int efe_destroy(efe_handle* h);

/* Message of the last failing call on h (static string if h is NULL). */
const char* efe_last_error(const efe_handle* h);

/* Sizes: grid nodes (incl. boundary), enrichment functions, quadrature points,
 * cells, and nonzeros of the enrichment-classical coupling M^ec (function-node
 * pairs).  Any output pointer may be NULL. */
int efe_sizes(const efe_handle* h, int64_t* n_nodes, int64_t* n_enrich,
              int64_t* n_qpoints, int64_t* n_cells, int64_t* n_coupling);

/* Copy the quadrature points to xyzw_dev (device, 4 doubles per point: x, y, z,
 * weight), ordered cell by cell (cell index i + nx*(j + ny*k)). */
int efe_qpoints(efe_handle* h, double* xyzw_dev, void* stream);

/* Set the effective potential from its values at the quadrature points
 * (device, n_qpoints doubles, efe_qpoints order) and rebuild, on the device,
 * every V-dependent block: per-cell H^cc_e (Eq. Hcc), H^ec (Eq. Hec) and
 * H^ee (Eq. Hee), plus the FP32/BF16 copies of H^cc_e used by the mixed
 * modes.  Returns EFE_ERR_NAN if V holds a non-finite value. */
int efe_set_potential(efe_handle* h, const double* V_qpts_dev, void* stream);

/* Evaluate the analytic potential of `pot` at the quadrature points on the
 * device, then proceed as efe_set_potential. */
int efe_set_potential_analytic(efe_handle* h, const efe_potential_desc* pot, void* stream);

/* Allocate workspace for blocks of up to N vectors (optional; the block calls
 * below reserve on first use). */
int efe_reserve(efe_handle* h, int32_t N);

/* Y = H^E X (Eq. H2x2): matrix-free cell products of H^cc plus the
 * enrichment coupling, boundary rows zeroed.  X, Y in X layout (FP64 device).
 * X and Y must not overlap (EFE_ERR_ARG): Y is written while X is read. */
int efe_apply_H(efe_handle* h, const double* X, int64_t ldx, int32_t N,
                double* Y, int64_t ldy, void* stream);

/* Y = M^E X (Eq. M2x2) with the GLL-diagonal M^cc.  X and Y must not
 * overlap (EFE_ERR_ARG). */
int efe_apply_M(efe_handle* h, const double* X, int64_t ldx, int32_t N,
                double* Y, int64_t ldy, void* stream);

/* Y = (M^E)^-1 X by the block-wise (Banachiewicz) formula of Sec. IV.D,
 * applied matrix-free: x_e = S^-1 (W_e - M^ec D^-1 W_c), x_c = D^-1 (W_c - M^ec^T x_e).
 * X is copied to the workspace first, so Y may be X. */
int efe_apply_Minv(efe_handle* h, const double* X, int64_t ldx, int32_t N,
                   double* Y, int64_t ldy, void* stream);

/* Upper bound b of the spectrum of H~ = (M^E)^-1 H^E (Sec. V, "a few Arnoldi
 * iterations"): k Lanczos steps in the M-inner product from the device start
 * vector v0 (X layout, one column), b = largest Ritz value + |beta_k|.
 * Synchronises `stream`; writes *b_out on the host. */
int efe_upper_bound(efe_handle* h, const double* v0, int32_t k, double* b_out, void* stream);

/* Chebyshev filter of Sec. V in place: X <- T_m(t(H~)) X / T_m(t(a0)), with
 * t(x) = (2x - a - b)/(b - a) and the three-term recurrence in its scaled
 * form.  a: upper end of the wanted spectrum (largest Ritz value), b: upper
 * bound of the spectrum, a0 < a: lower bound used for scaling.  precision is
 * an EFE_PREC_* mode; the last `fp64_tail` degrees always run in FP64.
 * X in X layout (FP64 device), N >= 1, m >= 1. */
int efe_chfsi_step(efe_handle* h, double* X, int64_t ldx, int32_t N, int32_t m,
                   double a, double b, double a0, int32_t precision, int32_t fp64_tail,
                   void* stream);

/* Cholesky-QR (G = X^T X = R^T R, Q = X R^-1) and Rayleigh-Ritz
 * (Q^T H Q Psi = eps Q^T M Q Psi, Sec. V) in FP64 on the device; X <- Q Psi
 * (M-orthonormal Ritz vectors, ascending eps), N <= 4096.  eig_host / resid_host
 * (host, N doubles each; resid_host may be NULL, which skips the residual
 * work) receive the Ritz values and ||H x_i - eps_i M x_i||_2.  Large blocks
 * (a third R x N FP64 block above 16 GiB) form H Q, M Q and the residuals in
 * two column panels inside the workspace.  A numerically rank-deficient X (G not
 * positive definite in FP64, or a column keeping less than 1e-14 of its
 * squared norm outside the span of the columns before it) is first made well
 * conditioned by up to five shifted Cholesky-QR passes (G + s I, s = 11 (rows
 * N + N (N + 1)) u ||X||_F^2; Fukaya et al., SIAM J. Sci. Comput. 42, 2020);
 * directions lost to rounding come back as rounding noise.  Returns
 * EFE_ERR_CHOL if X is not finite, if G stays rank deficient after those
 * passes, or if Q^T M Q is not positive definite; EFE_ERR_NOCONV if the
 * dense eigensolver does not converge.  Synchronises `stream`. */
int efe_rayleigh_ritz(efe_handle* h, double* X, int64_t ldx, int32_t N,
                      double* eig_host, double* resid_host, void* stream);

/* Number of shifted Cholesky-QR passes efe_rayleigh_ritz has taken on this
 * handle (host counter). */
int efe_rr_shifted_passes(efe_handle* h, int64_t* count);

/* Engine for the FP64 products (the FP64 filter degrees, the H apply and the
 * tall N x N products of Rayleigh-Ritz): 0 = FP64 DFMA (default, the plain
 * FP64 path); 1 = FP64-grade products on the BF16 tensor cores by error-free
 * operand slicing (Ozaki scheme: seven 7-bit digits per operand, exact FP32
 * accumulation of the leading digit products; error within a few units of
 * 2^-48 of sum |a||b|).  Applies to N > 8 cell products, to the tall and Gram
 * products of Rayleigh-Ritz and to its dense N x N products for N > 512.  With
 * engine 1 and N > 8 the enrichment coupling of the FP64 applies also leaves the
 * FP64 pipe: double-float arithmetic on the FP32 pipe (coefficients and vector
 * values as pairs of floats; error within a few units of 2^-48 of sum |a||x|;
 * vector values must stay below 2^126 in magnitude, parts below FP32's normal
 * range are dropped).  Other cases keep DFMA; efe_apply_M_noalloc always does.
 * Host setting, no device work. */
int efe_set_fp64_engine(efe_handle* h, int32_t engine);

/* Test and tuning controls (no counterpart in the paper).  Host settings, no
 * device work; EFE_ERR_ARG for an unknown option or a value out of range.
 * Every default (0) picks by size; the settings exist so that the tests can
 * drive each code path on small inputs. */
#define EFE_OPT_GRID_CAP 1       /* the persistent tensor-core kernels (tcgen05 cell kernel, FP64 engine) run at most
                                    this many CTAs, so each CTA walks several work items (0: one CTA per SM);
                                    results do not depend on it */
#define EFE_OPT_IMAGE_ROWS 2     /* FP64 engine: rows per panel of the operand digit images of the tall products
                                    (0: panels whose images fit 8 GiB) */
#define EFE_OPT_RR_PANELS 3      /* 1: Rayleigh-Ritz forms H Q and M Q in two column panels (and the residuals by
                                    fresh H and M applies) whatever the size; 0: only when a third R x N FP64 block
                                    would exceed 16 GiB.  Takes effect at the next workspace reservation */
#define EFE_OPT_DENSE_BLOCKED 4  /* 1: the blocked multi-CTA dense N x N kernels (Cholesky, triangular inverse,
                                    block Jacobi eigensolver) whatever the size; 0: for N > 512 (Cholesky:
                                    N > 2048) */
#define EFE_OPT_COUPLING_SPARSE 5 /* 1: the mixed degrees take the many-function enrichment coupling (node-major FP32
                                    columns products, rows products over function groups with FP64 partial sums)
                                    whatever the size; 0: only when the dense-tile kernels' n_E x N FP32 array
                                    exceeds 200 KB of shared memory */
#define EFE_OPT_TEST_STALL 6      /* tests of the failure path only: 1 makes every tensor-core launch (tcgen05 cell
                                    kernel, FP64 engine) first wait on a barrier that nothing completes, so the
                                    bounded wait runs out; the launch drains its copies and MMAs, frees its TMEM and
                                    the call returns EFE_ERR_TIMEOUT.  0 (default): off */
#define EFE_OPT_COUPLING_COLS 7   /* the columns product W_c += (H^ec)^T Y_e of the many-function coupling:
                                    0 (default): dense tiles of 32-node blocks; 1: each node's own entries only.
                                    Same products, FP32 sums in another order */
int efe_set_option(efe_handle* h, int32_t option, int64_t value);

/* Kernel timing: when enabled, the library brackets every launch of its
 * classical cell-apply kernel (any precision) with CUDA events on the
 * launching stream.  efe_kernel_stats synchronises the device, then returns
 * the number of launches, their summed duration (ms) and the number of cell
 * products they performed (cells x N-column blocks counted as cells * N), and
 * optionally resets the counters. */
int efe_enable_timing(efe_handle* h, int32_t enable);
int efe_kernel_stats(efe_handle* h, int64_t* launches, double* total_ms, int64_t* cell_columns,
                     int32_t reset);

/* Second timing channel: the FP64 tensor-engine products (efe_set_fp64_engine
 * 1: the FP64 cell products, tall rotations and A^T B products), bracketed by
 * events while timing is enabled.  Returns their launches, summed duration
 * (ms) and algorithmic FP64 flops (2 * 125^2 * N per cell product, 2 rows N^2
 * per rotation, rows N (N + 1) per symmetric A^T B, 2 rows N^2 otherwise). */
int efe_kernel_stats_fp64(efe_handle* h, int64_t* launches, double* total_ms, double* flops, int32_t reset);

/* Y = M^E X exactly as efe_apply_M, but allocation-free (no counterpart in the
 * paper: it exists for callers that cannot allocate device memory at call
 * time -- latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree imply, and hosts that hand the GPU a
 * fixed, pre-planned memory budget).  The call allocates
 * nothing: its one scratch buffer (the partial sums of the enrichment row
 * products, n_segments x N doubles) is a file-scope device array of 2^21
 * doubles (16 MiB) that every GPU loading the library holds until the process
 * exits; the handle's own operator storage was allocated by efe_create.
 * efe_create maps the library's device module and looks up the array's device
 * address (cudaGetSymbolAddress) with the handle's device current, so this call
 * itself loads nothing and looks nothing up.  Sizes needing more than 2^21
 * scratch doubles return EFE_ERR_ARG before any device work.  All calls share
 * the array and it keeps the last call's contents (every entry a call reads is
 * written by that call first), so calls that overlap on the GPU -- on
 * different streams or from different threads -- race and must be serialised
 * by the caller.  X and Y must not overlap (EFE_ERR_ARG).  Arguments as
 * efe_apply_M. */
int efe_apply_M_noalloc(efe_handle* h, const double* X, int64_t ldx, int32_t N,
                        double* Y, int64_t ldy, void* stream);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * handles, all threads); a diagnostic counter for benchmarks. */
int efe_launch_count(int64_t* total);

/* ------------------------------------------------------------------------
 * Self-consistent field (Sec. V): rho_in -> V_eff (Eq. veff) -> ChFSI ->
 * Fermi-Dirac occupations (Eqs. FermiDirac, Mu) -> rho_out (Eq. Rho) ->
 * energy (Sec. II) -> n-stage Anderson mixing (Sec. VI).
 *
 * Quadrature-point layout ("Q layout"): FP64 device arrays of n_qpoints values
 * in the order of efe_qpoints (cell by cell; within a cell the rule's tensor
 * Gauss boxes in order, x fastest).  Densities are electrons per bohr^3,
 * potentials and energies Hartree.
 * Readings of what the paper leaves open: LDA = Slater exchange + Ceperley-
 * Alder correlation in the Perdew-Zunger (1981) parametrisation, spin-
 * unpolarised; the Hartree problem (Eq. Poisson) is solved in the classical
 * basis with Dirichlet data from the monopole and dipole of rho about its
 * centre of charge; the energy of a pair (rho_in, rho_out) is the Kohn-Sham
 * functional at rho_out with the potential of rho_in (equal to the paper's
 * expression at self-consistency); Anderson mixing acts on rho at the points
 * with the quadrature-weighted L2 inner product.
 * ------------------------------------------------------------------------ */
typedef struct {
  double n_electrons;        /* N_e of Eq. Mu */
  double kT;                 /* k_B T (Hartree); 500 K = 1.5834e-3 */
  double mix_beta;           /* Anderson mixing parameter (0, 1] */
  int32_t n_hist;            /* Anderson stages, 1 .. 8 (1 = linear mixing) */
  double poisson_tol;        /* relative residual |b - A phi| / |b| of each Hartree solve */
  int32_t poisson_max_steps; /* cap on exact-solve correction steps per Hartree solve (2 is ample) */
  int32_t lanczos_k;         /* Lanczos steps of the upper bound b per SCF step */
} efe_scf_params;

typedef struct {
  double band;               /* 2 sum_i f_i eps_i */
  double xc;                 /* int rho_out eps_xc(rho_out) */
  double hartree;            /* 1/2 int rho_out V_H[rho_out] */
  double zz;                 /* nuclear repulsion 1/2 sum_{I!=J} Z_I Z_J / |R_I - R_J| */
  double double_counting;    /* int rho_out (V_H[rho_in] + V_xc[rho_in]) */
  double total;              /* band - double_counting + hartree + xc + zz */
  double fermi_level;        /* mu of Eq. Mu */
  double drho;               /* |rho_out - rho_in|_L2 */
  double n_out;              /* int rho_out */
  double upper_bound;        /* b used by the filter */
  int32_t poisson_steps;     /* correction steps of the step's two Hartree solves */
  int32_t filter_passes;
} efe_scf_result;

/* rho(x_q) = 2 sum_i occ_i psi_i(x_q)^2 (Eq. Rho) at every quadrature point,
 * psi_i the FE function with coefficients X[:, i] (X layout, N columns).
 * occ: N FP64 device values.  rho: Q layout, written.  precision:
 * EFE_PREC_FP64, or EFE_PREC_FP32 (orbital values in FP32 arithmetic, the
 * squares and their sums in FP64; efe_scf_step uses it in the mixed modes). */
int efe_density(efe_handle* h, const double* X, int64_t ldx, int32_t N, const double* occ, double* rho,
                int32_t precision, void* stream);

/* LDA energy per electron eps_xc(rho) and potential v_xc = d(rho eps_xc)/d rho
 * at every point (Q layout); exc or vxc may be NULL.  rho is clamped below at
 * 1e-30. */
int efe_xc_lda(efe_handle* h, const double* rho, double* exc, double* vxc, void* stream);

/* Hartree potential of rho (Q layout): -lap V_H / (4 pi) = rho (Eq. Poisson),
 * classical basis, Dirichlet data Q/r + d.r/r^3 on the box faces.  The
 * interior block of the stiffness of the tensor-product mesh is a Kronecker
 * sum of 1-D operators and is solved exactly by fast diagonalisation; the
 * call repeats phi += A_ii^-1 (b - A phi)_i until |b - A phi| <= tol |b| or
 * max_steps corrections.  phi: nodal potential (n_nodes FP64, device) -- on
 * entry the interior values are the starting guess, on exit the solution;
 * NULL uses an internal zero start.  vh: V_H at the points (Q layout),
 * written.  steps: corrections taken (host, may be NULL).  Returns
 * EFE_ERR_NOCONV if the relative residual stays above 1e3 * tol. */
int efe_hartree(efe_handle* h, const double* rho, double* vh, double* phi, double tol, int32_t max_steps,
                int32_t* steps, void* stream);

/* Fermi-Dirac occupations (Eq. FermiDirac) with mu from 2 sum_i f_i = N_e
 * (Eq. Mu) by bisection.  Host arrays; EFE_ERR_ARG if the N states cannot hold
 * N_e electrons. */
int efe_fermi(const double* eps, int32_t N, double n_electrons, double kT, double* occ, double* mu);

/* One n-stage Anderson update from n (rho_in, rho_out) pairs (n x n_qpoints,
 * device, oldest first; n = 1 .. 8): writes the next rho_in to rho_next. */
int efe_anderson(efe_handle* h, const double* rho_in_hist, const double* rho_out_hist, int32_t n, double beta,
                 double* rho_next, void* stream);

/* Start an SCF run: checks the parameters, allocates the SCF buffers, forms
 * V_ext = -sum_I Z_I / |x - R_I| at the points and clears the mixing history
 * and the Ritz values. */
int efe_scf_init(efe_handle* h, const efe_scf_params* params, void* stream);

/* One SCF iteration on the subspace X (X layout, N columns, filtered in place):
 * V_eff(rho_in) -> efe_set_potential -> Lanczos bound b -> `passes` x
 * (degree-m filter + Rayleigh-Ritz; multiple passes re-orthonormalise between
 * them, Sec. VI.B.2) -> occupations -> rho_out -> V_H[rho_out] -> energies ->
 * Anderson.  In the mixed precisions the density's orbital values are FP32
 * (efe_density).  rho_in (Q layout) is read and then overwritten with the next
 * mixed input density; rho_out (Q layout) is written.  eig, occ: N host
 * values written (may be NULL); res: the energies.  The first step after
 * efe_scf_init runs a Rayleigh-Ritz step on X first to obtain the filter
 * interval. */
int efe_scf_step(efe_handle* h, double* X, int64_t ldx, int32_t N, int32_t m, int32_t passes, int32_t precision,
                 int32_t fp64_tail, double* rho_in, double* rho_out, double* eig, double* occ, efe_scf_result* res,
                 void* stream);

/* ------------------------------------------------------------------------
 * Learned initial density (not in the paper; the SCF of Sec. V needs a
 * starting rho_in).  Plain start: superposition of atomic densities (SAD)
 * from normalised Slater shells.  Learned start: rho = (rho_sad + floor)
 * exp(y) - floor (clipped at 0, rescaled to N_e) with y the output of a fully
 * connected network on atom-centred descriptors at each quadrature point.
 * Training and inference run on the device through the calls below.
 * precision arguments: EFE_PREC_FP32 (training / inference) or EFE_PREC_FP64
 * (checks); arrays are then float or double.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_shells;          /* 1 .. 3 */
  int32_t n[3];              /* principal quantum numbers (radial r^(n-1) exp(-zeta r)) */
  double zeta[3];
  double occ[3];             /* electrons per shell */
} efe_atom_shells;

/* rho_sad at the points (Q layout), one efe_atom_shells per atom (host array,
 * n_atoms entries, atom order of efe_create); scaled to n_electrons
 * electrons on the quadrature if n_electrons > 0. */
int efe_sad_density(efe_handle* h, const efe_atom_shells* shells, double n_electrons, double* rho, void* stream);

typedef struct {
  int32_t n_species;         /* species slots, 1 .. 4 */
  double species_Z[4];       /* an atom with charge species_Z[s] uses slot s */
  int32_t n_radial;          /* radial centres, 1 .. 16 */
  double radial_mu[16];
  double radial_sigma;
  int32_t n_ang;             /* angular bands, 0 .. 8 */
  double ang_mu[8];
  double ang_sigma;
  double r_cut;              /* smooth cutoff (1 + cos(pi r / r_cut)) / 2 */
  int32_t standardise;       /* 1: feature f is written as (f - offset[f]) * scale[f] */
  double offset[96];
  double scale[96];
} efe_desc_params;

/* Descriptors at every point: D (n_qpoints x F row-major, F = n_species *
 * (n_radial + n_ang)) with, per species slot s, the radial features
 * sum_I exp(-(r_I - mu_k)^2 / (2 sigma^2)) fc(r_I) and the angular features
 * |sum_I exp(-(r_I - mu_k)^2 / (2 sigma_a^2)) fc(r_I) (x - R_I) / r_I|^2. */
int efe_descriptors(efe_handle* h, const efe_desc_params* p, void* D, int32_t precision, void* stream);

/* rho = max((rho_sad + floor) exp(y) - floor, 0), rescaled to n_electrons
 * (Q layout; y float or double per precision). */
int efe_learned_density(efe_handle* h, const double* rho_sad, const void* y, double floor, double n_electrons,
                        double* rho, int32_t precision, void* stream);

/* Regression target y = log(rho + floor) - log(rho_sad + floor) at the points. */
int efe_density_log_ratio(efe_handle* h, const double* rho, const double* rho_sad, double floor, void* y,
                          int32_t precision, void* stream);

/* Fully connected network: n_layers linear layers dims[0] -> ... -> dims[n_layers]
 * (dims[n_layers] = 1), SiLU after every layer but the last.  Parameters are
 * one flat array: for each layer W (dims[l+1] x dims[l], row-major) then b. */
typedef struct {
  int32_t n_layers;          /* 1 .. 8 */
  int32_t dims[9];
} efe_mlp_shape;

int64_t efe_mlp_param_count(const efe_mlp_shape* s);
/* elements of the forward work array (pre-activations and activations) for n rows */
int64_t efe_mlp_work_elems(const efe_mlp_shape* s, int64_t n);
/* elements of the backward scratch array for n rows */
int64_t efe_mlp_scratch_elems(const efe_mlp_shape* s, int64_t n);
/* y (n) = net(X (n x dims[0])); work keeps what the backward pass needs */
int efe_mlp_forward(const efe_mlp_shape* s, const void* params, const void* X, int64_t n, void* y, void* work,
                    int32_t precision, void* stream);
/* grads = d(sum_i dy_i y_i)/d params for the X, work of the last forward call */
int efe_mlp_backward(const efe_mlp_shape* s, const void* params, const void* X, int64_t n, const void* work,
                     const void* dy, void* grads, void* scratch, int32_t precision, void* stream);
/* loss = sum c (yh - y)^2 / sum c (host), dy = d loss / d yh (device).  The two
 * sums go through a small file-scope device array shared by every call in the
 * process (per device), and the call synchronises `stream` to read them:
 * concurrent efe_wmse calls on one device race on that array and must be
 * serialised by the caller. */
int efe_wmse(const void* yh, const void* y, const void* c, int64_t n, void* dy, double* loss, int32_t precision,
             void* stream);
/* one Adam step (Kingma & Ba) on n parameters with moments m, v; t counts from 1 */
int efe_adam(void* p, const void* g, void* m, void* v, int64_t n, double lr, double beta1, double beta2, double eps,
             int32_t t, int32_t precision, void* stream);

/* ------------------------------------------------------------------------
 * Autotuner and batched systems
 * ------------------------------------------------------------------------ */
/* Times the tensor-core cell kernel's column tiles (64, 96, 160) on one full
 * cell apply for N columns in the given mixed precision (EFE_PREC_TF32,
 * EFE_PREC_TF32X3 or EFE_PREC_BF16) and keeps the fastest for this handle and N; tile_out: the
 * choice (host, may be NULL); ms_out: the three times in ms (host, may be NULL).
 * Needs a potential. */
int efe_autotune(efe_handle* h, int32_t N, int32_t precision, int32_t* tile_out, double* ms_out);

/* A batch of independent systems (handles on one device) whose ChFSI filter
 * steps run as one CUDA graph: each system's kernel sequence is a branch of
 * the graph, recorded once per (X pointers, ld, N, m, precision, fp64_tail)
 * and replayed; the recurrence coefficients of every system are copied by
 * nodes of the graph from pinned staging buffers refreshed before each launch,
 * so new filter bounds need no new recording.  The handles stay owned by the
 * caller and must outlive the batch. */
typedef struct efe_batch efe_batch;
int efe_batch_create(efe_handle* const* systems, int32_t n, efe_batch** out);
int efe_batch_destroy(efe_batch* b);
const char* efe_batch_last_error(const efe_batch* b);
/* graph size of the last recording (host, may be NULL) */
int efe_batch_graph_nodes(const efe_batch* b, int64_t* nodes, int64_t* kernel_nodes);
/* One efe_chfsi_step per system i (X[i], ldx[i], N[i], a[i], b[i], a0[i]; host
 * arrays of n entries).  use_graph = 0 runs the steps one after another on
 * `stream` (reference path); 1 replays the recorded graph.  Synchronises. */
int efe_batch_chfsi_step(efe_batch* b, double* const* X, const int64_t* ldx, const int32_t* N, int32_t m,
                         const double* a, const double* bnd, const double* a0, int32_t precision, int32_t fp64_tail,
                         int32_t use_graph, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EFE_H */
