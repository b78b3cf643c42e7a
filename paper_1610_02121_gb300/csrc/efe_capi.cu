// C ABI of the enriched finite-element ChFSI library: handle, device storage,
// and the orchestration of the filter (Sec. V), the block-wise overlap
// inverse (Sec. IV.D), Cholesky-QR and Rayleigh-Ritz.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "efe_internal.h"
#include "efe_kernels.h"

using namespace efe;

namespace {

constexpr int64_t SEG = 2048;  // nnz per segment of a long enrichment row

template <typename T>
struct DevBuf {
  T* p = nullptr;
  int64_t n = 0;
};

}  // namespace

struct efe_handle {
  int dev = 0;
  std::string err;
  RefElem re;
  MeshDev mesh;
  int64_t n_nodes = 0, n_cell = 0, nE = 0, nq = 0, n_enr = 0, rows = 0;
  int kmax = 0;
  bool potential_set = false;
  // device storage (all cudaMalloc'd, freed in efe_destroy)
  std::vector<void*> allocs;
  double* brk = nullptr;
  int n_atoms = 0;
  double *axyz = nullptr, *aZ = nullptr;
  double* qpts = nullptr;
  int64_t* qoff = nullptr;
  double* V = nullptr;
  int32_t* colour_cells = nullptr;
  int64_t colour_off[9] = {0};
  double *D = nullptr, *Dinv = nullptr, *mask = nullptr, *Dm = nullptr;
  double* Hcc = nullptr;
  float* Hcc32 = nullptr;
  float* Aimg32 = nullptr;  // FP32 images of H^cc_e in the tensor-core layout (chunk-major)
  int tc_mode = 0;          // 1: TF32 tcgen05 cell products, 2: 3-term split TF32 (FP32-grade), 3: BF16
  int tc_tile = 0, tc_tile_N = 0;  // autotuned column tile of the tensor-core cell kernel for N
  int n_sm = 148;
  int grid_cap = 0;         // test/tuning cap on the persistent tensor-core grids (0: one CTA per SM)
  int64_t opt_image_rows = 0;   // rows per operand-image panel of the FP64 engine's tall products (0: by budget)
  int opt_rr_panels = 0;        // 1: Rayleigh-Ritz in column panels whatever the size
  int opt_dense_blocked = 0;    // 1: blocked multi-CTA dense N x N kernels whatever the size
  double* noalloc_part = nullptr;  // device address of the static scratch of efe_apply_M_noalloc
  int fp64_engine = 0;      // 0: FP64 DFMA products; 1: FP64-grade products on the BF16 tensor cores
  int* hexp = nullptr;      // per-cell row exponents of H^cc_e (tensor-core FP64 products)
  unsigned char* oz_aimg = nullptr;  // pre-sliced BF16 digit images of H^cc_e (made on first use)
  bool oz_aimg_valid = false;
  int* oz_fexp = nullptr;   // per-column exponents (N)
  int* oz_bexp = nullptr;   // per-column exponents of small right-hand matrices (N)
  int* oz_aexp = nullptr;   // per-row exponents of tall left-hand matrices (rows)
  int2* oz_pairs = nullptr; // tile pairs of the tensor-core A^T B products
  unsigned char* oz_img[2] = {nullptr, nullptr};  // operand digit images of the tall products (grow-only)
  int64_t oz_img_bytes[2] = {0, 0};
  int64_t chol_shifted = 0;        // shifted Cholesky-QR passes taken by Rayleigh-Ritz
  double* chol_ratio = nullptr;    // device: min_j L_jj^2 / G_jj of the last Gram factorisation
  bool time_this = false;   // the cell-apply timer records only the filter's mixed-precision launches
  DevFunc* funcs = nullptr;
  int32_t *enr_cells = nullptr, *cf_ptr = nullptr, *cf_idx = nullptr;
  int64_t *blkP_off = nullptr, *blkQ_off = nullptr;
  int64_t nP = 0, nQ = 0;
  double *Pblk = nullptr, *Qblk = nullptr;
  int64_t nnz = 0;
  int32_t* ec_col = nullptr;
  double *mec = nullptr, *hec_kin = nullptr, *hec = nullptr;
  int64_t *ec_cptr = nullptr, *ec_cidx = nullptr;
  int64_t nseg = 0;
  int64_t *seg_start = nullptr, *seg_end = nullptr, *row_seg_ptr = nullptr;
  int64_t n_tn = 0;
  int32_t* t_nodes = nullptr;
  int64_t* t_ptr = nullptr;
  int32_t* t_col = nullptr;
  int64_t* t_perm = nullptr;
  double *mecT = nullptr, *hecT = nullptr;
  double *Mee = nullptr, *Hee_kin = nullptr, *Hee = nullptr, *Sinv = nullptr;
  int64_t *ee_cptr = nullptr, *ee_cidx = nullptr;
  int* info = nullptr;        // 8 ints
  // workspace
  int Nres = 0;
  double *B1 = nullptr, *B2 = nullptr, *W = nullptr, *xe = nullptr, *rb = nullptr, *part = nullptr;
  double* small = nullptr;    // 16 N x N blocks + vectors
  double* tnwork = nullptr;
  int64_t tnwork_elems = 0;
  double* rpart = nullptr;
  double* lz = nullptr;       // Lanczos vectors (6 * rows) + scalars
  int Nres32 = 0, ld32 = 0, ncb = 0;
  // FP32 classical blocks of the mixed degrees: two recurrence slots (each
  // degree overwrites Y_{k-2} in place) and the cell-product output; when the
  // rows need no padding they live inside the FP64 workspace (slots in W, the
  // output in B1), which the mixed degrees do not use
  float *Yf[2] = {nullptr, nullptr}, *Wf = nullptr, *cpart = nullptr;
  bool f32_alias = false;
  double* We = nullptr;       // n_E x N FP64 coupling rows of the mixed degrees
  void* dsc = nullptr;        // scratch of the blocked dense N x N kernels (grow-only)
  int64_t dsc_bytes = 0;
  bool whole_rr = true;       // Rayleigh-Ritz holds H Q and M Q whole (B2 exists); else column panels in W
  float *mecT32 = nullptr, *hecT32 = nullptr;
  // function groups sharing one support (the many-function mixed coupling):
  // items (first function, functions, node range) and per function its items and slot
  int n_gitems = 0;
  int4* gitems = nullptr;
  int32_t *f_it0 = nullptr, *f_it1 = nullptr, *f_slot = nullptr;
  float *hec32 = nullptr, *mecD32 = nullptr;   // row-pattern FP32 values of H^ec and M^ec D^-1
  int64_t* ec_rowptr = nullptr;               // start of each function's row in the row pattern
  int32_t* t_slot = nullptr;                  // slot of each transposed-pattern entry within its node block
  // (hi, lo) float pairs of the coupling values for the FP64-grade coupling on the
  // FP32 pipe (tensor-core FP64 engine): row pattern H^ec, M^ec, M^ec D^-1;
  // transposed pattern H^ec, M^ec; xe2: an enrichment block as pairs (n_E x N)
  float2 *hec2 = nullptr, *mec2 = nullptr, *mecD2 = nullptr, *hecT2 = nullptr, *mecT2 = nullptr, *xe2 = nullptr;
  double* gpart = nullptr;                    // n_gitems x grp_kmax() x N partial sums
  float* Xe32 = nullptr;                      // n_E x N FP32 copy of an enrichment block
  int opt_coup_sparse = 0;                    // 1: grouped sparse coupling whatever the size
  int opt_coup_cols = 0;                      // columns product: 0 dense tiles, 1 per-node entries
  int opt_test_stall = 0;                     // tests: tensor-core launches take their abort path
  // dense FP32 tiles of the pattern over blocks of pattern nodes (mixed filter)
  int64_t cb_nblk = 0, cb_nslots = 0;
  int64_t *cb_slot_off = nullptr, *cb_pos = nullptr, *cb_cta = nullptr, *cb_cta_cols = nullptr;
  int ncb_cols = 1;                    // CTAs of the columns product
  std::vector<int64_t> cb_soff_host;   // slot offsets of the node blocks (host copy)
  int32_t* cb_slots = nullptr;
  float *tileH = nullptr, *tileM = nullptr;
  double* Ye[2] = {nullptr, nullptr};
  // Chebyshev coefficients {alpha, c, beta} per degree: pinned host staging and device copy
  double* coefh = nullptr;
  double* coefd = nullptr;
  int coef_cap = 0;
  cudaEvent_t coef_ev = nullptr;
  bool coef_pending = false;
  // self-consistent field (Sec. V): quadrature leaves, Hartree operator, SCF state
  int64_t n_leaf = 0;
  int leaf_nmax = 1;
  int64_t *leaf_off = nullptr, *leaf_ptr = nullptr;
  int32_t *leaf_n = nullptr, *leaf_cell = nullptr, *cell_enr = nullptr;
  int64_t* eq_off = nullptr;
  int64_t eq_elems = 0;
  double* Eq = nullptr;                      // enrichment values at enriched-cell points (lazy)
  double* band[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // Kx Ky Kz Mx My Mz
  double* node_xyz = nullptr;                // node coordinates per axis
  double e_zz = 0.0;
  bool scf_ready = false;
  efe_scf_params scfp{};
  double *hb = nullptr, *hr64 = nullptr, *hlb = nullptr, *hphi = nullptr, *hpart_rr = nullptr;
  double *fdV[3] = {nullptr, nullptr, nullptr}, *fdVt[3] = {nullptr, nullptr, nullptr};
  double *fdlam[3] = {nullptr, nullptr, nullptr};
  double *fdU0 = nullptr, *fdU1 = nullptr;
  double *red_part = nullptr, *red_out = nullptr;
  double *vext = nullptr, *vh_in = nullptr, *vxc_in = nullptr, *vh_out = nullptr, *phi_in = nullptr,
         *phi_out = nullptr, *occ_dev = nullptr, *v0 = nullptr;
  double* hist[2 * ANDERSON_MAX] = {nullptr};  // rho_in ring, then rho_out ring
  int hist_count = 0, hist_head = 0, occ_cap = 0;
  std::vector<double> ritz;                  // Ritz values of the last Rayleigh-Ritz step
  int scf_iter = 0;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_free;                 // event pairs (even indices) ready for reuse
  struct TimedPair { int ev; int ch; double units; };
  std::vector<TimedPair> ev_pairs;
  // channel 0: mixed-precision cell products (units: cell columns);
  // channel 1: FP64 tensor-engine products (units: algorithmic FP64 flops)
  int64_t t_launches[2] = {0, 0};
  double t_ms[2] = {0.0, 0.0}, t_units[2] = {0.0, 0.0};
};

// tall FP64 product (defined with the Rayleigh-Ritz kernels below)
extern "C" int gemm_tall(efe_handle* h, int64_t rows, int K, int Nc, const double* A, int64_t lda, const double* B,
                         double* C, int64_t ldc, cudaStream_t st);

namespace {

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(_e);                 \
      return EFE_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

#define CKL()                                                                      \
  do {                                                                             \
    cudaError_t _e = cudaGetLastError();                                           \
    if (_e != cudaSuccess) {                                                       \
      h->err = std::string("kernel launch: ") + cudaGetErrorString(_e);            \
      return EFE_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

#define TRY(x)                 \
  do {                         \
    int _r = (x);              \
    if (_r != EFE_OK) return _r; \
  } while (0)

template <typename T>
int dalloc(efe_handle* h, T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return EFE_ERR_ALLOC;
  }
  h->allocs.push_back(q);
  *p = (T*)q;
  return EFE_OK;
}

template <typename T>
int upload(efe_handle* h, T** p, const std::vector<T>& v) {
  TRY(dalloc(h, p, (int64_t)v.size()));
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return EFE_OK;
}

void dfree(efe_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) h->allocs.erase(it);
  cudaFree(p);
}

int set_dev(efe_handle* h) {
  CK(cudaSetDevice(h->dev));
  return EFE_OK;
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

// CTAs of the persistent tensor-core kernels (cell kernel, FP64 engine): one per
// SM unless a cap is set (EFE_OPT_GRID_CAP)
inline int tc_grid(const efe_handle* h) {
  return (h->grid_cap > 0 && h->grid_cap < h->n_sm) ? h->grid_cap : h->n_sm;
}

// the mixed degrees' dense-tile coupling kernels keep an (n_E x N) FP32 array
// in shared memory: used when it fits, the sparse kernels otherwise
inline bool coup_tiles_fit(const efe_handle* h, int N) {
  return !h->opt_coup_sparse && coup_smem((int)h->nE, N, true) <= 200 * 1024;
}

// Byte size above which Rayleigh-Ritz no longer keeps H Q and M Q as whole
// blocks (a third FP64 block) but forms them in two column panels inside W.
constexpr int64_t WHOLE_RR_MAX_BYTES = 16ll << 30;

// FP32 blocks of the mixed degrees (see efe_handle): dropped before the FP64
// workspace they may live in is reallocated
void free32(efe_handle* h) {
  if (!h->f32_alias) {
    for (int i = 0; i < 2; ++i) dfree(h, h->Yf[i]);
    dfree(h, h->Wf);
  }
  for (int i = 0; i < 2; ++i) {
    dfree(h, h->Ye[i]);
    h->Yf[i] = nullptr;
    h->Ye[i] = nullptr;
  }
  dfree(h, h->cpart);
  dfree(h, h->We);
  dfree(h, h->gpart);
  dfree(h, h->Xe32);
  h->Wf = nullptr;
  h->cpart = nullptr;
  h->We = nullptr;
  h->gpart = nullptr;
  h->Xe32 = nullptr;
  h->f32_alias = false;
  h->Nres32 = 0;
}

int reserve(efe_handle* h, int N) {
  if (N <= h->Nres) return EFE_OK;
  free32(h);
  for (void* p : {(void*)h->B1, (void*)h->B2, (void*)h->W, (void*)h->xe, (void*)h->rb, (void*)h->part,
                  (void*)h->small, (void*)h->tnwork, (void*)h->rpart})
    dfree(h, p);
  h->B2 = nullptr;
  const int64_t R = h->rows;
  h->whole_rr = (int64_t)sizeof(double) * R * N <= WHOLE_RR_MAX_BYTES && !h->opt_rr_panels;
  TRY(dalloc(h, &h->B1, R * N));
  // W: in panel mode it holds two R x ceil(N/2) panels side by side
  TRY(dalloc(h, &h->W, R * (N + (h->whole_rr ? 0 : 1))));
  if (h->whole_rr) TRY(dalloc(h, &h->B2, R * N));
  TRY(dalloc(h, &h->xe, std::max<int64_t>(1, h->nE) * N));
  TRY(dalloc(h, &h->rb, std::max<int64_t>(1, h->nE) * N));
  TRY(dalloc(h, &h->part, std::max<int64_t>({1, h->nseg, (int64_t)h->n_gitems * grp_kmax()}) * N));
  dfree(h, h->xe2);
  h->xe2 = nullptr;
  TRY(dalloc(h, &h->xe2, std::max<int64_t>(1, h->nE) * N));
  TRY(dalloc(h, &h->small, 24 * (int64_t)N * N + 8 * (int64_t)N));
  // split-K partials of the DFMA A^T B products and the segment partials of the
  // tensor-core ones (both fit their split counts to this size)
  h->tnwork_elems = std::max<int64_t>(gemm_tn_work_elems(R, N, N), 4 * (int64_t)N * N);
  TRY(dalloc(h, &h->tnwork, h->tnwork_elems));
  TRY(dalloc(h, &h->rpart, ((R + 2047) / 2048 + 1) * (int64_t)N));
  dfree(h, h->oz_fexp);
  dfree(h, h->oz_bexp);
  dfree(h, h->oz_pairs);
  TRY(dalloc(h, &h->oz_fexp, N));
  TRY(dalloc(h, &h->oz_bexp, N));
  TRY(dalloc(h, &h->oz_pairs, oz_gram_max_pairs(N, N)));
  h->Nres = N;
  return EFE_OK;
}

int reserve32(efe_handle* h, int N) {
  if (N <= h->Nres32) return EFE_OK;
  TRY(reserve(h, std::max(N, h->Nres)));
  free32(h);
  // classical rows padded to a multiple of 8 elements: 16-byte aligned rows for
  // vector loads and bulk copies; the padding columns are zero and stay zero
  const int ld = (N + 7) / 8 * 8;
  const int64_t n32 = h->n_nodes * ld;
  if (ld == N) {
    // no padding to keep at zero: the two slots share W (R x N doubles hold
    // 2 n_nodes x N floats), the cell-product output lives in B1
    h->Yf[0] = reinterpret_cast<float*>(h->W);
    h->Yf[1] = h->Yf[0] + n32;
    h->Wf = reinterpret_cast<float*>(h->B1);
    h->f32_alias = true;
  } else {
    for (int i = 0; i < 2; ++i) {
      TRY(dalloc(h, &h->Yf[i], n32));
      CK(cudaMemset(h->Yf[i], 0, sizeof(float) * n32));
    }
    TRY(dalloc(h, &h->Wf, n32));
    CK(cudaMemset(h->Wf, 0, sizeof(float) * n32));
  }
  for (int i = 0; i < 2; ++i) TRY(dalloc(h, &h->Ye[i], std::max<int64_t>(1, h->nE) * N));
  TRY(dalloc(h, &h->We, std::max<int64_t>(1, h->nE) * N));
  // coupling products: one wave of CTAs each, node blocks split so that every
  // CTA holds about the same number of tile slots (plus a share for staging rows)
  auto partition = [&](bool rows, int64_t** dev, int* ncta_out) -> int {
    dfree(h, *dev);
    *dev = nullptr;
    *ncta_out = 1;
    // the dense-tile coupling kernels serve only blocks whose (n_E x N) array
    // fits in shared memory (the mixed degrees take the sparse kernels otherwise)
    if (h->nE <= 0 || h->cb_nblk <= 0 || !coup_tiles_fit(h, N)) return EFE_OK;
    const int64_t nblk = h->cb_nblk;
    const int ncta = (int)std::min<int64_t>(nblk, coup_resident_ctas((int)h->nE, N, h->n_sm, rows));
    const auto& so = h->cb_soff_host;
    const double wtot = (double)so[nblk] + 3.0 * (double)nblk;
    std::vector<int64_t> cb(ncta + 1, nblk);
    cb[0] = 0;
    int64_t b = 0;
    for (int c = 1; c < ncta; ++c) {
      const double target = wtot * c / ncta;
      while (b < nblk && (double)so[b] + 3.0 * (double)b < target) ++b;
      cb[c] = std::max(cb[c - 1], b);
    }
    TRY(upload(h, dev, cb));
    *ncta_out = ncta;
    return EFE_OK;
  };
  TRY(partition(true, &h->cb_cta, &h->ncb));
  TRY(partition(false, &h->cb_cta_cols, &h->ncb_cols));
  TRY(dalloc(h, &h->cpart, coup_tiles_fit(h, N) ? (int64_t)h->ncb * std::max<int64_t>(1, h->nE) * N : 1));
  if (h->nE > 0 && !coup_tiles_fit(h, N)) {
    TRY(dalloc(h, &h->gpart, (int64_t)std::max(1, h->n_gitems) * grp_kmax() * N));
    TRY(dalloc(h, &h->Xe32, h->nE * N));
  }
  h->ld32 = ld;
  h->Nres32 = N;
  return EFE_OK;
}

// --- timing of the classical cell-apply launches ---
int ev_get(efe_handle* h, int idx, cudaEvent_t* e) {
  while ((int)h->ev_pool.size() <= idx) {
    cudaEvent_t ev;
    CK(cudaEventCreate(&ev));
    h->ev_pool.push_back(ev);
  }
  *e = h->ev_pool[idx];
  return EFE_OK;
}

// channel 0 times only the filter's mixed-precision cell launches (time_this);
// channel 1 every FP64 tensor-engine product
int timed_begin(efe_handle* h, cudaStream_t st, int* slot, int ch = 0) {
  *slot = -1;
  if (!h->timing || (ch == 0 && !h->time_this)) return EFE_OK;
  int i;
  if (!h->ev_free.empty()) {
    i = h->ev_free.back();
    h->ev_free.pop_back();
  } else {
    i = (int)h->ev_pool.size();
  }
  cudaEvent_t a, b;
  TRY(ev_get(h, i, &a));
  TRY(ev_get(h, i + 1, &b));
  CK(cudaEventRecord(a, st));
  *slot = i;
  return EFE_OK;
}

// adds the finished pairs to their channels (waits for the last one)
int timed_fold(efe_handle* h) {
  if (h->ev_pairs.empty()) return EFE_OK;
  CK(cudaEventSynchronize(h->ev_pool[h->ev_pairs.back().ev + 1]));
  for (auto& pr : h->ev_pairs) {
    CK(cudaEventSynchronize(h->ev_pool[pr.ev + 1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_pool[pr.ev], h->ev_pool[pr.ev + 1]));
    h->t_ms[pr.ch] += ms;
    h->t_launches[pr.ch]++;
    h->t_units[pr.ch] += pr.units;
    h->ev_free.push_back(pr.ev);
  }
  h->ev_pairs.clear();
  return EFE_OK;
}

int timed_end(efe_handle* h, cudaStream_t st, int slot, double units, int ch = 0) {
  if (slot < 0) return EFE_OK;
  CK(cudaEventRecord(h->ev_pool[slot + 1], st));
  h->ev_pairs.push_back({slot, ch, units});
  if (h->ev_pairs.size() >= 4096) TRY(timed_fold(h));  // bound the event pool
  return EFE_OK;
}

// --- classical cell products, all 8 parity colours: W_c += H^cc Y_c ---
template <typename T>
int cell_apply_all(efe_handle* h, const T* Hc, const T* Y, int64_t ldy, T* Wc, int64_t ldw, int N, cudaStream_t st,
                   bool tc = false) {
  if constexpr (sizeof(T) == 8) {
    if (h->fp64_engine == 1 && N > 8) {
      if (!h->oz_aimg_valid) {
        if (!h->oz_aimg) TRY(dalloc(h, &h->oz_aimg, h->n_cell * oz_cell_image_bytes()));
        launch_oz_preslice(h->Hcc, h->hexp, h->n_cell, h->oz_aimg, st);
        h->oz_aimg_valid = true;
      }
      launch_oz_colexp((const double*)Y, ldy, h->n_nodes, N, h->oz_fexp, st);
      for (int c = 0; c < 8; ++c) {
        const int64_t nc = h->colour_off[c + 1] - h->colour_off[c];
        if (nc == 0) continue;
        int slot;
        TRY(timed_begin(h, st, &slot, 1));
        launch_oz_cell(h->Hcc, h->hexp, h->colour_cells + h->colour_off[c], nc, h->mesh, (const double*)Y, ldy,
                       h->oz_fexp, (double*)Wc, ldw, N, tc_grid(h), h->info + 4, st, h->oz_aimg, h->opt_test_stall);
        TRY(timed_end(h, st, slot, 2.0 * NL * NL * (double)N * (double)nc, 1));
      }
      CKL();
      return EFE_OK;
    }
  }
  for (int c = 0; c < 8; ++c) {
    const int64_t nc = h->colour_off[c + 1] - h->colour_off[c];
    if (nc == 0) continue;
    int slot;
    TRY(timed_begin(h, st, &slot));
    const int32_t* cl = h->colour_cells + h->colour_off[c];
    if constexpr (sizeof(T) == 8) {
      if (N <= 8)
        launch_cell_apply_narrow_f64((const double*)Hc, cl, nc, h->mesh, (const double*)Y, ldy, (double*)Wc, ldw, N, st);
      else
        launch_cell_apply_f64((const double*)Hc, cl, nc, h->mesh, (const double*)Y, ldy, (double*)Wc, ldw, N, st);
    } else {
      if (tc) {
        if (launch_cell_tc3(h->Aimg32, cl, nc, h->mesh, (const float*)Y, ldy, (float*)Wc, ldw, N,
                            h->tc_mode - 1, tc_grid(h), h->info + 4, st, h->tc_tile_N == N ? h->tc_tile : 0,
                            h->opt_test_stall)) {
          h->err = "tensor-core cell kernel needs 16-byte aligned rows";
          return EFE_ERR_ARG;
        }
      }
      else if (N <= 8)
        launch_cell_apply_narrow_f32((const float*)Hc, cl, nc, h->mesh, (const float*)Y, ldy, (float*)Wc, ldw, N, st);
      else
        launch_cell_apply_f32((const float*)Hc, cl, nc, h->mesh, (const float*)Y, ldy, (float*)Wc, ldw, N, st);
    }
    CKL();
    TRY(timed_end(h, st, slot, (double)(nc * (int64_t)N)));
  }
  return EFE_OK;
}

// The FP64 enrichment coupling runs in double-float arithmetic on the FP32 pipe
// (FP64-grade like the tensor-core engine it comes with) for blocks of N > 8
// vectors; the plain FP64 kernels otherwise.
bool use_df(const efe_handle* h, int N) { return h->fp64_engine == 1 && h->nE > 0 && N > 8; }

// --- H^E X: classical cell products + enrichment coupling (Eq. H2x2) ---
//   Wc = H^cc Xc + (H^ec)^T Xe ;  We = H^ec Xc + H^ee Xe
template <typename T>
int apply_H_generic(efe_handle* h, const T* Xc, int64_t ldx, const double* Xe, int64_t ldxe, T* Wc, int64_t ldw,
                    double* We, int64_t ldwe, int N, cudaStream_t st, const T* Hc) {
  if (ldw == N) {
    CK(cudaMemsetAsync(Wc, 0, sizeof(T) * h->n_nodes * N, st));
  } else {
    if constexpr (sizeof(T) == 8) launch_zero_rows(h->n_nodes, (double*)Wc, ldw, N, st);
    else launch_zero_rows_f32(h->n_nodes, (float*)Wc, ldw, N, st);
    CKL();
  }
  TRY(cell_apply_all<T>(h, Hc, Xc, ldx, Wc, ldw, N, st));
  if constexpr (sizeof(T) == 8) {
    if (use_df(h, N)) {
      launch_df_rows(h->nE, N, Xe, ldxe, h->xe2, st);
      launch_spmm_nodes_df(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->hecT2, 1.f, h->xe2, N, (double*)Wc, ldw, st);
      launch_grp_rows_df(h->n_gitems, h->gitems, h->ec_rowptr, h->ec_col, h->hec2, (const double*)Xc, ldx, h->part,
                         N, st);
      launch_grp_reduce((int)h->nE, h->f_it0, h->f_it1, h->f_slot, h->part, N, 1.0, nullptr, 0, 0.0, We, ldwe, st);
      launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Hee, h->nE, Xe, ldxe, 1.0, We, ldwe, st);
      CKL();
      return EFE_OK;
    }
  }
  if (h->nE > 0) {
    launch_spmm_nodes<T>(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->hecT, 1.0, Xe, ldxe, Wc, ldw, N, st);
    launch_spmm_segments<T>(h->nseg, h->seg_start, h->seg_end, h->ec_col, h->hec, nullptr, Xc, ldx, h->part, N, st);
    launch_seg_reduce((int)h->nE, h->row_seg_ptr, h->part, 1.0, nullptr, 0, 0.0, We, ldwe, N, st);
    launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Hee, h->nE, Xe, ldxe, 1.0, We, ldwe, st);
    CKL();
  }
  return EFE_OK;
}

// --- block-wise inverse on W (Sec. IV.D), in place on Wc, result x_e in h->xe ---
//   r = We - M^ec D^-1 Wc ; x_e = S^-1 r ; Wc <- Wc - (M^ec)^T x_e  (D^-1 applied later)
template <typename T>
int minv_core(efe_handle* h, T* Wc, int64_t ldw, const double* We, int64_t ldwe, int N, cudaStream_t st) {
  if (h->nE == 0) return EFE_OK;
  if constexpr (sizeof(T) == 8) {
    if (use_df(h, N)) {
      launch_grp_rows_df(h->n_gitems, h->gitems, h->ec_rowptr, h->ec_col, h->mecD2, (const double*)Wc, ldw, h->part,
                         N, st);
      launch_grp_reduce((int)h->nE, h->f_it0, h->f_it1, h->f_slot, h->part, N, -1.0, We, ldwe, 1.0, h->rb, N, st);
      launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Sinv, h->nE, h->rb, N, 0.0, h->xe, N, st);
      launch_df_rows(h->nE, N, h->xe, N, h->xe2, st);
      launch_spmm_nodes_df(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->mecT2, -1.f, h->xe2, N, (double*)Wc, ldw, st);
      CKL();
      return EFE_OK;
    }
  }
  launch_spmm_segments<T>(h->nseg, h->seg_start, h->seg_end, h->ec_col, h->mec, h->Dinv, Wc, ldw, h->part, N, st);
  launch_seg_reduce((int)h->nE, h->row_seg_ptr, h->part, -1.0, We, ldwe, 1.0, h->rb, N, N, st);
  launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Sinv, h->nE, h->rb, N, 0.0, h->xe, N, st);
  launch_spmm_nodes<T>(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->mecT, -1.0, h->xe, N, Wc, ldw, N, st);
  CKL();
  return EFE_OK;
}

int apply_M_impl(efe_handle* h, const double* X, int64_t ldx, int N, double* Y, int64_t ldy, cudaStream_t st) {
  const int64_t nn = h->n_nodes;
  launch_row_scale<double>(nn, h->Dm, X, ldx, Y, ldy, N, st);
  if (h->nE > 0 && use_df(h, N)) {
    launch_df_rows(h->nE, N, X + nn * ldx, ldx, h->xe2, st);
    launch_spmm_nodes_df(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->mecT2, 1.f, h->xe2, N, Y, ldy, st);
    launch_row_scale<double>(nn, h->mask, Y, ldy, Y, ldy, N, st);
    launch_grp_rows_df(h->n_gitems, h->gitems, h->ec_rowptr, h->ec_col, h->mec2, X, ldx, h->part, N, st);
    launch_grp_reduce((int)h->nE, h->f_it0, h->f_it1, h->f_slot, h->part, N, 1.0, nullptr, 0, 0.0, Y + nn * ldy, ldy,
                      st);
    launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Mee, h->nE, X + nn * ldx, ldx, 1.0, Y + nn * ldy, ldy, st);
  } else if (h->nE > 0) {
    launch_spmm_nodes<double>(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->mecT, 1.0, X + nn * ldx, ldx, Y, ldy, N, st);
    launch_row_scale<double>(nn, h->mask, Y, ldy, Y, ldy, N, st);
    launch_spmm_segments<double>(h->nseg, h->seg_start, h->seg_end, h->ec_col, h->mec, nullptr, X, ldx, h->part, N,
                                 st);
    launch_seg_reduce((int)h->nE, h->row_seg_ptr, h->part, 1.0, nullptr, 0, 0.0, Y + nn * ldy, ldy, N, st);
    launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Mee, h->nE, X + nn * ldx, ldx, 1.0, Y + nn * ldy, ldy, st);
  }
  CKL();
  return EFE_OK;
}

int apply_H_impl(efe_handle* h, const double* X, int64_t ldx, int N, double* Y, int64_t ldy, cudaStream_t st) {
  const int64_t nn = h->n_nodes;
  TRY(apply_H_generic<double>(h, X, ldx, X + nn * ldx, ldx, Y, ldy, Y + nn * ldy, ldy, N, st, h->Hcc));
  launch_row_scale<double>(nn, h->mask, Y, ldy, Y, ldy, N, st);
  CKL();
  return EFE_OK;
}

int apply_Minv_impl(efe_handle* h, const double* X, int64_t ldx, int N, double* Y, int64_t ldy, cudaStream_t st) {
  const int64_t nn = h->n_nodes;
  // W = X copied into the workspace so the core can work in place
  launch_copy_rows(h->rows, X, ldx, h->W, N, N, st);
  TRY(minv_core<double>(h, h->W, N, h->W + nn * N, N, N, st));
  launch_row_scale<double>(nn, h->Dinv, h->W, N, Y, ldy, N, st);
  if (h->nE > 0) launch_copy_rows(h->nE, h->xe, N, Y + nn * ldy, ldy, N, st);
  CKL();
  return EFE_OK;
}

// --- one filter degree in FP64: Ynew = alpha (H~ Ycur - c Ycur) + beta Yprev ---
int degree_f64(efe_handle* h, const double* Yc, int64_t ldc, const double* Yp, int64_t ldp, double* Yn, int64_t ldn,
               const double* coef, int N, cudaStream_t st) {
  const int64_t nn = h->n_nodes;
  double* Wc = h->W;
  double* We = h->W + nn * N;
  TRY(apply_H_generic<double>(h, Yc, ldc, Yc + nn * ldc, ldc, Wc, N, We, N, N, st, h->Hcc));
  TRY(minv_core<double>(h, Wc, N, We, N, N, st));
  launch_cheb_combine<double>(nn, h->Dinv, Wc, N, Yc, ldc, Yp, ldp, Yn, ldn, coef, N, st);
  if (h->nE > 0)
    launch_cheb_combine<double>(h->nE, nullptr, h->xe, N, Yc + nn * ldc, ldc, Yp ? Yp + nn * ldp : nullptr, ldp,
                                Yn + nn * ldn, ldn, coef, N, st);
  CKL();
  return EFE_OK;
}

// C (n_E x N, ld N) = A (n_E x n_E) B (n_E x N, ld N) in FP64: the FP64-grade
// tensor-core product when that engine is on and the product is large, DFMA
// otherwise
int gemm_ee(efe_handle* h, const double* A, const double* B, double* C, int N, cudaStream_t st) {
  const int nE = (int)h->nE;
  if (h->fp64_engine == 1 && (double)nE * nE * N >= 1e9) return gemm_tall(h, nE, nE, N, A, nE, B, C, N, st);
  launch_gemm_nn(nE, N, nE, 1.0, A, nE, B, N, 0.0, C, N, st);
  CKL();
  return EFE_OK;
}

// --- one filter degree with the classical block in FP32 (enrichment rows FP64) ---
// Classical rows use the padded leading dimension ld32; the enrichment
// coupling runs node-major with FP32 products and FP64 cross-block sums.
int degree_f32(efe_handle* h, const float* Yc, const double* Yce, const float* Yp, const double* Ype, float* Yn,
               double* Yne, const double* coef, int N, cudaStream_t st) {
  const int64_t nn = h->n_nodes;
  const int ld = h->ld32;
  double* We = h->We;  // nE x N FP64 scratch (W may hold the FP32 slots)
  CK(cudaMemsetAsync(h->Wf, 0, sizeof(float) * nn * ld, st));
  h->time_this = true;
  TRY(cell_apply_all<float>(h, h->Hcc32, Yc, ld, h->Wf, ld, N, st, h->tc_mode != 0));
  h->time_this = false;
  if (h->nE > 0) {
    const int nE = (int)h->nE;
    if (coup_tiles_fit(h, N)) {
      launch_coup_cols<float>(h->n_tn, h->ncb_cols, h->cb_cta_cols, h->t_nodes, h->cb_slot_off, h->cb_slots, h->tileH, 1.f, Yce, N, nE,
                              N, h->Wf, ld, st);
      launch_coup_rows<float>(h->n_tn, h->ncb, h->cb_cta, h->t_nodes, h->cb_slot_off, h->cb_slots, h->tileH, nullptr, Yc, ld,
                              nE, N, h->cpart, st);
      launch_coup_reduce(h->ncb, nE, N, h->cpart, 1.0, nullptr, 0, 0.0, We, N, st);
      launch_gemm_nn(nE, N, nE, 1.0, h->Hee, nE, Yce, N, 1.0, We, N, st);
      // block-wise inverse: r = We - M^ec D^-1 Wc, x_e = S^-1 r, Wc -= M^ec^T x_e
      launch_coup_rows<float>(h->n_tn, h->ncb, h->cb_cta, h->t_nodes, h->cb_slot_off, h->cb_slots, h->tileM, h->Dinv, h->Wf,
                              ld, nE, N, h->cpart, st);
      launch_coup_reduce(h->ncb, nE, N, h->cpart, -1.0, We, N, 1.0, h->rb, N, st);
      launch_gemm_nn(nE, N, nE, 1.0, h->Sinv, nE, h->rb, N, 0.0, h->xe, N, st);
      launch_coup_cols<float>(h->n_tn, h->ncb_cols, h->cb_cta_cols, h->t_nodes, h->cb_slot_off, h->cb_slots, h->tileM, -1.f, h->xe, N,
                              nE, N, h->Wf, ld, st);
    } else {
      // many enrichment functions: node-major FP32 columns products, grouped
      // FP32 rows products with FP64 partial sums, FP64 n_E x n_E products
      const int64_t nE64 = h->nE;
      launch_f64_to_f32_rows(nE64, Yce, N, h->Xe32, N, N, st);
      auto cols = [&](const float* tile, const float* valT, float sgn) {
        if (h->opt_coup_cols)
          launch_coup_cols_sparse(h->n_tn, h->t_nodes, h->t_ptr, h->t_slot, valT, h->cb_slot_off, h->cb_slots, sgn,
                                  h->Xe32, N, N, h->Wf, ld, st);
        else
          launch_coup_cols_chunk(h->n_tn, h->t_nodes, h->cb_slot_off, h->cb_slots, tile, sgn, h->Xe32, N, N, h->Wf, ld,
                                 st);
      };
      cols(h->tileH, h->hecT32, 1.f);
      TRY(gemm_ee(h, h->Hee, Yce, h->rb, N, st));                       // H^ee Y_e
      launch_grp_rows(h->n_gitems, h->gitems, h->ec_rowptr, h->ec_col, h->hec32, Yc, ld, h->gpart, N, st);
      launch_grp_reduce(nE, h->f_it0, h->f_it1, h->f_slot, h->gpart, N, 1.0, h->rb, N, 1.0, We, N, st);
      // block-wise inverse: r = We - M^ec D^-1 Wc, x_e = S^-1 r, Wc -= M^ec^T x_e
      launch_grp_rows(h->n_gitems, h->gitems, h->ec_rowptr, h->ec_col, h->mecD32, h->Wf, ld, h->gpart, N, st);
      launch_grp_reduce(nE, h->f_it0, h->f_it1, h->f_slot, h->gpart, N, -1.0, We, N, 1.0, h->rb, N, st);
      TRY(gemm_ee(h, h->Sinv, h->rb, h->xe, N, st));
      launch_f64_to_f32_rows(nE64, h->xe, N, h->Xe32, N, N, st);
      cols(h->tileM, h->mecT32, -1.f);
      CKL();
    }
  }
  launch_cheb_combine_f4(nn, ld, h->Dinv, h->Wf, Yc, Yp, Yn, coef, st);
  if (h->nE > 0) launch_cheb_combine<double>(h->nE, nullptr, h->xe, N, Yce, N, Ype, N, Yne, N, coef, N, st);
  CKL();
  return EFE_OK;
}

bool is_finite_d(double x) { return std::isfinite(x); }

// tiny host symmetric tridiagonal eigenvalues (Jacobi on a dense copy, k <= 64)
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int k = (int)a.size();
  std::vector<double> A((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) {
    A[(size_t)i * k + i] = a[i];
    if (i + 1 < k) A[(size_t)i * k + i + 1] = A[(size_t)(i + 1) * k + i] = b[i];
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
    if (off < 1e-30) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[(size_t)p * k + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * k + q] - A[(size_t)p * k + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int i = 0; i < k; ++i) {
          const double aip = A[(size_t)i * k + p], aiq = A[(size_t)i * k + q];
          A[(size_t)i * k + p] = c * aip - s * aiq;
          A[(size_t)i * k + q] = s * aip + c * aiq;
        }
        for (int j = 0; j < k; ++j) {
          const double apj = A[(size_t)p * k + j], aqj = A[(size_t)q * k + j];
          A[(size_t)p * k + j] = c * apj - s * aqj;
          A[(size_t)q * k + j] = s * apj + c * aqj;
        }
      }
  }
  double mx = -INFINITY;
  for (int i = 0; i < k; ++i) mx = std::max(mx, A[(size_t)i * k + i]);
  return mx;
}


// Symmetric eigenproblem A = W diag(w) W^T by cyclic Jacobi rotations (A row-major
// n x n, destroyed; W row-major, eigenvectors in columns).
void host_jacobi_eig(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& W) {
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) W[(size_t)i * n + i] = 1.0;
  double norm2 = 0.0;
  for (double v : A) norm2 += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off <= 1e-34 * norm2) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
        A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double wkp = W[(size_t)k * n + p], wkq = W[(size_t)k * n + q];
          W[(size_t)k * n + p] = c * wkp - sn * wkq;
          W[(size_t)k * n + q] = sn * wkp + c * wkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Fast-diagonalisation data of axis d: the interior blocks K_ii, M_ii of the
// assembled 1-D stiffness and mass give K V = M V diag(lam) with V^T M V = I
// (M = L L^T, C = L^-1 K L^-T = W diag(lam) W^T, V = L^-T W).
int fd_axis(efe_handle* h, int d, int nn, const std::vector<double>& Kb, const std::vector<double>& Mb) {
  const int m = nn - 2;
  if (m < 1) return EFE_OK;
  std::vector<double> K((size_t)m * m, 0.0), L((size_t)m * m, 0.0);
  for (int a = 0; a < m; ++a)
    for (int o = 0; o < 9; ++o) {
      const int b = a + o - 4;
      if (b < 0 || b >= m) continue;
      K[(size_t)a * m + b] = Kb[(size_t)(a + 1) * 9 + o];
      L[(size_t)a * m + b] = Mb[(size_t)(a + 1) * 9 + o];
    }
  if (host_cholesky_lower(L.data(), m) != 0) {
    h->err = "1-D mass matrix not positive definite";
    return EFE_ERR_CHOL;
  }
  for (int a = 0; a < m; ++a)
    for (int b = a + 1; b < m; ++b) L[(size_t)a * m + b] = 0.0;
  // Y = L^-1 K (columns by forward substitution), C = L^-1 Y^T  (= L^-1 K L^-T, K symmetric)
  auto fwd = [&](std::vector<double>& X) {
    for (int c = 0; c < m; ++c)
      for (int a = 0; a < m; ++a) {
        double v = X[(size_t)a * m + c];
        for (int k = 0; k < a; ++k) v -= L[(size_t)a * m + k] * X[(size_t)k * m + c];
        X[(size_t)a * m + c] = v / L[(size_t)a * m + a];
      }
  };
  fwd(K);
  std::vector<double> C((size_t)m * m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) C[(size_t)a * m + b] = K[(size_t)b * m + a];
  fwd(C);
  for (int a = 0; a < m; ++a)
    for (int b = a + 1; b < m; ++b) {
      const double v = 0.5 * (C[(size_t)a * m + b] + C[(size_t)b * m + a]);
      C[(size_t)a * m + b] = C[(size_t)b * m + a] = v;
    }
  std::vector<double> lam, W;
  host_jacobi_eig(C, m, lam, W);
  // V = L^-T W (back substitution, column by column)
  for (int c = 0; c < m; ++c)
    for (int a = m - 1; a >= 0; --a) {
      double v = W[(size_t)a * m + c];
      for (int k = a + 1; k < m; ++k) v -= L[(size_t)k * m + a] * W[(size_t)k * m + c];
      W[(size_t)a * m + c] = v / L[(size_t)a * m + a];
    }
  std::vector<double> Wt((size_t)m * m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) Wt[(size_t)b * m + a] = W[(size_t)a * m + b];
  TRY(upload(h, &h->fdV[d], W));
  TRY(upload(h, &h->fdVt[d], Wt));
  TRY(upload(h, &h->fdlam[d], lam));
  return EFE_OK;
}

// Quadrature leaves, enrichment-value offsets, the assembled 1-D operators of
// the Hartree stiffness and the node coordinates (self-consistent field).
int scf_setup_upload(efe_handle* h, const Setup& s) {
  h->n_leaf = (int64_t)s.leaf_n.size();
  for (int32_t n : s.leaf_n) h->leaf_nmax = std::max(h->leaf_nmax, (int)n);
  TRY(upload(h, &h->leaf_off, s.leaf_off));
  TRY(upload(h, &h->leaf_ptr, s.leaf_ptr));
  TRY(upload(h, &h->leaf_n, s.leaf_n));
  TRY(upload(h, &h->leaf_cell, s.leaf_cell));
  TRY(upload(h, &h->cell_enr, s.cell_enr));
  {
    std::vector<int64_t> eo(s.enr_cells.size() + 1, 0);
    for (size_t ei = 0; ei < s.enr_cells.size(); ++ei) {
      const int64_t e = s.enr_cells[ei];
      eo[ei + 1] = eo[ei] + (s.qoff[e + 1] - s.qoff[e]) * (int64_t)(s.cf_ptr[ei + 1] - s.cf_ptr[ei]);
    }
    h->eq_elems = eo.back();
    TRY(upload(h, &h->eq_off, eo));
  }
  // K_d = sum_cells (2/h) K1, M_d = sum_cells (h/2) M1 on the nodes of axis d,
  // stored as 9-entry bands (column offsets -4 .. 4)
  std::vector<double> xyz;
  for (int d = 0; d < 3; ++d) {
    const int nn = s.nn[d];
    std::vector<double> K((size_t)nn * 9, 0.0), M((size_t)nn * 9, 0.0);
    for (int c = 0; c < s.nc[d]; ++c) {
      const double hc = s.brk[d][c + 1] - s.brk[d][c];
      for (int a = 0; a < NP1; ++a)
        for (int b = 0; b < NP1; ++b) {
          const size_t idx = (size_t)(P * c + a) * 9 + (b - a + 4);
          K[idx] += (2.0 / hc) * s.K1[a * NP1 + b];
          M[idx] += (hc / 2.0) * s.M1[a * NP1 + b];
        }
    }
    TRY(upload(h, &h->band[d], K));
    TRY(upload(h, &h->band[3 + d], M));
    TRY(fd_axis(h, d, nn, K, M));
    xyz.push_back(s.brk[d][0]);
    for (int c = 0; c < s.nc[d]; ++c) {
      const double lo = s.brk[d][c], hc = s.brk[d][c + 1] - s.brk[d][c];
      for (int a = 1; a < NP1; ++a) xyz.push_back(lo + 0.5 * (s.gll_z[a] + 1.0) * hc);
    }
  }
  TRY(upload(h, &h->node_xyz, xyz));
  // nuclear repulsion E_ZZ
  h->e_zz = 0.0;
  const int na = (int)s.atom_Z.size();
  for (int a = 0; a < na; ++a)
    for (int b = a + 1; b < na; ++b) {
      double d2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double t = s.atom_xyz[3 * a + d] - s.atom_xyz[3 * b + d];
        d2 += t * t;
      }
      h->e_zz += s.atom_Z[a] * s.atom_Z[b] / sqrt(d2);
    }
  return EFE_OK;
}

LeafDev leaf_dev(const efe_handle* h) {
  return LeafDev{h->leaf_off, h->leaf_n, h->leaf_cell, h->qpts, h->leaf_nmax};
}

BandsDev bands_dev(const efe_handle* h) {
  BandsDev b;
  for (int d = 0; d < 3; ++d) {
    b.K[d] = h->band[d];
    b.M[d] = h->band[3 + d];
    b.nn[d] = h->mesh.nn[d];
  }
  return b;
}

// enrichment values at the enriched cells' points, computed on first use
int ensure_eq(efe_handle* h, cudaStream_t st) {
  if (h->Eq || h->nE == 0) return EFE_OK;
  TRY(dalloc(h, &h->Eq, h->eq_elems));
  EnrDev en{h->cell_enr, h->cf_ptr, h->cf_idx, h->qoff, h->eq_off, h->Eq, h->n_nodes};
  launch_enr_values(en, h->enr_cells, h->qoff, h->qpts, h->funcs, h->n_enr, st);
  CKL();
  return EFE_OK;
}

EnrDev enr_dev(const efe_handle* h) {
  if (h->nE == 0) return EnrDev{nullptr, nullptr, nullptr, h->qoff, nullptr, nullptr, h->n_nodes};
  return EnrDev{h->cell_enr, h->cf_ptr, h->cf_idx, h->qoff, h->eq_off, h->Eq, h->n_nodes};
}

// Hartree work buffers (allocated once)
int hartree_alloc(efe_handle* h) {
  if (h->hb) return EFE_OK;
  const int64_t nn = h->n_nodes;
  const int64_t nt = stiff_tiles(bands_dev(h));
  const int64_t nint = std::max<int64_t>(1, (int64_t)(h->mesh.nn[0] - 2) * (h->mesh.nn[1] - 2) * (h->mesh.nn[2] - 2));
  TRY(dalloc(h, &h->hb, nn));
  TRY(dalloc(h, &h->hr64, nn));
  TRY(dalloc(h, &h->hphi, nn));
  TRY(dalloc(h, &h->hlb, std::max<int64_t>(1, h->n_leaf) * NL));
  TRY(dalloc(h, &h->hpart_rr, nt));
  TRY(dalloc(h, &h->fdU0, nint));
  TRY(dalloc(h, &h->fdU1, nint));
  TRY(dalloc(h, &h->red_part, 64 * (int64_t)reduce_blocks()));
  TRY(dalloc(h, &h->red_out, 64));
  CK(cudaMemset(h->hphi, 0, sizeof(double) * nn));
  return EFE_OK;
}

// -lap phi / (4 pi) = rho with multipole Dirichlet data: load vector, boundary
// values, then defect correction phi += A_ii^-1 (b - A phi)_i with the exact
// fast-diagonalisation solve (one correction reaches rounding level; a second
// runs only if the FP64 residual is still above tol).
int hartree_solve(efe_handle* h, const double* rho, double* vh, double* phi, double tol, int max_corr, int* iters,
                  double* relres, cudaStream_t st) {
  TRY(hartree_alloc(h));
  const int64_t nn = h->n_nodes;
  const LeafDev lf = leaf_dev(h);
  const BandsDev bd = bands_dev(h);
  const int64_t nt = stiff_tiles(bd);
  launch_hartree_load(lf, h->n_leaf, h->mesh, h->re, h->leaf_ptr, rho, h->mask, nn, h->hlb, h->hb, st);
  launch_moments(h->qpts, rho, h->nq, h->red_part, h->red_out, st);
  launch_hartree_bc(h->mesh, h->node_xyz, h->mask, h->red_out, nn, phi, st);
  launch_dot(nn, h->hb, h->hb, h->red_part, h->red_out + 8, st);
  CKL();
  double bb = 0.0;
  CK(cudaMemcpyAsync(&bb, h->red_out + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double* V[3] = {h->fdV[0], h->fdV[1], h->fdV[2]};
  const double* Vt[3] = {h->fdVt[0], h->fdVt[1], h->fdVt[2]};
  const double* lam[3] = {h->fdlam[0], h->fdlam[1], h->fdlam[2]};
  int corr = 0;
  double rr = 0.0;
  for (;;) {
    if (launch_stiff_resid(bd, phi, h->hb, h->mask, h->hr64, h->hpart_rr, st)) {
      h->err = "Hartree residual kernel: shared-memory configuration failed";
      return EFE_ERR_CUDA;
    }
    launch_finish(h->hpart_rr, (int)nt, 1, h->red_out + 9, st);
    CKL();
    CK(cudaMemcpyAsync(&rr, h->red_out + 9, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!std::isfinite(rr)) {
      h->err = "non-finite Hartree residual";
      return EFE_ERR_NAN;
    }
    if (rr <= tol * tol * bb || corr >= max_corr) break;
    launch_fd_solve(bd, V, Vt, lam, h->hr64, h->fdU0, h->fdU1, phi, st);
    CKL();
    ++corr;
  }
  if (relres) *relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  if (iters) *iters = corr;
  launch_leaf_interp(lf, h->n_leaf, h->mesh, h->re, phi, vh, st);
  CKL();
  if (bb > 0.0 && rr > 1e6 * tol * tol * bb) {
    h->err = "Hartree solve did not reach the requested residual";
    return EFE_ERR_NOCONV;
  }
  return EFE_OK;
}

// host: occupations by bisection on mu (same steps as the electron-count condition)
int fermi_host(const double* eps, int N, double ne, double kT, double* occ, double* mu_out) {
  if (N < 1 || !(kT > 0.0) || !(ne >= 0.0)) return EFE_ERR_ARG;
  double emin = eps[0], emax = eps[0];
  for (int i = 1; i < N; ++i) {
    emin = std::min(emin, eps[i]);
    emax = std::max(emax, eps[i]);
  }
  auto count = [&](double mu) {
    double c = 0.0;
    for (int i = 0; i < N; ++i) {
      const double x = std::min(700.0, std::max(-700.0, (eps[i] - mu) / kT));
      c += 1.0 / (1.0 + exp(x));
    }
    return 2.0 * c;
  };
  double lo = emin - 50.0 * kT - 1.0, hi = emax + 50.0 * kT + 1.0;
  if (count(hi) < ne) return EFE_ERR_ARG;
  for (int k = 0; k < 400; ++k) {
    const double mid = 0.5 * (lo + hi);
    if (count(mid) < ne) lo = mid; else hi = mid;
    if (hi - lo < 1e-14) break;
  }
  const double mu = 0.5 * (lo + hi);
  for (int i = 0; i < N; ++i) {
    const double x = std::min(700.0, std::max(-700.0, (eps[i] - mu) / kT));
    occ[i] = 1.0 / (1.0 + exp(x));
  }
  if (mu_out) *mu_out = mu;
  return EFE_OK;
}

// Anderson: weighted Gram of the residual differences on the device, the
// (n-1) x (n-1) system on the host (Gaussian elimination with partial pivoting;
// a pivot below 1e-14 of the largest diagonal drops that stage), then the mix.
int anderson_apply(efe_handle* h, const HistDev& hs, double beta, double* out, cudaStream_t st) {
  const int n = hs.n, m = n - 1;
  AndersonCoef th;
  for (int k = 0; k < ANDERSON_MAX; ++k) th.t[k] = 0.0;
  if (m > 0) {
    const int nv = anderson_values(n);
    launch_anderson_gram(h->qpts, h->nq, hs, h->red_part, h->red_out, st);
    CKL();
    double v[64];
    CK(cudaMemcpyAsync(v, h->red_out, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double A[ANDERSON_MAX][ANDERSON_MAX + 1];
    int c = 0;
    for (int k = 0; k < m; ++k)
      for (int l = k; l < m; ++l) A[k][l] = A[l][k] = v[c++];
    for (int k = 0; k < m; ++k) A[k][m] = v[c++];
    double dmax = 0.0;
    for (int k = 0; k < m; ++k) dmax = std::max(dmax, fabs(A[k][k]));
    bool use[ANDERSON_MAX];
    for (int k = 0; k < m; ++k) use[k] = true;
    for (int col = 0; col < m; ++col) {
      int piv = -1;
      double best = 0.0;
      for (int r = col; r < m; ++r)
        if (fabs(A[r][col]) > best) { best = fabs(A[r][col]); piv = r; }
      if (piv < 0 || best <= 1e-14 * dmax) { use[col] = false; continue; }
      if (piv != col)
        for (int j = 0; j <= m; ++j) std::swap(A[piv][j], A[col][j]);
      for (int r = col + 1; r < m; ++r) {
        const double f = A[r][col] / A[col][col];
        for (int j = col; j <= m; ++j) A[r][j] -= f * A[col][j];
      }
    }
    for (int col = m - 1; col >= 0; --col) {
      if (!use[col]) { th.t[col] = 0.0; continue; }
      double sv = A[col][m];
      for (int j = col + 1; j < m; ++j) sv -= A[col][j] * th.t[j];
      th.t[col] = sv / A[col][col];
    }
  }
  launch_anderson_mix(h->nq, hs, th, beta, out, st);
  CKL();
  return EFE_OK;
}

// device address of the allocation-free entry point's static scratch (defined
// with that entry point below)
int noalloc_scratch(efe_handle* h, int dev, double** out);

}  // namespace

extern "C" {

int efe_create(const efe_mesh_desc* mesh, const efe_atoms_desc* atoms, const efe_basis_desc* basis,
               efe_handle** out) {
  if (!out) return EFE_ERR_ARG;
  *out = nullptr;
  efe_handle* h = new (std::nothrow) efe_handle();
  if (!h) return EFE_ERR_ALLOC;
  *out = h;
  CK(cudaGetDevice(&h->dev));
  {
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev));
    h->n_sm = nsm > 0 ? nsm : 148;
  }
  // map this library's device module and look up the static scratch of
  // efe_apply_M_noalloc now, so that the entry point itself never loads a
  // module or allocates
  TRY(noalloc_scratch(h, h->dev, &h->noalloc_part));
  Setup s;
  int rc;
  try {
    rc = build_setup(mesh, atoms, basis, s);
  } catch (...) {
    h->err = "host allocation failed during set-up";
    return EFE_ERR_ALLOC;
  }
  if (rc != EFE_OK) {
    h->err = s.err;
    return rc;
  }
  h->n_nodes = s.n_nodes;
  h->n_cell = s.n_cell;
  h->nE = s.nE;
  h->nq = s.n_q;
  h->rows = s.n_nodes + s.nE;
  h->n_enr = (int64_t)s.enr_cells.size();
  std::memcpy(h->re.z, s.gll_z, sizeof(h->re.z));
  std::memcpy(h->re.w, s.gll_w, sizeof(h->re.w));
  std::memcpy(h->re.M1, s.M1, sizeof(h->re.M1));
  std::memcpy(h->re.K1, s.K1, sizeof(h->re.K1));
  for (int d = 0; d < 3; ++d) {
    h->mesh.nc[d] = s.nc[d];
    h->mesh.nn[d] = s.nn[d];
  }
  std::vector<double> brk;
  for (int d = 0; d < 3; ++d) brk.insert(brk.end(), s.brk[d].begin(), s.brk[d].end());
  TRY(upload(h, &h->brk, brk));
  h->mesh.brk = h->brk;
  h->n_atoms = (int)s.atom_Z.size();
  TRY(upload(h, &h->axyz, s.atom_xyz));
  TRY(upload(h, &h->aZ, s.atom_Z));
  TRY(upload(h, &h->qpts, s.qpts));
  TRY(upload(h, &h->qoff, s.qoff));
  TRY(scf_setup_upload(h, s));
  TRY(dalloc(h, &h->V, h->nq));
  // parity colours of the cells
  {
    std::vector<int32_t> cc;
    h->colour_off[0] = 0;
    for (int c = 0; c < 8; ++c) {
      for (int64_t e = 0; e < s.n_cell; ++e) {
        const int i = (int)(e % s.nc[0]), j = (int)((e / s.nc[0]) % s.nc[1]),
                  k = (int)(e / ((int64_t)s.nc[0] * s.nc[1]));
        if ((i & 1) + 2 * (j & 1) + 4 * (k & 1) == c) cc.push_back((int32_t)e);
      }
      h->colour_off[c + 1] = (int64_t)cc.size();
    }
    TRY(upload(h, &h->colour_cells, cc));
  }
  TRY(upload(h, &h->D, s.D));
  TRY(upload(h, &h->Dinv, s.Dinv));
  {
    std::vector<double> mask(s.n_nodes), Dm(s.n_nodes);
    for (int64_t g = 0; g < s.n_nodes; ++g) {
      mask[g] = s.Dinv[g] != 0.0 ? 1.0 : 0.0;
      Dm[g] = mask[g] * s.D[g];
    }
    TRY(upload(h, &h->mask, mask));
    TRY(upload(h, &h->Dm, Dm));
  }
  TRY(dalloc(h, &h->Hcc, h->n_cell * NL * NL));
  TRY(dalloc(h, &h->Hcc32, h->n_cell * NL * NL));
  TRY(dalloc(h, &h->hexp, oz_hexp_elems(h->n_cell)));
  TRY(dalloc(h, &h->oz_aexp, h->rows));
  TRY(dalloc(h, &h->Aimg32, tc3_image_elems(h->n_cell)));
  TRY(dalloc(h, &h->info, 8));
  TRY(dalloc(h, &h->chol_ratio, 1));
  if (h->nE > 0) {
    TRY(upload(h, &h->funcs, s.funcs));
    TRY(upload(h, &h->enr_cells, s.enr_cells));
    TRY(upload(h, &h->cf_ptr, s.cf_ptr));
    TRY(upload(h, &h->cf_idx, s.cf_idx));
    for (int64_t ei = 0; ei < h->n_enr; ++ei) h->kmax = std::max(h->kmax, s.cf_ptr[ei + 1] - s.cf_ptr[ei]);
    if (h->kmax > 64) {
      h->err = "more than 64 enrichment functions meet one cell";
      return EFE_ERR_ARG;
    }
    TRY(upload(h, &h->blkP_off, s.blkP_off));
    TRY(upload(h, &h->blkQ_off, s.blkQ_off));
    h->nP = s.blkP_off.back();
    h->nQ = s.blkQ_off.back();
    TRY(dalloc(h, &h->Pblk, h->nP));
    TRY(dalloc(h, &h->Qblk, h->nQ));
    h->nnz = (int64_t)s.ec_col.size();
    TRY(upload(h, &h->ec_col, s.ec_col));
    TRY(upload(h, &h->mec, s.mec_val));
    TRY(upload(h, &h->hec_kin, s.hec_kin));
    TRY(dalloc(h, &h->hec, h->nnz));
    TRY(upload(h, &h->ec_cptr, s.ec_contrib_ptr));
    TRY(upload(h, &h->ec_cidx, s.ec_contrib_idx));
    // segments of the long rows
    std::vector<int64_t> ss, se, rsp(1, 0);
    for (int a = 0; a < s.nE; ++a) {
      for (int64_t q = s.ec_ptr[a]; q < s.ec_ptr[a + 1]; q += SEG) {
        ss.push_back(q);
        se.push_back(std::min(q + SEG, s.ec_ptr[a + 1]));
      }
      rsp.push_back((int64_t)ss.size());
    }
    h->nseg = (int64_t)ss.size();
    TRY(upload(h, &h->seg_start, ss));
    TRY(upload(h, &h->seg_end, se));
    TRY(upload(h, &h->row_seg_ptr, rsp));
    {
      // function groups sharing one support: consecutive functions of one atom
      // with one cutoff and identical row patterns (at most grp_kmax() each),
      // cut into items of GRP_SEG nodes for the many-function mixed coupling
      constexpr int GRP_SEG = 1024;
      std::vector<int4> items;
      std::vector<int32_t> it0(s.nE), it1(s.nE), slot(s.nE);
      int a = 0;
      while (a < s.nE) {
        const int64_t len = s.ec_ptr[a + 1] - s.ec_ptr[a];
        int kg = 1;
        while (a + kg < s.nE && kg < grp_kmax()) {
          const int b = a + kg;
          const bool same = s.funcs[b].Rx == s.funcs[a].Rx && s.funcs[b].Ry == s.funcs[a].Ry &&
                            s.funcs[b].Rz == s.funcs[a].Rz && s.funcs[b].r0 == s.funcs[a].r0 &&
                            s.funcs[b].t == s.funcs[a].t && s.ec_ptr[b + 1] - s.ec_ptr[b] == len &&
                            std::equal(s.ec_col.begin() + s.ec_ptr[a], s.ec_col.begin() + s.ec_ptr[a + 1],
                                       s.ec_col.begin() + s.ec_ptr[b]);
          if (!same) break;
          ++kg;
        }
        const int first = (int)items.size();
        for (int64_t j = 0; j < len; j += GRP_SEG)
          items.push_back(make_int4(a, kg, (int)j, (int)std::min<int64_t>(len, j + GRP_SEG)));
        for (int k = 0; k < kg; ++k) {
          it0[a + k] = first;
          it1[a + k] = (int)items.size();
          slot[a + k] = k;
        }
        a += kg;
      }
      h->n_gitems = (int)items.size();
      TRY(upload(h, &h->gitems, items));
      TRY(upload(h, &h->f_it0, it0));
      TRY(upload(h, &h->f_it1, it1));
      TRY(upload(h, &h->f_slot, slot));
      TRY(upload(h, &h->ec_rowptr, s.ec_ptr));
      std::vector<float> md(s.ec_col.size());
      for (size_t q = 0; q < md.size(); ++q) md[q] = (float)(s.mec_val[q] * s.Dinv[s.ec_col[q]]);
      TRY(upload(h, &h->mecD32, md));
    }
    h->n_tn = (int64_t)s.t_nodes.size();
    TRY(upload(h, &h->t_nodes, s.t_nodes));
    TRY(upload(h, &h->t_ptr, s.t_ptr));
    TRY(upload(h, &h->t_col, s.t_col));
    TRY(upload(h, &h->t_perm, s.t_perm));
    TRY(dalloc(h, &h->mecT, h->nnz));
    TRY(dalloc(h, &h->hecT, h->nnz));
    TRY(dalloc(h, &h->mecT32, h->nnz));
    TRY(dalloc(h, &h->hecT32, h->nnz));
    TRY(dalloc(h, &h->hec32, h->nnz));
    launch_permute(h->nnz, h->mec, h->t_perm, h->mecT, 0);
    launch_to_f32(h->mecT, h->mecT32, h->nnz, 0);
    TRY(dalloc(h, &h->mec2, h->nnz));
    TRY(dalloc(h, &h->mecD2, h->nnz));
    TRY(dalloc(h, &h->mecT2, h->nnz));
    TRY(dalloc(h, &h->hec2, h->nnz));
    TRY(dalloc(h, &h->hecT2, h->nnz));
    launch_df_coef(h->nnz, h->mec, nullptr, nullptr, h->mec2, 0);
    launch_df_coef(h->nnz, h->mec, h->Dinv, h->ec_col, h->mecD2, 0);
    launch_df_coef(h->nnz, h->mecT, nullptr, nullptr, h->mecT2, 0);
    CKL();
    {
      // blocks of consecutive pattern nodes: their function slots and the tile
      // position of every pattern entry
      const int B = coup_block_nodes();
      const int64_t nblk = (h->n_tn + B - 1) / B;
      std::vector<int64_t> soff(nblk + 1, 0), pos(h->nnz);
      std::vector<int32_t> slots, tslot(h->nnz);
      std::vector<int32_t> fs;
      for (int64_t b = 0; b < nblk; ++b) {
        const int64_t r0 = b * B, r1 = std::min<int64_t>(h->n_tn, r0 + B);
        fs.assign(s.t_col.begin() + s.t_ptr[r0], s.t_col.begin() + s.t_ptr[r1]);
        std::sort(fs.begin(), fs.end());
        fs.erase(std::unique(fs.begin(), fs.end()), fs.end());
        for (int64_t r = r0; r < r1; ++r)
          for (int64_t q = s.t_ptr[r]; q < s.t_ptr[r + 1]; ++q) {
            const int64_t k = std::lower_bound(fs.begin(), fs.end(), s.t_col[q]) - fs.begin();
            pos[q] = (soff[b] + k) * B + (r - r0);
            tslot[q] = (int32_t)k;
          }
        slots.insert(slots.end(), fs.begin(), fs.end());
        soff[b + 1] = soff[b] + (int64_t)fs.size();
      }
      h->cb_nblk = nblk;
      h->cb_nslots = soff[nblk];
      TRY(upload(h, &h->cb_slot_off, soff));
      h->cb_soff_host = soff;
      TRY(upload(h, &h->cb_slots, slots));
      TRY(upload(h, &h->cb_pos, pos));
      TRY(upload(h, &h->t_slot, tslot));
      TRY(dalloc(h, &h->tileM, h->cb_nslots * B));
      TRY(dalloc(h, &h->tileH, h->cb_nslots * B));
      CK(cudaMemset(h->tileM, 0, sizeof(float) * h->cb_nslots * B));
      CK(cudaMemset(h->tileH, 0, sizeof(float) * h->cb_nslots * B));
      launch_tile_scatter(h->nnz, h->cb_pos, h->mecT32, h->tileM, 0);
      CKL();
    }
    TRY(upload(h, &h->Mee, s.Mee));
    TRY(upload(h, &h->Hee_kin, s.Hee_kin));
    TRY(dalloc(h, &h->Hee, h->nE * h->nE));
    TRY(upload(h, &h->Sinv, s.Sinv));
    TRY(upload(h, &h->ee_cptr, s.ee_contrib_ptr));
    TRY(upload(h, &h->ee_cidx, s.ee_contrib_idx));
  }
  CK(cudaDeviceSynchronize());
  return EFE_OK;
}

int efe_destroy(efe_handle* h) {
  if (!h) return EFE_OK;
  cudaSetDevice(h->dev);
  if (h->coef_ev) cudaEventSynchronize(h->coef_ev);
  if (h->coefh) cudaFreeHost(h->coefh);
  if (h->coef_ev) cudaEventDestroy(h->coef_ev);
  for (void* p : h->allocs) cudaFree(p);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return EFE_OK;
}

const char* efe_last_error(const efe_handle* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

int efe_sizes(const efe_handle* h, int64_t* n_nodes, int64_t* n_enrich, int64_t* n_qpoints, int64_t* n_cells,
              int64_t* n_coupling) {
  if (!h) return EFE_ERR_ARG;
  if (n_coupling) *n_coupling = h->nnz;
  if (n_nodes) *n_nodes = h->n_nodes;
  if (n_enrich) *n_enrich = h->nE;
  if (n_qpoints) *n_qpoints = h->nq;
  if (n_cells) *n_cells = h->n_cell;
  return EFE_OK;
}

int efe_qpoints(efe_handle* h, double* xyzw, void* stream) {
  if (!h || !xyzw) return EFE_ERR_ARG;
  TRY(set_dev(h));
  CK(cudaMemcpyAsync(xyzw, h->qpts, sizeof(double) * 4 * h->nq, cudaMemcpyDeviceToDevice, S(stream)));
  return EFE_OK;
}

int efe_set_potential(efe_handle* h, const double* Vq, void* stream) {
  if (!h || !Vq) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  if (Vq != h->V) CK(cudaMemcpyAsync(h->V, Vq, sizeof(double) * h->nq, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(h->info, 0, sizeof(int), st));
  launch_check_finite(h->V, h->nq, h->info, st);
  CKL();
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, h->info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) {
    h->err = "non-finite potential value";
    return EFE_ERR_NAN;
  }
  if (launch_hcc_sf(h->re, h->mesh, leaf_dev(h), h->leaf_ptr, h->V, h->n_cell, h->Hcc, st)) {
    h->err = "cell-matrix kernel: shared-memory configuration failed";
    return EFE_ERR_CUDA;
  }
  CKL();
  if (h->nE > 0) {
    TRY(ensure_eq(h, st));
    if (launch_enr_sf(h->re, h->mesh, leaf_dev(h), h->leaf_ptr, enr_dev(h), h->enr_cells, h->n_enr, h->V,
                      h->blkP_off, h->blkQ_off, h->Pblk, h->Qblk, st)) {
      h->err = "enrichment-block kernel: shared-memory configuration failed";
      return EFE_ERR_CUDA;
    }
    CKL();
    launch_gather_sum(h->nnz, h->hec_kin, h->ec_cptr, h->ec_cidx, h->Pblk, h->hec, st);
    launch_permute(h->nnz, h->hec, h->t_perm, h->hecT, st);
    launch_to_f32(h->hecT, h->hecT32, h->nnz, st);
    launch_to_f32(h->hec, h->hec32, h->nnz, st);
    launch_df_coef(h->nnz, h->hec, nullptr, nullptr, h->hec2, st);
    launch_df_coef(h->nnz, h->hecT, nullptr, nullptr, h->hecT2, st);
    launch_tile_scatter(h->nnz, h->cb_pos, h->hecT32, h->tileH, st);
    launch_gather_sum(h->nE * h->nE, h->Hee_kin, h->ee_cptr, h->ee_cidx, h->Qblk, h->Hee, st);
    launch_symmetrize(h->Hee, (int)h->nE, (int)h->nE, st);
    CKL();
  }
  launch_to_f32(h->Hcc, h->Hcc32, h->n_cell * NL * NL, st);
  launch_build_aimg(h->Hcc, h->n_cell, h->Aimg32, st);
  launch_oz_hexp(h->Hcc, h->n_cell, h->hexp, st);
  CKL();
  h->oz_aimg_valid = false;   // the digit images follow H^cc_e (remade on first use)
  h->potential_set = true;
  return EFE_OK;
}

int efe_set_potential_analytic(efe_handle* h, const efe_potential_desc* pot, void* stream) {
  if (!h || !pot || pot->n_terms < 0) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  double *dA = nullptr, *ds = nullptr, *dc = nullptr;
  const int nt = pot->n_terms;
  if (nt > 0) {
    TRY(dalloc(h, &dA, nt));
    TRY(dalloc(h, &ds, nt));
    TRY(dalloc(h, &dc, 3 * nt));
    CK(cudaMemcpy(dA, pot->A, sizeof(double) * nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ds, pot->s, sizeof(double) * nt, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dc, pot->c, sizeof(double) * 3 * nt, cudaMemcpyHostToDevice));
  }
  launch_potential_analytic(h->qpts, h->nq, h->axyz, h->aZ, h->n_atoms, pot->nuclear, dA, ds, dc,
                            nt, pot->omega, h->V, st);
  CKL();
  int rc = efe_set_potential(h, h->V, stream);
  CK(cudaStreamSynchronize(st));
  dfree(h, dA);
  dfree(h, ds);
  dfree(h, dc);
  return rc;
}

int efe_reserve(efe_handle* h, int32_t N) {
  if (!h || N < 1) return EFE_ERR_ARG;
  TRY(set_dev(h));
  return reserve(h, N);
}

static int check_block(efe_handle* h, const void* X, int64_t ldx, int N) {
  if (!X || N < 1 || ldx < N) {
    h->err = "bad block argument (null pointer, N < 1 or ld < N)";
    return EFE_ERR_ARG;
  }
  if (!h->potential_set) {
    h->err = "no potential set (call efe_set_potential first)";
    return EFE_ERR_STATE;
  }
  return EFE_OK;
}

// The products below write Y while they still read X: the two blocks (rows x N
// with their leading dimensions) must not share any byte.
static int check_disjoint(efe_handle* h, const double* X, int64_t ldx, const double* Y, int64_t ldy, int N) {
  const uintptr_t x0 = (uintptr_t)X, y0 = (uintptr_t)Y;
  const uintptr_t x1 = x0 + sizeof(double) * (uintptr_t)((h->rows - 1) * ldx + N);
  const uintptr_t y1 = y0 + sizeof(double) * (uintptr_t)((h->rows - 1) * ldy + N);
  if (x0 < y1 && y0 < x1) {
    h->err = "X and Y overlap (in-place products are not supported)";
    return EFE_ERR_ARG;
  }
  return EFE_OK;
}

int efe_apply_H(efe_handle* h, const double* X, int64_t ldx, int32_t N, double* Y, int64_t ldy, void* stream) {
  if (!h) return EFE_ERR_ARG;
  TRY(check_block(h, X, ldx, N));
  TRY(check_block(h, Y, ldy, N));
  TRY(check_disjoint(h, X, ldx, Y, ldy, N));
  TRY(set_dev(h));
  TRY(reserve(h, N));
  return apply_H_impl(h, X, ldx, N, Y, ldy, S(stream));
}

int efe_apply_M(efe_handle* h, const double* X, int64_t ldx, int32_t N, double* Y, int64_t ldy, void* stream) {
  if (!h) return EFE_ERR_ARG;
  TRY(check_block(h, X, ldx, N));
  TRY(check_block(h, Y, ldy, N));
  TRY(check_disjoint(h, X, ldx, Y, ldy, N));
  TRY(set_dev(h));
  TRY(reserve(h, N));
  return apply_M_impl(h, X, ldx, N, Y, ldy, S(stream));
}

int efe_apply_Minv(efe_handle* h, const double* X, int64_t ldx, int32_t N, double* Y, int64_t ldy, void* stream) {
  if (!h) return EFE_ERR_ARG;
  TRY(check_block(h, X, ldx, N));
  TRY(check_block(h, Y, ldy, N));
  TRY(set_dev(h));
  TRY(reserve(h, N));
  return apply_Minv_impl(h, X, ldx, N, Y, ldy, S(stream));
}

int efe_upper_bound(efe_handle* h, const double* v0, int32_t k, double* b_out, void* stream) {
  if (!h || !b_out || k < 1 || k > 64) return EFE_ERR_ARG;
  TRY(check_block(h, v0, 1, 1));
  TRY(set_dev(h));
  TRY(reserve(h, 1));
  cudaStream_t st = S(stream);
  const int64_t R = h->rows;
  if (!h->lz) TRY(dalloc(h, &h->lz, 6 * R + 512));
  double *v = h->lz, *vp = v + R, *w = vp + R, *Mv = w + R, *tmp = Mv + R, *scal = tmp + R, *part = scal + 8;
  auto dot = [&](const double* x, const double* y, double* out) -> int {
    launch_dot(R, x, y, part, scal, st);
    CKL();
    CK(cudaMemcpyAsync(out, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return EFE_OK;
  };
  TRY(apply_M_impl(h, v0, 1, 1, Mv, 1, st));
  double nrm2;
  TRY(dot(v0, Mv, &nrm2));
  if (!(nrm2 > 0.0) || !is_finite_d(nrm2)) {
    h->err = "start vector has zero or non-finite M-norm";
    return EFE_ERR_ARG;
  }
  launch_scale(R, v0, 1.0 / sqrt(nrm2), v, st);
  CK(cudaMemsetAsync(vp, 0, sizeof(double) * R, st));
  std::vector<double> al, be;
  double beta = 0.0;
  for (int j = 0; j < k; ++j) {
    TRY(apply_H_impl(h, v, 1, 1, tmp, 1, st));
    TRY(apply_Minv_impl(h, tmp, 1, 1, w, 1, st));
    TRY(apply_M_impl(h, v, 1, 1, Mv, 1, st));
    double alpha;
    TRY(dot(w, Mv, &alpha));
    launch_axpby3(R, w, v, vp, alpha, beta, st);
    CKL();
    TRY(apply_M_impl(h, w, 1, 1, Mv, 1, st));
    double b2;
    TRY(dot(w, Mv, &b2));
    if (!is_finite_d(alpha) || !is_finite_d(b2)) {
      h->err = "non-finite value in the Lanczos bound";
      return EFE_ERR_NAN;
    }
    beta = sqrt(std::max(b2, 0.0));
    al.push_back(alpha);
    be.push_back(beta);
    if (beta == 0.0) break;
    CK(cudaMemcpyAsync(vp, v, sizeof(double) * R, cudaMemcpyDeviceToDevice, st));
    launch_scale(R, w, 1.0 / beta, v, st);
    CKL();
  }
  *b_out = tridiag_max_eig(al, be) + fabs(be.back());
  return EFE_OK;
}

// Scaled three-term recurrence coefficients of degrees 1..m (Sec. V):
// Y_k = alpha_k (H~ Y_{k-1} - c Y_{k-1}) + beta_k Y_{k-2}.
static void fill_coefs(double* out, int m, double a, double b, double a0) {
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  double sig = s1;
  for (int k = 1; k <= m; ++k) {
    double al, be;
    if (k == 1) {
      al = s1 / e;
      be = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / s1 - sig);
      al = 2.0 * sn / e;
      be = -sig * sn;
      sig = sn;
    }
    out[3 * (k - 1)] = al;
    out[3 * (k - 1) + 1] = c;
    out[3 * (k - 1) + 2] = be;
  }
}

// Stage the recurrence coefficients of the m degrees ({alpha, c, beta} each) in
// pinned host memory and copy them to the device.  Outside a graph capture the
// previous copy is waited for first, so the staging buffer is never rewritten
// while a copy reads it; inside a capture the copy becomes a graph node that
// reads the staging buffer at every launch (the caller refreshes it).
static int stage_coefs(efe_handle* h, int m, double a, double b, double a0, cudaStream_t st, bool in_graph) {
  if (m > h->coef_cap) {
    if (in_graph) {
      h->err = "coefficient buffers must exist before a graph capture";
      return EFE_ERR_STATE;
    }
    if (h->coef_ev) CK(cudaEventSynchronize(h->coef_ev));
    if (h->coefh) cudaFreeHost(h->coefh);
    dfree(h, h->coefd);
    h->coefh = nullptr;
    CK(cudaMallocHost(&h->coefh, sizeof(double) * 3 * m));
    TRY(dalloc(h, &h->coefd, 3 * (int64_t)m));
    h->coef_cap = m;
    if (!h->coef_ev) CK(cudaEventCreateWithFlags(&h->coef_ev, cudaEventDisableTiming));
  }
  if (!in_graph && h->coef_pending) CK(cudaEventSynchronize(h->coef_ev));
  fill_coefs(h->coefh, m, a, b, a0);
  CK(cudaMemcpyAsync(h->coefd, h->coefh, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, st));
  if (!in_graph) {
    CK(cudaEventRecord(h->coef_ev, st));
    h->coef_pending = true;
  }
  return EFE_OK;
}

// Enqueue one ChFSI filter step on `st` without any host synchronisation
// (graph-capturable when in_graph and the workspaces already exist).
static int chfsi_enqueue(efe_handle* h, double* X, int64_t ldx, int32_t N, int32_t m, double a, double b,
                         double a0, int32_t precision, int32_t fp64_tail, cudaStream_t st, bool in_graph) {
  TRY(check_block(h, X, ldx, N));
  if (m < 1 || !(b > a) || !(a > a0) || !is_finite_d(a) || !is_finite_d(b) || !is_finite_d(a0) || fp64_tail < 0) {
    h->err = "bad filter parameters (need m >= 1, a0 < a < b, finite)";
    return EFE_ERR_ARG;
  }
  if (precision != EFE_PREC_FP64 && precision != EFE_PREC_FP32 && precision != EFE_PREC_TF32 &&
      precision != EFE_PREC_TF32X3 && precision != EFE_PREC_BF16) {
    h->err = "precision mode not available in this build";
    return EFE_ERR_ARG;
  }
  const int n_low = (precision == EFE_PREC_FP64) ? 0 : std::max(0, m - fp64_tail);
  if (in_graph) {
    if (N > h->Nres || (n_low > 0 && N > h->Nres32)) {
      h->err = "workspaces must be reserved before a graph capture";
      return EFE_ERR_STATE;
    }
  } else {
    TRY(reserve(h, N));
    if (n_low > 0) TRY(reserve32(h, N));
  }
  TRY(stage_coefs(h, m, a, b, a0, st, in_graph));
  const int64_t nn = h->n_nodes;
  h->tc_mode = (precision == EFE_PREC_TF32) ? 1 : (precision == EFE_PREC_TF32X3 ? 2 : (precision == EFE_PREC_BF16 ? 3 : 0));
  CK(cudaMemsetAsync(h->info + 4, 0, sizeof(int), st));
  // Two slots per precision: degree k writes Y_k over Y_{k-2} (the combine is
  // elementwise), degree 1 into the free slot.  FP64 slots: 0 = X (user, ldx),
  // 1 = B1 (ld N).
  double* buf[2] = {X, h->B1};
  int64_t ld[2] = {ldx, N};
  int prev = -1, cur = 0;
  int k = 1;
  if (n_low > 0) {
    // load Y_0 into FP32 slot 0
    launch_f64_to_f32_rows(nn, X, ldx, h->Yf[0], h->ld32, N, st);
    if (h->nE > 0) launch_copy_rows(h->nE, X + nn * ldx, ldx, h->Ye[0], N, N, st);
    CKL();
    int p32 = -1, c32 = 0;
    for (; k <= n_low; ++k) {
      const int nx = 1 - c32;
      TRY(degree_f32(h, h->Yf[c32], h->Ye[c32], p32 >= 0 ? h->Yf[p32] : nullptr, p32 >= 0 ? h->Ye[p32] : nullptr,
                     h->Yf[nx], h->Ye[nx], h->coefd + 3 * (k - 1), N, st));
      p32 = c32;
      c32 = nx;
    }
    // hand the last two degrees to FP64 storage: current -> X (free since Y_0
    // was loaded), previous -> B1 (the FP32 slots may live in W and B1 holds
    // only the dead cell-product output)
    launch_f32_to_f64_rows(nn, h->Yf[c32], h->ld32, X, ldx, N, st);
    if (h->nE > 0) launch_copy_rows(h->nE, h->Ye[c32], N, X + nn * ldx, ldx, N, st);
    cur = 0;
    launch_f32_to_f64_rows(nn, h->Yf[p32], h->ld32, h->B1, N, N, st);
    if (h->nE > 0) launch_copy_rows(h->nE, h->Ye[p32], N, h->B1 + nn * N, N, N, st);
    prev = 1;
    CKL();
  }
  for (; k <= m; ++k) {
    const int nx = prev >= 0 ? prev : 1 - cur;
    TRY(degree_f64(h, buf[cur], ld[cur], prev >= 0 ? buf[prev] : nullptr, prev >= 0 ? ld[prev] : 0, buf[nx], ld[nx],
                   h->coefd + 3 * (k - 1), N, st));
    prev = cur;
    cur = nx;
  }
  if (cur != 0) {
    launch_copy_rows(h->rows, buf[cur], ld[cur], X, ldx, N, st);
    CKL();
  }
  return EFE_OK;
}

static int chfsi_check_flags(efe_handle* h, cudaStream_t st) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, h->info + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) {
    h->err = "tensor-core kernel: bounded mbarrier wait ran out";
    return EFE_ERR_TIMEOUT;
  }
  return EFE_OK;
}

int efe_chfsi_step(efe_handle* h, double* X, int64_t ldx, int32_t N, int32_t m, double a, double b, double a0,
                   int32_t precision, int32_t fp64_tail, void* stream) {
  if (!h) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  TRY(chfsi_enqueue(h, X, ldx, N, m, a, b, a0, precision, fp64_tail, st, false));
  const int n_low = (precision == EFE_PREC_FP64) ? 0 : std::max(0, m - fp64_tail);
  if ((n_low > 0 && h->tc_mode) || h->fp64_engine == 1) TRY(chfsi_check_flags(h, st));
  return EFE_OK;
}

// grow-only device buffer i of the operand images (at least `bytes`)
int oz_img_buf(efe_handle* h, int i, int64_t bytes) {
  if (bytes <= h->oz_img_bytes[i]) return EFE_OK;
  dfree(h, h->oz_img[i]);
  h->oz_img[i] = nullptr;
  h->oz_img_bytes[i] = 0;
  TRY(dalloc(h, &h->oz_img[i], bytes));
  h->oz_img_bytes[i] = bytes;
  return EFE_OK;
}

// Device bytes the digit images of one tall product may take: the operands are
// sliced in row panels of at most this size (14 bytes per FP64 value).
constexpr int64_t OZ_IMAGE_BUDGET = 8ll << 30;

// rows per image panel: `unit`-row multiples whose image (bytes_per_row each)
// fits the budget, or the test override
int64_t image_panel_rows(const efe_handle* h, int64_t rows, int64_t bytes_per_row, int64_t unit) {
  int64_t pr = h->opt_image_rows > 0 ? h->opt_image_rows : OZ_IMAGE_BUDGET / std::max<int64_t>(1, bytes_per_row);
  pr = std::max<int64_t>(unit, pr / unit * unit);
  return std::min(pr, (rows + unit - 1) / unit * unit);
}

// C = A B for a tall A (rows x K) and a small B (K x Nc, ld Nc): FP64-grade
// tensor-core products when enabled (A sliced in row panels whose digit image
// fits the budget; K in exact groups of 256 inside the kernel), FP64 DFMA
// otherwise.
int gemm_tall_ld(efe_handle* h, int64_t rows, int K, int Nc, const double* A, int64_t lda, const double* B,
                 int64_t ldb, double* C, int64_t ldc, cudaStream_t st);

int gemm_tall(efe_handle* h, int64_t rows, int K, int Nc, const double* A, int64_t lda, const double* B, double* C,
              int64_t ldc, cudaStream_t st) {
  return gemm_tall_ld(h, rows, K, Nc, A, lda, B, Nc, C, ldc, st);
}

// C = A R for an upper-triangular R (N x N, ld N): column panels of C need only
// the leading rows of R, so each panel is a tall product with K = its last
// column + 1 (about 0.6 of the full product's work at N ~ 2000)
int gemm_tall_upper(efe_handle* h, int64_t rows, int N, const double* A, int64_t lda, const double* R, double* C,
                    int64_t ldc, cudaStream_t st) {
  constexpr int CPW = 384;   // four 96-column tiles of the tensor-core product
  if (N <= CPW) return gemm_tall(h, rows, N, N, A, lda, R, C, ldc, st);
  for (int c0 = 0; c0 < N; c0 += CPW) {
    const int c1 = std::min(N, c0 + CPW);
    TRY(gemm_tall_ld(h, rows, c1, c1 - c0, A, lda, R + c0, N, C + c0, ldc, st));
  }
  return EFE_OK;
}

// C = A B, B: K x Nc with leading dimension ldb
int gemm_tall_ld(efe_handle* h, int64_t rows, int K, int Nc, const double* A, int64_t lda, const double* B,
                 int64_t ldb, double* C, int64_t ldc, cudaStream_t st) {
  if (h->fp64_engine == 1) {
    launch_oz_rowexp(A, lda, rows, K, h->oz_aexp, st);
    launch_oz_colexp(B, ldb, K, Nc, h->oz_bexp, st);
    const int64_t nchk = (K + 15) / 16;
    TRY(oz_img_buf(h, 1, oz_img_cols_bytes(nchk, Nc)));
    launch_oz_img_cols(B, ldb, K, Nc, h->oz_bexp, nchk, h->oz_img[1], st);
    const int64_t pr = image_panel_rows(h, rows, oz_img_rows_bytes(128, K) / 128, 128);
    TRY(oz_img_buf(h, 0, oz_img_rows_bytes(pr, K)));
    for (int64_t r0 = 0; r0 < rows; r0 += pr) {
      const int64_t n = std::min(pr, rows - r0);
      // both operands sliced once into digit images; the product kernel then only
      // streams them (bulk copies) through the tensor cores
      launch_oz_img_rows(A + r0 * lda, lda, n, K, h->oz_aexp + r0, h->oz_img[0], st);
      int slot;
      TRY(timed_begin(h, st, &slot, 1));
      launch_oz_rows(A + r0 * lda, lda, n, K, h->oz_aexp + r0, B, ldb, h->oz_bexp, C + r0 * ldc, ldc, Nc, tc_grid(h),
                     h->info + 4, st, h->oz_img[0], h->oz_img[1], h->opt_test_stall);
      TRY(timed_end(h, st, slot, 2.0 * (double)n * K * Nc, 1));
    }
  } else {
    launch_gemm_nn(rows, Nc, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, st);
  }
  CKL();
  return EFE_OK;
}

// C (Na x Nb, ldc) = A^T B for tall A (rows x Na), B (rows x Nb): FP64 DFMA
// split-K, or with the tensor-core FP64 engine the sliced A^T B (exponents per
// column over all rows; the rows in panels whose column images fit the budget,
// each panel's product added to C).  sym: C is symmetric (Na = Nb): only the
// tiles that meet the upper triangle are formed, the rest mirrored.
int gemm_gram(efe_handle* h, int64_t rows, int Na, int Nb, const double* A, int64_t lda, const double* B,
              int64_t ldb, double* C, int64_t ldc, bool sym, cudaStream_t st) {
  if (h->fp64_engine == 1) {
    launch_oz_colexp(A, lda, rows, Na, h->oz_fexp, st);
    if (B != A) launch_oz_colexp(B, ldb, rows, Nb, h->oz_bexp, st);
    const int* bexp = B != A ? h->oz_bexp : h->oz_fexp;
    // column digit images: per 16 rows, 28 KB per 128 columns of each operand
    const int64_t per16 = oz_img_cols_bytes(1, Na) + (B != A ? oz_img_cols_bytes(1, Nb) : 0);
    const int64_t kp = image_panel_rows(h, rows, (per16 + 15) / 16, 256);
    // image chunks of a panel: enough for any segmentation (the segments, at
    // most 2 n_sm of them, are multiples of 256 rows)
    const int64_t nch = (std::min(kp, rows) + 15) / 16 + 16 * (2 * (int64_t)tc_grid(h) + 1);
    TRY(oz_img_buf(h, 0, oz_img_cols_bytes(nch, Na)));
    if (B != A) TRY(oz_img_buf(h, 1, oz_img_cols_bytes(nch, Nb)));
    bool ok = true;
    for (int64_t k0 = 0; k0 < rows && ok; k0 += kp) {
      const int64_t kn = std::min(kp, rows - k0);
      int slot;
      TRY(timed_begin(h, st, &slot, 1));
      ok = launch_oz_gram(kn, Na, Nb, A + k0 * lda, lda, h->oz_fexp, B + k0 * ldb, ldb, bexp, C, ldc, sym, h->tnwork,
                          h->tnwork_elems, h->oz_pairs, tc_grid(h), h->info + 4, st, h->oz_img[0],
                          h->oz_img_bytes[0], h->oz_img[1], h->oz_img_bytes[1], k0 > 0, h->opt_test_stall) == 0;
      TRY(timed_end(h, st, slot, ok ? (sym ? 1.0 : 2.0) * (double)kn * Na * (Nb + (sym ? 1 : 0)) : 0.0, 1));
    }
    if (ok) {
      CKL();
      return EFE_OK;
    }
  }
  launch_gemm_tn(rows, Na, Nb, A, lda, B, ldb, C, ldc, h->tnwork, h->tnwork_elems, st, sym);
  CKL();
  return EFE_OK;
}

// Largest block of vectors Rayleigh-Ritz takes (its dense N x N work).
constexpr int RR_MAX_N = 4096;

// grow-only scratch of the blocked dense kernels
int dense_scratch(efe_handle* h, int64_t bytes) {
  if (bytes <= h->dsc_bytes) return EFE_OK;
  dfree(h, h->dsc);
  h->dsc = nullptr;
  h->dsc_bytes = 0;
  unsigned char* p = nullptr;
  TRY(dalloc(h, &p, bytes));
  h->dsc = p;
  h->dsc_bytes = bytes;
  return EFE_OK;
}

// the one-CTA dense kernels up to these sizes, the blocked multi-CTA ones above
constexpr int CHOL_ONE_CTA_MAX = 2048;
constexpr int DENSE_SMALL_MAX = 512;

// A = L L^T in place (lower, n x n, ld n); *info: 0 or j + 1 of the first breakdown
int chol_lower(efe_handle* h, double* A, int n, cudaStream_t st, double* min_ratio, int* info = nullptr) {
  if (!info) info = h->info;
  if (n <= CHOL_ONE_CTA_MAX && !h->opt_dense_blocked) {
    launch_chol(A, n, n, info, st, min_ratio);
  } else {
    TRY(dense_scratch(h, (int64_t)sizeof(double) * chol_blocked_scratch(n)));
    launch_chol_blocked(A, n, n, info, min_ratio, (double*)h->dsc, st);
  }
  CKL();
  return EFE_OK;
}

// Li = L^-1 (lower, n x n, ld n)
int trinv_lower(efe_handle* h, const double* L, int n, double* Li, cudaStream_t st) {
  if (n <= DENSE_SMALL_MAX && !h->opt_dense_blocked) {
    launch_trinv_lower(L, n, n, Li, n, st);
  } else {
    TRY(dense_scratch(h, (int64_t)sizeof(double) * ((int64_t)n * n / 4 + 64 * (int64_t)n)));
    launch_trinv_blocked(L, n, n, Li, n, (double*)h->dsc, st);
  }
  CKL();
  return EFE_OK;
}

// C = A B for N x N FP64 matrices (ld N) of the dense Rayleigh-Ritz steps: on the
// tensor-core FP64 engine when it is selected and N takes the blocked dense path
// (the DFMA pipe needs ~20 ms per product at N = 2200), else the DFMA kernel
int dense_nn(efe_handle* h, int N, const double* A, const double* B, double* C, cudaStream_t st) {
  if (h->fp64_engine == 1 && (N > DENSE_SMALL_MAX || h->opt_dense_blocked))
    return gemm_tall_ld(h, N, N, N, A, N, B, N, C, N, st);
  launch_gemm_nn(N, N, N, 1.0, A, N, B, N, 0.0, C, N, st);
  return EFE_OK;
}

// Dense symmetric eigenproblem C = V diag(w) V^T of Rayleigh-Ritz (N x N, FP64).
// FP64 rotations run at the FP64 rate of one SM, so C is first diagonalised in
// FP32 (to a relative off-diagonal size ~1e-6); the FP32 vectors are made
// orthonormal in FP64 (Q = V32 L^-T, L L^T = V32^T V32), C' = Q^T C Q is then
// nearly diagonal and FP64 Jacobi finishes it in two or three sweeps
// (quadratic convergence); V = Q V'.  Falls back to FP64 Jacobi from scratch
// if the FP32 stage fails.  Scratch: 9 N x N blocks at E.
int sym_eig_blocked(efe_handle* h, const double* C, int N, double* V, double* w, double* E, cudaStream_t st);

int sym_eig(efe_handle* h, const double* C, int N, double* V, double* w, double* E, cudaStream_t st) {
  if (N > DENSE_SMALL_MAX || h->opt_dense_blocked) return sym_eig_blocked(h, C, N, V, w, E, st);
  const int64_t NN = (int64_t)N * N;
  float* C32 = reinterpret_cast<float*>(E);
  float* V32 = C32 + NN;
  double* Q0 = E + NN;
  double* G = Q0 + NN;
  double* Li = G + NN;
  double* LiT = Li + NN;
  double* Q = LiT + NN;
  double* T1 = Q + NN;
  double* C2 = T1 + NN;
  double* V2 = C2 + NN;
  float* w32 = reinterpret_cast<float*>(V);  // scratch until V is written
  CK(cudaMemsetAsync(h->info + 1, 0, 2 * sizeof(int), st));
  launch_f64_to_f32_rows(N, C, N, C32, N, N, st);
  launch_jacobi_f32(C32, N, N, V32, N, w32, 60, h->info + 2, st);
  launch_f32_to_f64_rows(N, V32, N, Q0, N, N, st);
  launch_gemm_tn(N, N, N, Q0, N, Q0, N, G, N, h->tnwork, h->tnwork_elems, st, true);
  launch_symmetrize(G, N, N, st);
  launch_chol(G, N, N, h->info + 2, st);
  CKL();
  int inf = 0;
  CK(cudaMemcpyAsync(&inf, h->info + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (inf) {  // FP32 stage unusable: plain FP64 Jacobi
    CK(cudaMemcpyAsync(C2, C, sizeof(double) * NN, cudaMemcpyDeviceToDevice, st));
    launch_jacobi(C2, N, N, V, N, w, 60, h->info + 1, st);
    CKL();
    return EFE_OK;
  }
  launch_trinv_lower(G, N, N, Li, N, st);
  launch_transpose(Li, N, N, LiT, N, st);
  launch_gemm_nn(N, N, N, 1.0, Q0, N, LiT, N, 0.0, Q, N, st);
  launch_gemm_tn(N, N, N, Q, N, C, N, T1, N, h->tnwork, h->tnwork_elems, st, false);
  launch_gemm_nn(N, N, N, 1.0, T1, N, Q, N, 0.0, C2, N, st);
  launch_symmetrize(C2, N, N, st);
  launch_jacobi(C2, N, N, V2, N, w, 40, h->info + 1, st);
  launch_gemm_nn(N, N, N, 1.0, Q, N, V2, N, 0.0, V, N, st);
  CKL();
  return EFE_OK;
}

// The same two stages for large N on many SMs: block Jacobi in FP32 to an
// off-diagonal size ~1e-6, the FP32 vectors made orthonormal in FP64 (blocked
// Cholesky and triangular inverse), then FP64 block Jacobi on the nearly
// diagonal Q^T C Q (two or three sweeps).
int sym_eig_blocked(efe_handle* h, const double* C, int N, double* V, double* w, double* E, cudaStream_t st) {
  const int64_t NN = (int64_t)N * N;
  float* V32 = reinterpret_cast<float*>(E);
  float* w32 = V32 + NN;
  double* Q0 = E + NN;
  double* G = Q0 + NN;
  double* Li = G + NN;
  double* LiT = Li + NN;
  double* Q = LiT + NN;
  double* T1 = Q + NN;
  double* C2 = T1 + NN;
  double* V2 = C2 + NN;
  CK(cudaMemsetAsync(h->info + 1, 0, 2 * sizeof(int), st));
  TRY(dense_scratch(h, block_jacobi_scratch_bytes(N, (int)sizeof(double))));
  double ratio = 0.0;
  const int r32 = block_jacobi<float>(C, N, N, V32, N, w32, 40, 1e-12, h->dsc, st, &ratio);
  if (r32 < 0) {
    h->err = "block Jacobi (FP32 stage): CUDA error";
    return EFE_ERR_CUDA;
  }
  bool refine = true;
  if (r32 == 0) {
    launch_f32_to_f64_rows(N, V32, N, Q0, N, N, st);
    if (h->fp64_engine == 1) {
      TRY(gemm_gram(h, N, N, N, Q0, N, Q0, N, G, N, true, st));
    } else {
      launch_gemm_tn(N, N, N, Q0, N, Q0, N, G, N, h->tnwork, h->tnwork_elems, st, true);
    }
    launch_symmetrize(G, N, N, st);
    TRY(chol_lower(h, G, N, st, nullptr, h->info + 2));
    int inf = 0;
    CK(cudaMemcpyAsync(&inf, h->info + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    refine = inf == 0;
  }
  auto mm = [&](const double* A, const double* B, double* Cm) { return dense_nn(h, N, A, B, Cm, st); };
  const double* C64 = C;
  if (refine && r32 == 0) {
    TRY(trinv_lower(h, G, N, Li, st));
    launch_transpose(Li, N, N, LiT, N, st);
    TRY(mm(Q0, LiT, Q));
    if (h->fp64_engine == 1) {
      TRY(gemm_gram(h, N, N, N, Q, N, C, N, T1, N, false, st));
    } else {
      launch_gemm_tn(N, N, N, Q, N, C, N, T1, N, h->tnwork, h->tnwork_elems, st, false);
    }
    TRY(mm(T1, Q, C2));
    launch_symmetrize(C2, N, N, st);
    C64 = C2;
  }
  // FP64 stage: on the nearly diagonal C2, or on C itself if the FP32 stage failed
  // off-diagonal Frobenius norm <= 1e-13 of the total: eigenvalue errors of
  // order 1e-26 relative, far below FP64 rounding of the projected matrix
  const int r64 = block_jacobi<double>(C64, N, N, C64 == C ? V : V2, N, w, C64 == C ? 60 : 20, 1e-26, h->dsc, st,
                                       &ratio);
  if (r64 < 0) {
    h->err = "block Jacobi (FP64 stage): CUDA error";
    return EFE_ERR_CUDA;
  }
  if (r64 == 1 && ratio > 1e-20) {
    h->err = "block Jacobi eigensolver did not converge";
    return EFE_ERR_NOCONV;
  }
  if (C64 != C) TRY(mm(Q, V2, V));
  CKL();
  return EFE_OK;
}

int efe_rr_shifted_passes(efe_handle* h, int64_t* count) {
  if (!h || !count) return EFE_ERR_ARG;
  *count = h->chol_shifted;
  return EFE_OK;
}

int efe_rayleigh_ritz(efe_handle* h, double* X, int64_t ldx, int32_t N, double* eig_host, double* resid_host,
                      void* stream) {
  if (!h || !eig_host) return EFE_ERR_ARG;
  TRY(check_block(h, X, ldx, N));
  if (N > RR_MAX_N) {
    h->err = "N above the dense eigensolver's limit (" + std::to_string(RR_MAX_N) + ")";
    return EFE_ERR_ARG;
  }
  TRY(set_dev(h));
  TRY(reserve(h, N));
  cudaStream_t st = S(stream);
  const int64_t R = h->rows;
  const int64_t NN = (int64_t)N * N;
  double* G = h->small;
  double* Linv = G + NN;
  double* Rinv = Linv + NN;
  double* Hp = Rinv + NN;
  double* Mp = Hp + NN;
  double* Lm = Mp + NN;
  double* Lminv = Lm + NN;
  double* LminvT = Lminv + NN;
  double* T1 = LminvT + NN;
  double* C = T1 + NN;
  double* Vj = C + NN;
  double* Z = Vj + NN;
  double* Psi = Z + NN;
  double* wv = Psi + NN;
  double* eps = wv + N;
  double* res = eps + N;
  double* E0 = res + N + 5 * (int64_t)N;   // eigensolver scratch: 9 blocks
  double* Q = h->B1;
  int inf[2] = {0, 0};
  // Cholesky-QR: G = X^T X = L L^T, Q = X L^-T
  CK(cudaMemsetAsync(h->info + 4, 0, sizeof(int), st));
  // factorise the Gram matrix of X; ok if X is numerically full rank: G is
  // positive definite and every column keeps a fraction >= 1e-14 of its squared
  // norm outside the span of the columns before it (X L^-T is then orthogonal
  // to ~1e-2, well conditioned enough for the generalised problem below; the
  // filter's spread of amplifications over an all-electron spectrum routinely
  // leaves blocks between 1e-14 and 1e-10)
  auto gram_chol = [&](bool& ok) -> int {
    TRY(gemm_gram(h, R, N, N, X, ldx, X, ldx, G, N, true, st));
    launch_symmetrize(G, N, N, st);
    TRY(chol_lower(h, G, N, st, h->chol_ratio));
    int fl[5] = {0, 0, 0, 0, 0};
    double ratio = 0.0;
    CK(cudaMemcpyAsync(fl, h->info, sizeof(fl), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ratio, h->chol_ratio, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (fl[4]) {
      h->err = "tensor-core FP64 product: bounded wait ran out";
      return EFE_ERR_TIMEOUT;
    }
    ok = fl[0] == 0 && ratio >= 1e-14;
    return EFE_OK;
  };
  bool ok = false;
  TRY(gram_chol(ok));
  // numerically rank-deficient block (a high filter degree from a poor start
  // collapses columns onto the lowest states): shifted Cholesky-QR (Fukaya,
  // Kannan, Nakatsukasa, Yamamoto & Yanagisawa, SIAM J. Sci. Comput. 42, 2020).
  // G + s I with s = 11 (R N + N (N + 1)) u ||X||_F^2 is safely positive
  // definite and X <- X R_s^-1 divides the condition number by about
  // ||X||_2 / sqrt(s) (at least ~200 on a million-row block); after at most
  // five such passes the plain factorisation is accurate (directions lost to
  // rounding come back as rounding noise, which the next filter pass treats
  // like any other start vector).
  for (int pass = 0; !ok; ++pass) {
    if (pass == 5) {
      h->err = "Cholesky-QR breakdown: Gram matrix X^T X is not positive definite (non-finite or rank-deficient block)";
      return EFE_ERR_CHOL;
    }
    TRY(gemm_gram(h, R, N, N, X, ldx, X, ldx, G, N, true, st));
    launch_symmetrize(G, N, N, st);
    launch_shift_diag(G, N, N, 11.0 * ((double)R * N + (double)N * (N + 1)) * 0x1p-53, st);
    TRY(chol_lower(h, G, N, st, nullptr));
    int fl[5] = {0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(fl, h->info, sizeof(fl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (fl[4]) {
      h->err = "tensor-core FP64 product: bounded wait ran out";
      return EFE_ERR_TIMEOUT;
    }
    if (fl[0]) {
      h->err = "Cholesky-QR breakdown: shifted Gram matrix is not positive definite (non-finite block)";
      return EFE_ERR_CHOL;
    }
    TRY(trinv_lower(h, G, N, Linv, st));
    launch_transpose(Linv, N, N, Rinv, N, st);
    TRY(gemm_tall_upper(h, R, N, X, ldx, Rinv, Q, N, st));
    launch_copy_rows(R, Q, N, X, ldx, N, st);
    h->chol_shifted++;
    TRY(gram_chol(ok));
  }
  TRY(trinv_lower(h, G, N, Linv, st));
  launch_transpose(Linv, N, N, Rinv, N, st);
  TRY(gemm_tall_upper(h, R, N, X, ldx, Rinv, Q, N, st));
  // projections H_p = Q^T H Q, M_p = Q^T M Q
  const bool whole = h->whole_rr && h->B2 != nullptr;
  if (whole) {
    double *HQ = h->B2, *MQ = h->W;
    TRY(apply_H_impl(h, Q, N, N, HQ, N, st));
    TRY(apply_M_impl(h, Q, N, N, MQ, N, st));
    TRY(gemm_gram(h, R, N, N, Q, N, HQ, N, Hp, N, true, st));
    TRY(gemm_gram(h, R, N, N, Q, N, MQ, N, Mp, N, true, st));
    launch_symmetrize(Hp, N, N, st);
    launch_symmetrize(Mp, N, N, st);
  } else {
    // two column panels [0, n1) and [n1, N): H Q_p and M Q_p side by side in W;
    // the panel's block column of H_p above its diagonal block in full, the
    // (symmetric) diagonal block by its upper tiles, then the lower triangle
    // mirrored
    const int n1 = N / 2;
    for (int pnl = 0; pnl < 2; ++pnl) {
      const int c0 = pnl == 0 ? 0 : n1, c1 = pnl == 0 ? n1 : N, w = c1 - c0;
      if (w <= 0) continue;
      double *HQp = h->W, *MQp = h->W + R * w;
      TRY(apply_H_impl(h, Q + c0, N, w, HQp, w, st));
      TRY(apply_M_impl(h, Q + c0, N, w, MQp, w, st));
      if (c0 > 0) {
        TRY(gemm_gram(h, R, c0, w, Q, N, HQp, w, Hp + c0, N, false, st));
        TRY(gemm_gram(h, R, c0, w, Q, N, MQp, w, Mp + c0, N, false, st));
      }
      TRY(gemm_gram(h, R, w, w, Q + c0, N, HQp, w, Hp + (int64_t)c0 * N + c0, N, true, st));
      TRY(gemm_gram(h, R, w, w, Q + c0, N, MQp, w, Mp + (int64_t)c0 * N + c0, N, true, st));
    }
    launch_mirror_upper(Hp, N, N, st);
    launch_mirror_upper(Mp, N, N, st);
  }
  CK(cudaMemcpyAsync(Lm, Mp, sizeof(double) * NN, cudaMemcpyDeviceToDevice, st));
  TRY(chol_lower(h, Lm, N, st, nullptr));
  CK(cudaMemcpyAsync(inf, h->info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (inf[0]) {
    h->err = "projected overlap Q^T M Q is not positive definite";
    return EFE_ERR_CHOL;
  }
  // C = Lm^-1 Hp Lm^-T, eig(C) = (eps, Z), Psi = Lm^-T Z
  TRY(trinv_lower(h, Lm, N, Lminv, st));
  launch_transpose(Lminv, N, N, LminvT, N, st);
  TRY(dense_nn(h, N, Lminv, Hp, T1, st));
  TRY(dense_nn(h, N, T1, LminvT, C, st));
  launch_symmetrize(C, N, N, st);
  TRY(sym_eig(h, C, N, Vj, wv, E0, st));
  launch_sort_eig(wv, Vj, N, N, eps, Z, N, st);
  TRY(dense_nn(h, N, LminvT, Z, Psi, st));
  // rotation and residuals
  TRY(gemm_tall(h, R, N, N, Q, N, Psi, X, ldx, st));
  if (resid_host) {
    if (whole) {
      TRY(gemm_tall(h, R, N, N, h->B2, N, Psi, Q, N, st));     // H X = (H Q) Psi
      TRY(gemm_tall(h, R, N, N, h->W, N, Psi, h->B2, N, st));  // M X = (M Q) Psi
      launch_resid_norms(R, Q, N, h->B2, N, eps, N, h->rpart, res, st);
    } else {
      // H X and M X of each panel of the rotated block, applied afresh (an H
      // apply costs far less than rotating H Q at large N)
      const int n1 = N / 2;
      for (int pnl = 0; pnl < 2; ++pnl) {
        const int c0 = pnl == 0 ? 0 : n1, c1 = pnl == 0 ? n1 : N, w = c1 - c0;
        if (w <= 0) continue;
        double *HXp = h->W, *MXp = h->W + R * w;
        TRY(apply_H_impl(h, X + c0, ldx, w, HXp, w, st));
        TRY(apply_M_impl(h, X + c0, ldx, w, MXp, w, st));
        launch_resid_norms(R, HXp, w, MXp, w, eps + c0, w, h->rpart, res + c0, st);
      }
    }
    CKL();
  }
  CK(cudaMemcpyAsync(inf + 1, h->info + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(eig_host, eps, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  if (resid_host) CK(cudaMemcpyAsync(resid_host, res, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(inf, h->info + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (inf[0]) {
    h->err = "tensor-core FP64 product: bounded wait ran out";
    return EFE_ERR_TIMEOUT;
  }
  if (inf[1]) {
    h->err = "dense eigensolver did not converge";
    return EFE_ERR_NOCONV;
  }
  for (int i = 0; i < N; ++i)
    if (!is_finite_d(eig_host[i])) {
      h->err = "non-finite Ritz value";
      return EFE_ERR_NAN;
    }
  return EFE_OK;
}

int efe_set_fp64_engine(efe_handle* h, int32_t engine) {
  if (!h || (engine != 0 && engine != 1)) return EFE_ERR_ARG;
  h->fp64_engine = engine;
  return EFE_OK;
}

int efe_set_option(efe_handle* h, int32_t option, int64_t value) {
  if (!h || value < 0) return EFE_ERR_ARG;
  switch (option) {
    case EFE_OPT_GRID_CAP:
      if (value > (1 << 20)) return EFE_ERR_ARG;
      h->grid_cap = (int)value;
      return EFE_OK;
    case EFE_OPT_IMAGE_ROWS:
      h->opt_image_rows = value;
      return EFE_OK;
    case EFE_OPT_RR_PANELS:
      if (value > 1) return EFE_ERR_ARG;
      if (h->opt_rr_panels != (int)value) {
        h->opt_rr_panels = (int)value;
        h->Nres = 0;   // the workspace layout changes at the next reservation
      }
      return EFE_OK;
    case EFE_OPT_DENSE_BLOCKED:
      if (value > 1) return EFE_ERR_ARG;
      h->opt_dense_blocked = (int)value;
      return EFE_OK;
    case EFE_OPT_TEST_STALL:
      if (value > 1) return EFE_ERR_ARG;
      h->opt_test_stall = (int)value;
      return EFE_OK;
    case EFE_OPT_COUPLING_SPARSE:
      if (value > 1) return EFE_ERR_ARG;
      if (h->opt_coup_sparse != (int)value) {
        h->opt_coup_sparse = (int)value;
        h->Nres32 = 0;   // the mixed workspace is remade at the next filter call
      }
      return EFE_OK;
    case EFE_OPT_COUPLING_COLS:
      if (value > 1) return EFE_ERR_ARG;
      h->opt_coup_cols = (int)value;
      return EFE_OK;
    default:
      h->err = "unknown option";
      return EFE_ERR_ARG;
  }
}

int efe_launch_count(int64_t* total) {
  if (!total) return EFE_ERR_ARG;
  *total = g_launches.load();
  return EFE_OK;
}

int efe_enable_timing(efe_handle* h, int32_t enable) {
  if (!h) return EFE_ERR_ARG;
  h->timing = enable != 0;
  return EFE_OK;
}

static int kernel_stats(efe_handle* h, int ch, int64_t* launches, double* total_ms, double* units, int32_t reset) {
  if (!h) return EFE_ERR_ARG;
  TRY(set_dev(h));
  CK(cudaDeviceSynchronize());
  TRY(timed_fold(h));
  if (launches) *launches = h->t_launches[ch];
  if (total_ms) *total_ms = h->t_ms[ch];
  if (units) *units = h->t_units[ch];
  if (reset) {
    h->t_launches[ch] = 0;
    h->t_ms[ch] = 0.0;
    h->t_units[ch] = 0.0;
  }
  return EFE_OK;
}

int efe_kernel_stats(efe_handle* h, int64_t* launches, double* total_ms, int64_t* cell_columns, int32_t reset) {
  double u = 0.0;
  TRY(kernel_stats(h, 0, launches, total_ms, &u, reset));
  if (cell_columns) *cell_columns = (int64_t)u;
  return EFE_OK;
}

int efe_kernel_stats_fp64(efe_handle* h, int64_t* launches, double* total_ms, double* flops, int32_t reset) {
  return kernel_stats(h, 1, launches, total_ms, flops, reset);
}

// ---------------------------------------------------------------------------
// self-consistent field
int efe_density(efe_handle* h, const double* X, int64_t ldx, int32_t N, const double* occ, double* rho,
                int32_t precision, void* stream) {
  if (!h || !X || !occ || !rho || N < 1 || ldx < N) return EFE_ERR_ARG;
  if (precision != EFE_PREC_FP64 && precision != EFE_PREC_FP32) {
    h->err = "density precision must be EFE_PREC_FP64 or EFE_PREC_FP32";
    return EFE_ERR_ARG;
  }
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  TRY(ensure_eq(h, st));
  if (launch_leaf_density(leaf_dev(h), h->n_leaf, h->mesh, h->re, enr_dev(h), h->kmax, X, ldx, N, occ, rho,
                          precision == EFE_PREC_FP32, st)) {
    h->err = "density kernel: shared-memory request too large (enrichment functions per cell)";
    return EFE_ERR_ARG;
  }
  CKL();
  return EFE_OK;
}

int efe_xc_lda(efe_handle* h, const double* rho, double* exc, double* vxc, void* stream) {
  if (!h || !rho || (!exc && !vxc)) return EFE_ERR_ARG;
  TRY(set_dev(h));
  launch_lda(h->nq, rho, exc, vxc, S(stream));
  CKL();
  return EFE_OK;
}

int efe_hartree(efe_handle* h, const double* rho, double* vh, double* phi, double tol, int32_t max_steps,
                int32_t* steps, void* stream) {
  if (!h || !rho || !vh || !(tol > 0.0) || max_steps < 1) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  TRY(hartree_alloc(h));
  if (!phi) {
    phi = h->hphi;
    CK(cudaMemsetAsync(phi, 0, sizeof(double) * h->n_nodes, st));
  }
  int it = 0;
  const int rc = hartree_solve(h, rho, vh, phi, tol, max_steps, &it, nullptr, st);
  if (steps) *steps = it;
  return rc;
}

int efe_fermi(const double* eps, int32_t N, double n_electrons, double kT, double* occ, double* mu) {
  if (!eps || !occ) return EFE_ERR_ARG;
  return fermi_host(eps, N, n_electrons, kT, occ, mu);
}

int efe_anderson(efe_handle* h, const double* rho_in_hist, const double* rho_out_hist, int32_t n, double beta,
                 double* rho_next, void* stream) {
  if (!h || !rho_in_hist || !rho_out_hist || !rho_next || n < 1 || n > ANDERSON_MAX) return EFE_ERR_ARG;
  TRY(set_dev(h));
  TRY(hartree_alloc(h));
  HistDev hs;
  hs.n = n;
  for (int k = 0; k < n; ++k) {
    hs.rin[k] = rho_in_hist + (int64_t)k * h->nq;
    hs.rout[k] = rho_out_hist + (int64_t)k * h->nq;
  }
  return anderson_apply(h, hs, beta, rho_next, S(stream));
}

int efe_scf_init(efe_handle* h, const efe_scf_params* p, void* stream) {
  if (!h || !p) return EFE_ERR_ARG;
  if (!(p->n_electrons > 0.0) || !(p->kT > 0.0) || !(p->mix_beta > 0.0) || p->mix_beta > 1.0 || p->n_hist < 1 ||
      p->n_hist > ANDERSON_MAX || !(p->poisson_tol > 0.0) || p->poisson_max_steps < 1 || p->lanczos_k < 2) {
    h->err = "SCF parameters out of range";
    return EFE_ERR_ARG;
  }
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  if (!h->vext) {
    TRY(dalloc(h, &h->vext, h->nq));
    TRY(dalloc(h, &h->vh_in, h->nq));
    TRY(dalloc(h, &h->vxc_in, h->nq));
    TRY(dalloc(h, &h->vh_out, h->nq));
    TRY(dalloc(h, &h->phi_in, h->n_nodes));
    TRY(dalloc(h, &h->phi_out, h->n_nodes));
    TRY(dalloc(h, &h->v0, h->rows));
    for (int k = 0; k < 2 * ANDERSON_MAX; ++k) TRY(dalloc(h, &h->hist[k], h->nq));
  }
  CK(cudaMemsetAsync(h->phi_in, 0, sizeof(double) * h->n_nodes, st));
  CK(cudaMemsetAsync(h->phi_out, 0, sizeof(double) * h->n_nodes, st));
  launch_potential_analytic(h->qpts, h->nq, h->axyz, h->aZ, h->n_atoms, 1, nullptr, nullptr, nullptr, 0, 0.0,
                            h->vext, st);
  CKL();
  TRY(ensure_eq(h, st));
  TRY(hartree_alloc(h));
  h->scfp = *p;
  h->hist_count = 0;
  h->hist_head = 0;
  h->ritz.clear();
  h->scf_iter = 0;
  h->scf_ready = true;
  CK(cudaStreamSynchronize(st));
  return EFE_OK;
}

int efe_scf_step(efe_handle* h, double* X, int64_t ldx, int32_t N, int32_t m, int32_t passes, int32_t precision,
                 int32_t fp64_tail, double* rho_in, double* rho_out, double* eig, double* occ, efe_scf_result* res,
                 void* stream) {
  if (!h || !X || !rho_in || !rho_out || !res || N < 1 || ldx < N || m < 1 || passes < 1) return EFE_ERR_ARG;
  if (!h->scf_ready) {
    h->err = "call efe_scf_init first";
    return EFE_ERR_STATE;
  }
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  const efe_scf_params& p = h->scfp;
  std::memset(res, 0, sizeof(*res));
  // V_eff = V_ext + V_H[rho_in] + v_xc(rho_in)   (Eq. veff)
  int it1 = 0, it2 = 0;
  TRY(hartree_solve(h, rho_in, h->vh_in, h->phi_in, p.poisson_tol, p.poisson_max_steps, &it1, nullptr, st));
  launch_veff(h->nq, rho_in, h->vext, h->vh_in, h->vxc_in, h->V, st);
  CKL();
  TRY(efe_set_potential(h, h->V, stream));
  std::vector<double> ev(N), fv(N);
  // the SCF step uses only the Ritz values (no residuals)
  if ((int)h->ritz.size() != N) {
    TRY(efe_rayleigh_ritz(h, X, ldx, N, ev.data(), nullptr, stream));
    h->ritz = ev;
  }
  // Lanczos start: the last column of X
  CK(cudaMemcpy2DAsync(h->v0, sizeof(double), X + (N - 1), sizeof(double) * ldx, sizeof(double), h->rows,
                       cudaMemcpyDeviceToDevice, st));
  double b = 0.0;
  TRY(efe_upper_bound(h, h->v0, p.lanczos_k, &b, stream));
  for (int pass = 0; pass < passes; ++pass) {
    const double a = *std::max_element(h->ritz.begin(), h->ritz.end());
    const double a0 = *std::min_element(h->ritz.begin(), h->ritz.end());
    TRY(efe_chfsi_step(h, X, ldx, N, m, a, b, a0, precision, fp64_tail, stream));
    TRY(efe_rayleigh_ritz(h, X, ldx, N, ev.data(), nullptr, stream));
    h->ritz = ev;
  }
  double mu = 0.0;
  if (fermi_host(h->ritz.data(), N, p.n_electrons, p.kT, fv.data(), &mu) != EFE_OK) {
    h->err = "the subspace holds fewer than N_e / 2 states";
    return EFE_ERR_ARG;
  }
  if (h->occ_cap < N) {
    if (h->occ_dev) dfree(h, h->occ_dev);
    TRY(dalloc(h, &h->occ_dev, N));
    h->occ_cap = N;
  }
  CK(cudaMemcpyAsync(h->occ_dev, fv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
  TRY(efe_density(h, X, ldx, N, h->occ_dev, rho_out, precision == EFE_PREC_FP64 ? EFE_PREC_FP64 : EFE_PREC_FP32,
                  stream));
  TRY(hartree_solve(h, rho_out, h->vh_out, h->phi_out, p.poisson_tol, p.poisson_max_steps, &it2, nullptr, st));
  launch_scf_sums(h->qpts, h->nq, rho_in, rho_out, h->vh_in, h->vxc_in, h->vh_out, h->red_part, h->red_out + 16, st);
  CKL();
  double sums[5];
  CK(cudaMemcpyAsync(sums, h->red_out + 16, sizeof(sums), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double band = 0.0;
  for (int i = 0; i < N; ++i) band += 2.0 * fv[i] * h->ritz[i];
  res->band = band;
  res->xc = sums[0];
  res->hartree = 0.5 * sums[1];
  res->double_counting = sums[2];
  res->drho = sqrt(sums[3]);
  res->n_out = sums[4];
  res->zz = h->e_zz;
  res->total = res->band - res->double_counting + res->hartree + res->xc + res->zz;
  res->fermi_level = mu;
  res->upper_bound = b;
  res->poisson_steps = it1 + it2;
  res->filter_passes = passes;
  if (eig) std::memcpy(eig, h->ritz.data(), sizeof(double) * N);
  if (occ) std::memcpy(occ, fv.data(), sizeof(double) * N);
  // n-stage Anderson mixing: push (rho_in, rho_out), then overwrite rho_in
  const int nh = p.n_hist;
  const int slot = h->hist_head;
  CK(cudaMemcpyAsync(h->hist[slot], rho_in, sizeof(double) * h->nq, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->hist[ANDERSON_MAX + slot], rho_out, sizeof(double) * h->nq, cudaMemcpyDeviceToDevice, st));
  h->hist_head = (slot + 1) % nh;
  h->hist_count = std::min(h->hist_count + 1, nh);
  HistDev hs;
  hs.n = h->hist_count;
  for (int k = 0; k < hs.n; ++k) {
    const int sk = ((h->hist_head - hs.n + k) % nh + nh) % nh;
    hs.rin[k] = h->hist[sk];
    hs.rout[k] = h->hist[ANDERSON_MAX + sk];
  }
  TRY(anderson_apply(h, hs, p.mix_beta, rho_in, st));
  h->scf_iter++;
  return EFE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free overlap product.
//
// efe_apply_M_noalloc computes the same Y = M^E X as efe_apply_M, but its only
// scratch (the per-segment partial sums of the M^ec row products) lives in
// the file-scope device array below instead of the handle's workspace, so the
// call performs no device allocation of any kind.  Every GPU that loads this
// library holds the array until the process exits.
// ---------------------------------------------------------------------------
#define EFE_NOALLOC_SCRATCH_DOUBLES (1 << 21)  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[EFE_NOALLOC_SCRATCH_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};
}  // namespace

namespace {
// Device address of the scratch array on `dev` (which must be current).  Looked
// up once per device (by efe_create); host code may not use the array's name as
// an address.
int noalloc_scratch(efe_handle* h, int dev, double** out) {
  if (dev < 0 || dev >= 256) {
    h->err = "device ordinal out of range for the allocation-free scratch table";
    return EFE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      h->err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
      return EFE_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return EFE_OK;
}
}  // namespace

extern "C" int efe_apply_M_noalloc(efe_handle* h, const double* X, int64_t ldx, int32_t N, double* Y, int64_t ldy,
                                   void* stream) {
  if (!h) return EFE_ERR_ARG;
  TRY(check_block(h, X, ldx, N));
  TRY(check_block(h, Y, ldy, N));
  TRY(check_disjoint(h, X, ldx, Y, ldy, N));
  if (h->nE > 0 && h->nseg * (int64_t)N > EFE_NOALLOC_SCRATCH_DOUBLES) {
    h->err = "efe_apply_M_noalloc: segments x N exceeds the static scratch of 2^21 doubles";
    return EFE_ERR_ARG;
  }
  TRY(set_dev(h));
  // looked up by efe_create (with this handle's device current)
  double* part = h->noalloc_part;
  cudaStream_t st = S(stream);
  const int64_t nn = h->n_nodes;
  launch_row_scale<double>(nn, h->Dm, X, ldx, Y, ldy, N, st);
  if (h->nE > 0) {
    launch_spmm_nodes<double>(h->n_tn, h->t_nodes, h->t_ptr, h->t_col, h->mecT, 1.0, X + nn * ldx, ldx, Y, ldy, N, st);
    launch_row_scale<double>(nn, h->mask, Y, ldy, Y, ldy, N, st);
    // every partial is written before it is read: nothing to clear
    launch_spmm_segments<double>(h->nseg, h->seg_start, h->seg_end, h->ec_col, h->mec, nullptr, X, ldx, part, N, st);
    launch_seg_reduce((int)h->nE, h->row_seg_ptr, part, 1.0, nullptr, 0, 0.0, Y + nn * ldy, ldy, N, st);
    launch_gemm_nn(h->nE, N, (int)h->nE, 1.0, h->Mee, h->nE, X + nn * ldx, ldx, 1.0, Y + nn * ldy, ldy, st);
  }
  CKL();
  return EFE_OK;
}

// ---------------------------------------------------------------------------
// Learned initial density: SAD start, descriptors, network, loss, optimiser.
// The loss reduction uses a file-scope device array (no handle needed).
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_learn_red[2 * 1024 + 8];

namespace {
std::mutex g_learn_mu;
double* g_learn_ptr[256] = {nullptr};

double* learn_red(int dev) {
  if (dev < 0 || dev >= 256) return nullptr;
  std::lock_guard<std::mutex> lk(g_learn_mu);
  if (!g_learn_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_learn_red) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_learn_ptr[dev] = (double*)p;
  }
  return g_learn_ptr[dev];
}

bool valid_shape(const efe_mlp_shape* s) {
  if (!s || s->n_layers < 1 || s->n_layers > 8) return false;
  for (int l = 0; l <= s->n_layers; ++l)
    if (s->dims[l] < 1 || s->dims[l] > 4096) return false;
  return s->dims[s->n_layers] == 1;
}

bool valid_prec(int32_t p) { return p == EFE_PREC_FP32 || p == EFE_PREC_FP64; }
}  // namespace

extern "C" {

int efe_sad_density(efe_handle* h, const efe_atom_shells* shells, double n_electrons, double* rho, void* stream) {
  if (!h || !shells || !rho) return EFE_ERR_ARG;
  TRY(set_dev(h));
  std::vector<SadShellDev> sd(std::max(1, h->n_atoms));
  for (int a = 0; a < h->n_atoms; ++a) {
    const efe_atom_shells& s = shells[a];
    if (s.n_shells < 1 || s.n_shells > 3) {
      h->err = "efe_atom_shells.n_shells must be 1 .. 3";
      return EFE_ERR_ARG;
    }
    sd[a].n_shells = s.n_shells;
    for (int k = 0; k < s.n_shells; ++k) {
      if (s.n[k] < 1 || s.n[k] > 7 || !(s.zeta[k] > 0.0) || !(s.occ[k] >= 0.0)) {
        h->err = "bad Slater shell (n in 1..7, zeta > 0, occ >= 0)";
        return EFE_ERR_ARG;
      }
      double fact = 1.0;
      for (int i = 2; i <= 2 * s.n[k]; ++i) fact *= i;
      sd[a].n[k] = s.n[k];
      sd[a].zeta[k] = s.zeta[k];
      sd[a].occ[k] = s.occ[k];
      sd[a].c[k] = sqrt(pow(2.0 * s.zeta[k], 2 * s.n[k] + 1) / fact);
    }
  }
  cudaStream_t st = S(stream);
  SadShellDev* dsh = nullptr;
  TRY(dalloc(h, &dsh, (int64_t)sd.size()));
  CK(cudaMemcpyAsync(dsh, sd.data(), sizeof(SadShellDev) * sd.size(), cudaMemcpyHostToDevice, st));
  launch_sad(h->qpts, h->nq, h->axyz, h->n_atoms, dsh, rho, st);
  if (n_electrons > 0.0) {
    double* red = learn_red(h->dev);
    if (!red) {
      h->err = "reduction scratch unavailable";
      return EFE_ERR_CUDA;
    }
    launch_scale_count(h->qpts, h->nq, n_electrons, rho, red, st);
  }
  CKL();
  CK(cudaStreamSynchronize(st));
  dfree(h, dsh);
  return EFE_OK;
}

int efe_descriptors(efe_handle* h, const efe_desc_params* p, void* D, int32_t precision, void* stream) {
  if (!h || !p || !D || !valid_prec(precision)) return EFE_ERR_ARG;
  if (p->n_species < 1 || p->n_species > DESC_MAX_SPECIES || p->n_radial < 1 || p->n_radial > DESC_MAX_RADIAL ||
      p->n_ang < 0 || p->n_ang > DESC_MAX_ANG || !(p->radial_sigma > 0.0) || !(p->r_cut > 0.0) ||
      (p->n_ang > 0 && !(p->ang_sigma > 0.0))) {
    h->err = "descriptor parameters out of range";
    return EFE_ERR_ARG;
  }
  TRY(set_dev(h));
  DescDev dd;
  dd.n_species = p->n_species;
  dd.n_radial = p->n_radial;
  dd.n_ang = p->n_ang;
  for (int k = 0; k < DESC_MAX_RADIAL; ++k) dd.radial_mu[k] = k < p->n_radial ? p->radial_mu[k] : 0.0;
  for (int k = 0; k < DESC_MAX_ANG; ++k) dd.ang_mu[k] = k < p->n_ang ? p->ang_mu[k] : 0.0;
  dd.radial_sigma = p->radial_sigma;
  dd.ang_sigma = p->ang_sigma;
  dd.r_cut = p->r_cut;
  dd.standardise = p->standardise ? 1 : 0;
  const int nfeat = p->n_species * (p->n_radial + p->n_ang);
  for (int f = 0; f < DESC_MAX_SPECIES * (DESC_MAX_RADIAL + DESC_MAX_ANG); ++f) {
    dd.offset[f] = (p->standardise && f < nfeat) ? p->offset[f] : 0.0;
    dd.scale[f] = (p->standardise && f < nfeat) ? p->scale[f] : 1.0;
  }
  // species slot of every atom (-1: not described)
  std::vector<double> Z(h->n_atoms);
  if (h->n_atoms > 0) CK(cudaMemcpy(Z.data(), h->aZ, sizeof(double) * h->n_atoms, cudaMemcpyDeviceToHost));
  std::vector<int32_t> slot(std::max(1, h->n_atoms), -1);
  for (int a = 0; a < h->n_atoms; ++a)
    for (int s = 0; s < p->n_species; ++s)
      if (fabs(Z[a] - p->species_Z[s]) < 1e-9) slot[a] = s;
  cudaStream_t st = S(stream);
  int32_t* dslot = nullptr;
  TRY(dalloc(h, &dslot, (int64_t)slot.size()));
  CK(cudaMemcpyAsync(dslot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice, st));
  if (precision == EFE_PREC_FP32)
    launch_descriptors<float>(h->qpts, h->nq, h->axyz, dslot, h->n_atoms, dd, (float*)D, st);
  else
    launch_descriptors<double>(h->qpts, h->nq, h->axyz, dslot, h->n_atoms, dd, (double*)D, st);
  CKL();
  CK(cudaStreamSynchronize(st));
  dfree(h, dslot);
  return EFE_OK;
}

int efe_learned_density(efe_handle* h, const double* rho_sad, const void* y, double floor, double n_electrons,
                        double* rho, int32_t precision, void* stream) {
  if (!h || !rho_sad || !y || !rho || !(floor > 0.0) || !valid_prec(precision)) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  if (precision == EFE_PREC_FP32)
    launch_apply_correction<float>(h->nq, rho_sad, (const float*)y, floor, rho, st);
  else
    launch_apply_correction<double>(h->nq, rho_sad, (const double*)y, floor, rho, st);
  if (n_electrons > 0.0) {
    double* red = learn_red(h->dev);
    if (!red) {
      h->err = "reduction scratch unavailable";
      return EFE_ERR_CUDA;
    }
    launch_scale_count(h->qpts, h->nq, n_electrons, rho, red, st);
  }
  CKL();
  return EFE_OK;
}

int efe_density_log_ratio(efe_handle* h, const double* rho, const double* rho_sad, double floor, void* y,
                          int32_t precision, void* stream) {
  if (!h || !rho || !rho_sad || !y || !(floor > 0.0) || !valid_prec(precision)) return EFE_ERR_ARG;
  TRY(set_dev(h));
  cudaStream_t st = S(stream);
  if (precision == EFE_PREC_FP32)
    launch_log_ratio<float>(h->nq, rho, rho_sad, floor, (float*)y, st);
  else
    launch_log_ratio<double>(h->nq, rho, rho_sad, floor, (double*)y, st);
  CKL();
  return EFE_OK;
}

int64_t efe_mlp_param_count(const efe_mlp_shape* s) {
  return valid_shape(s) ? mlp_param_count(s->dims, s->n_layers) : -1;
}

int64_t efe_mlp_work_elems(const efe_mlp_shape* s, int64_t n) {
  return valid_shape(s) && n >= 0 ? mlp_work_elems(s->dims, s->n_layers, n) : -1;
}

int64_t efe_mlp_scratch_elems(const efe_mlp_shape* s, int64_t n) {
  return valid_shape(s) && n >= 0 ? mlp_scratch_elems(s->dims, s->n_layers, n) : -1;
}

int efe_mlp_forward(const efe_mlp_shape* s, const void* params, const void* X, int64_t n, void* y, void* work,
                    int32_t precision, void* stream) {
  if (!valid_shape(s) || !params || !X || !y || !work || n < 1 || !valid_prec(precision)) return EFE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == EFE_PREC_FP32)
    mlp_forward<float>(s->dims, s->n_layers, (const float*)params, (const float*)X, n, (float*)y, (float*)work, st);
  else
    mlp_forward<double>(s->dims, s->n_layers, (const double*)params, (const double*)X, n, (double*)y,
                        (double*)work, st);
  return cudaGetLastError() == cudaSuccess ? EFE_OK : EFE_ERR_CUDA;
}

int efe_mlp_backward(const efe_mlp_shape* s, const void* params, const void* X, int64_t n, const void* work,
                     const void* dy, void* grads, void* scratch, int32_t precision, void* stream) {
  if (!valid_shape(s) || !params || !X || !work || !dy || !grads || !scratch || n < 1 || !valid_prec(precision))
    return EFE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == EFE_PREC_FP32)
    mlp_backward<float>(s->dims, s->n_layers, (const float*)params, (const float*)X, n, (const float*)work,
                        (const float*)dy, (float*)grads, (float*)scratch, st);
  else
    mlp_backward<double>(s->dims, s->n_layers, (const double*)params, (const double*)X, n, (const double*)work,
                         (const double*)dy, (double*)grads, (double*)scratch, st);
  return cudaGetLastError() == cudaSuccess ? EFE_OK : EFE_ERR_CUDA;
}

int efe_wmse(const void* yh, const void* y, const void* c, int64_t n, void* dy, double* loss, int32_t precision,
             void* stream) {
  if (!yh || !y || !c || !dy || n < 1 || !valid_prec(precision)) return EFE_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EFE_ERR_CUDA;
  double* red = learn_red(dev);
  if (!red) return EFE_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  double* stats = red + 2 * 1024;
  if (precision == EFE_PREC_FP32)
    launch_wmse<float>((const float*)yh, (const float*)y, (const float*)c, n, (float*)dy, red, stats, st);
  else
    launch_wmse<double>((const double*)yh, (const double*)y, (const double*)c, n, (double*)dy, red, stats, st);
  if (loss) {
    if (cudaMemcpyAsync(loss, stats, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return EFE_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return EFE_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? EFE_OK : EFE_ERR_CUDA;
}

int efe_adam(void* p, const void* g, void* m, void* v, int64_t n, double lr, double beta1, double beta2, double eps,
             int32_t t, int32_t precision, void* stream) {
  if (!p || !g || !m || !v || n < 1 || t < 1 || !valid_prec(precision) || !(lr > 0.0)) return EFE_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == EFE_PREC_FP32)
    launch_adam<float>(n, (float*)p, (const float*)g, (float*)m, (float*)v, lr, beta1, beta2, eps, t, st);
  else
    launch_adam<double>(n, (double*)p, (const double*)g, (double*)m, (double*)v, lr, beta1, beta2, eps, t, st);
  return cudaGetLastError() == cudaSuccess ? EFE_OK : EFE_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner of the tensor-core cell kernel and batched multi-system filter steps
// ---------------------------------------------------------------------------
extern "C" {

int efe_autotune(efe_handle* h, int32_t N, int32_t precision, int32_t* tile_out, double* ms_out) {
  if (!h || N < 1 || (precision != EFE_PREC_TF32 && precision != EFE_PREC_TF32X3 && precision != EFE_PREC_BF16))
    return EFE_ERR_ARG;
  if (!h->potential_set) {
    h->err = "no potential set (call efe_set_potential first)";
    return EFE_ERR_STATE;
  }
  TRY(set_dev(h));
  TRY(reserve(h, N));
  TRY(reserve32(h, N));
  cudaStream_t st = nullptr;
  const int64_t nn = h->n_nodes;
  CK(cudaMemsetAsync(h->Yf[0], 0, sizeof(float) * nn * h->ld32, st));
  CK(cudaMemsetAsync(h->Wf, 0, sizeof(float) * nn * h->ld32, st));
  CK(cudaMemsetAsync(h->info + 4, 0, sizeof(int), st));
  int ntile = 0;
  const int* tiles = tc3_tiles(&ntile);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 0;
  double best_ms = 1e300;
  for (int i = 0; i < ntile; ++i) {
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {  // rep 0 warms up
      CK(cudaEventRecord(e0, st));
      for (int c = 0; c < 8; ++c) {
        const int64_t nc = h->colour_off[c + 1] - h->colour_off[c];
        if (nc == 0) continue;
        if (launch_cell_tc3(h->Aimg32, h->colour_cells + h->colour_off[c], nc, h->mesh, h->Yf[0], h->ld32, h->Wf,
                            h->ld32, N, precision == EFE_PREC_TF32X3 ? 1 : (precision == EFE_PREC_BF16 ? 2 : 0),
                            tc_grid(h), h->info + 4, st, tiles[i])) {
          h->err = "tensor-core cell kernel needs 16-byte aligned rows";
          return EFE_ERR_ARG;
        }
      }
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      if (rep == 1 || (rep > 1 && t < ms)) ms = t;
    }
    if (ms_out) ms_out[i] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = tiles[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int flag = 0;
  CK(cudaMemcpy(&flag, h->info + 4, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    h->err = "tensor-core cell kernel: bounded mbarrier wait ran out";
    return EFE_ERR_TIMEOUT;
  }
  h->tc_tile = best;
  h->tc_tile_N = N;
  if (tile_out) *tile_out = best;
  return EFE_OK;
}

}  // extern "C"

struct efe_batch {
  std::vector<efe_handle*> hs;
  int dev = 0;
  cudaStream_t s0 = nullptr;
  std::vector<cudaStream_t> st;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  int64_t kernel_nodes = 0, nodes = 0;
  // what the captured graph was recorded for
  std::vector<double*> X;
  std::vector<int64_t> ldx;
  std::vector<int32_t> N;
  int m = 0, precision = -1, fp64_tail = -1, engine = -1;
  std::string err;
};

namespace {
void batch_clear_graph(efe_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->X.clear();
}
}  // namespace

extern "C" {

int efe_batch_create(efe_handle* const* systems, int32_t n, efe_batch** out) {
  if (!out || !systems || n < 1) return EFE_ERR_ARG;
  *out = nullptr;
  efe_batch* b = new (std::nothrow) efe_batch();
  if (!b) return EFE_ERR_ALLOC;
  *out = b;
  b->dev = systems[0]->dev;
  for (int i = 0; i < n; ++i) {
    if (!systems[i] || systems[i]->dev != b->dev) {
      b->err = "batch systems must be valid handles on one device";
      return EFE_ERR_ARG;
    }
    b->hs.push_back(systems[i]);
  }
  if (cudaSetDevice(b->dev) != cudaSuccess || cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    b->err = "stream / event creation failed";
    return EFE_ERR_CUDA;
  }
  b->st.resize(n, nullptr);
  b->join.resize(n, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) {
      b->err = "stream / event creation failed";
      return EFE_ERR_CUDA;
    }
  return EFE_OK;
}

int efe_batch_destroy(efe_batch* b) {
  if (!b) return EFE_OK;
  cudaSetDevice(b->dev);
  batch_clear_graph(b);
  for (auto s : b->st)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
  return EFE_OK;
}

const char* efe_batch_last_error(const efe_batch* b) { return b ? b->err.c_str() : "null batch"; }

int efe_batch_graph_nodes(const efe_batch* b, int64_t* nodes, int64_t* kernel_nodes) {
  if (!b) return EFE_ERR_ARG;
  if (nodes) *nodes = b->nodes;
  if (kernel_nodes) *kernel_nodes = b->kernel_nodes;
  return EFE_OK;
}

int efe_batch_chfsi_step(efe_batch* b, double* const* X, const int64_t* ldx, const int32_t* N, int32_t m,
                         const double* a, const double* bnd, const double* a0, int32_t precision, int32_t fp64_tail,
                         int32_t use_graph, void* stream) {
  if (!b || !X || !ldx || !N || !a || !bnd || !a0 || m < 1) return EFE_ERR_ARG;
  const int n = (int)b->hs.size();
  if (cudaSetDevice(b->dev) != cudaSuccess) return EFE_ERR_CUDA;
  cudaStream_t caller = (cudaStream_t)stream;
  auto fail = [&](int i, int rc) {
    b->err = "system " + std::to_string(i) + ": " + b->hs[i]->err;
    return rc;
  };
  if (!use_graph) {
    for (int i = 0; i < n; ++i) {
      const int rc = efe_chfsi_step(b->hs[i], X[i], ldx[i], N[i], m, a[i], bnd[i], a0[i], precision, fp64_tail,
                                    stream);
      if (rc != EFE_OK) return fail(i, rc);
    }
    return EFE_OK;
  }
  const int n_low = (precision == EFE_PREC_FP64) ? 0 : std::max(0, m - fp64_tail);
  // workspaces and coefficient buffers exist before any capture
  for (int i = 0; i < n; ++i) {
    efe_handle* h = b->hs[i];
    int rc = reserve(h, N[i]);
    if (rc == EFE_OK && n_low > 0) rc = reserve32(h, N[i]);
    if (rc != EFE_OK) return fail(i, rc);
    if (h->coef_cap < m) {
      rc = stage_coefs(h, m, a[i], bnd[i], a0[i], caller, false);
      if (rc != EFE_OK) return fail(i, rc);
    }
    if (h->coef_pending) cudaEventSynchronize(h->coef_ev);
    h->coef_pending = false;
  }
  bool same = b->exec && b->m == m && b->precision == precision && b->fp64_tail == fp64_tail &&
              (int)b->X.size() == n && b->engine == b->hs[0]->fp64_engine;
  for (int i = 0; same && i < n; ++i) same = b->X[i] == X[i] && b->ldx[i] == ldx[i] && b->N[i] == N[i];
  if (!same) {
    batch_clear_graph(b);
    const int64_t l0 = g_launches.load();
    std::vector<bool> timing(n);
    for (int i = 0; i < n; ++i) {
      timing[i] = b->hs[i]->timing;
      b->hs[i]->timing = false;
    }
    if (cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      b->err = "cudaStreamBeginCapture failed";
      return EFE_ERR_CUDA;
    }
    int rc = EFE_OK, bad = -1;
    cudaEventRecord(b->fork, b->s0);
    for (int i = 0; i < n && rc == EFE_OK; ++i) {
      cudaStreamWaitEvent(b->st[i], b->fork, 0);
      rc = chfsi_enqueue(b->hs[i], X[i], ldx[i], N[i], m, a[i], bnd[i], a0[i], precision, fp64_tail, b->st[i], true);
      if (rc != EFE_OK) bad = i;
      cudaEventRecord(b->join[i], b->st[i]);
      cudaStreamWaitEvent(b->s0, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->s0, &graph);
    for (int i = 0; i < n; ++i) b->hs[i]->timing = timing[i];
    g_launches.store(l0);  // capture records, it does not launch
    if (rc != EFE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return fail(bad, rc);
    }
    if (ce != cudaSuccess || !graph) {
      cudaGetLastError();
      b->err = std::string("graph capture failed: ") + cudaGetErrorString(ce);
      return EFE_ERR_CUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int64_t nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      b->err = std::string("graph instantiation failed: ") + cudaGetErrorString(ie);
      return EFE_ERR_CUDA;
    }
    b->nodes = (int64_t)nn;
    b->kernel_nodes = nk;
    b->X.assign(X, X + n);
    b->ldx.assign(ldx, ldx + n);
    b->N.assign(N, N + n);
    b->m = m;
    b->precision = precision;
    b->fp64_tail = fp64_tail;
    b->engine = b->hs[0]->fp64_engine;
  }
  // refresh the staged coefficients (read by the graph's copy nodes), then replay
  for (int i = 0; i < n; ++i) {
    fill_coefs(b->hs[i]->coefh, m, a[i], bnd[i], a0[i]);
    b->hs[i]->tc_mode = (precision == EFE_PREC_TF32) ? 1 : (precision == EFE_PREC_TF32X3 ? 2 : (precision == EFE_PREC_BF16 ? 3 : 0));
  }
  if (cudaStreamSynchronize(caller) != cudaSuccess || cudaGraphLaunch(b->exec, b->s0) != cudaSuccess) {
    cudaGetLastError();
    b->err = "graph launch failed";
    return EFE_ERR_CUDA;
  }
  g_launches += b->kernel_nodes;
  if (cudaStreamSynchronize(b->s0) != cudaSuccess) {
    b->err = "graph execution failed";
    return EFE_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    const int rc = chfsi_check_flags(b->hs[i], b->s0);
    if (rc != EFE_OK) return fail(i, rc);
  }
  return EFE_OK;
}

}  // extern "C"
