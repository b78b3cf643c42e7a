// Dense N x N kernels of Cholesky-QR and Rayleigh-Ritz for large blocks of
// vectors (N in the thousands, Sec. V on the 280-atom cluster), spread over
// many SMs:
//   * blocked right-looking Cholesky (64-column panels: one-CTA diagonal block,
//     row-parallel triangular solve of the panel, trailing update as an FP64
//     GEMM);
//   * the inverse of a lower triangle by 2 x 2 block recursion (two half-size
//     inverses and two GEMMs);
//   * a two-sided block Jacobi eigensolver for symmetric matrices: the matrix
//     is cut into blocks of B rows/columns, a round-robin tournament pairs the
//     blocks, every pair's 2B x 2B subproblem is diagonalised in shared memory
//     by one CTA (cyclic Jacobi), and the pair's rotation is applied to its 2B
//     rows and columns of the whole matrix and to the eigenvector matrix by
//     many CTAs (row-times-2B x 2B products), B = 16.  Float (the fast first
//     stage) and double (the refinement).
// No atomics: every result has a fixed order of operations.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "efe_kernels.h"

namespace efe {

extern std::atomic<int64_t> g_launches;

namespace {

constexpr int CB = 64;        // Cholesky panel width
// block Jacobi: block size BJ_B (a template parameter), subproblems of
// BJ_S = 2 BJ_B, shared rows of BJ_S + 1

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- Cholesky
// Diagonal block A[j0:j0+b, j0:j0+b] (already updated by the panels before it)
// factorised in place by one CTA; info = j + 1 of the first breakdown (global
// index), left alone if it is already set.
__global__ void __launch_bounds__(1024) k_chol_diag(double* A, int lda, int j0, int b, int* info) {
  __shared__ double S[CB][CB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int t = tid; t < b * b; t += blockDim.x) S[t / b][t % b] = A[(int64_t)(j0 + t / b) * lda + j0 + t % b];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const double d = S[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = j + 1;
        S[j][j] = 1.0;
      } else {
        S[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double piv = S[j][j];
    for (int i = j + 1 + tid; i < b; i += blockDim.x) S[i][j] /= piv;
    __syncthreads();
    for (int t = tid; t < (b - j - 1) * (b - j - 1); t += blockDim.x) {
      const int i = j + 1 + t / (b - j - 1), c = j + 1 + t % (b - j - 1);
      if (c <= i) S[i][c] -= S[i][j] * S[c][j];
    }
    __syncthreads();
  }
  for (int t = tid; t < b * b; t += blockDim.x) {
    const int i = t / b, c = t % b;
    A[(int64_t)(j0 + i) * lda + j0 + c] = c <= i ? S[i][c] : 0.0;
  }
  if (tid == 0 && bad && *info == 0) *info = j0 + bad;
}

// Panel below the diagonal block: L21 = A21 L11^-T, one row per thread
// (forward substitution against the diagonal block held in shared memory).
__global__ void __launch_bounds__(128) k_chol_panel(double* A, int lda, int j0, int b, int n) {
  __shared__ double L[CB][CB + 1];
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) L[t / b][t % b] = A[(int64_t)(j0 + t / b) * lda + j0 + t % b];
  __syncthreads();
  const int r = j0 + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double x[CB];
  double* row = A + (int64_t)r * lda + j0;
#pragma unroll 4
  for (int k = 0; k < b; ++k) {
    double v = row[k];
    for (int i = 0; i < k; ++i) v -= x[i] * L[k][i];
    x[k] = v / L[k][k];
  }
  for (int k = 0; k < b; ++k) row[k] = x[k];
}

// T (b x m, ld m) = transpose of the panel rows j0+b .. n-1, columns j0 .. j0+b-1
__global__ void k_panel_transpose(const double* A, int lda, int j0, int b, int n, double* T) {
  const int m = n - j0 - b;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * b) return;
  const int r = (int)(t / b), c = (int)(t % b);
  T[(int64_t)c * m + r] = A[(int64_t)(j0 + b + r) * lda + j0 + c];
}

__global__ void k_zero_upper(double* A, int n, int lda) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), c = (int)(t % n);
  if (c > i) A[(int64_t)i * lda + c] = 0.0;
}

__global__ void k_copy_diag(const double* A, int n, int lda, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[(int64_t)i * lda + i];
}

// min_j L_jj^2 / d0_j (one CTA): the smallest fraction of a column's squared
// norm outside the span of the columns before it
__global__ void k_chol_ratio(const double* L, int n, int lda, const double* d0, const int* info, double* out) {
  __shared__ double red[1024];
  double m = 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double l = L[(int64_t)i * lda + i];
    m = fmin(m, l * l / d0[i]);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = *info ? 0.0 : red[0];
}

__global__ void k_zero_block(double* A, int rows, int cols, int lda) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * cols) return;
  A[(t / cols) * lda + t % cols] = 0.0;
}

// ---------------------------------------------------------------- block Jacobi
// Position of block slot s in round r of the round-robin tournament over nb
// blocks (slot 0 fixed, the others rotate).
__device__ __forceinline__ int rr_block(int s, int r, int nb) { return s == 0 ? 0 : ((s - 1 + r) % (nb - 1)) + 1; }

__device__ __forceinline__ void bj_pair(int k, int r, int nb, int& p, int& q) {
  const int a = rr_block(k, r, nb), b = rr_block(nb - 1 - k, r, nb);
  p = min(a, b);
  q = max(a, b);
}

template <int BJ_B>
__device__ __forceinline__ int bj_index(int i, int p, int q) { return i < BJ_B ? p * BJ_B + i : q * BJ_B + (i - BJ_B); }

template <typename T>
__global__ void k_bj_pad(const double* __restrict__ C, int n, int ldc, T* __restrict__ A, T* __restrict__ V, int np) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)np * np) return;
  const int i = (int)(t / np), j = (int)(t % np);
  A[t] = (i < n && j < n) ? (T)C[(int64_t)i * ldc + j] : T(0);
  V[t] = i == j ? T(1) : T(0);
}

// One CTA per block pair of round r: diagonalise the BJ_S x BJ_S subproblem
// [[A_pp, A_pq], [A_qp, A_qq]] in shared memory by cyclic Jacobi; write the
// rotation J (BJ_S x BJ_S, row-major), the subproblem's eigenvalues, and whether
// any rotation was applied.
template <typename T, int BJ_B>
__global__ void __launch_bounds__(256) k_bj_solve(const T* __restrict__ A, int np, int nb, int r, T* __restrict__ Jb,
                                                  T* __restrict__ lam, int* __restrict__ rotated, int max_sweeps) {
  constexpr int BJ_S = 2 * BJ_B, BJ_LD = BJ_S + 1;
  extern __shared__ double smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  T* J = S + BJ_S * BJ_LD;
  __shared__ T cs[BJ_B], sn[BJ_B];
  __shared__ int pp[BJ_B], qq[BJ_B];
  __shared__ int any, any_sweep;
  const int k = blockIdx.x, tid = threadIdx.x;
  int p, q;
  bj_pair(k, r, nb, p, q);
  for (int t = tid; t < BJ_S * BJ_S; t += blockDim.x) {
    const int i = t / BJ_S, j = t % BJ_S;
    S[i * BJ_LD + j] = A[(int64_t)bj_index<BJ_B>(i, p, q) * np + bj_index<BJ_B>(j, p, q)];
    J[i * BJ_LD + j] = i == j ? T(1) : T(0);
  }
  if (tid == 0) any = 0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) any_sweep = 0;
    __syncthreads();
    for (int rd = 0; rd < BJ_S - 1; ++rd) {
      if (tid < BJ_B) {
        const int a = tid == 0 ? 0 : ((tid - 1 + rd) % (BJ_S - 1)) + 1;
        const int b2 = ((BJ_S - 1 - tid - 1 + rd) % (BJ_S - 1)) + 1;
        const int i = min(a, b2), j = max(a, b2);
        const T aij = S[i * BJ_LD + j], aii = S[i * BJ_LD + i], ajj = S[j * BJ_LD + j];
        T c = T(1), s = T(0);
        // negligible off-diagonal entry (below the rounding of both diagonal
        // entries): no rotation
        const T g = T(100) * fabs(aij);
        if (aij != T(0) && !(fabs(aii) + g == fabs(aii) && fabs(ajj) + g == fabs(ajj))) {
          const T tau = (ajj - aii) / (T(2) * aij);
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + t * t);
          s = t * c;
          any_sweep = 1;
        }
        pp[tid] = i;
        qq[tid] = j;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // rows i, j of S
      for (int t = tid; t < BJ_B * BJ_S; t += blockDim.x) {
        const int e = t / BJ_S, col = t % BJ_S;
        if (sn[e] == T(0)) continue;
        const int i = pp[e], j = qq[e];
        const T c = cs[e], s = sn[e];
        const T x = S[i * BJ_LD + col], y = S[j * BJ_LD + col];
        S[i * BJ_LD + col] = c * x - s * y;
        S[j * BJ_LD + col] = s * x + c * y;
      }
      __syncthreads();
      // columns i, j of S and of J
      for (int t = tid; t < BJ_B * BJ_S; t += blockDim.x) {
        const int e = t / BJ_S, row = t % BJ_S;
        if (sn[e] == T(0)) continue;
        const int i = pp[e], j = qq[e];
        const T c = cs[e], s = sn[e];
        const T x = S[row * BJ_LD + i], y = S[row * BJ_LD + j];
        S[row * BJ_LD + i] = c * x - s * y;
        S[row * BJ_LD + j] = s * x + c * y;
        const T u = J[row * BJ_LD + i], v = J[row * BJ_LD + j];
        J[row * BJ_LD + i] = c * u - s * v;
        J[row * BJ_LD + j] = s * u + c * v;
      }
      __syncthreads();
      if (tid < BJ_B && sn[tid] != T(0)) {
        S[pp[tid] * BJ_LD + qq[tid]] = T(0);
        S[qq[tid] * BJ_LD + pp[tid]] = T(0);
      }
      __syncthreads();
    }
    if (tid == 0 && any_sweep) any = 1;
    __syncthreads();
    if (!any_sweep) break;
  }
  T* Jo = Jb + (int64_t)k * BJ_S * BJ_S;
  for (int t = tid; t < BJ_S * BJ_S; t += blockDim.x) Jo[t] = J[(t / BJ_S) * BJ_LD + t % BJ_S];
  for (int t = tid; t < BJ_S; t += blockDim.x) lam[(int64_t)k * BJ_S + t] = S[t * BJ_LD + t];
  if (tid == 0) rotated[k] = any;
}

// M[:, idx(p,q)] <- M[:, idx(p,q)] J_k for every pair k (rows in chunks of 32).
template <typename T, int BJ_B>
__global__ void __launch_bounds__(256) k_bj_cols(T* __restrict__ M, int np, int nb, int r, const T* __restrict__ Jb,
                                                 const int* __restrict__ rotated) {
  constexpr int BJ_S = 2 * BJ_B;
  const int k = blockIdx.y;
  if (!rotated[k]) return;
  __shared__ T Js[BJ_S][BJ_S + 1];
  __shared__ T Xs[32][BJ_S + 1];
  int p, q;
  bj_pair(k, r, nb, p, q);
  const T* Jk = Jb + (int64_t)k * BJ_S * BJ_S;
  for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) Js[t / BJ_S][t % BJ_S] = Jk[t];
  const int r0 = blockIdx.x * 32;
  for (int t = threadIdx.x; t < 32 * BJ_S; t += blockDim.x) {
    const int rr = t / BJ_S, c = t % BJ_S;
    Xs[rr][c] = (r0 + rr < np) ? M[(int64_t)(r0 + rr) * np + bj_index<BJ_B>(c, p, q)] : T(0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * BJ_S; t += blockDim.x) {
    const int rr = t / BJ_S, c = t % BJ_S;
    if (r0 + rr >= np) continue;
    T acc = T(0);
#pragma unroll 8
    for (int l = 0; l < BJ_S; ++l) acc = fma(Xs[rr][l], Js[l][c], acc);
    M[(int64_t)(r0 + rr) * np + bj_index<BJ_B>(c, p, q)] = acc;
  }
}

// A[idx(p,q), :] <- J_k^T A[idx(p,q), :] for every pair k (columns in chunks
// of one block); the pair's own BJ_S x BJ_S block becomes diag(lambda_k).
template <typename T, int BJ_B>
__global__ void __launch_bounds__(256) k_bj_rows(T* __restrict__ A, int np, int nb, int r, const T* __restrict__ Jb,
                                                 const T* __restrict__ lam, const int* __restrict__ rotated) {
  constexpr int BJ_S = 2 * BJ_B;
  const int k = blockIdx.y;
  if (!rotated[k]) return;
  __shared__ T Js[BJ_S][BJ_S + 1];
  __shared__ T Xs[BJ_S][BJ_B + 1];
  int p, q;
  bj_pair(k, r, nb, p, q);
  const int cblk = blockIdx.x, c0 = cblk * BJ_B;
  if (cblk == p || cblk == q) {
    // own block columns: diag(lambda) in rows idx(p,q), columns of this block
    const int off = cblk == p ? 0 : BJ_B;
    for (int t = threadIdx.x; t < BJ_S * BJ_B; t += blockDim.x) {
      const int i = t / BJ_B, c = t % BJ_B;
      A[(int64_t)bj_index<BJ_B>(i, p, q) * np + c0 + c] = (i == off + c) ? lam[(int64_t)k * BJ_S + i] : T(0);
    }
    return;
  }
  const T* Jk = Jb + (int64_t)k * BJ_S * BJ_S;
  for (int t = threadIdx.x; t < BJ_S * BJ_S; t += blockDim.x) Js[t / BJ_S][t % BJ_S] = Jk[t];
  for (int t = threadIdx.x; t < BJ_S * BJ_B; t += blockDim.x) {
    const int i = t / BJ_B, c = t % BJ_B;
    Xs[i][c] = A[(int64_t)bj_index<BJ_B>(i, p, q) * np + c0 + c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < BJ_S * BJ_B; t += blockDim.x) {
    const int i = t / BJ_B, c = t % BJ_B;
    T acc = T(0);
#pragma unroll 8
    for (int l = 0; l < BJ_S; ++l) acc = fma(Js[l][i], Xs[l][c], acc);
    A[(int64_t)bj_index<BJ_B>(i, p, q) * np + c0 + c] = acc;
  }
}

// partial sums of the squared off-diagonal and total entries of the leading n x n part
template <typename T>
__global__ void k_bj_norms(const T* __restrict__ A, int np, int n, double* __restrict__ part) {
  __shared__ double so[256], st[256];
  double o = 0.0, a = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const double v = (double)A[(int64_t)i * np + j];
    a += v * v;
    if (i != j) o += v * v;
  }
  so[threadIdx.x] = o;
  st[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      so[threadIdx.x] += so[threadIdx.x + w];
      st[threadIdx.x] += st[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = so[0];
    part[2 * blockIdx.x + 1] = st[0];
  }
}

template <typename T>
__global__ void k_bj_out(const T* __restrict__ A, const T* __restrict__ V, int np, int n, T* __restrict__ Vo, int ldv,
                         T* __restrict__ w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  Vo[(int64_t)i * ldv + j] = V[(int64_t)i * np + j];
  if (i == j) w[i] = A[(int64_t)i * np + i];
}

constexpr int BJ_NORM_BLOCKS = 128;

}  // namespace

// ------------------------------------------------------------------ host side
void launch_chol_blocked(double* A, int n, int lda, int* info, double* min_ratio, double* scratch,
                         cudaStream_t st) {
  // scratch: n (original diagonal) + CB * n (transposed panel) doubles
  double* d0 = scratch;
  double* T = scratch + n;
  cudaMemsetAsync(info, 0, sizeof(int), st);
  if (min_ratio) {
    k_copy_diag<<<nblk(n, 256), 256, 0, st>>>(A, n, lda, d0);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  for (int j0 = 0; j0 < n; j0 += CB) {
    const int b = std::min(CB, n - j0);
    const int m = n - j0 - b;
    k_chol_diag<<<1, 1024, 0, st>>>(A, lda, j0, b, info);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (m <= 0) break;
    k_chol_panel<<<nblk(m, 128), 128, 0, st>>>(A, lda, j0, b, n);
    k_panel_transpose<<<nblk((int64_t)m * b, 256), 256, 0, st>>>(A, lda, j0, b, n, T);
    g_launches.fetch_add(2, std::memory_order_relaxed);
    // A22 -= L21 L21^T (the whole square; only its lower triangle is used)
    double* A22 = A + (int64_t)(j0 + b) * lda + j0 + b;
    launch_gemm_nn(m, m, b, -1.0, A + (int64_t)(j0 + b) * lda + j0, lda, T, m, 1.0, A22, lda, st);
  }
  k_zero_upper<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(A, n, lda);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (min_ratio) {
    k_chol_ratio<<<1, 1024, 0, st>>>(A, n, lda, d0, info, min_ratio);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
}

int64_t chol_blocked_scratch(int n) { return (int64_t)n + (int64_t)CB * n; }

// Li = L^-1 (lower, n x n, ld ldi), 2 x 2 block recursion down to 128-wide
// diagonal blocks, which the column-per-thread kernel inverts.
// scratch: n * n / 4 doubles (the largest off-diagonal block).
void launch_trinv_blocked(const double* L, int n, int lda, double* Li, int ldi, double* scratch, cudaStream_t st) {
  if (n <= 128) {
    launch_trinv_lower(L, n, lda, Li, ldi, st);
    return;
  }
  const int n1 = (n / 2 + 63) / 64 * 64, n2 = n - n1;
  launch_trinv_blocked(L, n1, lda, Li, ldi, scratch, st);
  launch_trinv_blocked(L + (int64_t)n1 * lda + n1, n2, lda, Li + (int64_t)n1 * ldi + n1, ldi, scratch, st);
  // Li21 = -Li22 (L21 Li11); T = L21 Li11 is n2 x n1
  launch_gemm_nn(n2, n1, n1, 1.0, L + (int64_t)n1 * lda, lda, Li, ldi, 0.0, scratch, n1, st);
  launch_gemm_nn(n2, n1, n2, -1.0, Li + (int64_t)n1 * ldi + n1, ldi, scratch, n1, 0.0, Li + (int64_t)n1 * ldi, ldi,
                 st);
  k_zero_block<<<nblk((int64_t)n1 * n2, 256), 256, 0, st>>>(Li + n1, n1, n2, ldi);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

constexpr int BJ_BLOCK = 16;   // block Jacobi block size of both stages

static int64_t bj_scratch_bytes(int n, int elem, int B) {
  const int S = 2 * B;
  const int nb0 = (n + B - 1) / B;
  const int nb = std::max(2, nb0 + (nb0 & 1));
  const int64_t np = (int64_t)nb * B;
  const int64_t pairs = nb / 2;
  return elem * (2 * np * np + pairs * S * S + pairs * S) + (int64_t)sizeof(int) * pairs +
         (int64_t)sizeof(double) * 2 * BJ_NORM_BLOCKS + 1024;
}

int64_t block_jacobi_scratch_bytes(int n, int elem) { return bj_scratch_bytes(n, elem, BJ_BLOCK); }

// Symmetric C (n x n, FP64, ldc) = V diag(w) V^T by block Jacobi in precision T.
// Sweeps until the off-diagonal square sum is <= tol2 times the total or
// max_sweeps; returns 0 on convergence, 1 if the sweeps ran out, -1 on a CUDA
// error.  The only host synchronisation is the norm check after each sweep.
namespace {
template <typename T, int BJ_B>
int block_jacobi_b(const double* C, int n, int ldc, T* V, int ldv, T* w, int max_sweeps, double tol2, void* scratch,
                   cudaStream_t st, double* ratio_out) {
  constexpr int BJ_S = 2 * BJ_B, BJ_LD = BJ_S + 1;
  const int nb0 = (n + BJ_B - 1) / BJ_B;
  const int nb = std::max(2, nb0 + (nb0 & 1));
  const int np = nb * BJ_B;
  const int pairs = nb / 2;
  T* A = reinterpret_cast<T*>(scratch);
  T* Vp = A + (int64_t)np * np;
  T* Jb = Vp + (int64_t)np * np;
  T* lam = Jb + (int64_t)pairs * BJ_S * BJ_S;
  int* rot = reinterpret_cast<int*>(lam + (int64_t)pairs * BJ_S);
  double* part = reinterpret_cast<double*>(((uintptr_t)(rot + pairs) + 255) & ~(uintptr_t)255);
  k_bj_pad<T><<<nblk((int64_t)np * np, 256), 256, 0, st>>>(C, n, ldc, A, Vp, np);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const size_t smem = sizeof(T) * 2 * BJ_S * BJ_LD;
  if (cudaFuncSetAttribute(k_bj_solve<T, BJ_B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  std::vector<double> hp(2 * BJ_NORM_BLOCKS);
  int rc = 1;
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    k_bj_norms<T><<<BJ_NORM_BLOCKS, 256, 0, st>>>(A, np, n, part);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1;
    double off = 0.0, tot = 0.0;
    for (int b = 0; b < BJ_NORM_BLOCKS; ++b) {
      off += hp[2 * b];
      tot += hp[2 * b + 1];
    }
    if (ratio_out) *ratio_out = tot > 0.0 ? off / tot : 0.0;
    if (off <= tol2 * tot) {
      rc = 0;
      break;
    }
    if (sweep == max_sweeps) break;
    for (int r = 0; r < nb - 1; ++r) {
      k_bj_solve<T, BJ_B><<<pairs, 256, smem, st>>>(A, np, nb, r, Jb, lam, rot, 30);
      k_bj_cols<T, BJ_B><<<dim3(nblk(np, 32), pairs), 256, 0, st>>>(A, np, nb, r, Jb, rot);
      k_bj_rows<T, BJ_B><<<dim3(nb, pairs), 256, 0, st>>>(A, np, nb, r, Jb, lam, rot);
      k_bj_cols<T, BJ_B><<<dim3(nblk(np, 32), pairs), 256, 0, st>>>(Vp, np, nb, r, Jb, rot);
      g_launches.fetch_add(4, std::memory_order_relaxed);
    }
  }
  k_bj_out<T><<<nblk((int64_t)n * n, 256), 256, 0, st>>>(A, Vp, np, n, V, ldv, w);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return rc;
}
}  // namespace

// Both stages in 16-wide blocks: the subproblem solves run on one SM each (the
// FP64 ones at that SM's FP64 rate), so halving the block halves the solve work
// per sweep at the same update flops (measured: 280-atom Rayleigh-Ritz 5.41 s with
// 32-wide blocks, 4.95 s with 16)
template <typename T>
int block_jacobi(const double* C, int n, int ldc, T* V, int ldv, T* w, int max_sweeps, double tol2, void* scratch,
                 cudaStream_t st, double* ratio_out) {
  return block_jacobi_b<T, BJ_BLOCK>(C, n, ldc, V, ldv, w, max_sweeps, tol2, scratch, st, ratio_out);
}

template int block_jacobi<float>(const double*, int, int, float*, int, float*, int, double, void*, cudaStream_t,
                                 double*);
template int block_jacobi<double>(const double*, int, int, double*, int, double*, int, double, void*, cudaStream_t,
                                  double*);

}  // namespace efe
