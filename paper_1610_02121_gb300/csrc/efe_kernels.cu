// CUDA kernels of the enriched finite-element ChFSI library (sm_103a).
//
// Set-up kernels (efe_set_potential), FP64 / FP32-storage hot-path kernels of
// the Chebyshev filter (Sec. V) -- cell products of H^cc (Eq. Hcc) with a
// deterministic parity-coloured scatter, enrichment coupling H^ec / M^ec
// (Eqs. Hec, Mec) as sparse row products, the block-wise overlap inverse
// (Sec. IV.D) and the scaled three-term recurrence -- and the FP64 dense kernels
// of Cholesky-QR and Rayleigh-Ritz.  No FP atomics anywhere: every reduction
// has a fixed order, so results are bitwise reproducible run to run.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <atomic>

#include "efe_func.h"
#include "efe_kernels.h"

namespace efe {

std::atomic<int64_t> g_launches{0};

// SM count of the current device, looked up once per device ordinal
static std::atomic<int> g_sm_count[64];
int current_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 148;
  }
  int n = g_sm_count[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
    g_sm_count[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {
}  // namespace

namespace {

inline unsigned grid1(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// set_potential
// ---------------------------------------------------------------------------
__global__ void k_potential(const double* __restrict__ qpts, int64_t nq, const double* __restrict__ axyz,
                            const double* __restrict__ aZ, int na, int nuclear, const double* __restrict__ gA,
                            const double* __restrict__ gs, const double* __restrict__ gc, int nt, double omega,
                            double* __restrict__ V) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double x = qpts[4 * q], y = qpts[4 * q + 1], z = qpts[4 * q + 2];
  double v = 0.0;
  if (nuclear)
    for (int a = 0; a < na; ++a) {
      const double dx = x - axyz[3 * a], dy = y - axyz[3 * a + 1], dz = z - axyz[3 * a + 2];
      v -= aZ[a] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  for (int g = 0; g < nt; ++g) {
    const double dx = x - gc[3 * g], dy = y - gc[3 * g + 1], dz = z - gc[3 * g + 2];
    v += gA[g] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * gs[g] * gs[g]));
  }
  if (omega != 0.0) v += 0.5 * omega * omega * (x * x + y * y + z * z);
  V[q] = v;
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 1;
}

__global__ void k_gather_sum(int64_t n, const double* __restrict__ base, const int64_t* __restrict__ cptr,
                             const int64_t* __restrict__ cidx, const double* __restrict__ blk,
                             double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = base ? base[i] : 0.0;
  for (int64_t q = cptr[i]; q < cptr[i + 1]; ++q) v += blk[cidx[q]];
  out[i] = v;
}

__global__ void k_permute(int64_t n, const double* __restrict__ src, const int64_t* __restrict__ perm,
                          double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

__global__ void k_to_f32(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}

// ---------------------------------------------------------------------------
// hot path
// ---------------------------------------------------------------------------
// W_c(nodes of e) += H_e Y_e for every cell e of one parity colour.  Cells of
// one colour share no node, so the read-modify-write scatter needs no atomics.
// CTA = (cell, 32-column tile); 256 threads in 4 x 4 register blocks.
template <typename T>
__global__ void __launch_bounds__(256) k_cell_apply(const T* __restrict__ Hcc, const int32_t* __restrict__ cells,
                                                    MeshDev m, const T* __restrict__ Y, int64_t ldy,
                                                    T* __restrict__ W, int64_t ldw, int N) {
  const int64_t e = cells[blockIdx.x];
  const int c0 = blockIdx.y * 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  int64_t* gnode = reinterpret_cast<int64_t*>(smraw);                          // NL
  T(*Ys)[33] = reinterpret_cast<T(*)[33]>(smraw + sizeof(int64_t) * 128);       // NL x 33
  T(*Hs)[26] = reinterpret_cast<T(*)[26]>(smraw + sizeof(int64_t) * 128 + sizeof(T) * NL * 33);  // 128 x 26
  const int tid = threadIdx.x;
  const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]), k = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const int64_t NX = m.nn[0], NY = m.nn[1];
  if (tid < NL) {
    const int a = tid % NP1, b = (tid / NP1) % NP1, c = tid / (NP1 * NP1);
    gnode[tid] = (int64_t)(P * i + a) + NX * ((int64_t)(P * j + b) + NY * (int64_t)(P * k + c));
  }
  if (tid < 3 * 26) Hs[125 + tid / 26][tid % 26] = T(0);
  __syncthreads();
  for (int idx = tid; idx < NL * 32; idx += 256) {
    const int r = idx / 32, cc = idx % 32;
    const int col = c0 + cc;
    Ys[r][cc] = (col < N) ? Y[gnode[r] * ldy + col] : T(0);
  }
  const int ty = tid / 8, tx = tid % 8;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const T* He = Hcc + e * (int64_t)(NL * NL);
  for (int kc = 0; kc < NL; kc += 25) {
    __syncthreads();
    for (int idx = tid; idx < NL * 25; idx += 256) {
      const int r = idx / 25, kk = idx % 25;
      Hs[r][kk] = He[r * NL + kc + kk];
    }
    __syncthreads();
#pragma unroll 5
    for (int kk = 0; kk < 25; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Hs[ty * 4 + a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Ys[kc + kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = ty * 4 + a;
    if (r >= NL) continue;
    T* wr = W + gnode[r] * ldw;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int col = c0 + tx * 4 + b;
      if (col < N) wr[col] += acc[a][b];
    }
  }
}

template <typename T>
__global__ void k_spmm_nodes(int64_t nrows, const int32_t* __restrict__ rnode, const int64_t* __restrict__ ptr,
                             const int32_t* __restrict__ col, const double* __restrict__ val, double sgn,
                             const double* __restrict__ Xe, int64_t ldxe, T* __restrict__ out, int64_t ldo, int N) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int64_t g = rnode[w];
  const int64_t q0 = ptr[w], q1 = ptr[w + 1];
  for (int c = lane; c < N; c += 32) {
    double s = 0.0;
    for (int64_t q = q0; q < q1; ++q) s = fma(val[q], Xe[(int64_t)col[q] * ldxe + c], s);
    T* o = out + g * ldo + c;
    *o = (T)((double)(*o) + sgn * s);
  }
}

template <typename T>
__global__ void k_spmm_segments(const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_end,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                const double* __restrict__ scale, const T* __restrict__ Xc, int64_t ldx,
                                double* __restrict__ part, int N) {
  const int64_t seg = blockIdx.x;
  const int64_t q0 = seg_start[seg], q1 = seg_end[seg];
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    double s = 0.0;
    for (int64_t q = q0; q < q1; ++q) {
      const int64_t g = col[q];
      const double v = scale ? val[q] * scale[g] : val[q];
      s = fma(v, (double)Xc[g * ldx + c], s);
    }
    part[seg * N + c] = s;
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision enrichment coupling for many enrichment functions (the
// (n_E x N) array of the dense-tile kernels no longer fits in shared memory):
// FP32 products, FP64 sums across node chunks.
//
// Rows product W_e = C X_c over function groups: the functions of one atom
// with one cutoff share a support, hence one node list, so a CTA reads each
// node row of its column tile once for the whole group (k_g <= GRP_KMAX
// functions).  Work item = (group, node range); FP32 sums over chunks of 64
// nodes are added into FP64 per-item partials; a fixed-order reduction over
// the items of a function finishes.
constexpr int GRP_KMAX = 8;
constexpr int GRP_CHUNK = 64;
constexpr int GRP_CT = 128;   // columns per CTA (one per thread)

__global__ void __launch_bounds__(GRP_CT, 8) k_grp_rows(const int4* __restrict__ items, const int64_t* __restrict__ ec_ptr,
                                                    const int32_t* __restrict__ ec_col, const float* __restrict__ coef,
                                                    const float* __restrict__ Xc, int64_t ldx, double* __restrict__ part,
                                                    int N) {
  __shared__ int64_t nd[GRP_CHUNK];
  __shared__ float cf[GRP_KMAX][GRP_CHUNK];
  __shared__ int64_t rowp[GRP_KMAX];
  const int4 it = items[blockIdx.x];   // first function, functions, node positions [j0, j1)
  const int f0 = it.x, kg = it.y, j0 = it.z, j1 = it.w;
  const int c = blockIdx.y * GRP_CT + threadIdx.x;
  if (threadIdx.x < kg) rowp[threadIdx.x] = ec_ptr[f0 + threadIdx.x];
  double acc[GRP_KMAX];
#pragma unroll
  for (int k = 0; k < GRP_KMAX; ++k) acc[k] = 0.0;
  for (int j = j0; j < j1; j += GRP_CHUNK) {
    const int n = min(GRP_CHUNK, j1 - j);
    __syncthreads();
    const int64_t base = rowp[0];
    if (threadIdx.x < n) nd[threadIdx.x] = ec_col[base + j + threadIdx.x];
#pragma unroll
    for (int u = 0; u < GRP_KMAX * GRP_CHUNK / GRP_CT; ++u) {
      const int t = threadIdx.x + u * GRP_CT;
      const int k = t / GRP_CHUNK, jj = t % GRP_CHUNK;
      if (k < kg) cf[k][jj] = jj < n ? coef[rowp[k] + j + jj] : 0.f;
    }
    __syncthreads();
    if (c < N) {
      float s[GRP_KMAX];
#pragma unroll
      for (int k = 0; k < GRP_KMAX; ++k) s[k] = 0.f;
#pragma unroll 16
      for (int jj = 0; jj < n; ++jj) {
        const float x = Xc[nd[jj] * ldx + c];
#pragma unroll
        for (int k = 0; k < GRP_KMAX; ++k)
          if (k < kg) s[k] = fmaf(cf[k][jj], x, s[k]);
      }
#pragma unroll
      for (int k = 0; k < GRP_KMAX; ++k) acc[k] += (double)s[k];
    }
  }
  if (c < N) {
    double* o = part + (int64_t)blockIdx.x * GRP_KMAX * N + c;
#pragma unroll
    for (int k = 0; k < GRP_KMAX; ++k)
      if (k < kg) o[(int64_t)k * N] = acc[k];
  }
}

// out[f][c] = sgn * sum over the items of f's group (fixed order) + alpha * base[f][c]
__global__ void k_grp_reduce(int nE, const int32_t* __restrict__ f_it0, const int32_t* __restrict__ f_it1,
                             const int32_t* __restrict__ f_slot, const double* __restrict__ part, int N, double sgn,
                             const double* __restrict__ base, int64_t ldb, double alpha, double* __restrict__ out,
                             int64_t ldo) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nE * N) return;
  const int f = (int)(idx / N), c = (int)(idx % N);
  double s = 0.0;
  for (int it = f_it0[f]; it < f_it1[f]; ++it) s += part[((int64_t)it * GRP_KMAX + f_slot[f]) * N + c];
  double v = sgn * s;
  if (base) v += alpha * base[(int64_t)f * ldb + c];
  out[(int64_t)f * ldo + c] = v;
}

// Columns product W_c[node] += sgn * sum_f C[f][node] X_e[f] (node-major, FP32
// products and sums over the node's few functions; X_e in FP32, L2-resident).
__global__ void k_spmm_nodes_f32(int64_t nrows, const int32_t* __restrict__ rnode, const int64_t* __restrict__ ptr,
                                 const int32_t* __restrict__ col, const float* __restrict__ val, float sgn,
                                 const float* __restrict__ Xe, int64_t ldxe, float* __restrict__ out, int64_t ldo,
                                 int N) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int64_t g = rnode[w];
  const int64_t q0 = ptr[w], q1 = ptr[w + 1];
  for (int c = lane; c < N; c += 32) {
    float s = 0.f;
    for (int64_t q = q0; q < q1; ++q) s = fmaf(val[q], Xe[(int64_t)col[q] * ldxe + c], s);
    float* o = out + g * ldo + c;
    *o = fmaf(sgn, s, *o);
  }
}

// Narrow blocks (N <= 4: the Lanczos vector): the threads of a block split the
// entries of a segment instead of the columns, and the partials are added by a
// fixed shuffle tree and a fixed-order sum over the warps (reproducible).
constexpr int SPMM_NARROW = 4;

// one row per thread (N <= 4): the rows' few entries are walked by consecutive
// threads instead of one lane of a warp per row
template <typename T>
__global__ void k_spmm_nodes_rowthread(int64_t nrows, const int32_t* __restrict__ rnode,
                                       const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                       const double* __restrict__ val, double sgn, const double* __restrict__ Xe,
                                       int64_t ldxe, T* __restrict__ out, int64_t ldo, int N) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= nrows) return;
  const int64_t q0 = ptr[w], q1 = ptr[w + 1];
  double s[SPMM_NARROW] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t q = q0; q < q1; ++q) {
    const double v = val[q];
    const double* xr = Xe + (int64_t)col[q] * ldxe;
#pragma unroll
    for (int c = 0; c < SPMM_NARROW; ++c)
      if (c < N) s[c] = fma(v, xr[c], s[c]);
  }
  const int64_t g = rnode[w];
#pragma unroll
  for (int c = 0; c < SPMM_NARROW; ++c)
    if (c < N) {
      T* o = out + g * ldo + c;
      *o = (T)((double)(*o) + sgn * s[c]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_spmm_segments_narrow(const int64_t* __restrict__ seg_start,
                                                              const int64_t* __restrict__ seg_end,
                                                              const int32_t* __restrict__ col,
                                                              const double* __restrict__ val,
                                                              const double* __restrict__ scale,
                                                              const T* __restrict__ Xc, int64_t ldx,
                                                              double* __restrict__ part, int N) {
  __shared__ double red[8][SPMM_NARROW];
  const int64_t seg = blockIdx.x;
  const int64_t q0 = seg_start[seg], q1 = seg_end[seg];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double s[SPMM_NARROW] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int64_t g = col[q];
    const double v = scale ? val[q] * scale[g] : val[q];
#pragma unroll
    for (int c = 0; c < SPMM_NARROW; ++c)
      if (c < N) s[c] = fma(v, (double)Xc[g * ldx + c], s[c]);
  }
#pragma unroll
  for (int c = 0; c < SPMM_NARROW; ++c) {
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
    if (lane == 0) red[wp][c] = s[c];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k][threadIdx.x];
    part[seg * N + threadIdx.x] = t;
  }
}

__global__ void k_seg_reduce(int nrows, const int64_t* __restrict__ row_seg_ptr, const double* __restrict__ part,
                             double sgn, const double* __restrict__ base, int64_t ldb, double alpha_base,
                             double* __restrict__ out, int64_t ldo, int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nrows * N) return;
  const int r = (int)(idx / N), c = (int)(idx % N);
  double s = 0.0;
  for (int64_t sg = row_seg_ptr[r]; sg < row_seg_ptr[r + 1]; ++sg) s += part[sg * N + c];
  double v = sgn * s;
  if (base) v += alpha_base * base[(int64_t)r * ldb + c];
  out[(int64_t)r * ldo + c] = v;
}

// coef = {alpha, c, beta} of this degree, read from device memory (so a captured
// graph of the filter stays valid when the filter bounds change)
template <typename T>
// Yn may be Yp (the recurrence writes Y_k over Y_{k-2}; each element is read
// before it is written by the same thread), so those two are not restrict.
__global__ void k_cheb_combine(int64_t nrows, const double* __restrict__ rowscale, const T* __restrict__ X,
                               int64_t ldx, const T* __restrict__ Yc, int64_t ldc, const T* Yp,
                               int64_t ldp, T* Yn, int64_t ldn, const double* __restrict__ coef, int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * N) return;
  const double alpha = coef[0], cc = coef[1], beta = coef[2];
  const int64_t r = idx / N;
  const int c = (int)(idx % N);
  double x = (double)X[r * ldx + c];
  if (rowscale) x *= rowscale[r];
  double y = alpha * (x - cc * (double)Yc[r * ldc + c]);
  if (Yp) y += beta * (double)Yp[r * ldp + c];
  Yn[r * ldn + c] = (T)y;
}

template <typename T>
__global__ void k_row_scale(int64_t nrows, const double* __restrict__ s, const T* __restrict__ X, int64_t ldx,
                            T* __restrict__ Y, int64_t ldy, int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * N) return;
  const int64_t r = idx / N;
  const int c = (int)(idx % N);
  Y[r * ldy + c] = (T)(s[r] * (double)X[r * ldx + c]);
}

template <typename S, typename D>
__global__ void k_convert_rows(int64_t nrows, const S* __restrict__ X, int64_t ldx, D* __restrict__ Y, int64_t ldy,
                               int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * N) return;
  const int64_t r = idx / N;
  const int c = (int)(idx % N);
  Y[r * ldy + c] = (D)X[r * ldx + c];
}

template <typename T>
__global__ void k_zero_rows(int64_t nrows, T* __restrict__ X, int64_t ldx, int N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * N) return;
  X[(idx / N) * ldx + idx % N] = T(0);
}

// Cell products for a narrow block (N <= 8 columns, e.g. the single-vector
// Lanczos bound): one CTA per cell, each warp takes rows of H_e, lanes split
// the 125 columns and reduce with shuffles, so the cell matrix is read once
// with coalesced row loads and no work is spent on empty column tiles.
template <typename T, int NMAX>
__global__ void __launch_bounds__(256) k_cell_apply_narrow(const T* __restrict__ Hcc, const int32_t* __restrict__ cells,
                                                           MeshDev m, const T* __restrict__ Y, int64_t ldy,
                                                           T* __restrict__ W, int64_t ldw, int N) {
  const int64_t e = cells[blockIdx.x];
  __shared__ T ys[NL][NMAX];
  __shared__ int64_t gnode[NL];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]), k = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const int64_t NX = m.nn[0], NY = m.nn[1];
  if (tid < NL) {
    const int a = tid % NP1, b = (tid / NP1) % NP1, c = tid / (NP1 * NP1);
    const int64_t g = (int64_t)(P * i + a) + NX * ((int64_t)(P * j + b) + NY * (int64_t)(P * k + c));
    gnode[tid] = g;
#pragma unroll
    for (int cc = 0; cc < NMAX; ++cc) ys[tid][cc] = (cc < N) ? Y[g * ldy + cc] : T(0);
  }
  __syncthreads();
  const T* He = Hcc + e * (int64_t)(NL * NL);
  // four rows per warp at a time: sixteen independent loads in flight per lane,
  // and lane i writes row r0 + i
  for (int r0 = warp * 4; r0 < NL; r0 += 32) {
    T acc[4][NMAX];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int cc = 0; cc < NMAX; ++cc) acc[i][cc] = T(0);
    for (int kk = lane; kk < NL; kk += 32) {
      T h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) h[i] = (r0 + i < NL) ? He[(r0 + i) * NL + kk] : T(0);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int cc = 0; cc < NMAX; ++cc) acc[i][cc] = fma(h[i], ys[kk][cc], acc[i][cc]);
    }
    T mine[NMAX];
#pragma unroll
    for (int cc = 0; cc < NMAX; ++cc) mine[cc] = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int cc = 0; cc < NMAX; ++cc) {
        T v = acc[i][cc];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        v = __shfl_sync(0xffffffffu, v, 0);
        if (lane == i) mine[cc] = v;
      }
    if (lane < 4 && r0 + lane < NL) {
      T* wr = W + gnode[r0 + lane] * ldw;
#pragma unroll
      for (int cc = 0; cc < NMAX; ++cc)
        if (cc < N) wr[cc] += mine[cc];
    }
  }
}

// Node-major enrichment products (FP32 arithmetic, mixed-precision filter).
// The pattern nodes (the nodes that meet a support) form blocks of CPB
// consecutive nodes.  The functions touching a block are few (neighbouring
// nodes lie in the same supports); for each block the set-up lists them
// ("slots") and the values of H^ec and M^ec are kept as dense FP32 tiles
// (slots x CPB, slot-major), so a block's product is a small dense GEMM (4 x 4
// register tiles) over contiguous tile data, and each vector row is read once.
constexpr int CPB = 32;     // nodes per block
constexpr int CPF = 64;     // slots per GEMM pass (more: further passes)

// tile[pos[q]] = val[q]   (tiles zeroed beforehand)
__global__ void k_tile_scatter(int64_t nnz, const int64_t* __restrict__ pos, const float* __restrict__ val,
                               float* __restrict__ tile) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < nnz) tile[pos[q]] = val[q];
}

// Rows product: part[b][a][c] = sum over the blocks of CTA b of
//   sum_u tile[slot][u] * scale[g_u] * X[g_u][c]  accumulated at a = f(slot),
// in a CTA-private (n_E x N) shared-memory array.  CTA b takes the blocks
// cta_blk[b] .. cta_blk[b + 1] (a one-wave partition balanced by slot count).
// Shared rows are padded to a multiple of four floats so that every thread
// reads and updates its four columns with one 16-byte access.
template <typename T>
__global__ void __launch_bounds__(256) k_coup_rows(int64_t n_tn, const int64_t* __restrict__ cta_blk,
                                                   const int32_t* __restrict__ t_nodes,
                                                   const int64_t* __restrict__ slot_off,
                                                   const int32_t* __restrict__ slots, const float* __restrict__ tile,
                                                   const double* __restrict__ scale, const T* __restrict__ X,
                                                   int64_t ldx, int nE, int N, float* __restrict__ part) {
  extern __shared__ __align__(16) float smf[];
  const int ldy = (N + 3) & ~3;
  float* acc = smf;                                  // nE x ldy
  float* Ys = acc + (size_t)nE * ldy;                // CPB x ldy
  float* Ps = Ys + CPB * ldy;                        // CPF x CPB
  __shared__ int sf[CPF];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < nE * ldy; i += bd) acc[i] = 0.f;
  const int64_t b0 = cta_blk[blockIdx.x], b1 = cta_blk[blockIdx.x + 1];
  const int ncb = ldy / 4;
  for (int64_t bb = b0; bb < b1; ++bb) {
    const int64_t r0 = bb * CPB;
    const int nb = (int)min((int64_t)CPB, n_tn - r0);
    __syncthreads();
    if (sizeof(T) == 4 && (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0 && ldy <= ldx) {
      // padded FP32 rows: four columns per 16-byte load (columns past N are zero)
      const int q4 = ldy / 4;
      for (int i = tid; i < CPB * q4; i += bd) {
        const int u = i / q4, c4 = i % q4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u < nb) {
          const int64_t g = t_nodes[r0 + u];
          v = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + g * ldx + 4 * c4);
          if (scale) {
            const float sc = (float)scale[g];
            v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
          }
        }
        *reinterpret_cast<float4*>(Ys + u * ldy + 4 * c4) = v;
      }
    } else {
      for (int i = tid; i < CPB * ldy; i += bd) {
        const int u = i / ldy, c = i % ldy;
        float v = 0.f;
        if (u < nb && c < N) {
          const int64_t g = t_nodes[r0 + u];
          v = (float)X[g * ldx + c];
          if (scale) v *= (float)scale[g];
        }
        Ys[i] = v;
      }
    }
    const int64_t s0 = slot_off[bb], s1 = slot_off[bb + 1];
    for (int64_t sp = s0; sp < s1; sp += CPF) {
      const int nf = (int)min((int64_t)CPF, s1 - sp);
      __syncthreads();
      for (int i = tid; i < CPF * CPB; i += bd) Ps[i] = (i < nf * CPB) ? tile[sp * CPB + i] : 0.f;
      if (tid < nf) sf[tid] = slots[sp + tid];
      __syncthreads();
      const int nsb = (nf + 3) / 4;
      for (int t = tid; t < nsb * ncb; t += bd) {
        const int sb = t / ncb, cb = t % ncb;
        float r[4][4] = {};
#pragma unroll 8
        for (int u = 0; u < CPB; ++u) {
          float pv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) pv[i] = Ps[(sb * 4 + i) * CPB + u];
          const float4 y4 = *reinterpret_cast<const float4*>(Ys + u * ldy + cb * 4);
          const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) r[i][j] = fmaf(pv[i], yv[j], r[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int sl = sb * 4 + i;
          if (sl >= nf) break;
          float4* ar = reinterpret_cast<float4*>(acc + (size_t)sf[sl] * ldy + cb * 4);
          float4 a4 = *ar;
          a4.x += r[i][0];
          a4.y += r[i][1];
          a4.z += r[i][2];
          a4.w += r[i][3];
          *ar = a4;
        }
      }
    }
  }
  __syncthreads();
  float* Pp = part + (int64_t)blockIdx.x * nE * N;
  for (int i = tid; i < nE * N; i += bd) Pp[i] = acc[(i / N) * ldy + i % N];
}

// out[a][c] = alpha_base * base[a][c] + sgn * sum_b part[b][a][c]  (fixed order, FP64).
// A block takes 32 consecutive outputs; its 8 thread rows sum the partials
// b = y, y + 8, ... and the 8 row sums are added in order.
__global__ void __launch_bounds__(256) k_coup_reduce(int nb, int nE, int N, const float* __restrict__ part,
                                                     double sgn, const double* __restrict__ base, int64_t ldb,
                                                     double alpha_base, double* __restrict__ out, int64_t ldo) {
  __shared__ double rs[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int64_t idx = blockIdx.x * 32LL + x;
  const int64_t tot = (int64_t)nE * N;
  double s = 0.0;
  if (idx < tot)
    for (int b = y; b < nb; b += 8) s += (double)part[(int64_t)b * tot + idx];
  rs[y][x] = s;
  __syncthreads();
  if (y == 0 && idx < tot) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += rs[k][x];
    const int a = (int)(idx / N), c = (int)(idx % N);
    v *= sgn;
    if (base) v += alpha_base * base[(int64_t)a * ldb + c];
    out[(int64_t)a * ldo + c] = v;
  }
}

// Columns product for many enrichment functions, over the node blocks of the
// dense tiles: a CTA takes one block of CPB consecutive pattern nodes and one
// chunk of GRP_CT columns, stages the block's (slots x CPB) tile and the X_e
// rows of its slots (FP32) in shared memory -- each X_e row is read once per
// block instead of once per node -- and adds sgn * tile^T X_e into the block's
// W rows (FP32 products and sums over the block's functions).
__global__ void __launch_bounds__(GRP_CT) k_coup_cols_chunk(int64_t n_tn, const int32_t* __restrict__ t_nodes,
                                                           const int64_t* __restrict__ slot_off,
                                                           const int32_t* __restrict__ slots,
                                                           const float* __restrict__ tile, float sgn,
                                                           const float* __restrict__ Xe, int64_t ldxe, int N,
                                                           float* __restrict__ W, int64_t ldw) {
  __shared__ __align__(16) float T[CPF][CPB];
  __shared__ __align__(16) float Xs[CPF][GRP_CT];
  __shared__ int64_t nd[CPB];
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const int c = blockIdx.y * GRP_CT + tid;
  const int64_t r0 = b * CPB;
  const int nb = (int)min((int64_t)CPB, n_tn - r0);
  if (tid < nb) nd[tid] = t_nodes[r0 + tid];
  float acc[CPB];
#pragma unroll
  for (int i = 0; i < CPB; ++i) acc[i] = 0.f;
  const int64_t s0 = slot_off[b], s1 = slot_off[b + 1];
  for (int64_t sp = s0; sp < s1; sp += CPF) {
    const int nf = (int)min((int64_t)CPF, s1 - sp);
    __syncthreads();
    // independent loads, several in flight per thread
#pragma unroll 4
    for (int i = tid; i < nf * CPB; i += GRP_CT) T[i / CPB][i % CPB] = tile[sp * CPB + i];
#pragma unroll 8
    for (int k = 0; k < nf; ++k) Xs[k][tid] = c < N ? Xe[(int64_t)slots[sp + k] * ldxe + c] : 0.f;
    __syncthreads();
    for (int k = 0; k < nf; ++k) {
      const float x = Xs[k][tid];
      const float4* t4 = reinterpret_cast<const float4*>(T[k]);
#pragma unroll
      for (int i4 = 0; i4 < CPB / 4; ++i4) {
        const float4 tv = t4[i4];
        acc[4 * i4] = fmaf(tv.x, x, acc[4 * i4]);
        acc[4 * i4 + 1] = fmaf(tv.y, x, acc[4 * i4 + 1]);
        acc[4 * i4 + 2] = fmaf(tv.z, x, acc[4 * i4 + 2]);
        acc[4 * i4 + 3] = fmaf(tv.w, x, acc[4 * i4 + 3]);
      }
    }
  }
  // The block's results leave through shared memory: one bulk reduce-add per W
  // row segment, performed in L2, so no W value travels back to the SM (W rows
  // are padded to a multiple of 8 values; columns at or past N add zeros).
  __syncthreads();                 // every thread is done with Xs
  float* res = &Xs[0][0];          // CPB x GRP_CT results (CPB <= CPF)
#pragma unroll
  for (int i = 0; i < CPB; ++i) res[i * GRP_CT + tid] = sgn * acc[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid < nb) {
    const int c0 = blockIdx.y * GRP_CT;
    const uint32_t bytes = (uint32_t)((min(GRP_CT, N - c0) + 3) / 4 * 16);
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(res + tid * GRP_CT);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(
                     W + nd[tid] * ldw + c0),
                 "r"(src), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

// The same columns product with each node's own entries only (the transposed
// pattern: node rows, FP32 values and each entry's slot within its block)
// instead of the block's dense tile, which is mostly zeros when many functions
// meet a block (about 8 of 40 slots per node at 280 atoms).
constexpr int CPE = 1024;   // entries of a block staged at a time
__global__ void __launch_bounds__(GRP_CT) k_coup_cols_sparse(int64_t n_tn, const int32_t* __restrict__ t_nodes,
                                                            const int64_t* __restrict__ t_ptr,
                                                            const int32_t* __restrict__ t_slot,
                                                            const float* __restrict__ val,
                                                            const int64_t* __restrict__ slot_off,
                                                            const int32_t* __restrict__ slots, float sgn,
                                                            const float* __restrict__ Xe, int64_t ldxe, int N,
                                                            float* __restrict__ W, int64_t ldw) {
  __shared__ float Xs[CPF][GRP_CT];
  __shared__ float2 ent[CPE];          // (value, slot as int bits)
  __shared__ int64_t nd[CPB];
  __shared__ int eoff[CPB + 1];
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const int c = blockIdx.y * GRP_CT + tid;
  const int64_t r0 = b * CPB;
  const int nb = (int)min((int64_t)CPB, n_tn - r0);
  const int64_t q0 = t_ptr[r0];
  if (tid <= nb) eoff[tid] = (int)(t_ptr[r0 + tid] - q0);
  if (tid < nb) nd[tid] = t_nodes[r0 + tid];
  const int64_t s0 = slot_off[b];
  const int ns = (int)(slot_off[b + 1] - s0);
  float acc[CPB];
#pragma unroll
  for (int i = 0; i < CPB; ++i) acc[i] = 0.f;
  // slots in passes of CPF; entries whose slot falls in the pass are summed
  for (int sp = 0; sp < ns; sp += CPF) {
    const int nf = min(CPF, ns - sp);
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < nf; ++k) Xs[k][tid] = c < N ? Xe[(int64_t)slots[s0 + sp + k] * ldxe + c] : 0.f;
    const int ne = eoff[nb];
    for (int e0 = 0; e0 < ne; e0 += CPE) {
      const int m = min(CPE, ne - e0);
      __syncthreads();
      for (int e = tid; e < m; e += GRP_CT) ent[e] = make_float2(val[q0 + e0 + e], __int_as_float(t_slot[q0 + e0 + e]));
      __syncthreads();
#pragma unroll
      for (int i = 0; i < CPB; ++i) {
        if (i >= nb) break;
        const int a0 = max(eoff[i] - e0, 0), a1 = min(eoff[i + 1] - e0, m);
        float s = acc[i];
        for (int e = a0; e < a1; ++e) {
          const float2 v = ent[e];
          const int k = __float_as_int(v.y) - sp;
          if (k >= 0 && k < nf) s = fmaf(v.x, Xs[k][tid], s);
        }
        acc[i] = s;
      }
    }
  }
  if (c < N) {
    // read-modify-write in two halves of 16 rows (loads batched per half)
#pragma unroll
    for (int h = 0; h < CPB; h += CPB / 2) {
      float wv[CPB / 2];
#pragma unroll
      for (int i = 0; i < CPB / 2; ++i) wv[i] = h + i < nb ? W[nd[h + i] * ldw + c] : 0.f;
#pragma unroll
      for (int i = 0; i < CPB / 2; ++i)
        if (h + i < nb) W[nd[h + i] * ldw + c] = fmaf(sgn, acc[h + i], wv[i]);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64-grade enrichment coupling on the FP32 pipe (with the tensor-core FP64
// engine selected; this part retires FP64 instructions at about 1/64 of the
// FP32 rate, which bounds the plain FP64 coupling).  Every FP64 coefficient is
// kept as an unevaluated sum of two floats (hi = nearest float, lo = the
// rounded remainder) and every FP64 vector value is cut into two floats by its
// bits; a product takes its high part exactly (the fma error term) plus the
// two cross terms, and the sums run in double-float arithmetic (error-free
// two-sum of the high words, low words added).  Error: a few units of 2^-48 of
// sum |a||x| (the dropped lo*lo term and the 24-bit low words).  Values must
// lie below 2^126 in magnitude (larger ones become infinite); parts below the
// FP32 normal range are dropped (relative size below 2^-126).

// FP32 value with the bits of the unbiased exponent ex and the 24-bit significand
// m (leading bit set, given as an integer); 0 below the normal range.
__device__ __forceinline__ float df_make(uint32_t sgn, int ex, uint32_t m24) {
  const int be = ex + 127;
  if (be <= 0) return 0.f;
  if (be >= 255) return __uint_as_float(sgn | 0x7F800000u);
  return __uint_as_float(sgn | ((uint32_t)be << 23) | (m24 & 0x7FFFFFu));
}

// x = hi + lo: hi = the leading 24 significant bits of x, lo = the next 29
// bits truncated to 24 (integer operations only)
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const uint32_t sgn = (uint32_t)(b >> 63) << 31;
  if (e == 0) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  const int ex = e - 1023;
  hi = df_make(sgn, ex, (uint32_t)(b >> 29) | 0x800000u);
  const uint32_t r = (uint32_t)(b & 0x1FFFFFFFull);
  if (r == 0) {
    lo = 0.f;
    return;
  }
  const int nb = 32 - __clz(r);   // significant bits of r (1..29)
  const uint32_t m = nb > 24 ? (r >> (nb - 24)) : (r << (24 - nb));
  lo = df_make(sgn, ex - 52 + nb - 1, m);
}

// exact FP64 value of a float (integer operations only; 0 for subnormal floats)
__device__ __forceinline__ double df_f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t be = (u >> 23) & 0xFFu;
  if (be == 0) return 0.0;
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                  ((unsigned long long)(be == 255 ? 2047u : be - 127u + 1023u) << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// (S, C) += (ah + al) (xh + xl)
__device__ __forceinline__ void df_fma(float ah, float al, float xh, float xl, float& S, float& C) {
  const float p = ah * xh;
  const float c = fmaf(ah, xl, fmaf(al, xh, fmaf(ah, xh, -p)));
  const float s = S + p;
  const float bb = s - S;
  const float err = (S - (s - bb)) + (p - bb);
  S = s;
  C += err + c;
}

// FP64 coefficients -> (hi, lo) float pairs, optionally times scale[col[q]]
__global__ void k_df_coef(int64_t n, const double* __restrict__ v, const double* __restrict__ scale,
                          const int32_t* __restrict__ col, float2* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double a = scale ? v[q] * scale[col[q]] : v[q];
  const float hi = (float)a;
  out[q] = make_float2(hi, (float)(a - (double)hi));
}

// rows of an FP64 block -> (hi, lo) pairs by bits (rows x N, ld in, N out)
__global__ void k_df_rows(int64_t rows, int N, const double* __restrict__ X, int64_t ldx, float2* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * N) return;
  float hi, lo;
  df_split(X[(i / N) * ldx + i % N], hi, lo);
  out[i] = make_float2(hi, lo);
}

// Columns product out[node] = out[node] + sgn sum_q val[q] Xe[col[q]] (one warp
// per pattern node, lanes over the columns); Xe2: the enrichment rows as (hi, lo)
// pairs (k_df_rows).  The FP64 sum is added to out by a reduction performed in L2
// (each out value receives one addition per launch: the pattern nodes are distinct)
__global__ void k_spmm_nodes_df(int64_t nrows, const int32_t* __restrict__ rnode, const int64_t* __restrict__ ptr,
                                const int32_t* __restrict__ col, const float2* __restrict__ val, float sgn,
                                const float2* __restrict__ Xe2, int N, double* __restrict__ out, int64_t ldo) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int64_t g = rnode[w];
  const int64_t q0 = ptr[w], q1 = ptr[w + 1];
  for (int c = lane; c < N; c += 32) {
    float S = 0.f, C = 0.f;
    for (int64_t q = q0; q < q1; ++q) {
      const float2 a = val[q];
      const float2 x = Xe2[(int64_t)col[q] * N + c];
      df_fma(sgn * a.x, sgn * a.y, x.x, x.y, S, C);
    }
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(out + g * ldo + c), "d"(df_f2d(S) + df_f2d(C))
                 : "memory");
  }
}

// Rows product over function groups (the items of k_grp_rows): part[item][k][c]
// = sum over the item's nodes of coef[k][node] Xc[node][c], FP64 Xc, double-float
// sums over the whole item
__global__ void __launch_bounds__(GRP_CT) k_grp_rows_df(const int4* __restrict__ items, const int64_t* __restrict__ ec_ptr,
                                                       const int32_t* __restrict__ ec_col, const float2* __restrict__ coef,
                                                       const double* __restrict__ Xc, int64_t ldx, double* __restrict__ part,
                                                       int N) {
  __shared__ int64_t nd[GRP_CHUNK];
  __shared__ float2 cf[GRP_KMAX][GRP_CHUNK];
  __shared__ int64_t rowp[GRP_KMAX];
  const int4 it = items[blockIdx.x];
  const int f0 = it.x, kg = it.y, j0 = it.z, j1 = it.w;
  const int c = blockIdx.y * GRP_CT + threadIdx.x;
  if (threadIdx.x < kg) rowp[threadIdx.x] = ec_ptr[f0 + threadIdx.x];
  float S[GRP_KMAX], C[GRP_KMAX];
#pragma unroll
  for (int k = 0; k < GRP_KMAX; ++k) {
    S[k] = 0.f;
    C[k] = 0.f;
  }
  for (int j = j0; j < j1; j += GRP_CHUNK) {
    const int n = min(GRP_CHUNK, j1 - j);
    __syncthreads();
    const int64_t base = rowp[0];
    if (threadIdx.x < n) nd[threadIdx.x] = ec_col[base + j + threadIdx.x];
#pragma unroll
    for (int u = 0; u < GRP_KMAX * GRP_CHUNK / GRP_CT; ++u) {
      const int t = threadIdx.x + u * GRP_CT;
      const int k = t / GRP_CHUNK, jj = t % GRP_CHUNK;
      if (k < kg) cf[k][jj] = jj < n ? coef[rowp[k] + j + jj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (c < N) {
#pragma unroll 4
      for (int jj = 0; jj < n; ++jj) {
        float xh, xl;
        df_split(Xc[nd[jj] * ldx + c], xh, xl);
#pragma unroll
        for (int k = 0; k < GRP_KMAX; ++k)
          if (k < kg) df_fma(cf[k][jj].x, cf[k][jj].y, xh, xl, S[k], C[k]);
      }
    }
  }
  if (c < N) {
    double* o = part + (int64_t)blockIdx.x * GRP_KMAX * N + c;
#pragma unroll
    for (int k = 0; k < GRP_KMAX; ++k)
      if (k < kg) o[(int64_t)k * N] = df_f2d(S[k]) + df_f2d(C[k]);
  }
}

// Columns product: W[g_u][c] += sgn * sum_slot tile[slot][u] * Xe[f(slot)][c]
// (Xe staged in shared memory as FP32, rows padded to four floats), same block
// tiles and CTA partition as the rows product.
template <typename T>
__global__ void __launch_bounds__(256) k_coup_cols(int64_t n_tn, const int64_t* __restrict__ cta_blk,
                                                   const int32_t* __restrict__ t_nodes,
                                                   const int64_t* __restrict__ slot_off,
                                                   const int32_t* __restrict__ slots, const float* __restrict__ tile,
                                                   float sgn, const double* __restrict__ Xe, int64_t ldxe, int nE,
                                                   int N, T* __restrict__ W, int64_t ldw) {
  extern __shared__ __align__(16) float smf[];
  const int ldx = (N + 3) & ~3;
  float* xs = smf;                                   // nE x ldx
  float* Ps = xs + (size_t)nE * ldx;                 // CPF x CPB
  __shared__ int sf[CPF];
  __shared__ int64_t sg[CPB];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < nE * ldx; i += bd) {
    const int a = i / ldx, c = i % ldx;
    xs[i] = c < N ? (float)Xe[(int64_t)a * ldxe + c] : 0.f;
  }
  const int64_t b0 = cta_blk[blockIdx.x], b1 = cta_blk[blockIdx.x + 1];
  const int ncb = ldx / 4;
  for (int64_t bb = b0; bb < b1; ++bb) {
    const int64_t r0 = bb * CPB;
    const int nb = (int)min((int64_t)CPB, n_tn - r0);
    const int64_t s0 = slot_off[bb], s1 = slot_off[bb + 1];
    // thread t owns output tiles (4 nodes x 4 columns) t and t + bd of each group of
    // 2 bd tiles; results summed over the slot passes
    const int ntile = (CPB / 4) * ncb;
    __syncthreads();
    if (tid < nb) sg[tid] = t_nodes[r0 + tid];
    for (int tg = 0; tg < ntile; tg += 2 * bd) {
      float r[2][4][4] = {};
      for (int64_t sp = s0; sp < s1; sp += CPF) {
        const int nf = (int)min((int64_t)CPF, s1 - sp);
        __syncthreads();
        for (int i = tid; i < CPF * CPB; i += bd) Ps[i] = (i < nf * CPB) ? tile[sp * CPB + i] : 0.f;
        if (tid < nf) sf[tid] = slots[sp + tid];
        __syncthreads();
        for (int k = 0; k < 2; ++k) {
          const int t = tg + tid + k * bd;
          if (t >= ntile) break;
          const int ub = t / ncb, cb = t % ncb;
          for (int sl = 0; sl < nf; ++sl) {
            const float4 x4 = *reinterpret_cast<const float4*>(xs + (size_t)sf[sl] * ldx + cb * 4);
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
            const float4 p4 = *reinterpret_cast<const float4*>(Ps + sl * CPB + ub * 4);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) r[k][i][j] = fmaf(pv[i], xv[j], r[k][i][j]);
          }
        }
      }
      for (int k = 0; k < 2; ++k) {
        const int t = tg + tid + k * bd;
        if (t >= ntile) break;
        const int ub = t / ncb, cb = t % ncb;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int u = ub * 4 + i;
          if (u >= nb) break;
          T* wr = W + sg[u] * ldw + cb * 4;
          if (sizeof(T) == 4 && (ldw & 3) == 0 && ((uintptr_t)W & 15) == 0 && cb * 4 + 4 <= ldw) {
            // padded FP32 rows: one 16-byte update (columns past N add zero)
            float4* w4 = reinterpret_cast<float4*>(wr);
            float4 o = *w4;
            o.x += sgn * r[k][i][0];
            o.y += sgn * r[k][i][1];
            o.z += sgn * r[k][i][2];
            o.w += sgn * r[k][i][3];
            *w4 = o;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (cb * 4 + j < N) wr[j] = (T)((float)wr[j] + sgn * r[k][i][j]);
          }
        }
      }
    }
  }
}

// Chebyshev combine on 16-byte aligned FP32 rows (ld multiple of 4): four columns per thread.
// as k_cheb_combine: Yn may be Yp.  X (the cell-product output of this degree)
// is zeroed after it is read, ready to accumulate the next degree's products.
__global__ void k_cheb_combine_f4(int64_t nrows, int ld4, const double* __restrict__ rowscale,
                                  const float4* __restrict__ X, const float4* __restrict__ Yc,
                                  const float4* Yp, float4* Yn,
                                  const double* __restrict__ coef) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * ld4) return;
  const float alpha = (float)coef[0], cc = (float)coef[1], beta = (float)coef[2];
  const int64_t r = idx / ld4;
  const float sc = rowscale ? (float)rowscale[r] : 1.f;
  const float4 x = X[idx], y = Yc[idx];
  float4 o;
  o.x = alpha * (sc * x.x - cc * y.x);
  o.y = alpha * (sc * x.y - cc * y.y);
  o.z = alpha * (sc * x.z - cc * y.z);
  o.w = alpha * (sc * x.w - cc * y.w);
  if (Yp) {
    const float4 p = Yp[idx];
    o.x += beta * p.x;
    o.y += beta * p.y;
    o.z += beta * p.z;
    o.w += beta * p.w;
  }
  Yn[idx] = o;
}

// ---------------------------------------------------------------------------
// dense FP64
// ---------------------------------------------------------------------------
constexpr int GT = 48;  // output tile (16 x 16 threads, 3 x 3 each)

__global__ void __launch_bounds__(256) k_gemm_nn(int64_t M, int Nc, int K, double alpha,
                                                 const double* __restrict__ A, int64_t lda,
                                                 const double* __restrict__ B, int64_t ldb, double beta,
                                                 double* __restrict__ C, int64_t ldc, int64_t sA, int64_t sB,
                                                 int64_t sC) {
  __shared__ double As[16][GT + 1];
  __shared__ double Bs[16][GT + 1];
  // batch member blockIdx.z (strides 0 for a single product)
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;
  const int64_t row0 = (int64_t)blockIdx.x * GT;
  const int col0 = blockIdx.y * GT;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  double acc[3][3] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int idx = tid; idx < 16 * GT; idx += 256) {
      const int r = idx / 16, kk = idx % 16;
      As[kk][r] = (row0 + r < M && k0 + kk < K) ? A[(row0 + r) * lda + k0 + kk] : 0.0;
      const int kb = idx / GT, cc = idx % GT;
      Bs[kb][cc] = (k0 + kb < K && col0 + cc < Nc) ? B[(int64_t)(k0 + kb) * ldb + col0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[3], bv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) av[a] = As[kk][ty * 3 + a];
#pragma unroll
      for (int b = 0; b < 3; ++b) bv[b] = Bs[kk][tx * 3 + b];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t r = row0 + ty * 3 + a;
    if (r >= M) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int c = col0 + tx * 3 + b;
      if (c >= Nc) continue;
      double v = alpha * acc[a][b];
      if (beta != 0.0) v += beta * C[r * ldc + c];
      C[r * ldc + c] = v;
    }
  }
}

// Small products (fewer 48 x 48 tiles than SMs: the n_E x N coupling solves and
// the N x N Rayleigh-Ritz products): one output per thread in 16 x 16 tiles, so
// that several times more SMs share the FP64 work.  Same summation order (k
// ascending, one fused multiply-add each) as k_gemm_nn, hence the same bits.
__global__ void __launch_bounds__(256) k_gemm_nn_small(int64_t M, int Nc, int K, double alpha,
                                                       const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb, double beta,
                                                       double* __restrict__ C, int64_t ldc) {
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int64_t r = (int64_t)blockIdx.x * 16 + ty;
  const int c = blockIdx.y * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    As[ty][tx] = (r < M && k0 + tx < K) ? A[r * lda + k0 + tx] : 0.0;
    Bs[ty][tx] = (k0 + ty < K && c < Nc) ? B[(int64_t)(k0 + ty) * ldb + c] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (r < M && c < Nc) {
    double v = alpha * acc;
    if (beta != 0.0) v += beta * C[r * ldc + c];
    C[r * ldc + c] = v;
  }
}

constexpr int64_t TN_KC = 8192;

__global__ void __launch_bounds__(256) k_gemm_tn_part(int64_t K, int64_t kc, int Na, int Nb,
                                                      const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ B, int64_t ldb,
                                                      double* __restrict__ part, int sym) {
  // symmetric products: only tiles on or above the diagonal are formed
  if (sym && blockIdx.x > blockIdx.y) return;
  __shared__ double As[16][GT + 1];
  __shared__ double Bs[16][GT + 1];
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  const int64_t kb = (int64_t)blockIdx.z * kc;
  const int64_t ke = min(K, kb + kc);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  double acc[3][3] = {};
  for (int64_t k0 = kb; k0 < ke; k0 += 16) {
    for (int idx = tid; idx < 16 * GT; idx += 256) {
      const int kk = idx / GT, c = idx % GT;
      const bool okk = k0 + kk < ke;
      As[kk][c] = (okk && i0 + c < Na) ? A[(k0 + kk) * lda + i0 + c] : 0.0;
      Bs[kk][c] = (okk && j0 + c < Nb) ? B[(k0 + kk) * ldb + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[3], bv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) av[a] = As[kk][ty * 3 + a];
#pragma unroll
      for (int b = 0; b < 3; ++b) bv[b] = Bs[kk][tx * 3 + b];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  double* Pp = part + (int64_t)blockIdx.z * Na * Nb;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int r = i0 + ty * 3 + a;
    if (r >= Na) continue;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int c = j0 + tx * 3 + b;
      if (c < Nb) Pp[(int64_t)r * Nb + c] = acc[a][b];
    }
  }
}

__global__ void k_gemm_tn_reduce(int nsplit, int Na, int Nb, const double* __restrict__ part, double* __restrict__ C,
                                 int64_t ldc, int sym) {
  const int64_t idx0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx0 >= (int64_t)Na * Nb) return;
  const int64_t idx = idx0;
  int64_t src = idx;
  if (sym) {
    const int i = (int)(idx / Nb), j = (int)(idx % Nb);
    if (i / GT > j / GT) src = (int64_t)j * Nb + i;  // mirrored from the tile above the diagonal
  }
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * Na * Nb + src];
  C[(idx / Nb) * ldc + idx % Nb] = s;
}

// Right-looking Cholesky A = L L^T in one CTA (lower triangle; upper zeroed),
// n <= 2048.  Column j is scaled, kept in shared memory, and the trailing lower
// triangle is updated with one (row, column) pair per thread and step.
// min_ratio (optional): min_j L_jj^2 / A_jj, the smallest fraction of a
// column's squared norm outside the span of the columns before it (scale
// invariant; 1 / its square root bounds the column-scaled condition number).
__global__ void __launch_bounds__(1024) k_chol(double* A, int n, int lda, int* info, double* min_ratio) {
  __shared__ double piv, rmin;
  __shared__ int bad;
  __shared__ double d0[2048];
  __shared__ double lj[2048];
  const int tid = threadIdx.x, bd = blockDim.x;
  const bool track = min_ratio != nullptr;
  if (tid == 0) { bad = n > 2048 ? 1 : 0; rmin = 1.0; }
  __syncthreads();
  if (!bad && track)
    for (int i = tid; i < n; i += bd) d0[i] = A[(int64_t)i * lda + i];
  for (int j = 0; j < n && !bad; ++j) {
    __syncthreads();
    if (tid == 0) {
      const double d = A[(int64_t)j * lda + j];
      if (!(d > 0.0) || !isfinite(d)) bad = j + 1;
      else {
        piv = sqrt(d);
        A[(int64_t)j * lda + j] = piv;
        if (track) rmin = fmin(rmin, d / d0[j]);
      }
    }
    __syncthreads();
    if (bad) break;
    const int m = n - j - 1;
    for (int i = tid; i < m; i += bd) {
      const double v = A[(int64_t)(j + 1 + i) * lda + j] / piv;
      A[(int64_t)(j + 1 + i) * lda + j] = v;
      lj[i] = v;
    }
    __syncthreads();
    const int64_t tot = (int64_t)m * m;
    for (int64_t t = tid; t < tot; t += bd) {
      const int i = (int)(t / m), c = (int)(t % m);
      if (c <= i) A[(int64_t)(j + 1 + i) * lda + (j + 1 + c)] -= lj[i] * lj[c];
    }
  }
  __syncthreads();
  for (int64_t t = tid; t < (int64_t)n * n; t += bd) {
    const int i = (int)(t / n), c = (int)(t % n);
    if (c > i) A[(int64_t)i * lda + c] = 0.0;
  }
  if (tid == 0) {
    *info = bad;
    if (min_ratio) *min_ratio = bad ? 0.0 : rmin;
  }
}

// A += shift I, shift = coef * trace(A) (one CTA; the trace bounds ||X||_2^2 for A = X^T X).
__global__ void k_shift_diag(double* A, int n, int lda, double coef) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += A[(int64_t)i * lda + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double shift = coef * red[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * lda + i] += shift;
}

// Li = L^-1 (lower), one column per thread by forward substitution.
__global__ void k_trinv_lower(const double* __restrict__ L, int n, int lda, double* __restrict__ Li, int ldi) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    for (int i = 0; i < j; ++i) Li[(int64_t)i * ldi + j] = 0.0;
    for (int i = j; i < n; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) v -= L[(int64_t)i * lda + k] * Li[(int64_t)k * ldi + j];
      Li[(int64_t)i * ldi + j] = v / L[(int64_t)i * lda + i];
    }
  }
}

__global__ void k_transpose(const double* __restrict__ A, int n, int lda, double* __restrict__ B, int ldb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  B[(int64_t)j * ldb + i] = A[(int64_t)i * lda + j];
}

__global__ void k_symmetrize(double* A, int n, int lda) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (j <= i) return;
  const double v = 0.5 * (A[(int64_t)i * lda + j] + A[(int64_t)j * lda + i]);
  A[(int64_t)i * lda + j] = v;
  A[(int64_t)j * lda + i] = v;
}

__global__ void k_mirror_upper(double* A, int n, int lda) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  if (i > j) A[(int64_t)i * lda + j] = A[(int64_t)j * lda + i];
}

// Parallel cyclic Jacobi (round-robin pairing) for a symmetric n x n matrix in
// one CTA: A <- J^T A J with disjoint rotations per round, V <- V J.
// T = double, or float for the pre-diagonalisation of the mixed eigensolver;
// stops when the off-diagonal square sum is <= tol2 times the total.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(1024) k_jacobi(T* Ag, int n, int ldag, T* V, int ldv, T* w, int max_sweeps,
                                                 double tol2, int* info) {
  __shared__ T cs[1024], sn[1024];
  __shared__ int pp[1024], qq[1024];
  __shared__ double red[2][32];
  __shared__ int done;
  extern __shared__ double As_raw[];
  T* As_dyn = reinterpret_cast<T*>(As_raw);
  const int tid = threadIdx.x, bd = blockDim.x;
  // the working matrix lives in shared memory when it fits (n <= 150), else in global memory
  T* A = SMEM ? As_dyn : Ag;
  const int lda = SMEM ? n : ldag;
  if (SMEM) {
    for (int64_t t = tid; t < (int64_t)n * n; t += bd) As_dyn[t] = Ag[(t / n) * (int64_t)ldag + t % n];
    __syncthreads();
  }
  const int n2 = n + (n & 1);
  const int np = n2 / 2;
  for (int64_t t = tid; t < (int64_t)n * n; t += bd) V[(t / n) * ldv + t % n] = (t / n == t % n) ? T(1) : T(0);
  if (tid == 0) done = 0;
  int sweep = 0;
  for (; sweep <= max_sweeps; ++sweep) {
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int64_t t = tid; t < (int64_t)n * n; t += bd) {
      const double a = (double)A[(t / n) * lda + t % n];
      tot += a * a;
      if (t / n != t % n) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = off; red[1][tid >> 5] = tot; }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, st = 0.0;
      for (int i = 0; i < (bd + 31) / 32; ++i) { so += red[0][i]; st += red[1][i]; }
      done = (so <= tol2 * st) ? 1 : 0;
    }
    __syncthreads();
    if (done || sweep == max_sweeps) break;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int k = tid; k < np; k += bd) {
        const int s1 = k, s2 = n2 - 1 - k;
        const int pl1 = (s1 == 0) ? 0 : ((s1 - 1 + r) % (n2 - 1)) + 1;
        const int pl2 = (s2 == 0) ? 0 : ((s2 - 1 + r) % (n2 - 1)) + 1;
        const int p = min(pl1, pl2), q = max(pl1, pl2);
        if (q >= n) { pp[k] = -1; continue; }
        const T apq = A[(int64_t)p * lda + q];
        T c = T(1), s = T(0);
        if (apq != T(0)) {
          const T app = A[(int64_t)p * lda + p], aqq = A[(int64_t)q * lda + q];
          const T tau = (aqq - app) / (T(2) * apq);
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + t * t);
          s = t * c;
        }
        pp[k] = p; qq[k] = q; cs[k] = c; sn[k] = s;
      }
      __syncthreads();
      for (int64_t t = tid; t < (int64_t)n * np; t += bd) {
        const int i = (int)(t / np), k = (int)(t % np);
        const int p = pp[k];
        if (p < 0) continue;
        const int q = qq[k];
        const T c = cs[k], s = sn[k];
        T* Ai = A + (int64_t)i * lda;
        const T aip = Ai[p], aiq = Ai[q];
        Ai[p] = c * aip - s * aiq;
        Ai[q] = s * aip + c * aiq;
        T* Vi = V + (int64_t)i * ldv;
        const T vip = Vi[p], viq = Vi[q];
        Vi[p] = c * vip - s * viq;
        Vi[q] = s * vip + c * viq;
      }
      __syncthreads();
      for (int64_t t = tid; t < (int64_t)n * np; t += bd) {
        const int j = (int)(t / np), k = (int)(t % np);
        const int p = pp[k];
        if (p < 0) continue;
        const int q = qq[k];
        const T c = cs[k], s = sn[k];
        const T apj = A[(int64_t)p * lda + j], aqj = A[(int64_t)q * lda + j];
        A[(int64_t)p * lda + j] = c * apj - s * aqj;
        A[(int64_t)q * lda + j] = s * apj + c * aqj;
      }
      __syncthreads();
      for (int k = tid; k < np; k += bd) {
        const int p = pp[k];
        if (p < 0) continue;
        A[(int64_t)p * lda + qq[k]] = T(0);
        A[(int64_t)qq[k] * lda + p] = T(0);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += bd) w[i] = A[(int64_t)i * lda + i];
  if (tid == 0) *info = done ? 0 : 1;
}

__global__ void k_sort_eig(const double* __restrict__ w, const double* __restrict__ V, int n, int ldv,
                           double* __restrict__ ws, double* __restrict__ Vs, int ldvs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int rank = 0;
    const double wi = w[i];
    for (int j = 0; j < n; ++j) rank += (w[j] < wi || (w[j] == wi && j < i)) ? 1 : 0;
    ws[rank] = wi;
    for (int r = 0; r < n; ++r) Vs[(int64_t)r * ldvs + rank] = V[(int64_t)r * ldv + i];
  }
}

constexpr int RN_ROWS = 2048;

__global__ void k_resid_part(int64_t nrows, const double* __restrict__ HX, int64_t ldh, const double* __restrict__ MX,
                             int64_t ldm, const double* __restrict__ eps, int N, double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * RN_ROWS;
  const int64_t r1 = min(nrows, r0 + RN_ROWS);
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const double ec = eps[c];
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double d = HX[r * ldh + c] - ec * MX[r * ldm + c];
      s = fma(d, d, s);
    }
    part[(int64_t)blockIdx.x * N + c] = s;
  }
}

__global__ void k_resid_final(int nb, int N, const double* __restrict__ part, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * N + c];
  out[c] = sqrt(s);
}

__global__ void k_dot_part(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                           double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

__global__ void k_dot_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = s;
  }
}

__global__ void k_axpby3(int64_t n, double* __restrict__ w, const double* __restrict__ v,
                         const double* __restrict__ vp, double a, double b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) w[i] = w[i] - a * v[i] - b * vp[i];
}

__global__ void k_scale(int64_t n, const double* __restrict__ x, double s, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = s * x[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_potential_analytic(const double* qpts, int64_t nq, const double* axyz, const double* aZ, int na,
                               int nuclear, const double* gA, const double* gs, const double* gc, int nt,
                               double omega, double* V, cudaStream_t st) {
  if (nq <= 0) return;
  k_potential<<<grid1(nq, 256), 256, 0, st>>>(qpts, nq, axyz, aZ, na, nuclear, gA, gs, gc, nt, omega, V);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return;
  k_check_finite<<<(grid1(n, 256) < 4096u ? grid1(n, 256) : 4096u), 256, 0, st>>>(x, n, flag);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_gather_sum(int64_t n_out, const double* base, const int64_t* cptr, const int64_t* cidx,
                       const double* blk, double* out, cudaStream_t st) {
  if (n_out <= 0) return;
  k_gather_sum<<<grid1(n_out, 256), 256, 0, st>>>(n_out, base, cptr, cidx, blk, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_permute(int64_t n, const double* src, const int64_t* perm, double* dst, cudaStream_t st) {
  if (n <= 0) return;
  k_permute<<<grid1(n, 256), 256, 0, st>>>(n, src, perm, dst);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_to_f32<<<grid1(n, 256), 256, 0, st>>>(src, dst, n);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_cell_apply_f64(const double* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                           const double* Y, int64_t ldy, double* W, int64_t ldw, int N, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return;
  dim3 g((unsigned)ncells, (unsigned)((N + 31) / 32));
  const size_t smem = sizeof(int64_t) * 128 + sizeof(double) * (NL * 33 + 128 * 26);
  cudaFuncSetAttribute(k_cell_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_cell_apply<double><<<g, 256, smem, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_cell_apply_f32(const float* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                           const float* Y, int64_t ldy, float* W, int64_t ldw, int N, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return;
  dim3 g((unsigned)ncells, (unsigned)((N + 31) / 32));
  const size_t smem = sizeof(int64_t) * 128 + sizeof(float) * (NL * 33 + 128 * 26);
  cudaFuncSetAttribute(k_cell_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_cell_apply<float><<<g, 256, smem, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
void launch_spmm_nodes(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                       const double* val, double sgn, const double* Xe, int64_t ldxe, T* out, int64_t ldo, int N,
                       cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  if (N <= SPMM_NARROW)
    k_spmm_nodes_rowthread<T><<<grid1(nrows, 256), 256, 0, st>>>(nrows, rnode, ptr, col, val, sgn, Xe, ldxe, out,
                                                                 ldo, N);
  else
    k_spmm_nodes<T><<<grid1(nrows * 32, 256), 256, 0, st>>>(nrows, rnode, ptr, col, val, sgn, Xe, ldxe, out, ldo, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_spmm_nodes<double>(int64_t, const int32_t*, const int64_t*, const int32_t*, const double*,
                                        double, const double*, int64_t, double*, int64_t, int, cudaStream_t);
template void launch_spmm_nodes<float>(int64_t, const int32_t*, const int64_t*, const int32_t*, const double*,
                                       double, const double*, int64_t, float*, int64_t, int, cudaStream_t);

template <typename T>
void launch_spmm_segments(int64_t nseg, const int64_t* seg_start, const int64_t* seg_end, const int32_t* col,
                          const double* val, const double* scale, const T* Xc, int64_t ldx, double* part, int N,
                          cudaStream_t st) {
  if (nseg <= 0 || N <= 0) return;
  if (N <= SPMM_NARROW) {
    k_spmm_segments_narrow<T><<<(unsigned)nseg, 256, 0, st>>>(seg_start, seg_end, col, val, scale, Xc, ldx, part, N);
  } else {
    const int t = N >= 128 ? 128 : ((N + 31) / 32) * 32;
    k_spmm_segments<T><<<(unsigned)nseg, t, 0, st>>>(seg_start, seg_end, col, val, scale, Xc, ldx, part, N);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_spmm_segments<double>(int64_t, const int64_t*, const int64_t*, const int32_t*, const double*,
                                           const double*, const double*, int64_t, double*, int, cudaStream_t);
template void launch_spmm_segments<float>(int64_t, const int64_t*, const int64_t*, const int32_t*, const double*,
                                          const double*, const float*, int64_t, double*, int, cudaStream_t);

void launch_seg_reduce(int nrows, const int64_t* row_seg_ptr, const double* part, double sgn, const double* base,
                       int64_t ldb, double alpha_base, double* out, int64_t ldo, int N, cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_seg_reduce<<<grid1((int64_t)nrows * N, 256), 256, 0, st>>>(nrows, row_seg_ptr, part, sgn, base, ldb, alpha_base,
                                                                out, ldo, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
void launch_cheb_combine(int64_t nrows, const double* rowscale, const T* Xsrc, int64_t ldx, const T* Ycur,
                         int64_t ldc, const T* Yprev, int64_t ldp, T* Ynew, int64_t ldn, const double* coef, int N,
                         cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_cheb_combine<T><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, rowscale, Xsrc, ldx, Ycur, ldc, Yprev, ldp, Ynew,
                                                           ldn, coef, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_cheb_combine<double>(int64_t, const double*, const double*, int64_t, const double*, int64_t,
                                          const double*, int64_t, double*, int64_t, const double*, int, cudaStream_t);
template void launch_cheb_combine<float>(int64_t, const double*, const float*, int64_t, const float*, int64_t,
                                         const float*, int64_t, float*, int64_t, const double*, int, cudaStream_t);

template <typename T>
void launch_row_scale(int64_t nrows, const double* rowscale, const T* X, int64_t ldx, T* Y, int64_t ldy, int N,
                      cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_row_scale<T><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, rowscale, X, ldx, Y, ldy, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_row_scale<double>(int64_t, const double*, const double*, int64_t, double*, int64_t, int,
                                       cudaStream_t);
template void launch_row_scale<float>(int64_t, const double*, const float*, int64_t, float*, int64_t, int,
                                      cudaStream_t);

void launch_f64_to_f32_rows(int64_t nrows, const double* X, int64_t ldx, float* Y, int64_t ldy, int N,
                            cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_convert_rows<double, float><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, X, ldx, Y, ldy, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_f32_to_f64_rows(int64_t nrows, const float* X, int64_t ldx, double* Y, int64_t ldy, int N,
                            cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_convert_rows<float, double><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, X, ldx, Y, ldy, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_copy_rows(int64_t nrows, const double* X, int64_t ldx, double* Y, int64_t ldy, int N, cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_convert_rows<double, double><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, X, ldx, Y, ldy, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_zero_rows(int64_t nrows, double* X, int64_t ldx, int N, cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_zero_rows<double><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, X, ldx, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_zero_rows_f32(int64_t nrows, float* X, int64_t ldx, int N, cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_zero_rows<float><<<grid1(nrows * N, 256), 256, 0, st>>>(nrows, X, ldx, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_gemm_nn(int64_t M, int Nc, int K, double alpha, const double* A, int64_t lda, const double* B,
                    int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t st) {
  if (M <= 0 || Nc <= 0) return;
  dim3 g((unsigned)((M + GT - 1) / GT), (unsigned)((Nc + GT - 1) / GT));
  // fewer 48 x 48 output tiles than SMs: one output per thread in 16 x 16 tiles
  if ((int64_t)g.x * g.y < current_sm_count()) {
    dim3 gs((unsigned)((M + 15) / 16), (unsigned)((Nc + 15) / 16));
    k_gemm_nn_small<<<gs, 256, 0, st>>>(M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc);
  } else {
    k_gemm_nn<<<g, 256, 0, st>>>(M, Nc, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, 0, 0);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_gemm_nn_batched(int64_t M, int Nc, int K, const double* A, int64_t lda, int64_t sA, const double* B,
                            int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC, int batch,
                            cudaStream_t st) {
  if (M <= 0 || Nc <= 0 || batch <= 0) return;
  dim3 g((unsigned)((M + GT - 1) / GT), (unsigned)((Nc + GT - 1) / GT), (unsigned)batch);
  k_gemm_nn<<<g, 256, 0, st>>>(M, Nc, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, sA, sB, sC);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// K splits of an A^T B product: enough for about four CTAs per SM over the
// output tiles, none shorter than TN_KC rows
int64_t gemm_tn_splits(int64_t K, int Na, int Nb) {
  const int64_t tiles = (int64_t)((Na + GT - 1) / GT) * ((Nb + GT - 1) / GT);
  const int64_t want = (4 * (int64_t)current_sm_count() + tiles - 1) / tiles;
  const int64_t most = (K + TN_KC - 1) / TN_KC;
  return std::max<int64_t>(1, std::min(want, most));
}

int64_t gemm_tn_work_elems(int64_t K, int Na, int Nb) { return gemm_tn_splits(K, Na, Nb) * (int64_t)Na * Nb; }

void launch_gemm_tn(int64_t K, int Na, int Nb, const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, double* work, int64_t work_elems, cudaStream_t st, bool sym) {
  if (Na <= 0 || Nb <= 0) return;
  int64_t nsplit = gemm_tn_splits(K, Na, Nb);
  nsplit = std::max<int64_t>(1, std::min(nsplit, work_elems / ((int64_t)Na * Nb)));
  const int64_t kc = ((K + nsplit - 1) / nsplit + 15) / 16 * 16;
  nsplit = std::max<int64_t>(1, (K + kc - 1) / kc);
  dim3 g((unsigned)((Na + GT - 1) / GT), (unsigned)((Nb + GT - 1) / GT), (unsigned)nsplit);
  const int sy = (sym && Na == Nb) ? 1 : 0;
  k_gemm_tn_part<<<g, 256, 0, st>>>(K, kc, Na, Nb, A, lda, B, ldb, work, sy);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_gemm_tn_reduce<<<grid1((int64_t)Na * Nb, 256), 256, 0, st>>>((int)nsplit, Na, Nb, work, C, ldc, sy);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_shift_diag(double* A, int n, int lda, double coef, cudaStream_t st) {
  k_shift_diag<<<1, 1024, 0, st>>>(A, n, lda, coef);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_chol(double* A, int n, int lda, int* info, cudaStream_t st, double* min_ratio) {
  k_chol<<<1, 1024, 0, st>>>(A, n, lda, info, min_ratio);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_trinv_lower(const double* L, int n, int lda, double* Li, int ldi, cudaStream_t st) {
  k_trinv_lower<<<grid1(n, 128), 128, 0, st>>>(L, n, lda, Li, ldi);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_transpose(const double* A, int n, int lda, double* B, int ldb, cudaStream_t st) {
  k_transpose<<<grid1((int64_t)n * n, 256), 256, 0, st>>>(A, n, lda, B, ldb);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_mirror_upper(double* A, int n, int lda, cudaStream_t st) {
  k_mirror_upper<<<grid1((int64_t)n * n, 256), 256, 0, st>>>(A, n, lda);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_symmetrize(double* A, int n, int lda, cudaStream_t st) {
  k_symmetrize<<<grid1((int64_t)n * n, 256), 256, 0, st>>>(A, n, lda);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
void launch_jacobi_t(T* A, int n, int lda, T* V, int ldv, T* w, int max_sweeps, double tol2, int* info,
                     cudaStream_t st) {
  const size_t smem = sizeof(T) * (size_t)n * n;
  if (smem <= 180 * 1024) {
    cudaFuncSetAttribute(k_jacobi<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobi<T, true><<<1, 1024, smem, st>>>(A, n, lda, V, ldv, w, max_sweeps, tol2, info);
  } else {
    k_jacobi<T, false><<<1, 1024, 0, st>>>(A, n, lda, V, ldv, w, max_sweeps, tol2, info);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_jacobi(double* A, int n, int lda, double* V, int ldv, double* w, int max_sweeps, int* info,
                   cudaStream_t st) {
  launch_jacobi_t<double>(A, n, lda, V, ldv, w, max_sweeps, 1e-30, info, st);
}

void launch_jacobi_f32(float* A, int n, int lda, float* V, int ldv, float* w, int max_sweeps, int* info,
                       cudaStream_t st) {
  launch_jacobi_t<float>(A, n, lda, V, ldv, w, max_sweeps, 1e-12, info, st);
}

void launch_sort_eig(const double* w, const double* V, int n, int ldv, double* ws, double* Vs, int ldvs,
                     cudaStream_t st) {
  k_sort_eig<<<grid1(n, 128), 128, 0, st>>>(w, V, n, ldv, ws, Vs, ldvs);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_resid_norms(int64_t nrows, const double* HX, int64_t ldh, const double* MX, int64_t ldm,
                        const double* eps, int N, double* part, double* out, cudaStream_t st) {
  const int nb = (int)((nrows + RN_ROWS - 1) / RN_ROWS);
  k_resid_part<<<nb, 128, 0, st>>>(nrows, HX, ldh, MX, ldm, eps, N, part);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_resid_final<<<grid1(N, 128), 128, 0, st>>>(nb, N, part, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_dot(int64_t n, const double* x, const double* y, double* part, double* out, cudaStream_t st) {
  k_dot_part<<<256, 256, 0, st>>>(n, x, y, part);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_dot_final<<<1, 32, 0, st>>>(256, part, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_axpby3(int64_t n, double* w, const double* v, const double* vp, double a, double b, cudaStream_t st) {
  k_axpby3<<<grid1(n, 256), 256, 0, st>>>(n, w, v, vp, a, b);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_scale(int64_t n, const double* x, double s, double* y, cudaStream_t st) {
  k_scale<<<grid1(n, 256), 256, 0, st>>>(n, x, s, y);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_cell_apply_narrow_f64(const double* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                                  const double* Y, int64_t ldy, double* W, int64_t ldw, int N, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return;
  if (N == 1) k_cell_apply_narrow<double, 1><<<(unsigned)ncells, 256, 0, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  else k_cell_apply_narrow<double, 8><<<(unsigned)ncells, 256, 0, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_cell_apply_narrow_f32(const float* Hcc, const int32_t* cells, int64_t ncells, const MeshDev& m,
                                  const float* Y, int64_t ldy, float* W, int64_t ldw, int N, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return;
  if (N == 1) k_cell_apply_narrow<float, 1><<<(unsigned)ncells, 256, 0, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  else k_cell_apply_narrow<float, 8><<<(unsigned)ncells, 256, 0, st>>>(Hcc, cells, m, Y, ldy, W, ldw, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

int coup_block_nodes() { return CPB; }

// shared memory of the node-major kernels: the (n_E x N) array, the rows
// kernel's CPB x (N + 4) vector tile and one CPF x CPB pattern tile
size_t coup_smem(int nE, int N, bool rows) {
  const size_t ld = (size_t)((N + 3) & ~3);
  return sizeof(float) * ((size_t)nE * ld + (rows ? (size_t)CPB * ld : 0) + (size_t)CPF * CPB);
}

// CTAs of the rows (or columns) product resident at once (one wave of its partition)
int coup_resident_ctas(int nE, int N, int n_sm, bool rows) {
  const size_t smem = coup_smem(nE, N, rows);
  int per_sm = 0;
  cudaError_t e;
  if (rows) {
    cudaFuncSetAttribute(k_coup_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coup_rows<float>, 256, smem);
  } else {
    cudaFuncSetAttribute(k_coup_cols<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coup_cols<float>, 256, smem);
  }
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  return per_sm * n_sm;
}

void launch_tile_scatter(int64_t nnz, const int64_t* pos, const float* val, float* tile, cudaStream_t st) {
  if (nnz <= 0) return;
  k_tile_scatter<<<grid1(nnz, 256), 256, 0, st>>>(nnz, pos, val, tile);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
void launch_coup_rows(int64_t n_tn, int ncta, const int64_t* cta_blk, const int32_t* t_nodes,
                      const int64_t* slot_off, const int32_t* slots, const float* tile, const double* scale,
                      const T* X, int64_t ldx, int nE, int N, float* part, cudaStream_t st) {
  if (n_tn <= 0 || N <= 0 || nE <= 0 || ncta <= 0) return;
  const size_t smem = coup_smem(nE, N, true);
  cudaFuncSetAttribute(k_coup_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_coup_rows<T><<<ncta, 256, smem, st>>>(n_tn, cta_blk, t_nodes, slot_off, slots, tile, scale, X, ldx, nE, N, part);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_coup_rows<float>(int64_t, int, const int64_t*, const int32_t*, const int64_t*, const int32_t*,
                                      const float*, const double*, const float*, int64_t, int, int, float*,
                                      cudaStream_t);

void launch_coup_reduce(int nb, int nE, int N, const float* part, double sgn, const double* base, int64_t ldb,
                        double alpha_base, double* out, int64_t ldo, cudaStream_t st) {
  if (nE <= 0 || N <= 0) return;
  k_coup_reduce<<<(unsigned)(((int64_t)nE * N + 31) / 32), 256, 0, st>>>(nb, nE, N, part, sgn, base, ldb, alpha_base,
                                                                         out, ldo);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
void launch_coup_cols(int64_t n_tn, int ncta, const int64_t* cta_blk, const int32_t* t_nodes,
                      const int64_t* slot_off, const int32_t* slots, const float* tile, float sgn, const double* Xe,
                      int64_t ldxe, int nE, int N, T* W, int64_t ldw, cudaStream_t st) {
  if (n_tn <= 0 || N <= 0 || nE <= 0 || ncta <= 0) return;
  const size_t smem = coup_smem(nE, N, false);
  cudaFuncSetAttribute(k_coup_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_coup_cols<T><<<ncta, 256, smem, st>>>(n_tn, cta_blk, t_nodes, slot_off, slots, tile, sgn, Xe, ldxe, nE, N, W,
                                          ldw);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void launch_coup_cols<float>(int64_t, int, const int64_t*, const int32_t*, const int64_t*, const int32_t*,
                                      const float*, float, const double*, int64_t, int, int, float*, int64_t,
                                      cudaStream_t);

int grp_kmax() { return GRP_KMAX; }

void launch_grp_rows(int n_items, const int4* items, const int64_t* ec_ptr, const int32_t* ec_col, const float* coef,
                     const float* Xc, int64_t ldx, double* part, int N, cudaStream_t st) {
  if (n_items <= 0 || N <= 0) return;
  dim3 g((unsigned)n_items, (unsigned)((N + GRP_CT - 1) / GRP_CT));
  k_grp_rows<<<g, GRP_CT, 0, st>>>(items, ec_ptr, ec_col, coef, Xc, ldx, part, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_grp_reduce(int nE, const int32_t* f_it0, const int32_t* f_it1, const int32_t* f_slot, const double* part,
                       int N, double sgn, const double* base, int64_t ldb, double alpha, double* out, int64_t ldo,
                       cudaStream_t st) {
  if (nE <= 0 || N <= 0) return;
  k_grp_reduce<<<grid1((int64_t)nE * N, 256), 256, 0, st>>>(nE, f_it0, f_it1, f_slot, part, N, sgn, base, ldb, alpha,
                                                          out, ldo);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_coup_cols_chunk(int64_t n_tn, const int32_t* t_nodes, const int64_t* slot_off, const int32_t* slots,
                            const float* tile, float sgn, const float* Xe, int64_t ldxe, int N, float* W, int64_t ldw,
                            cudaStream_t st) {
  const int64_t nblk = (n_tn + CPB - 1) / CPB;
  if (nblk <= 0 || N <= 0) return;
  dim3 g((unsigned)nblk, (unsigned)((N + GRP_CT - 1) / GRP_CT));
  k_coup_cols_chunk<<<g, GRP_CT, 0, st>>>(n_tn, t_nodes, slot_off, slots, tile, sgn, Xe, ldxe, N, W, ldw);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_coup_cols_sparse(int64_t n_tn, const int32_t* t_nodes, const int64_t* t_ptr, const int32_t* t_slot,
                             const float* val, const int64_t* slot_off, const int32_t* slots, float sgn,
                             const float* Xe, int64_t ldxe, int N, float* W, int64_t ldw, cudaStream_t st) {
  const int64_t nblk = (n_tn + CPB - 1) / CPB;
  if (nblk <= 0 || N <= 0) return;
  dim3 g((unsigned)nblk, (unsigned)((N + GRP_CT - 1) / GRP_CT));
  k_coup_cols_sparse<<<g, GRP_CT, 0, st>>>(n_tn, t_nodes, t_ptr, t_slot, val, slot_off, slots, sgn, Xe, ldxe, N, W,
                                           ldw);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_spmm_nodes_f32(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                           const float* val, float sgn, const float* Xe, int64_t ldxe, float* out, int64_t ldo, int N,
                           cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_spmm_nodes_f32<<<grid1(nrows * 32, 256), 256, 0, st>>>(nrows, rnode, ptr, col, val, sgn, Xe, ldxe, out, ldo, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_cheb_combine_f4(int64_t nrows, int ld, const double* rowscale, const float* X, const float* Yc,
                            const float* Yp, float* Yn, const double* coef, cudaStream_t st) {
  if (nrows <= 0) return;
  const int ld4 = ld / 4;
  k_cheb_combine_f4<<<grid1(nrows * ld4, 256), 256, 0, st>>>(nrows, ld4, rowscale, (const float4*)X,
                                                            (const float4*)Yc, (const float4*)Yp, (float4*)Yn, coef);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_df_coef(int64_t n, const double* v, const double* scale, const int32_t* col, float2* out,
                    cudaStream_t st) {
  if (n <= 0) return;
  k_df_coef<<<grid1(n, 256), 256, 0, st>>>(n, v, scale, col, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_df_rows(int64_t rows, int N, const double* X, int64_t ldx, float2* out, cudaStream_t st) {
  if (rows <= 0 || N <= 0) return;
  k_df_rows<<<grid1(rows * N, 256), 256, 0, st>>>(rows, N, X, ldx, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_spmm_nodes_df(int64_t nrows, const int32_t* rnode, const int64_t* ptr, const int32_t* col,
                          const float2* val, float sgn, const float2* Xe2, int N, double* out, int64_t ldo,
                          cudaStream_t st) {
  if (nrows <= 0 || N <= 0) return;
  k_spmm_nodes_df<<<grid1(nrows * 32, 256), 256, 0, st>>>(nrows, rnode, ptr, col, val, sgn, Xe2, N, out, ldo);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_grp_rows_df(int n_items, const int4* items, const int64_t* ec_ptr, const int32_t* ec_col,
                        const float2* coef, const double* Xc, int64_t ldx, double* part, int N, cudaStream_t st) {
  if (n_items <= 0 || N <= 0) return;
  dim3 g((unsigned)n_items, (unsigned)((N + GRP_CT - 1) / GRP_CT));
  k_grp_rows_df<<<g, GRP_CT, 0, st>>>(items, ec_ptr, ec_col, coef, Xc, ldx, part, N);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

}  // namespace efe

