// Learned initial density for the SCF (Sec. V starts from an input density):
//   * superposition of atomic densities (SAD) from normalised Slater shells,
//   * atom-centred descriptors at the quadrature points (radial Gaussians and
//     angular dipole magnitudes per species slot, smooth cosine cutoff),
//   * a fully connected network (SiLU hidden layers) with forward and backward
//     passes written as tiled GEMMs, a weighted squared-error loss and Adam,
//   * the corrected start rho = (rho_sad + floor) exp(y) - floor, rescaled.
// Every kernel is templated on the arithmetic type: float for training and
// inference, double for the gradient checks against the oracle.  All
// reductions use fixed-order partials (bitwise reproducible).
#include <math.h>

#include "efe_kernels.h"

namespace efe {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int RED_B = 512;  // blocks of the fixed-order reductions

template <typename T>
__device__ __forceinline__ T silu_d(T z) { return z / (T(1) + exp(-z)); }
template <typename T>
__device__ __forceinline__ T silu_grad_d(T z) {
  const T s = T(1) / (T(1) + exp(-z));
  return s * (T(1) + z * (T(1) - s));
}

// ---------------------------------------------------------------------------
// SAD: rho(x) = sum_I sum_s N_s C_s^2 r^(2 n_s - 2) exp(-2 zeta_s r) / (4 pi)
__global__ void k_sad(const double* __restrict__ qpts, int64_t nq, const double* __restrict__ axyz, int na,
                      const SadShellDev* __restrict__ sh, double* __restrict__ rho) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double x = qpts[4 * q], y = qpts[4 * q + 1], z = qpts[4 * q + 2];
  double s = 0.0;
  for (int a = 0; a < na; ++a) {
    const double dx = x - axyz[3 * a], dy = y - axyz[3 * a + 1], dz = z - axyz[3 * a + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const SadShellDev& S = sh[a];
    for (int k = 0; k < S.n_shells; ++k) {
      double rp = 1.0;
      for (int i = 1; i < S.n[k]; ++i) rp *= r;
      const double R = S.c[k] * rp * exp(-S.zeta[k] * r);
      s += S.occ[k] * R * R;
    }
  }
  rho[q] = s * 0.079577471545947667884;  // 1 / (4 pi)
}

// ---------------------------------------------------------------------------
// descriptors: per point, per species slot s: radial G[s][k], angular A[s][k]
template <typename T>
__global__ void k_descriptors(const double* __restrict__ qpts, int64_t nq, const double* __restrict__ axyz,
                              const int32_t* __restrict__ slot, int na, DescDev p, T* __restrict__ D) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double x = qpts[4 * q], y = qpts[4 * q + 1], z = qpts[4 * q + 2];
  constexpr double PI = 3.14159265358979323846;
  const int nr = p.n_radial, nang = p.n_ang, ns = p.n_species;
  const int nf = ns * (nr + nang);
  T* out = D + q * nf;
  for (int f = 0; f < nf; ++f) out[f] = T(0);
  double av[DESC_MAX_SPECIES][DESC_MAX_ANG][3];
  for (int s = 0; s < DESC_MAX_SPECIES; ++s)
    for (int k = 0; k < DESC_MAX_ANG; ++k) av[s][k][0] = av[s][k][1] = av[s][k][2] = 0.0;
  for (int a = 0; a < na; ++a) {
    const double dx = x - axyz[3 * a], dy = y - axyz[3 * a + 1], dz = z - axyz[3 * a + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r < p.r_cut)) continue;
    const int s = slot[a];
    if (s < 0 || s >= ns) continue;
    const double fc = 0.5 * (1.0 + cos(PI * r / p.r_cut));
    for (int k = 0; k < nr; ++k) {
      const double t = r - p.radial_mu[k];
      out[s * nr + k] += (T)(exp(-t * t / (2.0 * p.radial_sigma * p.radial_sigma)) * fc);
    }
    const double ir = 1.0 / fmax(r, 1e-12);
    for (int k = 0; k < nang; ++k) {
      const double t = r - p.ang_mu[k];
      const double g = exp(-t * t / (2.0 * p.ang_sigma * p.ang_sigma)) * fc * ir;
      av[s][k][0] += g * dx;
      av[s][k][1] += g * dy;
      av[s][k][2] += g * dz;
    }
  }
  T* ang = out + ns * nr;
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < nang; ++k)
      ang[s * nang + k] = (T)(av[s][k][0] * av[s][k][0] + av[s][k][1] * av[s][k][1] + av[s][k][2] * av[s][k][2]);
  if (p.standardise)
    for (int f = 0; f < nf; ++f) out[f] = (T)(((double)out[f] - p.offset[f]) * p.scale[f]);
}

// ---------------------------------------------------------------------------
// Generic tiled GEMM: C[z][m][n] = sum_{k in chunk z} A(m, k) B(k, n), element
// (m, k) of A at A[m * sam + k * sak] and (k, n) of B at B[k * sbk + n * sbn];
// one 64 x 64 output tile per CTA (256 threads, 4 x 4 each), K chunk of kch
// per blockIdx.z (split-K partials for the long reductions of the backward pass).
constexpr int GM = 64, GK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_g(int64_t M, int64_t Nn, int64_t K, int64_t kch, const T* __restrict__ A,
                                                int64_t sam, int64_t sak, const T* __restrict__ B, int64_t sbk,
                                                int64_t sbn, T* __restrict__ C, int64_t ldc) {
  __shared__ T As[GK][GM + 1];
  __shared__ T Bs[GK][GM + 1];
  const int64_t m0 = (int64_t)blockIdx.x * GM, n0 = (int64_t)blockIdx.y * GM;
  const int64_t kb = (int64_t)blockIdx.z * kch, ke = min(K, kb + kch);
  C += (int64_t)blockIdx.z * M * ldc;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const bool a_kfast = sak == 1;
  const bool b_nfast = sbn == 1;
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    for (int idx = tid; idx < GK * GM; idx += 256) {
      int kk, mm;
      if (a_kfast) { kk = idx % GK; mm = idx / GK; } else { mm = idx % GM; kk = idx / GM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : T(0);
      int kk2, nn;
      if (b_nfast) { nn = idx % GM; kk2 = idx / GM; } else { kk2 = idx % GK; nn = idx / GK; }
      const int64_t gn = n0 + nn, gk2 = k0 + kk2;
      Bs[kk2][nn] = (gn < Nn && gk2 < ke) ? B[gk2 * sbk + gn * sbn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx * 4 + j;
      if (n < Nn) C[m * ldc + n] = acc[i][j];
    }
  }
}

// Z = C + b (bias per column), A = act(Z) (SiLU or identity); Z, A row-major n x d
template <typename T>
__global__ void k_bias_act(int64_t n, int d, const T* __restrict__ b, T* __restrict__ Z, T* __restrict__ A, int act) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const T z = Z[i] + b[i % d];
  Z[i] = z;
  A[i] = act ? silu_d(z) : z;
}

// dZ = dA * silu'(Z)
template <typename T>
__global__ void k_act_back(int64_t n, const T* __restrict__ Z, T* __restrict__ dA) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dA[i] *= silu_grad_d(Z[i]);
}

// out[i] = sum_z part[z][i] (fixed order), i < nout
template <typename T>
__global__ void k_sum_parts(int nz, int64_t nout, const T* __restrict__ part, T* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nout) return;
  T s = T(0);
  for (int z = 0; z < nz; ++z) s += part[(int64_t)z * nout + i];
  out[i] = s;
}

// column sums of dZ (n x d) in fixed order: part[blk][j], then summed
template <typename T>
__global__ void k_colsum_part(int64_t n, int d, const T* __restrict__ dZ, int64_t rows_per_blk, T* __restrict__ part) {
  const int j = threadIdx.x + blockIdx.y * blockDim.x;
  if (j >= d) return;
  const int64_t r0 = blockIdx.x * rows_per_blk, r1 = min(n, r0 + rows_per_blk);
  T s = T(0);
  for (int64_t r = r0; r < r1; ++r) s += dZ[r * d + j];
  part[(int64_t)blockIdx.x * d + j] = s;
}

// weighted squared error: loss = sum c (yh - y)^2 / sum c; dy = 2 c (yh - y) / sum c
template <typename T>
__global__ void __launch_bounds__(256) k_wmse_part(int64_t n, const T* __restrict__ yh, const T* __restrict__ y,
                                                   const T* __restrict__ c, double* __restrict__ part) {
  __shared__ double r1[256], r2[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)yh[i] - (double)y[i];
    a += (double)c[i] * d * d;
    b += (double)c[i];
  }
  r1[threadIdx.x] = a;
  r2[threadIdx.x] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      r1[threadIdx.x] += r1[threadIdx.x + s];
      r2[threadIdx.x] += r2[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = r1[0];
    part[gridDim.x + blockIdx.x] = r2[0];
  }
}

__global__ void k_wmse_finish(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) { a += part[i]; b += part[nb + i]; }
  out[0] = a / b;
  out[1] = b;
}

template <typename T>
__global__ void k_wmse_grad(int64_t n, const T* __restrict__ yh, const T* __restrict__ y, const T* __restrict__ c,
                            const double* __restrict__ stats, T* __restrict__ dy) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dy[i] = (T)(2.0 * (double)c[i] * ((double)yh[i] - (double)y[i]) / stats[1]);
}

template <typename T>
__global__ void k_adam(int64_t n, T* __restrict__ p, const T* __restrict__ g, T* __restrict__ m, T* __restrict__ v,
                       double lr, double b1, double b2, double eps, double c1, double c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = (double)g[i];
  const double mi = b1 * (double)m[i] + (1.0 - b1) * gi;
  const double vi = b2 * (double)v[i] + (1.0 - b2) * gi * gi;
  m[i] = (T)mi;
  v[i] = (T)vi;
  p[i] = (T)((double)p[i] - lr * (mi / c1) / (sqrt(vi / c2) + eps));
}

// rho = max((rho_sad + floor) exp(y) - floor, 0)
template <typename T>
__global__ void k_apply_correction(int64_t n, const double* __restrict__ rs, const T* __restrict__ y, double floor,
                                   double* __restrict__ rho) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) rho[i] = fmax((rs[i] + floor) * exp((double)y[i]) - floor, 0.0);
}

// target y = log(rho + floor) - log(rho_sad + floor)
template <typename T>
__global__ void k_log_ratio(int64_t n, const double* __restrict__ rho, const double* __restrict__ rs, double floor,
                            T* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (T)(log(rho[i] + floor) - log(rs[i] + floor));
}

__global__ void __launch_bounds__(256) k_wsum_part(const double* __restrict__ qpts, int64_t nq, const double* __restrict__ x,
                                                   double* __restrict__ part) {
  __shared__ double r[256];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
    a += qpts[4 * i + 3] * x[i];
  r[threadIdx.x] = a;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) r[threadIdx.x] += r[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = r[0];
}

__global__ void k_scale_to_count(int nb, const double* __restrict__ part, int64_t n, double target,
                                 double* __restrict__ x) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    tot = s;
  }
  __syncthreads();
  const double f = tot > 0.0 ? target / tot : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

template <typename T>
void gemm_g(int64_t M, int64_t Nn, int64_t K, int nsplit, const T* A, int64_t sam, int64_t sak, const T* B,
            int64_t sbk, int64_t sbn, T* C, int64_t ldc, cudaStream_t st) {
  const int64_t kch = ((K + nsplit - 1) / nsplit + GK - 1) / GK * GK;
  const int nz = (int)((K + kch - 1) / kch);
  dim3 g((unsigned)((M + GM - 1) / GM), (unsigned)((Nn + GM - 1) / GM), (unsigned)std::max(nz, 1));
  k_gemm_g<T><<<g, 256, 0, st>>>(M, Nn, K, kch, A, sam, sak, B, sbk, sbn, C, ldc);
  g_launches++;
}

template <typename T>
int gemm_splits(int64_t K, int64_t kch_target) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(64, (K + kch_target - 1) / kch_target));
}

}  // namespace

// ---------------------------------------------------------------------------
void launch_sad(const double* qpts, int64_t nq, const double* axyz, int na, const SadShellDev* sh, double* rho,
                cudaStream_t st) {
  if (nq <= 0) return;
  k_sad<<<nblk(nq, 256), 256, 0, st>>>(qpts, nq, axyz, na, sh, rho);
  g_launches++;
}

template <typename T>
void launch_descriptors(const double* qpts, int64_t nq, const double* axyz, const int32_t* slot, int na,
                        const DescDev& p, T* D, cudaStream_t st) {
  if (nq <= 0) return;
  k_descriptors<T><<<nblk(nq, 128), 128, 0, st>>>(qpts, nq, axyz, slot, na, p, D);
  g_launches++;
}
template void launch_descriptors<float>(const double*, int64_t, const double*, const int32_t*, int, const DescDev&,
                                        float*, cudaStream_t);
template void launch_descriptors<double>(const double*, int64_t, const double*, const int32_t*, int, const DescDev&,
                                         double*, cudaStream_t);

int64_t mlp_param_count(const int* dims, int nl) {
  int64_t s = 0;
  for (int l = 0; l < nl; ++l) s += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
  return s;
}

int64_t mlp_work_elems(const int* dims, int nl, int64_t n) {
  int64_t s = 0;
  for (int l = 0; l < nl; ++l) s += 2 * (int64_t)dims[l + 1];
  return s * n;
}

int64_t mlp_scratch_elems(const int* dims, int nl, int64_t n) {
  int dmax = 0;
  int64_t wmax = 0;
  for (int l = 0; l < nl; ++l) {
    dmax = std::max(dmax, std::max(dims[l], dims[l + 1]));
    wmax = std::max(wmax, (int64_t)dims[l + 1] * (dims[l] + 1));
  }
  return 2 * n * dmax + 64 * wmax + (int64_t)RED_B * dmax;
}

// work layout per layer l: Z_l (n x d_{l+1}) then A_l (n x d_{l+1})
template <typename T>
void mlp_forward(const int* dims, int nl, const T* params, const T* X, int64_t n, T* y, T* work, cudaStream_t st) {
  const T* a = X;
  const T* p = params;
  T* w = work;
  for (int l = 0; l < nl; ++l) {
    const int din = dims[l], dout = dims[l + 1];
    const T* W = p;
    const T* b = p + (int64_t)dout * din;
    T* Z = w;
    T* A = w + n * dout;
    // Z = a W^T : (n x din) (din x dout), element (k, j) of W^T = W[j * din + k]
    gemm_g<T>(n, dout, din, 1, a, din, 1, W, 1, din, Z, dout, st);
    k_bias_act<T><<<nblk(n * dout, 256), 256, 0, st>>>(n, dout, b, Z, A, l < nl - 1 ? 1 : 0);
    g_launches++;
    a = A;
    p = b + dout;
    w = A + n * dout;
  }
  // output layer has dout = 1: y = A_last
  cudaMemcpyAsync(y, a, sizeof(T) * n, cudaMemcpyDeviceToDevice, st);
}

template <typename T>
void mlp_backward(const int* dims, int nl, const T* params, const T* X, int64_t n, const T* work, const T* dy,
                  T* grads, T* scratch, cudaStream_t st) {
  int dmax = 0;
  int64_t wmax = 0;
  for (int l = 0; l < nl; ++l) {
    dmax = std::max(dmax, std::max(dims[l], dims[l + 1]));
    wmax = std::max(wmax, (int64_t)dims[l + 1] * (dims[l] + 1));
  }
  T* dcur = scratch;                 // n x dmax
  T* dnext = scratch + n * dmax;     // n x dmax
  T* part = dnext + n * dmax;        // 64 x wmax
  T* cpart = part + 64 * wmax;       // RED_B x dmax
  // parameter and work offsets
  int64_t poff[16], woff[16];
  int64_t po = 0, wo = 0;
  for (int l = 0; l < nl; ++l) {
    poff[l] = po;
    woff[l] = wo;
    po += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    wo += 2 * n * dims[l + 1];
  }
  cudaMemcpyAsync(dcur, dy, sizeof(T) * n, cudaMemcpyDeviceToDevice, st);  // dZ of the output layer (identity)
  for (int l = nl - 1; l >= 0; --l) {
    const int din = dims[l], dout = dims[l + 1];
    const T* a_prev = (l == 0) ? X : work + woff[l - 1] + n * dims[l];
    T* gW = grads + poff[l];
    T* gb = gW + (int64_t)dout * din;
    // dW = dZ^T a_prev : (dout x n)(n x din), split over n
    const int ns = gemm_splits<T>(n, 4096);
    gemm_g<T>(dout, din, n, ns, dcur, 1, dout, a_prev, din, 1, part, din, st);
    const int64_t kch = ((n + ns - 1) / ns + GK - 1) / GK * GK;
    const int nz = (int)((n + kch - 1) / kch);
    k_sum_parts<T><<<nblk((int64_t)dout * din, 256), 256, 0, st>>>(nz, (int64_t)dout * din, part, gW);
    // db = column sums of dZ
    const int64_t rpb = (n + RED_B - 1) / RED_B;
    dim3 gc((unsigned)((n + rpb - 1) / rpb), (unsigned)((dout + 127) / 128));
    k_colsum_part<T><<<gc, 128, 0, st>>>(n, dout, dcur, rpb, cpart);
    k_sum_parts<T><<<nblk(dout, 256), 256, 0, st>>>((int)gc.x, dout, cpart, gb);
    g_launches += 4;
    if (l > 0) {
      // dA_prev = dZ W : (n x dout)(dout x din), then dZ_prev = dA_prev * silu'(Z_prev)
      gemm_g<T>(n, din, dout, 1, dcur, dout, 1, params + poff[l], din, 1, dnext, din, st);
      k_act_back<T><<<nblk(n * din, 256), 256, 0, st>>>(n * din, work + woff[l - 1], dnext);
      g_launches++;
      T* t = dcur;
      dcur = dnext;
      dnext = t;
    }
  }
}

template void mlp_forward<float>(const int*, int, const float*, const float*, int64_t, float*, float*, cudaStream_t);
template void mlp_forward<double>(const int*, int, const double*, const double*, int64_t, double*, double*,
                                  cudaStream_t);
template void mlp_backward<float>(const int*, int, const float*, const float*, int64_t, const float*, const float*,
                                  float*, float*, cudaStream_t);
template void mlp_backward<double>(const int*, int, const double*, const double*, int64_t, const double*,
                                   const double*, double*, double*, cudaStream_t);

template <typename T>
void launch_wmse(const T* yh, const T* y, const T* c, int64_t n, T* dy, double* part, double* stats, cudaStream_t st) {
  k_wmse_part<T><<<RED_B, 256, 0, st>>>(n, yh, y, c, part);
  k_wmse_finish<<<1, 32, 0, st>>>(RED_B, part, stats);
  k_wmse_grad<T><<<nblk(n, 256), 256, 0, st>>>(n, yh, y, c, stats, dy);
  g_launches += 3;
}
template void launch_wmse<float>(const float*, const float*, const float*, int64_t, float*, double*, double*,
                                 cudaStream_t);
template void launch_wmse<double>(const double*, const double*, const double*, int64_t, double*, double*, double*,
                                  cudaStream_t);

template <typename T>
void launch_adam(int64_t n, T* p, const T* g, T* m, T* v, double lr, double b1, double b2, double eps, int t,
                 cudaStream_t st) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  k_adam<T><<<nblk(n, 256), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  g_launches++;
}
template void launch_adam<float>(int64_t, float*, const float*, float*, float*, double, double, double, double, int,
                                 cudaStream_t);
template void launch_adam<double>(int64_t, double*, const double*, double*, double*, double, double, double, double,
                                  int, cudaStream_t);

template <typename T>
void launch_apply_correction(int64_t n, const double* rs, const T* y, double floor, double* rho, cudaStream_t st) {
  k_apply_correction<T><<<nblk(n, 256), 256, 0, st>>>(n, rs, y, floor, rho);
  g_launches++;
}
template void launch_apply_correction<float>(int64_t, const double*, const float*, double, double*, cudaStream_t);
template void launch_apply_correction<double>(int64_t, const double*, const double*, double, double*, cudaStream_t);

template <typename T>
void launch_log_ratio(int64_t n, const double* rho, const double* rs, double floor, T* y, cudaStream_t st) {
  k_log_ratio<T><<<nblk(n, 256), 256, 0, st>>>(n, rho, rs, floor, y);
  g_launches++;
}
template void launch_log_ratio<float>(int64_t, const double*, const double*, double, float*, cudaStream_t);
template void launch_log_ratio<double>(int64_t, const double*, const double*, double, double*, cudaStream_t);

void launch_scale_count(const double* qpts, int64_t nq, double target, double* x, double* part, cudaStream_t st) {
  k_wsum_part<<<RED_B, 256, 0, st>>>(qpts, nq, x, part);
  k_scale_to_count<<<RED_B, 256, 0, st>>>(RED_B, part, nq, target, x);
  g_launches += 2;
}

int learn_reduce_blocks() { return RED_B; }

}  // namespace efe
