// CUDA kernels of the self-consistent field (Sec. V) around the filter:
//   * values of FE fields at the quadrature points and the electron density
//     rho = 2 sum_i f_i |psi_i|^2 (Eq. Rho), by sum factorisation over the
//     tensor Gauss boxes ("leaves") that make up every cell's rule;
//   * the Hartree problem -lap V_H / (4 pi) = rho (Eq. Poisson) in the
//     classical basis (Sec. III.A): load vector b_j = int rho N_j, Dirichlet
//     data from the monopole + dipole of rho, the FP64 residual on the node
//     grid, and an exact solve of the interior block by fast diagonalisation
//     (the stiffness of a tensor-product mesh is a Kronecker sum of 1-D
//     operators; the dense mode products run as FP64 GEMMs);
//   * LDA exchange-correlation (Ceperley-Alder in the Perdew-Zunger 1981
//     parametrisation), V_eff = V_ext + V_H + V_xc (Eq. veff);
//   * energy integrals and n-stage Anderson mixing of rho.
// All reductions use fixed-order block partials: results are bitwise
// reproducible run to run.  FP64 throughout.
#include <math.h>

#include "efe_func.h"
#include "efe_kernels.h"

namespace efe {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int LT = 256;     // threads of the leaf kernels
constexpr int CW = 16;      // orbital columns per pass of the density kernel
constexpr int NB_RED = 608; // blocks of the point / node reductions (4 x 152 SMs)

__device__ __forceinline__ void gll_lagrange(const double* z, double xi, double* l) {
#pragma unroll
  for (int a = 0; a < NP1; ++a) {
    double v = 1.0;
#pragma unroll
    for (int b = 0; b < NP1; ++b)
      if (b != a) v *= (xi - z[b]) / (z[a] - z[b]);
    l[a] = v;
  }
}

__device__ __forceinline__ void cell_box(const MeshDev& m, int64_t e, int* ijk, double* lo, double* h) {
  ijk[0] = (int)(e % m.nc[0]);
  ijk[1] = (int)((e / m.nc[0]) % m.nc[1]);
  ijk[2] = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const double* bx = m.brk;
  const double* by = bx + m.nc[0] + 1;
  const double* bz = by + m.nc[1] + 1;
  lo[0] = bx[ijk[0]]; h[0] = bx[ijk[0] + 1] - lo[0];
  lo[1] = by[ijk[1]]; h[1] = by[ijk[1] + 1] - lo[1];
  lo[2] = bz[ijk[2]]; h[2] = bz[ijk[2] + 1] - lo[2];
}

// 1-D Lagrange values L[d][i][a] of the cell's GLL basis at the leaf's
// abscissae, read from the stored points (x fastest within a leaf).
__device__ void leaf_lagrange(const RefElem& re, const double* qpts, int64_t off, int n, int nm, const double* lo,
                              const double* h, double* L) {
  for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
    const int d = t / n, i = t % n;
    const int64_t q = off + (d == 0 ? i : (d == 1 ? (int64_t)i * n : (int64_t)i * n * n));
    const double xi = 2.0 * (qpts[4 * q + d] - lo[d]) / h[d] - 1.0;
    gll_lagrange(re.z, xi, L + (d * nm + i) * NP1);
  }
}

__device__ __forceinline__ int64_t cell_node(const MeshDev& m, const int* ijk, int jl) {
  const int a = jl % NP1, b = (jl / NP1) % NP1, c = jl / (NP1 * NP1);
  return (int64_t)(P * ijk[0] + a) + (int64_t)m.nn[0] * ((int64_t)(P * ijk[1] + b) + (int64_t)m.nn[1] * (P * ijk[2] + c));
}

// fixed-order block sum of one double per thread (blockDim.x == 256)
__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// every block sums the same partials in the same order
__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum(v, red);
}

// ---------------------------------------------------------------------------
// rho(x_q) = 2 sum_i f_i psi_i(x_q)^2, psi_i = sum_j N_j X_ji + sum_a E_a X_{n+a, i}
// One CTA per leaf.  Per CW-column pass: X_e (125 x CW) -> T1 = Lx X_e ->
// T2 = Ly T1 -> psi = Lz T2 (+ enrichment) with 2730 FMAs per column on a
// 6^3 leaf instead of 27000 for the dense 216 x 125 basis matrix.
// T: arithmetic of the orbital values (double, or float in the mixed mode);
// 2 f psi^2 and its sums over orbitals are always FP64.
template <typename T>
__global__ void __launch_bounds__(LT) k_leaf_density(LeafDev lf, MeshDev m, RefElem re, EnrDev en,
                                                     const double* __restrict__ X, int64_t ldx, int N,
                                                     const double* __restrict__ occ, double* __restrict__ rho) {
  extern __shared__ __align__(16) double sm[];
  const int64_t leaf = blockIdx.x;
  const int n = lf.n[leaf];
  const int64_t off = lf.off[leaf];
  const int64_t e = lf.cell[leaf];
  const int np = n * n * n;
  const int nm = lf.nmax;
  double* L = sm;                                   // 3 x nm x 5
  double* racc = L + 3 * nm * NP1;                  // nm^3
  T* Xs = reinterpret_cast<T*>(racc + nm * nm * nm);  // 125 x CW
  T* T1 = Xs + NL * CW;                             // n x 25 x CW
  T* T2 = T1 + nm * 25 * CW;                        // n x n x 5 x CW
  T* Xes = T2 + nm * nm * 5 * CW;                   // kmax x CW
  __shared__ int64_t gnode[NL];
  int ijk[3];
  double lo[3], h[3];
  cell_box(m, e, ijk, lo, h);
  leaf_lagrange(re, lf.qpts, off, n, nm, lo, h, L);
  for (int t = threadIdx.x; t < NL; t += blockDim.x) gnode[t] = cell_node(m, ijk, t);
  for (int t = threadIdx.x; t < np; t += blockDim.x) racc[t] = 0.0;
  const int ei = en.cell_enr ? en.cell_enr[e] : -1;
  const int ke = ei >= 0 ? en.cf_ptr[ei + 1] - en.cf_ptr[ei] : 0;
  const int32_t* fl = ei >= 0 ? en.cf_idx + en.cf_ptr[ei] : nullptr;
  const double* Eq = ei >= 0 ? en.Eq + en.eq_off[ei] + (off - en.qoff[e]) * ke : nullptr;
  const double* Lx = L;
  const double* Ly = L + nm * NP1;
  const double* Lz = L + 2 * nm * NP1;
  for (int c0 = 0; c0 < N; c0 += CW) {
    __syncthreads();
    for (int t = threadIdx.x; t < NL * CW; t += blockDim.x) {
      const int r = t / CW, c = t % CW;
      Xs[t] = (c0 + c < N) ? (T)X[gnode[r] * ldx + c0 + c] : T(0);
    }
    for (int t = threadIdx.x; t < ke * CW; t += blockDim.x) {
      const int a = t / CW, c = t % CW;
      Xes[t] = (c0 + c < N) ? (T)X[(en.n_nodes + fl[a]) * ldx + c0 + c] : T(0);
    }
    __syncthreads();
    // T1[ix][b + 5c][col] = sum_a Lx[ix][a] X[a + 5b + 25c][col]
    for (int t = threadIdx.x; t < n * 25 * CW; t += blockDim.x) {
      const int col = t % CW, bc = (t / CW) % 25, ix = t / (25 * CW);
      const T* xr = Xs + (bc * NP1) * CW + col;
      T s = T(0);
#pragma unroll
      for (int a = 0; a < NP1; ++a) s = fma((T)Lx[ix * NP1 + a], xr[a * CW], s);
      T1[t] = s;
    }
    __syncthreads();
    // T2[ix][iy][c][col] = sum_b Ly[iy][b] T1[ix][b + 5c][col]
    for (int t = threadIdx.x; t < n * n * 5 * CW; t += blockDim.x) {
      const int col = t % CW, c = (t / CW) % 5, iy = (t / (5 * CW)) % n, ix = t / (5 * CW * n);
      const T* tr = T1 + (ix * 25 + c * NP1) * CW + col;
      T s = T(0);
#pragma unroll
      for (int b = 0; b < NP1; ++b) s = fma((T)Ly[iy * NP1 + b], tr[b * CW], s);
      T2[t] = s;
    }
    __syncthreads();
    // psi[p][col] = sum_c Lz[iz][c] T2[ix][iy][c][col] + sum_a E[p][a] Xe[a][col]
    // (whole warps iterate together: the lane sum below needs all 32 lanes)
    for (int t0 = 0; t0 < np * CW; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      const bool act = t < np * CW;
      const int col = t % CW, p = act ? t / CW : 0;
      const int ix = p % n, iy = (p / n) % n, iz = p / (n * n);
      const T* tr = T2 + ((ix * n + iy) * 5) * CW + col;
      T psi = T(0);
#pragma unroll
      for (int c = 0; c < NP1; ++c) psi = fma((T)Lz[iz * NP1 + c], tr[c * CW], psi);
      for (int a = 0; a < ke; ++a) psi = fma((T)Eq[(int64_t)p * ke + a], Xes[a * CW + col], psi);
      const double f = (act && c0 + col < N) ? occ[c0 + col] : 0.0;
      const double pd = (double)psi;
      double v = 2.0 * f * pd * pd;
      // fixed-order sum over the CW lanes of this point (CW divides 32)
#pragma unroll
      for (int s = CW / 2; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if (act && col == 0) racc[p] += v;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np; t += blockDim.x) rho[off + t] = racc[t];
}

// u(x_q) = sum_j N_j(x_q) phi_j  (classical field, one column)
__global__ void __launch_bounds__(LT) k_leaf_interp(LeafDev lf, MeshDev m, RefElem re, const double* __restrict__ phi,
                                                    double* __restrict__ out) {
  extern __shared__ __align__(16) double sm[];
  const int64_t leaf = blockIdx.x;
  const int n = lf.n[leaf];
  const int64_t off = lf.off[leaf];
  const int64_t e = lf.cell[leaf];
  const int nm = lf.nmax;
  double* L = sm;
  double* Xs = L + 3 * nm * NP1;
  double* T1 = Xs + NL;
  double* T2 = T1 + nm * 25;
  int ijk[3];
  double lo[3], h[3];
  cell_box(m, e, ijk, lo, h);
  leaf_lagrange(re, lf.qpts, off, n, nm, lo, h, L);
  for (int t = threadIdx.x; t < NL; t += blockDim.x) Xs[t] = phi[cell_node(m, ijk, t)];
  __syncthreads();
  for (int t = threadIdx.x; t < n * 25; t += blockDim.x) {
    const int bc = t % 25, ix = t / 25;
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < NP1; ++a) s = fma(L[ix * NP1 + a], Xs[bc * NP1 + a], s);
    T1[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n * 5; t += blockDim.x) {
    const int c = t % 5, iy = (t / 5) % n, ix = t / (5 * n);
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < NP1; ++b) s = fma(L[(nm + iy) * NP1 + b], T1[ix * 25 + c * NP1 + b], s);
    T2[t] = s;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n * n * n; p += blockDim.x) {
    const int ix = p % n, iy = (p / n) % n, iz = p / (n * n);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NP1; ++c) s = fma(L[(2 * nm + iz) * NP1 + c], T2[(ix * n + iy) * 5 + c], s);
    out[off + p] = s;
  }
}

// per-leaf load contributions  lb[leaf][j] = sum_{q in leaf} w_q rho_q N_j(x_q)
__global__ void __launch_bounds__(LT) k_leaf_load(LeafDev lf, MeshDev m, RefElem re, const double* __restrict__ rho,
                                                  double* __restrict__ lb) {
  extern __shared__ __align__(16) double sm[];
  const int64_t leaf = blockIdx.x;
  const int n = lf.n[leaf];
  const int64_t off = lf.off[leaf];
  const int64_t e = lf.cell[leaf];
  const int np = n * n * n;
  const int nm = lf.nmax;
  double* L = sm;
  double* u = L + 3 * nm * NP1;                    // np
  double* S2 = u + nm * nm * nm;                   // n x n x 5
  double* S1 = S2 + nm * nm * 5;                   // n x 25
  int ijk[3];
  double lo[3], h[3];
  cell_box(m, e, ijk, lo, h);
  leaf_lagrange(re, lf.qpts, off, n, nm, lo, h, L);
  for (int p = threadIdx.x; p < np; p += blockDim.x) u[p] = lf.qpts[4 * (off + p) + 3] * rho[off + p];
  __syncthreads();
  // S2[ix][iy][c] = sum_iz Lz[iz][c] u[ix][iy][iz]
  for (int t = threadIdx.x; t < n * n * 5; t += blockDim.x) {
    const int c = t % 5, iy = (t / 5) % n, ix = t / (5 * n);
    double s = 0.0;
    for (int iz = 0; iz < n; ++iz) s = fma(L[(2 * nm + iz) * NP1 + c], u[ix + n * (iy + n * iz)], s);
    S2[t] = s;
  }
  __syncthreads();
  // S1[ix][b][c] = sum_iy Ly[iy][b] S2[ix][iy][c]
  for (int t = threadIdx.x; t < n * 25; t += blockDim.x) {
    const int c = t % 5, b = (t / 5) % 5, ix = t / 25;
    double s = 0.0;
    for (int iy = 0; iy < n; ++iy) s = fma(L[(nm + iy) * NP1 + b], S2[(ix * n + iy) * 5 + c], s);
    S1[t] = s;
  }
  __syncthreads();
  // lb[a + 5b + 25c] = sum_ix Lx[ix][a] S1[ix][b][c]
  for (int t = threadIdx.x; t < NL; t += blockDim.x) {
    const int a = t % NP1, b = (t / NP1) % NP1, c = t / (NP1 * NP1);
    double s = 0.0;
    for (int ix = 0; ix < n; ++ix) s = fma(L[ix * NP1 + a], S1[ix * 25 + b * 5 + c], s);
    lb[leaf * NL + t] = s;
  }
}

// b_g = mask_g * sum over the cells around node g (z, y, x order) and their
// leaves (stored order) of the leaf contributions.
__global__ void k_node_load(MeshDev m, const int64_t* __restrict__ leaf_ptr, const double* __restrict__ lb,
                            const double* __restrict__ mask, int64_t n_nodes, double* __restrict__ b) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_nodes) return;
  const int G[3] = {(int)(g % m.nn[0]), (int)((g / m.nn[0]) % m.nn[1]), (int)(g / ((int64_t)m.nn[0] * m.nn[1]))};
  int c_lo[3], c_hi[3];
  for (int d = 0; d < 3; ++d) {
    c_hi[d] = min(G[d] / P, m.nc[d] - 1);
    c_lo[d] = (G[d] % P == 0 && G[d] > 0) ? G[d] / P - 1 : c_hi[d];
  }
  double s = 0.0;
  for (int cz = c_lo[2]; cz <= c_hi[2]; ++cz)
    for (int cy = c_lo[1]; cy <= c_hi[1]; ++cy)
      for (int cx = c_lo[0]; cx <= c_hi[0]; ++cx) {
        const int64_t e = cx + (int64_t)m.nc[0] * (cy + (int64_t)m.nc[1] * cz);
        const int jl = (G[0] - P * cx) + NP1 * ((G[1] - P * cy) + NP1 * (G[2] - P * cz));
        for (int64_t l = leaf_ptr[e]; l < leaf_ptr[e + 1]; ++l) s += lb[l * NL + jl];
      }
  b[g] = mask[g] * s;
}

// enrichment values at the points of the enriched cells, [point][function]
__global__ void k_enr_values(EnrDev en, const int32_t* __restrict__ enr_cells, const int64_t* __restrict__ qoff,
                             const double* __restrict__ qpts, const DevFunc* __restrict__ funcs, int64_t n_enr) {
  const int64_t ei = blockIdx.x;
  if (ei >= n_enr) return;
  const int64_t e = enr_cells[ei];
  const int k = en.cf_ptr[ei + 1] - en.cf_ptr[ei];
  const int32_t* fl = en.cf_idx + en.cf_ptr[ei];
  const int64_t q0 = qoff[e], nq = qoff[e + 1] - q0;
  double* out = const_cast<double*>(en.Eq) + en.eq_off[ei];
  for (int64_t t = threadIdx.x; t < nq * k; t += blockDim.x) {
    const int64_t p = t / k;
    const int a = (int)(t % k);
    const double* x = qpts + 4 * (q0 + p);
    out[t] = eval_func_value(funcs[fl[a]], x[0], x[1], x[2]);
  }
}

// ---------------------------------------------------------------------------
// Hartree stiffness  A = (1/4pi) (Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz)
// on the tensor-product node grid: Kd, Md are the assembled 1-D stiffness and
// exact mass matrices of axis d (9-wide bands).  A CTA forms a 16 x 8 x 8 tile
// of A x from a (24 x 16 x 16) halo region by three 1-D passes in shared memory.
constexpr int TX = 16, TY = 8, TZ = 8;
constexpr int HXW = TX + 8, HYW = TY + 8, HZW = TZ + 8;
constexpr int STILE = TX * TY * TZ;

template <typename T>
struct StiffSmem {
  T x[HZW * HYW * HXW];            // input region; later reused for the y-pass results
  T u[2 * TZ * HYW * HXW];         // z-pass: Mz x, Kz x
  double band[(TX + TY + TZ) * 9 * 2];
  double red[256];
};

template <typename T>
__device__ void stiff_tile(const BandsDev& bd, int i0, int j0, int k0, StiffSmem<T>& s, T* yout) {
  // band rows of this tile: x rows i0..i0+15, y rows j0..j0+7, z rows k0..k0+7
  for (int t = threadIdx.x; t < (TX + TY + TZ) * 9; t += blockDim.x) {
    const int r = t / 9, o = t % 9;
    int d, g;
    if (r < TX) { d = 0; g = i0 + r; } else if (r < TX + TY) { d = 1; g = j0 + r - TX; } else { d = 2; g = k0 + r - TX - TY; }
    const bool ok = g < bd.nn[d];
    s.band[2 * t] = ok ? bd.K[d][(int64_t)g * 9 + o] : 0.0;
    s.band[2 * t + 1] = ok ? bd.M[d][(int64_t)g * 9 + o] : 0.0;
  }
  __syncthreads();
  const double* bx = s.band;
  const double* by = s.band + TX * 18;
  const double* bz = s.band + (TX + TY) * 18;
  // z pass: u0 = Mz x, u1 = Kz x  on (k in 8) x (jj in 16) x (ii in 24)
  T* u0 = s.u;
  T* u1 = s.u + TZ * HYW * HXW;
  for (int t = threadIdx.x; t < TZ * HYW * HXW; t += blockDim.x) {
    const int ii = t % HXW, jj = (t / HXW) % HYW, k = t / (HXW * HYW);
    const T* xr = s.x + (k * HYW + jj) * HXW + ii;
    const double* br = bz + k * 18;
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int o = 0; o < 9; ++o) {
      const T v = xr[o * HYW * HXW];
      a0 = fma(T(br[2 * o + 1]), v, a0);
      a1 = fma(T(br[2 * o]), v, a1);
    }
    u0[t] = a0;
    u1[t] = a1;
  }
  __syncthreads();
  // y pass: v0 = My u0, v1 = Ky u0 + My u1  on (k in 8) x (j in 8) x (ii in 24)
  T* v0 = s.x;
  T* v1 = s.x + TZ * TY * HXW;
  for (int t = threadIdx.x; t < TZ * TY * HXW; t += blockDim.x) {
    const int ii = t % HXW, j = (t / HXW) % TY, k = t / (HXW * TY);
    const T* r0 = u0 + (k * HYW + j) * HXW + ii;
    const T* r1 = u1 + (k * HYW + j) * HXW + ii;
    const double* br = by + j * 18;
    T a0 = T(0), a1 = T(0);
#pragma unroll
    for (int o = 0; o < 9; ++o) {
      const T w0 = r0[o * HXW], w1 = r1[o * HXW];
      a0 = fma(T(br[2 * o + 1]), w0, a0);
      a1 = fma(T(br[2 * o]), w0, a1);
      a1 = fma(T(br[2 * o + 1]), w1, a1);
    }
    v0[t] = a0;
    v1[t] = a1;
  }
  __syncthreads();
  // x pass: y = (Kx v0 + Mx v1) / (4 pi)  on (k in 8) x (j in 8) x (i in 16)
  const T inv4pi = T(0.079577471545947667884);
#pragma unroll
  for (int r = 0; r < STILE / 256; ++r) {
    const int t = threadIdx.x + 256 * r;
    const int i = t % TX, j = (t / TX) % TY, k = t / (TX * TY);
    const T* r0 = v0 + (k * TY + j) * HXW + i;
    const T* r1 = v1 + (k * TY + j) * HXW + i;
    const double* br = bx + i * 18;
    T a = T(0);
#pragma unroll
    for (int o = 0; o < 9; ++o) {
      a = fma(T(br[2 * o]), r0[o], a);
      a = fma(T(br[2 * o + 1]), r1[o], a);
    }
    yout[r] = a * inv4pi;
  }
}

__device__ __forceinline__ void tile_origin(const BandsDev& bd, int* i0, int* j0, int* k0, int64_t* tile) {
  const int tx = (bd.nn[0] + TX - 1) / TX, ty = (bd.nn[1] + TY - 1) / TY;
  const int64_t b = blockIdx.x;
  *i0 = (int)(b % tx) * TX;
  *j0 = (int)((b / tx) % ty) * TY;
  *k0 = (int)(b / ((int64_t)tx * ty)) * TZ;
  *tile = b;
}

__device__ __forceinline__ int64_t node_of(const BandsDev& bd, int i, int j, int k) {
  return (int64_t)i + (int64_t)bd.nn[0] * ((int64_t)j + (int64_t)bd.nn[1] * k);
}

// FP64 residual r = mask (b - A phi) on the node grid and partials of |r|^2
__global__ void __launch_bounds__(256) k_stiff_resid(BandsDev bd, const double* __restrict__ phi,
                                                     const double* __restrict__ b, const double* __restrict__ mask,
                                                     double* __restrict__ r64, double* __restrict__ part_rr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  StiffSmem<double>& s = *reinterpret_cast<StiffSmem<double>*>(smraw);
  int i0, j0, k0;
  int64_t tile;
  tile_origin(bd, &i0, &j0, &k0, &tile);
  for (int t = threadIdx.x; t < HZW * HYW * HXW; t += blockDim.x) {
    const int ii = t % HXW, jj = (t / HXW) % HYW, kk = t / (HXW * HYW);
    const int gi = i0 - 4 + ii, gj = j0 - 4 + jj, gk = k0 - 4 + kk;
    const bool ok = gi >= 0 && gj >= 0 && gk >= 0 && gi < bd.nn[0] && gj < bd.nn[1] && gk < bd.nn[2];
    s.x[t] = ok ? phi[node_of(bd, gi, gj, gk)] : 0.0;
  }
  __syncthreads();
  double y[STILE / 256];
  stiff_tile<double>(bd, i0, j0, k0, s, y);
  double rr = 0.0;
#pragma unroll
  for (int r = 0; r < STILE / 256; ++r) {
    const int t = threadIdx.x + 256 * r;
    const int i = i0 + t % TX, j = j0 + (t / TX) % TY, k = k0 + t / (TX * TY);
    if (i < bd.nn[0] && j < bd.nn[1] && k < bd.nn[2]) {
      const int64_t g = node_of(bd, i, j, k);
      const double rv = mask[g] * (b[g] - y[r]);
      r64[g] = rv;
      rr += rv * rv;
    }
  }
  rr = block_sum(rr, s.red);
  if (threadIdx.x == 0) part_rr[tile] = rr;
}

// interior nodes (1 .. nn_d - 2 on every axis) <-> compact array U[k][j][i]
__global__ void k_fd_gather(BandsDev bd, const double* __restrict__ r, double* __restrict__ U) {
  const int mi = bd.nn[0] - 2, mj = bd.nn[1] - 2, mk = bd.nn[2] - 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)mi * mj * mk) return;
  const int i = (int)(t % mi), j = (int)((t / mi) % mj), k = (int)(t / ((int64_t)mi * mj));
  U[t] = r[node_of(bd, i + 1, j + 1, k + 1)];
}

__global__ void k_fd_scatter_add(BandsDev bd, const double* __restrict__ U, double* __restrict__ phi) {
  const int mi = bd.nn[0] - 2, mj = bd.nn[1] - 2, mk = bd.nn[2] - 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)mi * mj * mk) return;
  const int i = (int)(t % mi), j = (int)((t / mi) % mj), k = (int)(t / ((int64_t)mi * mj));
  phi[node_of(bd, i + 1, j + 1, k + 1)] += U[t];
}

// U[k][j][i] *= 4 pi / (lx_i + ly_j + lz_k)   (inverse of the diagonalised operator)
__global__ void k_fd_scale(int mi, int mj, int mk, const double* __restrict__ lx, const double* __restrict__ ly,
                           const double* __restrict__ lz, double* __restrict__ U) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)mi * mj * mk) return;
  const int i = (int)(t % mi), j = (int)((t / mi) % mj), k = (int)(t / ((int64_t)mi * mj));
  U[t] *= 12.566370614359172954 / (lx[i] + ly[j] + lz[k]);
}

// ---------------------------------------------------------------------------
// monopole and first moments of rho over the quadrature points
__global__ void __launch_bounds__(256) k_moments(const double* __restrict__ qpts, const double* __restrict__ rho,
                                                 int64_t nq, double* __restrict__ part) {
  __shared__ double red[256];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    const double wr = qpts[4 * q + 3] * rho[q];
    s[0] += wr;
    s[1] += wr * qpts[4 * q];
    s[2] += wr * qpts[4 * q + 1];
    s[3] += wr * qpts[4 * q + 2];
  }
  for (int c = 0; c < 4; ++c) {
    const double v = block_sum(s[c], red);
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = v;
  }
}

// generic fixed-order finish of nv block-partial vectors: out[c] = sum_b part[c * nb + b]
__global__ void __launch_bounds__(256) k_finish(const double* __restrict__ part, int nb, int nv, double* __restrict__ out) {
  __shared__ double red[256];
  for (int c = 0; c < nv; ++c) {
    const double v = sum_partials(part + (int64_t)c * nb, nb, red);
    if (threadIdx.x == 0) out[c] = v;
  }
}

// Dirichlet data on the boundary nodes: Q / r + d . r / r^3 about the centre of charge
__global__ void k_hartree_bc(MeshDev m, const double* __restrict__ node_xyz, const double* __restrict__ mask,
                             const double* __restrict__ mom, int64_t n_nodes, double* __restrict__ phi) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_nodes || mask[g] != 0.0) return;
  const double Q = mom[0];
  double c[3] = {0.0, 0.0, 0.0}, dip[3] = {0.0, 0.0, 0.0};
  if (fabs(Q) > 1e-300)
    for (int d = 0; d < 3; ++d) {
      c[d] = mom[1 + d] / Q;
      dip[d] = mom[1 + d] - c[d] * Q;
    }
  const int G[3] = {(int)(g % m.nn[0]), (int)((g / m.nn[0]) % m.nn[1]), (int)(g / ((int64_t)m.nn[0] * m.nn[1]))};
  const double* ax[3] = {node_xyz, node_xyz + m.nn[0], node_xyz + m.nn[0] + m.nn[1]};
  double rv[3], r2 = 0.0, rd = 0.0;
  for (int d = 0; d < 3; ++d) {
    rv[d] = ax[d][G[d]] - c[d];
    r2 += rv[d] * rv[d];
    rd += rv[d] * dip[d];
  }
  const double rn = sqrt(r2);
  phi[g] = Q / rn + rd / (rn * rn * rn);
}

// ---------------------------------------------------------------------------
// LDA (spin-unpolarised): Slater exchange + Perdew-Zunger 1981 fit of the
// Ceperley-Alder correlation; eps_xc per electron, v_xc = d(rho eps_xc)/d rho.
__device__ __forceinline__ void lda_pz(double rho, double* exc, double* vxc) {
  constexpr double PI = 3.14159265358979323846;
  constexpr double G = -0.1423, B1 = 1.0529, B2 = 0.3334;
  constexpr double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
  rho = fmax(rho, 1e-30);
  const double ex = -0.75 * cbrt(3.0 * rho / PI);
  const double rs = cbrt(3.0 / (4.0 * PI * rho));
  double ec, vc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs);
    const double den = 1.0 + B1 * sq + B2 * rs;
    ec = G / den;
    vc = ec * (1.0 + (7.0 / 6.0) * B1 * sq + (4.0 / 3.0) * B2 * rs) / den;
  } else {
    const double lr = log(rs);
    ec = A * lr + B + C * rs * lr + D * rs;
    vc = A * lr + (B - A / 3.0) + (2.0 / 3.0) * C * rs * lr + ((2.0 * D - C) / 3.0) * rs;
  }
  *exc = ex + ec;
  *vxc = (4.0 / 3.0) * ex + vc;
}

__global__ void k_lda(int64_t nq, const double* __restrict__ rho, double* __restrict__ exc, double* __restrict__ vxc) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double e, v;
  lda_pz(rho[q], &e, &v);
  if (exc) exc[q] = e;
  if (vxc) vxc[q] = v;
}

// V_eff = V_ext + V_H + v_xc(rho)   (Eq. veff); also keeps v_xc
__global__ void k_veff(int64_t nq, const double* __restrict__ rho, const double* __restrict__ vext,
                       const double* __restrict__ vh, double* __restrict__ vxc, double* __restrict__ veff) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double e, v;
  lda_pz(rho[q], &e, &v);
  vxc[q] = v;
  veff[q] = vext[q] + vh[q] + v;
}

// energy integrals: [int rho_o eps_xc(rho_o), int rho_o V_H[rho_o],
//                    int rho_o (V_H[rho_i] + v_xc(rho_i)), int (rho_o - rho_i)^2, int rho_o]
__global__ void __launch_bounds__(256) k_scf_sums(const double* __restrict__ qpts, int64_t nq,
                                                  const double* __restrict__ rho_in, const double* __restrict__ rho_out,
                                                  const double* __restrict__ vh_in, const double* __restrict__ vxc_in,
                                                  const double* __restrict__ vh_out, double* __restrict__ part) {
  __shared__ double red[256];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    const double w = qpts[4 * q + 3];
    const double ro = rho_out[q];
    double e, v;
    lda_pz(ro, &e, &v);
    const double wr = w * ro;
    const double dr = ro - rho_in[q];
    s[0] += wr * e;
    s[1] += wr * vh_out[q];
    s[2] += wr * (vh_in[q] + vxc_in[q]);
    s[3] += w * dr * dr;
    s[4] += wr;
  }
  for (int c = 0; c < 5; ++c) {
    const double v = block_sum(s[c], red);
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = v;
  }
}

// ---------------------------------------------------------------------------
// n-stage Anderson mixing.  With F_k = rho_out_k - rho_in_k and dF_k = F_k - F_last:
// Gram G_kl = int dF_k dF_l and right-hand side -int dF_k F_last (k, l < n - 1).
__global__ void __launch_bounds__(256) k_anderson_gram(const double* __restrict__ qpts, int64_t nq, HistDev hs,
                                                       double* __restrict__ part) {
  __shared__ double red[256];
  const int n = hs.n, m = n - 1;
  double acc[ANDERSON_MAX * (ANDERSON_MAX + 1) / 2 + ANDERSON_MAX];
  const int nv = m * (m + 1) / 2 + m;
  for (int c = 0; c < nv; ++c) acc[c] = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    const double w = qpts[4 * q + 3];
    const double Fn = hs.rout[m][q] - hs.rin[m][q];
    double dF[ANDERSON_MAX];
    for (int k = 0; k < m; ++k) dF[k] = (hs.rout[k][q] - hs.rin[k][q]) - Fn;
    int c = 0;
    for (int k = 0; k < m; ++k)
      for (int l = k; l < m; ++l) acc[c++] += w * dF[k] * dF[l];
    for (int k = 0; k < m; ++k) acc[c++] -= w * dF[k] * Fn;
  }
  for (int c = 0; c < nv; ++c) {
    const double v = block_sum(acc[c], red);
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = v;
  }
}

// rho_next = rin_last + sum_k th_k (rin_k - rin_last) + beta (F_last + sum_k th_k dF_k)
__global__ void k_anderson_mix(int64_t nq, HistDev hs, AndersonCoef th, double beta, double* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int m = hs.n - 1;
  const double rl = hs.rin[m][q];
  const double Fn = hs.rout[m][q] - rl;
  double rin = 0.0, fb = 0.0;
  for (int k = 0; k < m; ++k) {
    rin += th.t[k] * (hs.rin[k][q] - rl);
    fb += th.t[k] * ((hs.rout[k][q] - hs.rin[k][q]) - Fn);
  }
  out[q] = (rl + rin) + beta * (Fn + fb);
}

__global__ void k_scale_f64(int64_t n, double* __restrict__ x, const double* __restrict__ num, double target) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= target / num[0];
}


// ---------------------------------------------------------------------------
// Potential parts of the Hamiltonian blocks by sum factorisation over the
// quadrature leaves (set_potential, Eqs. Hcc, Hec, Hee).
//
// H^cc_e[(a,b,c),(a',b',c')] = kinetic (closed form) +
//   sum_q w V  Lx[a] Lx[a'] Ly[b] Ly[b'] Lz[c] Lz[c']
// depends on the index pairs only through the symmetric products
// Lx[a]Lx[a'] (15 pairs per axis): a 15 x 15 x 15 tensor per cell, formed
// leaf by leaf in three passes (15 n^3 + 225 n^2 + 3375 n FMAs for an n^3
// leaf, against 15625 n^3 for the dense B^T diag(wV) B), then expanded.
__constant__ int c_pa[15] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 3, 3, 4};
__constant__ int c_pb[15] = {0, 1, 2, 3, 4, 1, 2, 3, 4, 2, 3, 4, 3, 4, 4};

__device__ __forceinline__ int pair_index(int a, int b) {
  if (a > b) { const int t = a; a = b; b = t; }
  return a * NP1 - a * (a - 1) / 2 + (b - a);
}

__global__ void __launch_bounds__(256) k_hcc_sf(RefElem re, MeshDev m, LeafDev lf, const int64_t* __restrict__ leaf_ptr,
                                                const double* __restrict__ V, double* __restrict__ Hcc) {
  extern __shared__ __align__(16) double sm[];
  const int nm = lf.nmax;
  double* S = sm;                          // 15^3
  double* L = S + 3375;                    // 3 x nm x 5
  double* Pp = L + 3 * nm * NP1;           // 3 x nm x 15
  double* u = Pp + 3 * nm * 15;            // nm^3
  double* T1 = u + nm * nm * nm;           // 15 x nm^2
  double* T2 = T1 + 15 * nm * nm;          // 225 x nm
  const int64_t e = blockIdx.x;
  int ijk[3];
  double lo[3], h[3];
  cell_box(m, e, ijk, lo, h);
  for (int t = threadIdx.x; t < 3375; t += blockDim.x) S[t] = 0.0;
  for (int64_t l = leaf_ptr[e]; l < leaf_ptr[e + 1]; ++l) {
    const int n = lf.n[l];
    const int64_t off = lf.off[l];
    const int np = n * n * n;
    __syncthreads();
    leaf_lagrange(re, lf.qpts, off, n, nm, lo, h, L);
    for (int p = threadIdx.x; p < np; p += blockDim.x) u[p] = lf.qpts[4 * (off + p) + 3] * V[off + p];
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * n * 15; t += blockDim.x) {
      const int d = t / (n * 15), i = (t / 15) % n, al = t % 15;
      const double* Li = L + (d * nm + i) * NP1;
      Pp[(d * nm + i) * 15 + al] = Li[c_pa[al]] * Li[c_pb[al]];
    }
    __syncthreads();
    // T1[al][iy][iz] = sum_ix Px[ix][al] u[ix][iy][iz]
    for (int t = threadIdx.x; t < 15 * n * n; t += blockDim.x) {
      const int al = t / (n * n), r = t % (n * n), iy = r / n, iz = r % n;
      const double* ur = u + n * (iy + n * iz);
      double sacc = 0.0;
      for (int ix = 0; ix < n; ++ix) sacc = fma(Pp[ix * 15 + al], ur[ix], sacc);
      T1[t] = sacc;
    }
    __syncthreads();
    // T2[al][be][iz] = sum_iy Py[iy][be] T1[al][iy][iz]
    for (int t = threadIdx.x; t < 225 * n; t += blockDim.x) {
      const int ab = t / n, iz = t % n, al = ab / 15, be = ab % 15;
      double sacc = 0.0;
      for (int iy = 0; iy < n; ++iy) sacc = fma(Pp[(nm + iy) * 15 + be], T1[al * n * n + iy * n + iz], sacc);
      T2[ab * nm + iz] = sacc;
    }
    __syncthreads();
    // S[al][be][ga] += sum_iz Pz[iz][ga] T2[al][be][iz]
    for (int t = threadIdx.x; t < 3375; t += blockDim.x) {
      const int ab = t / 15, ga = t % 15;
      double sacc = 0.0;
      for (int iz = 0; iz < n; ++iz) sacc = fma(Pp[(2 * nm + iz) * 15 + ga], T2[ab * nm + iz], sacc);
      S[t] += sacc;
    }
  }
  __syncthreads();
  const double cx = h[1] * h[2] / (2.0 * h[0]), cy = h[0] * h[2] / (2.0 * h[1]), cz = h[0] * h[1] / (2.0 * h[2]);
  double* He = Hcc + e * (int64_t)(NL * NL);
  for (int idx = threadIdx.x; idx < NL * NL; idx += blockDim.x) {
    const int r = idx / NL, c = idx % NL;
    const int ra = r % NP1, rb = (r / NP1) % NP1, rc = r / (NP1 * NP1);
    const int ca = c % NP1, cb = (c / NP1) % NP1, cc = c / (NP1 * NP1);
    const double kin =
        0.5 * (cx * re.K1[ra * NP1 + ca] * re.M1[rb * NP1 + cb] * re.M1[rc * NP1 + cc] +
               cy * re.M1[ra * NP1 + ca] * re.K1[rb * NP1 + cb] * re.M1[rc * NP1 + cc] +
               cz * re.M1[ra * NP1 + ca] * re.M1[rb * NP1 + cb] * re.K1[rc * NP1 + cc]);
    He[idx] = kin + S[(pair_index(ra, ca) * 15 + pair_index(rb, cb)) * 15 + pair_index(rc, cc)];
  }
}

// Potential blocks of one enriched cell (Eqs. Hec, Hee):
//   P[a][j] = sum_q w V E_a N_j   (per leaf and function: the load-vector passes)
//   Q[a][b] = sum_q w V E_a E_b   (a <= b, mirrored)
// accumulated in place in the cell's own output blocks (thread-owned entries).
constexpr int ENR_G = 8;   // functions per pass

__global__ void __launch_bounds__(256) k_enr_sf(RefElem re, MeshDev m, LeafDev lf, const int64_t* __restrict__ leaf_ptr,
                                                EnrDev en, const int32_t* __restrict__ enr_cells,
                                                const double* __restrict__ V, const int64_t* __restrict__ blkP_off,
                                                const int64_t* __restrict__ blkQ_off, double* __restrict__ Pblk,
                                                double* __restrict__ Qblk) {
  extern __shared__ __align__(16) double sm[];
  const int nm = lf.nmax;
  double* L = sm;                                  // 3 x nm x 5
  double* wv = L + 3 * nm * NP1;                   // nm^3
  double* U = wv + nm * nm * nm;                   // G x nm^3
  double* S2 = U + ENR_G * nm * nm * nm;           // G x nm^2 x 5
  double* S1 = S2 + ENR_G * nm * nm * 5;           // G x nm x 25
  const int ei = blockIdx.x;
  const int64_t e = enr_cells[ei];
  const int k = en.cf_ptr[ei + 1] - en.cf_ptr[ei];
  const double* E = en.Eq + en.eq_off[ei];         // [point of the cell][function]
  double* P = Pblk + blkP_off[ei];
  double* Q = Qblk + blkQ_off[ei];
  int ijk[3];
  double lo[3], h[3];
  cell_box(m, e, ijk, lo, h);
  for (int t = threadIdx.x; t < k * NL; t += blockDim.x) P[t] = 0.0;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Q[t] = 0.0;
  const int64_t q0 = en.qoff[e];
  for (int64_t l = leaf_ptr[e]; l < leaf_ptr[e + 1]; ++l) {
    const int n = lf.n[l];
    const int64_t off = lf.off[l];
    const int64_t p0 = off - q0;
    const int np = n * n * n;
    __syncthreads();
    leaf_lagrange(re, lf.qpts, off, n, nm, lo, h, L);
    for (int p = threadIdx.x; p < np; p += blockDim.x) wv[p] = lf.qpts[4 * (off + p) + 3] * V[off + p];
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
      const int a = t / k, b = t % k;
      if (a > b) continue;
      const double* Ep = E + p0 * k;
      double sacc = 0.0;
      for (int p = 0; p < np; ++p) sacc = fma(wv[p] * Ep[(int64_t)p * k + a], Ep[(int64_t)p * k + b], sacc);
      Q[t] += sacc;
    }
    for (int a0 = 0; a0 < k; a0 += ENR_G) {
      const int g = min(ENR_G, k - a0);
      __syncthreads();
      for (int t = threadIdx.x; t < g * np; t += blockDim.x) {
        const int gi = t / np, p = t % np;
        U[gi * np + p] = wv[p] * E[(p0 + p) * k + a0 + gi];
      }
      __syncthreads();
      for (int t = threadIdx.x; t < g * n * n * 5; t += blockDim.x) {
        const int gi = t / (n * n * 5), r = t % (n * n * 5);
        const int c = r % 5, iy = (r / 5) % n, ix = r / (5 * n);
        const double* ug = U + gi * np;
        double sacc = 0.0;
        for (int iz = 0; iz < n; ++iz) sacc = fma(L[(2 * nm + iz) * NP1 + c], ug[ix + n * (iy + n * iz)], sacc);
        S2[gi * nm * nm * 5 + r] = sacc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < g * n * 25; t += blockDim.x) {
        const int gi = t / (n * 25), r = t % (n * 25);
        const int c = r % 5, b = (r / 5) % 5, ix = r / 25;
        double sacc = 0.0;
        for (int iy = 0; iy < n; ++iy)
          sacc = fma(L[(nm + iy) * NP1 + b], S2[gi * nm * nm * 5 + (ix * n + iy) * 5 + c], sacc);
        S1[gi * nm * 25 + r] = sacc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < g * NL; t += blockDim.x) {
        const int gi = t / NL, jl = t % NL;
        const int a = jl % NP1, b = (jl / NP1) % NP1, c = jl / (NP1 * NP1);
        double sacc = 0.0;
        for (int ix = 0; ix < n; ++ix) sacc = fma(L[ix * NP1 + a], S1[gi * nm * 25 + ix * 25 + b * 5 + c], sacc);
        P[(a0 + gi) * NL + jl] += sacc;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int a = t / k, b = t % k;
    if (a > b) Q[t] = Q[b * k + a];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
size_t leaf_density_smem(int nm, int kmax) {
  return sizeof(double) * (3 * nm * NP1 + nm * nm * nm + NL * CW + nm * 25 * CW + nm * nm * 5 * CW + (size_t)kmax * CW);
}

int launch_leaf_density(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re, const EnrDev& en,
                        int kmax, const double* X, int64_t ldx, int N, const double* occ, double* rho, bool fp32,
                        cudaStream_t st) {
  if (n_leaf <= 0) return 0;
  const size_t sm = leaf_density_smem(lf.nmax, kmax);
  if (sm > 227 * 1024) return 1;
  static size_t set64 = 0, set32 = 0;
  size_t& set = fp32 ? set32 : set64;
  if (sm > set) {
    const cudaError_t e =
        fp32 ? cudaFuncSetAttribute(k_leaf_density<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
             : cudaFuncSetAttribute(k_leaf_density<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return 1;
    set = sm;
  }
  if (fp32)
    k_leaf_density<float><<<(unsigned)n_leaf, LT, sm, st>>>(lf, m, re, en, X, ldx, N, occ, rho);
  else
    k_leaf_density<double><<<(unsigned)n_leaf, LT, sm, st>>>(lf, m, re, en, X, ldx, N, occ, rho);
  g_launches++;
  return 0;
}

void launch_leaf_interp(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re, const double* phi,
                        double* out, cudaStream_t st) {
  if (n_leaf <= 0) return;
  const int nm = lf.nmax;
  const size_t sm = sizeof(double) * (3 * nm * NP1 + NL + nm * 25 + nm * nm * 5);
  k_leaf_interp<<<(unsigned)n_leaf, LT, sm, st>>>(lf, m, re, phi, out);
  g_launches++;
}

void launch_hartree_load(const LeafDev& lf, int64_t n_leaf, const MeshDev& m, const RefElem& re,
                         const int64_t* leaf_ptr, const double* rho, const double* mask, int64_t n_nodes,
                         double* lb, double* b, cudaStream_t st) {
  if (n_leaf > 0) {
    const int nm = lf.nmax;
    const size_t sm = sizeof(double) * (3 * nm * NP1 + nm * nm * nm + nm * nm * 5 + nm * 25);
    k_leaf_load<<<(unsigned)n_leaf, LT, sm, st>>>(lf, m, re, rho, lb);
    g_launches++;
  }
  k_node_load<<<nblk(n_nodes, 256), 256, 0, st>>>(m, leaf_ptr, lb, mask, n_nodes, b);
  g_launches++;
}

void launch_enr_values(const EnrDev& en, const int32_t* enr_cells, const int64_t* qoff, const double* qpts,
                       const DevFunc* funcs, int64_t n_enr, cudaStream_t st) {
  if (n_enr <= 0) return;
  k_enr_values<<<(unsigned)n_enr, 256, 0, st>>>(en, enr_cells, qoff, qpts, funcs, n_enr);
  g_launches++;
}

int launch_hcc_sf(const RefElem& re, const MeshDev& m, const LeafDev& lf, const int64_t* leaf_ptr, const double* V,
                  int64_t n_cell, double* Hcc, cudaStream_t st) {
  if (n_cell <= 0) return 0;
  const int nm = lf.nmax;
  const size_t sm = sizeof(double) * (3375 + 3 * nm * NP1 + 3 * nm * 15 + nm * nm * nm + 15 * nm * nm + 225 * nm);
  static size_t set = 0;
  if (sm > set) {
    if (cudaFuncSetAttribute(k_hcc_sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 1;
    set = sm;
  }
  k_hcc_sf<<<(unsigned)n_cell, 256, sm, st>>>(re, m, lf, leaf_ptr, V, Hcc);
  g_launches++;
  return 0;
}

int launch_enr_sf(const RefElem& re, const MeshDev& m, const LeafDev& lf, const int64_t* leaf_ptr, const EnrDev& en,
                  const int32_t* enr_cells, int64_t n_enr, const double* V, const int64_t* blkP_off,
                  const int64_t* blkQ_off, double* Pblk, double* Qblk, cudaStream_t st) {
  if (n_enr <= 0) return 0;
  const int nm = lf.nmax;
  const size_t sm = sizeof(double) * (3 * nm * NP1 + nm * nm * nm + ENR_G * nm * nm * nm + ENR_G * nm * nm * 5 +
                                      ENR_G * nm * 25);
  static size_t set = 0;
  if (sm > set) {
    if (cudaFuncSetAttribute(k_enr_sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 1;
    set = sm;
  }
  k_enr_sf<<<(unsigned)n_enr, 256, sm, st>>>(re, m, lf, leaf_ptr, en, enr_cells, V, blkP_off, blkQ_off, Pblk, Qblk);
  g_launches++;
  return 0;
}

int64_t stiff_tiles(const BandsDev& bd) {
  return (int64_t)((bd.nn[0] + TX - 1) / TX) * ((bd.nn[1] + TY - 1) / TY) * ((bd.nn[2] + TZ - 1) / TZ);
}

int reduce_blocks() { return NB_RED; }

int launch_stiff_resid(const BandsDev& bd, const double* phi, const double* b, const double* mask, double* r64,
                       double* part_rr, cudaStream_t st) {
  const size_t sm = sizeof(StiffSmem<double>);
  static bool set = false;
  if (!set) {
    if (cudaFuncSetAttribute(k_stiff_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return 1;
    set = true;
  }
  k_stiff_resid<<<(unsigned)stiff_tiles(bd), 256, sm, st>>>(bd, phi, b, mask, r64, part_rr);
  g_launches++;
  return 0;
}

// interior solve A_ii d = r_i by fast diagonalisation; phi_i += d.
// V[d] (m x m, row-major, V^T M V = I, V^T K V = diag(lam)), Vt[d] = V[d]^T.
void launch_fd_solve(const BandsDev& bd, const double* const* V, const double* const* Vt, const double* const* lam,
                     const double* r, double* U0, double* U1, double* phi, cudaStream_t st) {
  const int mi = bd.nn[0] - 2, mj = bd.nn[1] - 2, mk = bd.nn[2] - 2;
  const int64_t n = (int64_t)mi * mj * mk;
  if (n <= 0) return;
  const int64_t sl = (int64_t)mi * mj;
  k_fd_gather<<<nblk(n, 256), 256, 0, st>>>(bd, r, U0);
  // forward transform u = (Vx (x) Vy (x) Vz)^T r
  launch_gemm_nn_batched((int64_t)mj * mk, mi, mi, U0, mi, 0, V[0], mi, 0, U1, mi, 0, 1, st);
  launch_gemm_nn_batched(mj, mi, mj, Vt[1], mj, 0, U1, mi, sl, U0, mi, sl, mk, st);
  launch_gemm_nn_batched(mk, (int)sl, mk, Vt[2], mk, 0, U0, sl, 0, U1, sl, 0, 1, st);
  k_fd_scale<<<nblk(n, 256), 256, 0, st>>>(mi, mj, mk, lam[0], lam[1], lam[2], U1);
  // back transform d = (Vx (x) Vy (x) Vz) u
  launch_gemm_nn_batched(mk, (int)sl, mk, V[2], mk, 0, U1, sl, 0, U0, sl, 0, 1, st);
  launch_gemm_nn_batched(mj, mi, mj, V[1], mj, 0, U0, mi, sl, U1, mi, sl, mk, st);
  launch_gemm_nn_batched((int64_t)mj * mk, mi, mi, U1, mi, 0, Vt[0], mi, 0, U0, mi, 0, 1, st);
  k_fd_scatter_add<<<nblk(n, 256), 256, 0, st>>>(bd, U0, phi);
  g_launches += 4;
}

void launch_moments(const double* qpts, const double* rho, int64_t nq, double* part, double* mom, cudaStream_t st) {
  k_moments<<<NB_RED, 256, 0, st>>>(qpts, rho, nq, part);
  k_finish<<<1, 256, 0, st>>>(part, NB_RED, 4, mom);
  g_launches += 2;
}

void launch_finish(const double* part, int nb, int nv, double* out, cudaStream_t st) {
  k_finish<<<1, 256, 0, st>>>(part, nb, nv, out);
  g_launches++;
}

void launch_hartree_bc(const MeshDev& m, const double* node_xyz, const double* mask, const double* mom,
                       int64_t n_nodes, double* phi, cudaStream_t st) {
  k_hartree_bc<<<nblk(n_nodes, 256), 256, 0, st>>>(m, node_xyz, mask, mom, n_nodes, phi);
  g_launches++;
}

void launch_lda(int64_t nq, const double* rho, double* exc, double* vxc, cudaStream_t st) {
  k_lda<<<nblk(nq, 256), 256, 0, st>>>(nq, rho, exc, vxc);
  g_launches++;
}

void launch_veff(int64_t nq, const double* rho, const double* vext, const double* vh, double* vxc, double* veff,
                 cudaStream_t st) {
  k_veff<<<nblk(nq, 256), 256, 0, st>>>(nq, rho, vext, vh, vxc, veff);
  g_launches++;
}

void launch_scf_sums(const double* qpts, int64_t nq, const double* rho_in, const double* rho_out, const double* vh_in,
                     const double* vxc_in, const double* vh_out, double* part, double* out, cudaStream_t st) {
  k_scf_sums<<<NB_RED, 256, 0, st>>>(qpts, nq, rho_in, rho_out, vh_in, vxc_in, vh_out, part);
  k_finish<<<1, 256, 0, st>>>(part, NB_RED, 5, out);
  g_launches += 2;
}

int anderson_values(int n) { return (n - 1) * n / 2 + (n - 1); }

void launch_anderson_gram(const double* qpts, int64_t nq, const HistDev& hs, double* part, double* out,
                          cudaStream_t st) {
  k_anderson_gram<<<NB_RED, 256, 0, st>>>(qpts, nq, hs, part);
  k_finish<<<1, 256, 0, st>>>(part, NB_RED, anderson_values(hs.n), out);
  g_launches += 2;
}

void launch_anderson_mix(int64_t nq, const HistDev& hs, const AndersonCoef& th, double beta, double* out,
                         cudaStream_t st) {
  k_anderson_mix<<<nblk(nq, 256), 256, 0, st>>>(nq, hs, th, beta, out);
  g_launches++;
}

void launch_scale_to(int64_t n, double* x, const double* num, double target, cudaStream_t st) {
  k_scale_f64<<<nblk(n, 256), 256, 0, st>>>(n, x, num, target);
  g_launches++;
}

}  // namespace efe
