// Host set-up of the enriched finite-element discretisation (FP64, OpenMP).
//
// Paper references:
//   Sec. III.B  spectral elements: GLL nodes, GLL-lumped (diagonal) M^cc,
//               Gauss rule for every other integral;
//   Sec. IV.A   enrichment blocks M^ec, M^ee and the kinetic parts of H^ec, H^ee
//               (Eqs. Hec, Hee, Mec, Mee);
//   Sec. IV.B   compact support of the cut-off enrichment functions;
//   Sec. IV.C   adaptive divide-and-conquer quadrature on enriched cells;
//   Sec. IV.D   Schur complement S = M^ee - M^ec (M^cc)^-1 (M^ec)^T and S^-1.
// The V-dependent parts are built on the device (efe_set_potential).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "efe_func.h"
#include "efe_internal.h"

namespace efe {

namespace {

// Legendre P_n and P_{n-1} at x by the three-term recurrence.
void legendre_pair(int n, double x, double* pn, double* pn1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pn1 = p0;
}

// n-point Gauss-Legendre rule: Newton on P_n from the Chebyshev-like guesses.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double xi = -cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre_pair(n, xi, &pn, &pn1);
      double dp = n * (xi * pn - pn1) / (xi * xi - 1.0);
      double dx = pn / dp;
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double pn, pn1;
    legendre_pair(n, xi, &pn, &pn1);
    double dp = n * (xi * pn - pn1) / (xi * xi - 1.0);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

// n-point Gauss-Lobatto-Legendre rule (degree N = n-1): the points are the
// roots of x P_N(x) - P_{N-1}(x) (end points included), whose derivative is
// (N + 1) P_N(x); weights 2 / (N (N + 1) P_N(x)^2).
void gauss_lobatto(int n, double* x, double* w) {
  const int N = n - 1;
  for (int i = 0; i < n; ++i) {
    double xi = -cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre_pair(N, xi, &pn, &pn1);
      double dx = (xi * pn - pn1) / ((N + 1.0) * pn);
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double pn, pn1;
    legendre_pair(N, xi, &pn, &pn1);
    x[i] = xi;
    w[i] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
}

// Lagrange polynomials through the GLL nodes and their derivatives at xi.
void lagrange(const double* z, double xi, double* l, double* dl) {
  for (int a = 0; a < NP1; ++a) {
    double v = 1.0, d = 0.0;
    for (int b = 0; b < NP1; ++b) {
      if (b == a) continue;
      double f = (xi - z[b]) / (z[a] - z[b]);
      // product rule, accumulated: d(v f) = dv f + v df
      d = d * f + v / (z[a] - z[b]);
      v *= f;
    }
    l[a] = v;
    if (dl) dl[a] = d;
  }
}

struct Box {
  double lo[3], hi[3];
};

struct TrialCtx {
  const Setup* s;
  const int32_t* fl;
  int k;
  int n;
  const double* gx;
  const double* gw;
};

// Tensor Gauss rule on a box, x fastest: points (x, y, z, w).
void gauss_box(const Box& b, int n, const double* gx, const double* gw, std::vector<double>& out) {
  double half[3], hw[3];
  for (int d = 0; d < 3; ++d) {
    half[d] = 0.5 * (b.hi[d] - b.lo[d]);
    hw[d] = half[d];
  }
  for (int iz = 0; iz < n; ++iz)
    for (int iy = 0; iy < n; ++iy)
      for (int ix = 0; ix < n; ++ix) {
        out.push_back(b.lo[0] + half[0] * (gx[ix] + 1.0));
        out.push_back(b.lo[1] + half[1] * (gx[iy] + 1.0));
        out.push_back(b.lo[2] + half[2] * (gx[iz] + 1.0));
        out.push_back(hw[0] * gw[ix] * hw[1] * gw[iy] * hw[2] * gw[iz]);
      }
}

// Integrals of the trial functions f3 = sum N^2, f4 = sum |grad N|^2 and
// f5 = (sum_I Z_I / |x - R_I|) f3 over the points of a rule.
void trial_integrals(const TrialCtx& c, const double* pts, size_t np, double I[3]) {
  I[0] = I[1] = I[2] = 0.0;
  const Setup& s = *c.s;
  const int na = (int)s.atom_Z.size();
  constexpr int L = 8;   // points per pass of the nuclear sum (independent lanes, each in atom order)
  for (size_t q0 = 0; q0 < np; q0 += L) {
    const int nl = (int)std::min<size_t>(L, np - q0);
    double px[L], py[L], pz[L], vn[L];
    for (int t = 0; t < L; ++t) {
      const double* p = pts + 4 * (q0 + std::min(t, nl - 1));
      px[t] = p[0];
      py[t] = p[1];
      pz[t] = p[2];
      vn[t] = 0.0;
    }
    for (int a = 0; a < na; ++a) {
      const double ax = s.atom_xyz[3 * a], ay = s.atom_xyz[3 * a + 1], az = s.atom_xyz[3 * a + 2], Za = s.atom_Z[a];
      for (int t = 0; t < L; ++t) {
        const double dx = px[t] - ax, dy = py[t] - ay, dz = pz[t] - az;
        vn[t] += Za / sqrt(dx * dx + dy * dy + dz * dz);
      }
    }
    for (int t = 0; t < nl; ++t) {
      const double* p = pts + 4 * (q0 + t);
      double f3 = 0.0, f4 = 0.0;
      for (int i = 0; i < c.k; ++i) {
        double v, g[3];
        eval_func(s.funcs[c.fl[i]], p[0], p[1], p[2], &v, g);
        f3 += v * v;
        f4 += g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      }
      I[0] += p[3] * f3;
      I[1] += p[3] * f4;
      I[2] += p[3] * vn[t] * f3;
    }
  }
}

// Sec. IV.C: append the parent's Gauss points if |I^p - sum I^c| < tau for every
// trial function (or at the depth cap), otherwise recurse into the 8 children
// (child c = cx + 2 cy + 4 cz).
void push_box(const Box& b, std::vector<double>& boxes) {
  for (int d = 0; d < 3; ++d) boxes.push_back(b.lo[d]);
  for (int d = 0; d < 3; ++d) boxes.push_back(b.hi[d]);
}

// Ip_known: the trial integrals over this box's own points when the caller
// already formed them (a child's integrals of its parent's test), else NULL.
void adaptive(const TrialCtx& c, const Box& b, int depth, int max_depth, double tau,
              std::vector<double>& out, std::vector<double>& boxes, const double* Ip_known = nullptr) {
  std::vector<double> parent;
  gauss_box(b, c.n, c.gx, c.gw, parent);
  if (depth >= max_depth) {
    out.insert(out.end(), parent.begin(), parent.end());
    push_box(b, boxes);
    return;
  }
  double Ip[3];
  if (Ip_known) {
    for (int d = 0; d < 3; ++d) Ip[d] = Ip_known[d];
  } else {
    trial_integrals(c, parent.data(), parent.size() / 4, Ip);
  }
  double mid[3];
  for (int d = 0; d < 3; ++d) mid[d] = 0.5 * (b.lo[d] + b.hi[d]);
  Box kids[8];
  double Ic[3] = {0.0, 0.0, 0.0};
  double Ik_all[8][3];
  for (int k = 0; k < 8; ++k) {
    int bit[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    for (int d = 0; d < 3; ++d) {
      kids[k].lo[d] = bit[d] ? mid[d] : b.lo[d];
      kids[k].hi[d] = bit[d] ? b.hi[d] : mid[d];
    }
    std::vector<double> cp;
    gauss_box(kids[k], c.n, c.gx, c.gw, cp);
    double* Ik = Ik_all[k];
    trial_integrals(c, cp.data(), cp.size() / 4, Ik);
    for (int d = 0; d < 3; ++d) Ic[d] += Ik[d];
  }
  bool ok = true;
  for (int d = 0; d < 3; ++d) ok = ok && (fabs(Ip[d] - Ic[d]) < tau);
  if (ok) {
    out.insert(out.end(), parent.begin(), parent.end());
    push_box(b, boxes);
    return;
  }
  for (int k = 0; k < 8; ++k) adaptive(c, kids[k], depth + 1, max_depth, tau, out, boxes, Ik_all[k]);
}

}  // namespace

int host_cholesky_lower(double* A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return j + 1;
    d = sqrt(d);
    A[(size_t)j * n + j] = d;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = v / d;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[(size_t)i * n + j] = 0.0;
  return 0;
}

void host_spd_inverse_from_chol(const double* L, int n, double* inv) {
  // Linv by forward substitution, then inv = Linv^T Linv
  std::vector<double> Li((size_t)n * n, 0.0);
#pragma omp parallel for schedule(dynamic)
  for (int j = 0; j < n; ++j) {
    for (int i = j; i < n; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) v -= L[(size_t)i * n + k] * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = v / L[(size_t)i * n + i];
    }
  }
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double v = 0.0;
      for (int k = std::max(a, b); k < n; ++k) v += Li[(size_t)k * n + a] * Li[(size_t)k * n + b];
      inv[(size_t)a * n + b] = v;
    }
}

int build_setup(const efe_mesh_desc* mesh, const efe_atoms_desc* atoms, const efe_basis_desc* basis,
                Setup& s) {
  if (!mesh || !atoms || !basis) { s.err = "null descriptor"; return EFE_ERR_ARG; }
  if (mesh->degree != P) { s.err = "only degree 4 (HEX125SPEC) is supported"; return EFE_ERR_ARG; }
  if (mesh->n_gauss < 1 || mesh->n_gauss > 10) { s.err = "n_gauss out of range"; return EFE_ERR_ARG; }
  if (basis->n_funcs > 0 && (basis->quad_n < 1 || basis->quad_n > 10 || basis->quad_max_depth < 0 ||
                             basis->quad_max_depth > 16)) {
    s.err = "adaptive quadrature parameters out of range";
    return EFE_ERR_ARG;
  }
  s.ng = mesh->n_gauss;
  for (int d = 0; d < 3; ++d) {
    if (mesh->n_cells[d] < 1 || !mesh->breaks[d]) { s.err = "bad mesh axis"; return EFE_ERR_ARG; }
    s.nc[d] = mesh->n_cells[d];
    s.nn[d] = P * s.nc[d] + 1;
    s.brk[d].assign(mesh->breaks[d], mesh->breaks[d] + s.nc[d] + 1);
    for (int i = 0; i < s.nc[d]; ++i)
      if (!(s.brk[d][i + 1] > s.brk[d][i])) { s.err = "breaks must increase"; return EFE_ERR_ARG; }
  }
  s.n_nodes = (int64_t)s.nn[0] * s.nn[1] * s.nn[2];
  s.n_cell = (int64_t)s.nc[0] * s.nc[1] * s.nc[2];
  if (s.n_nodes >= (int64_t)1 << 31) { s.err = "too many nodes for 32-bit node ids"; return EFE_ERR_ARG; }
  const int na = atoms->n_atoms;
  s.atom_xyz.assign(atoms->xyz, atoms->xyz + 3 * na);
  s.atom_Z.assign(atoms->Z, atoms->Z + na);
  s.nE = basis->n_funcs;
  for (int i = 0; i < s.nE; ++i) {
    DevFunc f;
    const int a = basis->atom[i];
    if (a < 0 || a >= na) { s.err = "enrichment atom index out of range"; return EFE_ERR_ARG; }
    f.Rx = s.atom_xyz[3 * a];
    f.Ry = s.atom_xyz[3 * a + 1];
    f.Rz = s.atom_xyz[3 * a + 2];
    f.kind = basis->kind[i];
    f.n = basis->n[i];
    f.l = basis->l[i];
    f.m = basis->m[i];
    f.r0 = basis->r0[i];
    f.t = basis->t[i];
    if (!(f.r0 > 0.0) || !(f.t > 0.0) || f.l < 0 || f.l > 1 || f.m < -f.l || f.m > f.l) {
      s.err = "bad enrichment function parameters";
      return EFE_ERR_ARG;
    }
    if (f.kind == 0) {
      const double Z = s.atom_Z[a];
      f.zeta = Z;
      if (f.n == 1 && f.l == 0) f.norm = 2.0 * pow(Z, 1.5);
      else if (f.n == 2 && f.l == 0) f.norm = pow(Z, 1.5) / (2.0 * sqrt(2.0));
      else if (f.n == 2 && f.l == 1) f.norm = pow(Z, 2.5) / (2.0 * sqrt(6.0));
      else { s.err = "hydrogenic radial available for 1s, 2s, 2p only"; return EFE_ERR_ARG; }
    } else if (f.kind == 1) {
      f.zeta = basis->zeta[i];
      if (f.n - 1 - f.l < 0 || f.n > 4 || !(f.zeta > 0.0)) { s.err = "bad Slater radial"; return EFE_ERR_ARG; }
      double fact = 1.0;
      for (int k = 2; k <= 2 * f.n; ++k) fact *= k;
      f.norm = pow(2.0 * f.zeta, f.n + 0.5) / sqrt(fact);
    } else {
      s.err = "unknown radial kind";
      return EFE_ERR_ARG;
    }
    s.funcs.push_back(f);
  }

  // reference element: GLL nodes/weights, exact 1-D matrices by an 8-point Gauss rule
  gauss_lobatto(NP1, s.gll_z, s.gll_w);
  {
    double gx[8], gw[8];
    gauss_legendre(8, gx, gw);
    std::memset(s.M1, 0, sizeof(s.M1));
    std::memset(s.K1, 0, sizeof(s.K1));
    for (int q = 0; q < 8; ++q) {
      double l[NP1], dl[NP1];
      lagrange(s.gll_z, gx[q], l, dl);
      for (int a = 0; a < NP1; ++a)
        for (int b = 0; b < NP1; ++b) {
          s.M1[a * NP1 + b] += gw[q] * l[a] * l[b];
          s.K1[a * NP1 + b] += gw[q] * dl[a] * dl[b];
        }
    }
  }
  double gxo[16], gwo[16];
  gauss_legendre(s.ng, gxo, gwo);
  const int qn = basis->n_funcs > 0 ? basis->quad_n : 1;
  double gxa[16], gwa[16];
  gauss_legendre(qn, gxa, gwa);

  // cells meeting each support ball (distance from the centre to the box < r0 + r0/t)
  const int nx = s.nc[0], ny = s.nc[1], nz = s.nc[2];
  s.cell_enr.assign(s.n_cell, -1);
  std::vector<std::vector<int32_t>> cfl(s.n_cell);
  for (int fi = 0; fi < s.nE; ++fi) {
    const DevFunc& f = s.funcs[fi];
    const double rs = f.r0 + f.r0 / f.t;
    const double R[3] = {f.Rx, f.Ry, f.Rz};
    for (int64_t e = 0; e < s.n_cell; ++e) {
      int ijk[3] = {(int)(e % nx), (int)((e / nx) % ny), (int)(e / ((int64_t)nx * ny))};
      double d2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        double lo = s.brk[d][ijk[d]], hi = s.brk[d][ijk[d] + 1];
        double g = std::max(0.0, std::max(lo - R[d], R[d] - hi));
        d2 += g * g;
      }
      if (sqrt(d2) < rs) cfl[e].push_back(fi);
    }
  }
  s.cf_ptr.push_back(0);
  for (int64_t e = 0; e < s.n_cell; ++e) {
    if (cfl[e].empty()) continue;
    s.cell_enr[e] = (int32_t)s.enr_cells.size();
    s.enr_cells.push_back((int32_t)e);
    s.cf_idx.insert(s.cf_idx.end(), cfl[e].begin(), cfl[e].end());
    s.cf_ptr.push_back((int32_t)s.cf_idx.size());
  }
  const int64_t n_enr = (int64_t)s.enr_cells.size();

  // per-enriched-cell adaptive rule and overlap / kinetic blocks (parallel)
  std::vector<std::vector<double>> epts(n_enr), eboxes(n_enr);
  std::vector<std::vector<double>> bMec(n_enr), bHkin(n_enr), bMee(n_enr), bHkee(n_enr);
  int bad_alloc = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ei = 0; ei < n_enr; ++ei) {
    const int64_t e = s.enr_cells[ei];
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
    Box b;
    b.lo[0] = s.brk[0][i]; b.hi[0] = s.brk[0][i + 1];
    b.lo[1] = s.brk[1][j]; b.hi[1] = s.brk[1][j + 1];
    b.lo[2] = s.brk[2][k]; b.hi[2] = s.brk[2][k + 1];
    const int32_t* fl = s.cf_idx.data() + s.cf_ptr[ei];
    const int kf = s.cf_ptr[ei + 1] - s.cf_ptr[ei];
    TrialCtx c{&s, fl, kf, qn, gxa, gwa};
    try {
      adaptive(c, b, 0, basis->quad_max_depth, basis->quad_tau, epts[ei], eboxes[ei]);
      bMec[ei].assign((size_t)kf * NL, 0.0);
      bHkin[ei].assign((size_t)kf * NL, 0.0);
      bMee[ei].assign((size_t)kf * kf, 0.0);
      bHkee[ei].assign((size_t)kf * kf, 0.0);
    } catch (...) {
#pragma omp atomic write
      bad_alloc = 1;
      continue;
    }
    const double h[3] = {b.hi[0] - b.lo[0], b.hi[1] - b.lo[1], b.hi[2] - b.lo[2]};
    std::vector<double> E(kf), G(3 * kf);
    double Bv[NL], dB[3][NL];
    const size_t np = epts[ei].size() / 4;
    for (size_t q = 0; q < np; ++q) {
      const double* p = &epts[ei][4 * q];
      const double w = p[3];
      double l[3][NP1], dl[3][NP1];
      for (int d = 0; d < 3; ++d) {
        double xi = 2.0 * (p[d] - b.lo[d]) / h[d] - 1.0;
        lagrange(s.gll_z, xi, l[d], dl[d]);
        for (int a = 0; a < NP1; ++a) dl[d][a] *= 2.0 / h[d];
      }
      for (int cz = 0; cz < NP1; ++cz)
        for (int cy = 0; cy < NP1; ++cy)
          for (int cx = 0; cx < NP1; ++cx) {
            const int jl = cx + NP1 * (cy + NP1 * cz);
            Bv[jl] = l[0][cx] * l[1][cy] * l[2][cz];
            dB[0][jl] = dl[0][cx] * l[1][cy] * l[2][cz];
            dB[1][jl] = l[0][cx] * dl[1][cy] * l[2][cz];
            dB[2][jl] = l[0][cx] * l[1][cy] * dl[2][cz];
          }
      for (int a = 0; a < kf; ++a) eval_func(s.funcs[fl[a]], p[0], p[1], p[2], &E[a], &G[3 * a]);
      for (int a = 0; a < kf; ++a) {
        const double we = w * E[a];
        const double g0 = 0.5 * w * G[3 * a], g1 = 0.5 * w * G[3 * a + 1], g2 = 0.5 * w * G[3 * a + 2];
        double* rm = &bMec[ei][(size_t)a * NL];
        double* rk = &bHkin[ei][(size_t)a * NL];
        for (int jl = 0; jl < NL; ++jl) {
          rm[jl] += we * Bv[jl];
          rk[jl] += g0 * dB[0][jl] + g1 * dB[1][jl] + g2 * dB[2][jl];
        }
        for (int c2 = 0; c2 < kf; ++c2) {
          bMee[ei][(size_t)a * kf + c2] += we * E[c2];
          bHkee[ei][(size_t)a * kf + c2] +=
              g0 * G[3 * c2] + g1 * G[3 * c2 + 1] + g2 * G[3 * c2 + 2];
        }
      }
    }
  }
  if (bad_alloc) { s.err = "host allocation failed in adaptive quadrature"; return EFE_ERR_ALLOC; }

  // quadrature point table, cell by cell
  s.qoff.assign(s.n_cell + 1, 0);
  for (int64_t e = 0; e < s.n_cell; ++e) {
    int64_t nq = (s.cell_enr[e] >= 0) ? (int64_t)(epts[s.cell_enr[e]].size() / 4)
                                       : (int64_t)s.ng * s.ng * s.ng;
    s.qoff[e + 1] = s.qoff[e] + nq;
  }
  s.n_q = s.qoff[s.n_cell];
  s.qpts.assign((size_t)s.n_q * 4, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t e = 0; e < s.n_cell; ++e) {
    double* out = &s.qpts[(size_t)s.qoff[e] * 4];
    if (s.cell_enr[e] >= 0) {
      const auto& v = epts[s.cell_enr[e]];
      std::copy(v.begin(), v.end(), out);
    } else {
      const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
      Box b;
      b.lo[0] = s.brk[0][i]; b.hi[0] = s.brk[0][i + 1];
      b.lo[1] = s.brk[1][j]; b.hi[1] = s.brk[1][j + 1];
      b.lo[2] = s.brk[2][k]; b.hi[2] = s.brk[2][k + 1];
      std::vector<double> tmp;
      gauss_box(b, s.ng, gxo, gwo, tmp);
      std::copy(tmp.begin(), tmp.end(), out);
    }
  }
  epts.clear();
  epts.shrink_to_fit();

  // quadrature leaves: every rule above is a union of tensor Gauss boxes whose
  // points are stored contiguously, x fastest (an ordinary cell is one box)
  s.leaf_ptr.assign(s.n_cell + 1, 0);
  for (int64_t e = 0; e < s.n_cell; ++e)
    s.leaf_ptr[e + 1] = s.leaf_ptr[e] + (s.cell_enr[e] >= 0 ? (int64_t)(eboxes[s.cell_enr[e]].size() / 6) : 1);
  const int64_t n_leaf = s.leaf_ptr[s.n_cell];
  s.leaf_box.assign((size_t)n_leaf * 6, 0.0);
  s.leaf_off.assign(n_leaf + 1, 0);
  s.leaf_n.assign(n_leaf, 0);
  s.leaf_cell.assign(n_leaf, 0);
  for (int64_t e = 0; e < s.n_cell; ++e) {
    const int64_t l0 = s.leaf_ptr[e];
    if (s.cell_enr[e] >= 0) {
      const auto& bx = eboxes[s.cell_enr[e]];
      const int64_t nl = (int64_t)(bx.size() / 6);
      std::copy(bx.begin(), bx.end(), &s.leaf_box[(size_t)l0 * 6]);
      for (int64_t l = 0; l < nl; ++l) {
        s.leaf_n[l0 + l] = qn;
        s.leaf_cell[l0 + l] = (int32_t)e;
        s.leaf_off[l0 + l] = s.qoff[e] + l * (int64_t)qn * qn * qn;
      }
    } else {
      const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
      double* bx = &s.leaf_box[(size_t)l0 * 6];
      bx[0] = s.brk[0][i]; bx[1] = s.brk[1][j]; bx[2] = s.brk[2][k];
      bx[3] = s.brk[0][i + 1]; bx[4] = s.brk[1][j + 1]; bx[5] = s.brk[2][k + 1];
      s.leaf_n[l0] = s.ng;
      s.leaf_cell[l0] = (int32_t)e;
      s.leaf_off[l0] = s.qoff[e];
    }
  }
  s.leaf_off[n_leaf] = s.n_q;
  eboxes.clear();

  // GLL-diagonal overlap D (Sec. III.B); D^-1 zero on the Dirichlet faces
  const int NX = s.nn[0], NY = s.nn[1], NZ = s.nn[2];
  s.D.assign(s.n_nodes, 0.0);
  for (int64_t e = 0; e < s.n_cell; ++e) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
    const double vol8 = (s.brk[0][i + 1] - s.brk[0][i]) * (s.brk[1][j + 1] - s.brk[1][j]) *
                        (s.brk[2][k + 1] - s.brk[2][k]) / 8.0;
    for (int c = 0; c < NP1; ++c)
      for (int bb = 0; bb < NP1; ++bb)
        for (int a = 0; a < NP1; ++a) {
          int64_t g = (int64_t)(P * i + a) + NX * ((int64_t)(P * j + bb) + (int64_t)NY * (P * k + c));
          s.D[g] += s.gll_w[a] * s.gll_w[bb] * s.gll_w[c] * vol8;
        }
  }
  s.Dinv.assign(s.n_nodes, 0.0);
  for (int64_t g = 0; g < s.n_nodes; ++g) {
    const int ix = (int)(g % NX), iy = (int)((g / NX) % NY), iz = (int)(g / ((int64_t)NX * NY));
    const bool bnd = ix == 0 || iy == 0 || iz == 0 || ix == NX - 1 || iy == NY - 1 || iz == NZ - 1;
    s.Dinv[g] = bnd ? 0.0 : 1.0 / s.D[g];
  }

  // block storage offsets
  s.blkP_off.assign(n_enr + 1, 0);
  s.blkQ_off.assign(n_enr + 1, 0);
  for (int64_t ei = 0; ei < n_enr; ++ei) {
    const int64_t kf = s.cf_ptr[ei + 1] - s.cf_ptr[ei];
    s.blkP_off[ei + 1] = s.blkP_off[ei] + kf * NL;
    s.blkQ_off[ei + 1] = s.blkQ_off[ei] + kf * kf;
  }

  // M^ec / H^ec row pattern (rows = functions) with assembly contributions
  const int nE = s.nE;
  std::vector<std::vector<std::pair<int32_t, int64_t>>> rows(nE);
  for (int64_t ei = 0; ei < n_enr; ++ei) {
    const int64_t e = s.enr_cells[ei];
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
    const int kf = s.cf_ptr[ei + 1] - s.cf_ptr[ei];
    for (int a = 0; a < kf; ++a) {
      const int fi = s.cf_idx[s.cf_ptr[ei] + a];
      for (int c = 0; c < NP1; ++c)
        for (int bb = 0; bb < NP1; ++bb)
          for (int aa = 0; aa < NP1; ++aa) {
            const int jl = aa + NP1 * (bb + NP1 * c);
            int64_t g = (int64_t)(P * i + aa) + NX * ((int64_t)(P * j + bb) + (int64_t)NY * (P * k + c));
            rows[fi].push_back({(int32_t)g, s.blkP_off[ei] + (int64_t)a * NL + jl});
          }
    }
  }
  s.ec_ptr.assign(nE + 1, 0);
  s.ec_contrib_ptr.assign(1, 0);
  for (int fi = 0; fi < nE; ++fi) {
    auto& r = rows[fi];
    std::sort(r.begin(), r.end());
    size_t q = 0;
    while (q < r.size()) {
      const int32_t g = r[q].first;
      double mv = 0.0, hv = 0.0;
      while (q < r.size() && r[q].first == g) {
        const int64_t pos = r[q].second;
        const int64_t ei = std::upper_bound(s.blkP_off.begin(), s.blkP_off.end(), pos) - s.blkP_off.begin() - 1;
        const int64_t off = pos - s.blkP_off[ei];
        mv += bMec[ei][off];
        hv += bHkin[ei][off];
        s.ec_contrib_idx.push_back(pos);
        ++q;
      }
      s.ec_col.push_back(g);
      s.mec_val.push_back(mv);
      s.hec_kin.push_back(hv);
      s.ec_contrib_ptr.push_back((int64_t)s.ec_contrib_idx.size());
    }
    s.ec_ptr[fi + 1] = (int64_t)s.ec_col.size();
    r.clear();
    r.shrink_to_fit();
  }
  // transposed pattern over nodes
  {
    const int64_t nnz = (int64_t)s.ec_col.size();
    std::vector<std::pair<int32_t, int64_t>> tv(nnz);
    for (int fi = 0; fi < nE; ++fi)
      for (int64_t q = s.ec_ptr[fi]; q < s.ec_ptr[fi + 1]; ++q) tv[q] = {s.ec_col[q], q};
    std::stable_sort(tv.begin(), tv.end(),
                     [](const std::pair<int32_t, int64_t>& x, const std::pair<int32_t, int64_t>& y) {
                       return x.first < y.first;
                     });
    s.t_ptr.assign(1, 0);
    for (int64_t q = 0; q < nnz; ++q) {
      if (q == 0 || tv[q].first != tv[q - 1].first) {
        if (q > 0) s.t_ptr.push_back(q);
        s.t_nodes.push_back(tv[q].first);
      }
      const int64_t pos = tv[q].second;
      const int fi = (int)(std::upper_bound(s.ec_ptr.begin(), s.ec_ptr.end(), pos) - s.ec_ptr.begin() - 1);
      s.t_col.push_back(fi);
      s.t_perm.push_back(pos);
    }
    if (nnz > 0) s.t_ptr.push_back(nnz);
  }
  // M^ee, kinetic H^ee, and the H^ee assembly contributions
  s.Mee.assign((size_t)nE * nE, 0.0);
  s.Hee_kin.assign((size_t)nE * nE, 0.0);
  {
    std::vector<int64_t> cnt((size_t)nE * nE + 1, 0);
    for (int64_t ei = 0; ei < n_enr; ++ei) {
      const int kf = s.cf_ptr[ei + 1] - s.cf_ptr[ei];
      const int32_t* fl = s.cf_idx.data() + s.cf_ptr[ei];
      for (int a = 0; a < kf; ++a)
        for (int c = 0; c < kf; ++c) {
          const size_t ent = (size_t)fl[a] * nE + fl[c];
          s.Mee[ent] += bMee[ei][(size_t)a * kf + c];
          s.Hee_kin[ent] += bHkee[ei][(size_t)a * kf + c];
          cnt[ent + 1]++;
        }
    }
    for (size_t q = 0; q < (size_t)nE * nE; ++q) cnt[q + 1] += cnt[q];
    s.ee_contrib_ptr = cnt;
    s.ee_contrib_idx.assign(cnt[(size_t)nE * nE], 0);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t ei = 0; ei < n_enr; ++ei) {
      const int kf = s.cf_ptr[ei + 1] - s.cf_ptr[ei];
      const int32_t* fl = s.cf_idx.data() + s.cf_ptr[ei];
      for (int a = 0; a < kf; ++a)
        for (int c = 0; c < kf; ++c) {
          const size_t ent = (size_t)fl[a] * nE + fl[c];
          s.ee_contrib_idx[fill[ent]++] = s.blkQ_off[ei] + (int64_t)a * kf + c;
        }
    }
  }
  bMec.clear(); bHkin.clear(); bMee.clear(); bHkee.clear();

  // Schur complement and its inverse (Sec. IV.D)
  if (nE > 0) {
    std::vector<int32_t> node2t(s.n_nodes, -1);
    for (size_t r = 0; r < s.t_nodes.size(); ++r) node2t[s.t_nodes[r]] = (int32_t)r;
    s.S.assign((size_t)nE * nE, 0.0);
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < nE; ++a) {
      std::vector<double> row(nE, 0.0);
      for (int64_t q = s.ec_ptr[a]; q < s.ec_ptr[a + 1]; ++q) {
        const int32_t g = s.ec_col[q];
        const double v = s.mec_val[q] * s.Dinv[g];
        if (v == 0.0) continue;
        const int32_t tr = node2t[g];
        for (int64_t u = s.t_ptr[tr]; u < s.t_ptr[tr + 1]; ++u) row[s.t_col[u]] += v * s.mec_val[s.t_perm[u]];
      }
      for (int c = 0; c < nE; ++c) s.S[(size_t)a * nE + c] = s.Mee[(size_t)a * nE + c] - row[c];
    }
    for (int a = 0; a < nE; ++a)
      for (int c = a + 1; c < nE; ++c) {
        double v = 0.5 * (s.S[(size_t)a * nE + c] + s.S[(size_t)c * nE + a]);
        s.S[(size_t)a * nE + c] = s.S[(size_t)c * nE + a] = v;
      }
    std::vector<double> L = s.S;
    int info = host_cholesky_lower(L.data(), nE);
    if (info) {
      s.err = "Schur complement S is not positive definite (ill-conditioned enriched basis)";
      return EFE_ERR_CHOL;
    }
    s.Sinv.assign((size_t)nE * nE, 0.0);
    host_spd_inverse_from_chol(L.data(), nE, s.Sinv.data());
  }
  return EFE_OK;
}

}  // namespace efe
