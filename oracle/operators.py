"""Enriched finite-element operators -- oracle (test infrastructure only).

Builds, for a workload description from ``workloads``, every matrix of the
paper's discrete problem in plain FP64:

* Sec. III.A, Eq. Hjk / Eq. Hcc: per-cell classical Hamiltonian
  H^cc_e = 1/2 int grad N_j . grad N_k + int V N_j N_k (Gauss rule, adaptive rule
  in enriched cells); homogeneous Dirichlet on the box faces (boundary rows are
  kept as rows that stay zero).
* Sec. III.B: M^cc from the GLL rule, i.e. diagonal, D_j = sum_e w_a w_b w_c |J_e|.
* Sec. IV.A, Eqs. Hec, Hee, Mec, Mee: enrichment-classical and
  enrichment-enrichment blocks, integrated with the adaptive rule (Sec. IV.C).
* Sec. IV.D: the Schur complement S = M^ee - M^ec (M^cc)^-1 (M^ec)^T and the
  block-wise (Banachiewicz) inverse of M^E applied matrix-free.
* Sec. V (last paragraph): the elemental mat-vec, cell product then assembly.

Pins: tests/test_oracle_operators.py (GLL-lumped mass sums to the box volume,
kinetic block annihilates constants / reproduces the exact gradient energy of
polynomials, elemental apply equals the assembled sparse product, block-wise
inverse equals the dense inverse of the assembled M^E, S is SPD) and the
closed-form spectra in tests/test_oracle_chfsi.py.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .quadrature import gll_rule, gauss_rule, lagrange_values, lagrange_derivs, exact_1d_matrices
from .enrichment import eval_all, support_radius
from .adaptive import adaptive_rule, gauss_box


def potential(system, pts):
    """V(x) = -sum_I Z_I/|x-R_I| + sum_g A_g exp(-|x-c_g|^2 / (2 s_g^2)) + omega^2 |x|^2 / 2.

    Eq. vext for the nuclear term; the Gaussian sum and the harmonic term are
    the workloads' synthetic smooth parts."""
    pot = system["potential"]
    V = np.zeros(pts.shape[0])
    if pot["nuclear"]:
        for R, Z in zip(system["atoms"], system["Z"]):
            V -= Z / np.sqrt(np.sum((pts - R[None, :]) ** 2, axis=1))
    for A, s, c in zip(pot["gauss_A"], pot["gauss_s"], pot["gauss_c"]):
        V += A * np.exp(-np.sum((pts - c[None, :]) ** 2, axis=1) / (2.0 * s * s))
    if pot["omega"] != 0.0:
        V += 0.5 * pot["omega"] ** 2 * np.sum(pts * pts, axis=1)
    return V


class Discretisation:
    """All cells, node maps, quadrature lists and operator blocks of one system."""

    def __init__(self, system, build_matrices=True):
        self.system = system
        p = system["p"]
        self.p = p
        self.nl = (p + 1) ** 3
        self.z, self.wgll = gll_rule(p + 1)
        self.M1, self.K1 = exact_1d_matrices(self.z)
        self.breaks = system["breaks"]
        self.ncell_ax = [len(b) - 1 for b in self.breaks]
        self.nnode_ax = [p * n + 1 for n in self.ncell_ax]
        self.n_nodes = int(np.prod(self.nnode_ax))
        self.nE = len(system["funcs"])
        nx, ny, nz = self.ncell_ax
        NX, NY, _ = self.nnode_ax
        self.n_cell = nx * ny * nz
        # cell ordering e = i + nx*(j + ny*k); local node a + (p+1)(b + (p+1)c)
        self.cell_ijk = np.array([(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)])
        loc = np.array([(a, b, c) for c in range(p + 1) for b in range(p + 1) for a in range(p + 1)])
        gi = p * self.cell_ijk[:, None, 0] + loc[None, :, 0]
        gj = p * self.cell_ijk[:, None, 1] + loc[None, :, 1]
        gk = p * self.cell_ijk[:, None, 2] + loc[None, :, 2]
        self.cell_nodes = gi + NX * (gj + NY * gk)
        self.lo = np.stack([self.breaks[d][self.cell_ijk[:, d]] for d in range(3)], axis=1)
        self.hi = np.stack([self.breaks[d][self.cell_ijk[:, d] + 1] for d in range(3)], axis=1)
        self.h = self.hi - self.lo
        # boundary mask
        ix = np.arange(NX)
        iy = np.arange(NY)
        iz = np.arange(self.nnode_ax[2])
        bm = ((iz == 0) | (iz == self.nnode_ax[2] - 1))[:, None, None] | \
             ((iy == 0) | (iy == NY - 1))[None, :, None] | ((ix == 0) | (ix == NX - 1))[None, None, :]
        self.boundary = bm.reshape(-1)
        self.interior = ~self.boundary
        self._cell_funcs()
        self._diag_mass()
        if build_matrices:
            self.build()

    # -- geometry ------------------------------------------------------------
    def _cell_funcs(self):
        """Functions whose support ball meets each cell (Sec. IV.B locality)."""
        sysd = self.system
        self.funcs_of_cell = [[] for _ in range(self.n_cell)]
        for fi, f in enumerate(sysd["funcs"]):
            R = sysd["atoms"][f["atom"]]
            rs = support_radius(f)
            d = np.maximum(0.0, np.maximum(self.lo - R[None, :], R[None, :] - self.hi))
            dist = np.sqrt(np.sum(d * d, axis=1))
            for e in np.nonzero(dist < rs)[0]:
                self.funcs_of_cell[e].append(fi)
        self.enriched = np.array([len(f) > 0 for f in self.funcs_of_cell])

    def _diag_mass(self):
        """D = diag(M^cc) from the GLL rule (Sec. III.B)."""
        w = self.wgll
        w3 = (w[None, None, :] * w[None, :, None] * w[:, None, None]).reshape(-1)  # index a fastest
        D = np.zeros(self.n_nodes)
        for e in range(self.n_cell):
            D[self.cell_nodes[e]] += w3 * np.prod(self.h[e]) / 8.0
        self.D = D
        self.Dinv = np.where(self.interior, 1.0 / D, 0.0)

    def cell_quadrature(self, e):
        """Gauss tensor rule, or the adaptive rule in enriched cells (Sec. IV.C).
        Rules depend on the mesh and basis only and are cached."""
        cache = self.__dict__.setdefault("_quad", {})
        if e not in cache:
            if self.enriched[e]:
                q = self.system["quad"]
                cache[e] = adaptive_rule(self.system, self.lo[e], self.hi[e], self.funcs_of_cell[e],
                                         q["tau"], q["max_depth"], q["n"])
            else:
                cache[e] = gauss_box(self.lo[e], self.hi[e], self.system["n_gauss"])
        return cache[e]

    def basis_at(self, e, pts):
        """Classical basis values B (npt, 125) and physical gradients dB (npt, 125, 3)."""
        xi = 2.0 * (pts - self.lo[e][None, :]) / self.h[e][None, :] - 1.0
        L = [lagrange_values(self.z, xi[:, d]) for d in range(3)]
        dL = [lagrange_derivs(self.z, xi[:, d]) * (2.0 / self.h[e][d]) for d in range(3)]
        n1 = self.p + 1
        B = (L[2][:, :, None, None] * L[1][:, None, :, None] * L[0][:, None, None, :]).reshape(-1, n1 ** 3)
        gx = (L[2][:, :, None, None] * L[1][:, None, :, None] * dL[0][:, None, None, :]).reshape(-1, n1 ** 3)
        gy = (L[2][:, :, None, None] * dL[1][:, None, :, None] * L[0][:, None, None, :]).reshape(-1, n1 ** 3)
        gz = (dL[2][:, :, None, None] * L[1][:, None, :, None] * L[0][:, None, None, :]).reshape(-1, n1 ** 3)
        return B, np.stack([gx, gy, gz], axis=2)

    def kinetic_cell(self, e):
        """1/2 int grad N_j . grad N_k on an axis-aligned cell, exact (Eq. Hcc, first term).

        int dN/dx dN/dx = (hy hz / (2 hx)) K1 (x) M1 (x) M1, and cyclically."""
        hx, hy, hz = self.h[e]
        M1, K1 = self.M1, self.K1
        T = (hy * hz / (2.0 * hx)) * np.kron(M1, np.kron(M1, K1)) \
            + (hx * hz / (2.0 * hy)) * np.kron(M1, np.kron(K1, M1)) \
            + (hx * hy / (2.0 * hz)) * np.kron(K1, np.kron(M1, M1))
        return 0.5 * T

    # -- operator blocks ---------------------------------------------------------
    def build(self, V=None, Vq=None):
        """Per-cell H^cc_e, per-enriched-cell H^ec_e and M^ec_e, global H^ee and M^ee.

        ``V`` is an optional callable V(points); ``Vq`` optional values at every
        quadrature point in cell order; default is the workload's analytic potential."""
        if Vq is not None:
            offs = np.cumsum([0] + [len(self.cell_quadrature(e)[1]) for e in range(self.n_cell)])
            Vq = np.asarray(Vq, dtype=np.float64)
        Vf = V if V is not None else (lambda pts: potential(self.system, pts))
        self.Hcc = np.zeros((self.n_cell, self.nl, self.nl))
        self.Hec = {}
        self.Mec = {}
        self.Hee = np.zeros((self.nE, self.nE))
        self.Mee = np.zeros((self.nE, self.nE))
        self.nq = np.zeros(self.n_cell, dtype=np.int64)
        for e in range(self.n_cell):
            pts, w = self.cell_quadrature(e)
            self.nq[e] = len(w)
            B, dB = self.basis_at(e, pts)
            wV = w * (Vq[offs[e]:offs[e + 1]] if Vq is not None else Vf(pts))
            self.Hcc[e] = self.kinetic_cell(e) + B.T @ (wV[:, None] * B)
            fl = self.funcs_of_cell[e]
            if fl:
                E, G = eval_all(self.system, pts, fl)
                self.Mec[e] = E.T @ (w[:, None] * B)
                kin = sum(G[:, :, d].T @ (w[:, None] * dB[:, :, d]) for d in range(3))
                self.Hec[e] = 0.5 * kin + E.T @ (wV[:, None] * B)
                kin_ee = sum(G[:, :, d].T @ (w[:, None] * G[:, :, d]) for d in range(3))
                idx = np.array(fl)
                self.Mee[np.ix_(idx, idx)] += E.T @ (w[:, None] * E)
                self.Hee[np.ix_(idx, idx)] += 0.5 * kin_ee + E.T @ (wV[:, None] * E)
        self._assemble()
        self._schur()

    def _assemble(self):
        """Global sparse H^E and M^E over [all nodes; enrichment] (Eqs. H2x2, M2x2)."""
        nn, nE = self.n_nodes, self.nE
        rows, cols, hv = [], [], []
        for e in range(self.n_cell):
            cn = self.cell_nodes[e]
            rows.append(np.repeat(cn, self.nl))
            cols.append(np.tile(cn, self.nl))
            hv.append(self.Hcc[e].ravel())
        mr, mc, mv = [np.arange(nn)], [np.arange(nn)], [self.D]
        for e, blk in self.Hec.items():
            fl = np.array(self.funcs_of_cell[e]) + nn
            cn = self.cell_nodes[e]
            r = np.repeat(fl, self.nl)
            c = np.tile(cn, len(fl))
            rows += [r, c]
            cols += [c, r]
            hv += [blk.ravel(), blk.ravel()]
            mb = self.Mec[e]
            mr += [r, c]
            mc += [c, r]
            mv += [mb.ravel(), mb.ravel()]
        ee_r, ee_c = np.meshgrid(np.arange(nE) + nn, np.arange(nE) + nn, indexing="ij")
        rows.append(ee_r.ravel())
        cols.append(ee_c.ravel())
        hv.append(self.Hee.ravel())
        mr.append(ee_r.ravel())
        mc.append(ee_c.ravel())
        mv.append(self.Mee.ravel())
        n = nn + nE
        self.H = sp.coo_matrix((np.concatenate(hv), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(n, n)).tocsr()
        self.M = sp.coo_matrix((np.concatenate(mv), (np.concatenate(mr), np.concatenate(mc))),
                               shape=(n, n)).tocsr()
        # M^ec as its own sparse block (nE x n_nodes)
        self.Mec_global = self.M[nn:, :nn].tocsr()
        self.Hec_global = self.H[nn:, :nn].tocsr()
        self.active = np.concatenate([self.interior, np.ones(nE, dtype=bool)])

    def _schur(self):
        """S = M^ee - M^ec (M^cc)^-1 (M^ec)^T over the interior nodes (Sec. IV.D)."""
        if self.nE == 0:
            self.S = np.zeros((0, 0))
            self.S_chol = None
            return
        L = self.Mec_global @ sp.diags(self.Dinv)
        self.L = L.tocsr()
        self.S = self.Mee - (self.L @ self.Mec_global.T).toarray()
        self.S = 0.5 * (self.S + self.S.T)
        self.S_chol = sla.cho_factor(self.S, lower=True)

    # -- products -----------------------------------------------------------------
    def restrict(self, Y):
        Y = np.array(Y, copy=True)
        Y[:self.n_nodes][self.boundary] = 0.0
        return Y

    def apply_H_assembled(self, X):
        return self.restrict(self.H @ X)

    def apply_M_assembled(self, X):
        return self.restrict(self.M @ X)

    def apply_H_elemental(self, X):
        """H^E X by cell products then assembly (Sec. V, last paragraph)."""
        nn = self.n_nodes
        Xc, Xe = X[:nn], X[nn:]
        W = np.zeros_like(X)
        Wc, We = W[:nn], W[nn:]
        for e in range(self.n_cell):
            cn = self.cell_nodes[e]
            Wc[cn] += self.Hcc[e] @ Xc[cn]
            if e in self.Hec:
                fl = self.funcs_of_cell[e]
                Wc[cn] += self.Hec[e].T @ Xe[fl]
                We[fl] += self.Hec[e] @ Xc[cn]
        We += self.Hee @ Xe
        return self.restrict(W)

    def apply_Minv_block(self, W):
        """(M^E)^-1 W by the Banachiewicz block formula of Sec. IV.D, never formed:

            x_c = (D^-1 + L^T S^-1 L) W_c - L^T S^-1 W_e
            x_e = -S^-1 L W_c + S^-1 W_e,      L = M^ec D^-1."""
        nn = self.n_nodes
        Wc, We = W[:nn], W[nn:]
        Dinv = self.Dinv[:, None] if W.ndim == 2 else self.Dinv
        if self.nE == 0:
            return np.concatenate([Dinv * Wc, We])
        LW = self.L @ Wc
        SinvLW = sla.cho_solve(self.S_chol, LW)
        SinvWe = sla.cho_solve(self.S_chol, We)
        xc = Dinv * Wc + self.L.T @ SinvLW - self.L.T @ SinvWe
        xe = -SinvLW + SinvWe
        return np.concatenate([xc, xe])

    def apply_Htilde(self, X, elemental=True):
        """H~ X = (M^E)^-1 H^E X (Eq. SEPEFEM)."""
        HX = self.apply_H_elemental(X) if elemental else self.apply_H_assembled(X)
        return self.apply_Minv_block(HX)

    def dense_active(self):
        """Dense H^E, M^E restricted to interior nodes + enrichment rows."""
        a = np.nonzero(self.active)[0]
        return self.H[a][:, a].toarray(), self.M[a][:, a].toarray(), a
