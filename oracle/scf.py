"""Self-consistent field pieces -- oracle (test infrastructure only).

Paper, Sec. II: V_eff = V_xc + V_H + V_ext (Eq. veff); the Hartree potential
solves -lap V_H / (4 pi) = rho (Eq. Poisson), discretised with the classical
FE basis (Sec. III.A, A^C Phi = b^C with A_jk = (1/4pi) int grad N_j . grad N_k
and b_j = int rho N_j); rho = 2 sum_i f(eps_i, mu) |psi_i|^2 (Eq. Rho) with
Fermi-Dirac occupations (Eq. FermiDirac) and the electron-count constraint
(Eq. Mu); total energy E_tot = E_band + E_xc - int V_xc rho - 1/2 int rho V_H
+ E_ZZ.  Sec. V: SCF loop rho_in -> V_eff -> eigenpairs -> rho_out -> mixing;
Sec. VI: n-stage Anderson mixing, T = 500 K.

Readings (the paper is silent on these; listed in the design notes):
* LDA: Ceperley-Alder correlation in the Perdew-Zunger (1981) parametrisation,
  spin-unpolarised, with Slater exchange; constants from that published
  article (not in the paper).
* Dirichlet data of the Hartree problem: monopole + dipole of rho about its
  centre of charge, evaluated at the boundary nodes.
* Energy of a non-self-consistent pair (rho_in, rho_out): the Kohn-Sham
  functional at rho_out, E_band - int rho_out (V_H[rho_in] + V_xc[rho_in])
  + E_H[rho_out] + E_xc[rho_out] + E_ZZ, which equals the paper's expression
  at self-consistency.
* Anderson mixing on rho at the quadrature points, weighted L2 inner product.

Pins (tests/test_oracle_scf.py): sum_i 2 f_i = N_e; exchange energy per
electron of the uniform gas -0.458165 / r_s (independent constant route);
continuity of the PZ81 correlation at r_s = 1 (the parametrisation's own
matching condition) and V_xc = d(rho eps_xc)/d rho by finite differences;
FE Hartree potential and energy of a Gaussian charge (Q erf(r/(sqrt2 sigma))/r,
Q^2/(2 sqrt(pi) sigma)) and of the hydrogen 1s density (1/r - (1 + 1/r)
exp(-2r), 5/16) with their convergence under refinement; E_ZZ closed form;
Anderson mixing reduces to linear mixing for one stage and lands on the fixed
point of a linear map; the whole SCF for the LDA hydrogen atom against an
independent radial solver (total energy and 1s eigenvalue within 1 mHa).
LDA correlation beyond these identities: parity unpinned (no tabulated values).
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as ssl

from .enrichment import eval_all

KB_HA_PER_K = 3.166811563e-6   # Boltzmann constant (Ha/K)


# ---------------------------------------------------------------------- occupations
def fermi_occupations(eps, n_electrons, kT, tol=1e-14):
    """f_i of Eq. FermiDirac with mu from 2 sum_i f_i = N_e (Eq. Mu), by bisection."""
    eps = np.asarray(eps, dtype=np.float64)

    def count(mu):
        x = np.clip((eps - mu) / kT, -700.0, 700.0)
        return 2.0 * np.sum(1.0 / (1.0 + np.exp(x)))

    lo, hi = eps.min() - 50.0 * kT - 1.0, eps.max() + 50.0 * kT + 1.0
    if count(hi) < n_electrons:
        raise ValueError("not enough states for the electron count")
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    mu = 0.5 * (lo + hi)
    x = np.clip((eps - mu) / kT, -700.0, 700.0)
    return 1.0 / (1.0 + np.exp(x)), mu


# ---------------------------------------------------------------------- LDA
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_exchange(rho):
    """Slater exchange of the uniform gas: eps_x = -(3/4)(3 rho/pi)^(1/3), v_x = 4/3 eps_x."""
    rho = np.maximum(np.asarray(rho, dtype=np.float64), 1e-30)
    ex = -(3.0 / 4.0) * (3.0 * rho / math.pi) ** (1.0 / 3.0)
    return ex, (4.0 / 3.0) * ex


def lda_correlation(rho):
    """Perdew-Zunger parametrisation of the Ceperley-Alder correlation energy per
    electron and its potential (spin-unpolarised)."""
    rho = np.maximum(np.asarray(rho, dtype=np.float64), 1e-30)
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    ec = np.empty_like(rho)
    vc = np.empty_like(rho)
    hi = rs >= 1.0
    r = rs[hi]
    sq = np.sqrt(r)
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * r
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + (7.0 / 6.0) * PZ_BETA1 * sq + (4.0 / 3.0) * PZ_BETA2 * r) / den
    r = rs[~hi]
    lr = np.log(r)
    ec[~hi] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[~hi] = (PZ_A * lr + (PZ_B - PZ_A / 3.0) + (2.0 / 3.0) * PZ_C * r * lr
               + ((2.0 * PZ_D - PZ_C) / 3.0) * r)
    return ec, vc


def lda_pz81(rho):
    """eps_xc (energy per electron) and v_xc = d(rho eps_xc)/d rho, spin-unpolarised LDA."""
    ex, vx = lda_exchange(rho)
    ec, vc = lda_correlation(rho)
    return ex + ec, vx + vc


# ---------------------------------------------------------------------- quadrature cache
class QuadCache:
    """Per-cell quadrature points, weights, classical basis values and enrichment
    values of a Discretisation (the same rules the operators use)."""

    def __init__(self, disc):
        self.disc = disc
        self.pts, self.w, self.off = [], [], [0]
        for e in range(disc.n_cell):
            p, w = disc.cell_quadrature(e)
            self.pts.append(p)
            self.w.append(w)
            self.off.append(self.off[-1] + len(w))
        self.all_pts = np.concatenate(self.pts)
        self.all_w = np.concatenate(self.w)

    def psi_values(self, e, X):
        """Orbital values at the quadrature points of cell e: B X_c + E X_e."""
        d = self.disc
        B, _ = d.basis_at(e, self.pts[e])
        vals = B @ X[d.cell_nodes[e]]
        fl = d.funcs_of_cell[e]
        if fl:
            E, _ = eval_all(d.system, self.pts[e], fl)
            vals = vals + E @ X[d.n_nodes + np.array(fl)]
        return vals


def density(qc, X, f):
    """rho at every quadrature point, cell by cell: 2 sum_i f_i psi_i(x)^2 (Eq. Rho)."""
    out = np.empty(len(qc.all_w))
    for e in range(qc.disc.n_cell):
        psi = qc.psi_values(e, X)
        out[qc.off[e]:qc.off[e + 1]] = 2.0 * (psi * psi) @ f
    return out


# ---------------------------------------------------------------------- Hartree
def hartree(qc, rho):
    """FE solution of -lap V_H / (4 pi) = rho with multipole Dirichlet data.

    Returns (V_H at the quadrature points, nodal potential)."""
    d = qc.disc
    w = qc.all_w
    Q = np.sum(w * rho)
    centre = (w * rho) @ qc.all_pts / Q if abs(Q) > 1e-300 else np.zeros(3)
    dip = (w * rho) @ (qc.all_pts - centre[None, :])
    # stiffness A = (1/4pi) int grad N_j . grad N_k  (= 2 x kinetic block / 4pi), load b_j = int rho N_j
    rows, cols, vals = [], [], []
    b = np.zeros(d.n_nodes)
    for e in range(d.n_cell):
        cn = d.cell_nodes[e]
        Ke = 2.0 * d.kinetic_cell(e) / (4.0 * math.pi)
        rows.append(np.repeat(cn, d.nl))
        cols.append(np.tile(cn, d.nl))
        vals.append(Ke.ravel())
        B, _ = d.basis_at(e, qc.pts[e])
        b[cn] += B.T @ (qc.w[e] * rho[qc.off[e]:qc.off[e + 1]])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(d.n_nodes, d.n_nodes)).tocsr()
    # nodal coordinates
    ax = []
    for dd in range(3):
        br = d.breaks[dd]
        pts = [br[0]]
        for i in range(len(br) - 1):
            pts.extend(list(br[i] + 0.5 * (d.z[1:] + 1.0) * (br[i + 1] - br[i])))
        ax.append(np.array(pts))
    Zg, Yg, Xg = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    node_xyz = np.stack([Xg.ravel(), Yg.ravel(), Zg.ravel()], axis=1)
    phi = np.zeros(d.n_nodes)
    bnd = d.boundary
    rv = node_xyz[bnd] - centre[None, :]
    rn = np.sqrt(np.sum(rv * rv, axis=1))
    phi[bnd] = Q / rn + (rv @ dip) / rn ** 3
    inn = d.interior
    rhs = b[inn] - A[inn][:, bnd] @ phi[bnd]
    phi[inn] = ssl.spsolve(A[inn][:, inn].tocsc(), rhs)
    VH = np.empty(len(w))
    for e in range(d.n_cell):
        B, _ = d.basis_at(e, qc.pts[e])
        VH[qc.off[e]:qc.off[e + 1]] = B @ phi[d.cell_nodes[e]]
    return VH, phi


def nuclear_repulsion(atoms, Z):
    """E_ZZ = 1/2 sum_{I != J} Z_I Z_J / |R_I - R_J| (Eq. repulsiveEnergy)."""
    e = 0.0
    for i in range(len(Z)):
        for j in range(i + 1, len(Z)):
            e += Z[i] * Z[j] / np.linalg.norm(atoms[i] - atoms[j])
    return e


def energies(qc, rho_in, rho_out, VH_in, VH_out, eps, f, system):
    """Kohn-Sham energy terms at rho_out with potentials of rho_in (reading above)."""
    w = qc.all_w
    exc_in, vxc_in = lda_pz81(rho_in)
    exc_out, _ = lda_pz81(rho_out)
    e_band = 2.0 * np.sum(f * eps)
    e_xc = np.sum(w * rho_out * exc_out)
    e_h = 0.5 * np.sum(w * rho_out * VH_out)
    e_zz = nuclear_repulsion(system["atoms"], system["Z"])
    e_dc = np.sum(w * rho_out * (VH_in + vxc_in))
    total = e_band - e_dc + e_h + e_xc + e_zz
    return {"band": e_band, "xc": e_xc, "hartree": e_h, "zz": e_zz, "double_counting": e_dc, "total": total}


# ---------------------------------------------------------------------- mixing
def anderson(rho_ins, rho_outs, w, beta=0.5):
    """n-stage Anderson mixing of the densities (weighted least squares on the residuals)."""
    F = [ro - ri for ri, ro in zip(rho_ins, rho_outs)]
    n = len(F)
    if n == 1:
        return rho_ins[-1] + beta * F[-1]
    dF = [F[k] - F[-1] for k in range(n - 1)]
    Amat = np.array([[np.sum(w * a * c) for c in dF] for a in dF])
    rhs = np.array([-np.sum(w * a * F[-1]) for a in dF])
    theta = np.linalg.lstsq(Amat, rhs, rcond=None)[0]
    rin = rho_ins[-1] + sum(t * (rho_ins[k] - rho_ins[-1]) for k, t in enumerate(theta))
    fbar = F[-1] + sum(t * dF[k] for k, t in enumerate(theta))
    return rin + beta * fbar


def scf(disc, qc, system, rho0, X0, m, n_electrons, kT, beta=0.5, n_hist=5, tol_e=1e-8,
        tol_rho=1e-6, max_scf=60, chfsi_tol=1e-9, v0=None, verbose=False):
    """SCF loop of Sec. V: rho_in -> V_eff (Eq. veff) -> ChFSI eigenpairs ->
    Fermi occupations -> rho_out -> energy -> n-stage Anderson mixing."""
    from .chfsi import chfsi
    w = qc.all_w
    Vext = v_ext(system, qc.all_pts)
    rho_in = rho0.copy()
    ins, outs = [], []
    X = X0
    e_prev = None
    out = {}
    for it in range(max_scf):
        VH_in, _ = hartree(qc, rho_in)
        _, vxc = lda_pz81(rho_in)
        disc.build(Vq=vxc + VH_in + Vext)
        eps, X, res, b, hist = chfsi(disc, X, m, n_iter_max=200, tol=chfsi_tol, v0=v0,
                                     n_conv=X.shape[1] - 2)
        f, mu = fermi_occupations(eps, n_electrons, kT)
        rho_out = density(qc, X, f)
        VH_out, _ = hartree(qc, rho_out)
        E = energies(qc, rho_in, rho_out, VH_in, VH_out, eps, f, system)
        drho = math.sqrt(np.sum(w * (rho_out - rho_in) ** 2))
        if verbose:
            print(it, E["total"], drho)
        out = {"energies": E, "eps": eps, "f": f, "mu": mu, "rho": rho_out, "X": X, "iterations": it + 1,
               "drho": drho}
        if e_prev is not None and abs(E["total"] - e_prev) < tol_e and drho < tol_rho:
            break
        e_prev = E["total"]
        ins.append(rho_in)
        outs.append(rho_out)
        ins, outs = ins[-n_hist:], outs[-n_hist:]
        rho_in = anderson(ins, outs, w, beta)
    return out


def v_ext(system, pts):
    V = np.zeros(len(pts))
    for R, Z in zip(system["atoms"], system["Z"]):
        V -= Z / np.sqrt(np.sum((pts - R[None, :]) ** 2, axis=1))
    return V
