"""Chebyshev-filtered subspace iteration -- oracle (test infrastructure only).

Paper, Sec. V: the unwanted part [a, b] of the spectrum of H~ = (M^E)^-1 H^E is
mapped to [-1, 1] by t(x) = (2x - a - b)/(b - a); b comes from a few
Krylov iterations on H~, a is the largest Rayleigh quotient of the previous
subspace; the degree-m Chebyshev polynomial of the mapped operator is
applied through p_{k+1} = 2 x p_k - p_{k-1}; the filtered block is
orthonormalised and the Galerkin problem Q^T H Q Psi = eps Q^T M Q Psi is solved
by a direct dense solver; the subspace is rotated to Q Psi.

Readings where the paper is silent (each listed in the design notes):
* the plain recurrence is also given in its scaled form (dividing by
  T_k(t(a0)) at every degree, with a0 a lower bound of the spectrum), which
  spans the same space and cannot overflow; both are implemented and a test
  checks that they agree;
* "a few Arnoldi iterations" is read as a k-step Lanczos run in the
  M-inner product (H~ is self-adjoint there), with b = max Ritz value + |beta_k|;
* "orthonormalize" is read as Cholesky-QR in the Euclidean inner product;
* the residual of a Ritz pair is ||H x - eps M x||_2 with x^T M x = 1.

Pins (tests/test_oracle_chfsi.py): the filter equals V T_m(t(Lambda)) V^-1 X
from a dense eigendecomposition; CholQR gives Q^T Q = I and Q R = X; a
Rayleigh-Ritz step on the full space returns the dense generalised
eigenvalues; converged ChFSI reproduces the dense eigenvalues and the closed
form spectra of the hydrogen atom and the harmonic oscillator.
"""
import numpy as np
import scipy.linalg as sla


def chebyshev_filter_plain(apply_Ht, X, m, a, b):
    """T_m(t(H~)) X by the three-term recurrence of Sec. V (unscaled)."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    Yprev = X
    Y = (apply_Ht(X) - c * X) / e
    for _ in range(2, m + 1):
        Ynew = 2.0 * (apply_Ht(Y) - c * Y) / e - Yprev
        Yprev, Y = Y, Ynew
    return Y


def chebyshev_filter_scaled(apply_Ht, X, m, a, b, a0):
    """Scaled form of the same recurrence: returns T_m(t(H~)) X / T_m(t(a0)).

    With s_k = T_{k-1}(t(a0)) / T_k(t(a0)):  s_1 = e / (a0 - c),
    s_{k+1} = 1 / (2/s_1 - s_k), and
    Y_{k+1} = (2 s_{k+1} / e)(H~ Y_k - c Y_k) - s_k s_{k+1} Y_{k-1}."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    s1 = e / (a0 - c)
    s = s1
    Yprev = X
    Y = (s1 / e) * (apply_Ht(X) - c * X)
    for _ in range(2, m + 1):
        snew = 1.0 / (2.0 / s1 - s)
        Ynew = (2.0 * snew / e) * (apply_Ht(Y) - c * Y) - (s * snew) * Yprev
        Yprev, Y = Y, Ynew
        s = snew
    return Y


def chebyshev_scale_factors(m, a, b, a0):
    """T_k(t(a0)) for k = 0..m by the scalar recurrence (for cross checks)."""
    t0 = (2.0 * a0 - a - b) / (b - a)
    T = [1.0, t0]
    for _ in range(2, m + 1):
        T.append(2.0 * t0 * T[-1] - T[-2])
    return np.array(T[:m + 1])


def lanczos_upper_bound(apply_Ht, apply_M, v0, k):
    """Upper bound of the spectrum of H~ by k Lanczos steps in the M-inner product."""
    v = v0 / np.sqrt(v0 @ apply_M(v0))
    vprev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for j in range(k):
        w = apply_Ht(v)
        alpha = w @ apply_M(v)
        w = w - alpha * v - beta * vprev
        beta = np.sqrt(max(w @ apply_M(w), 0.0))
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        vprev, v = v, w / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    theta = np.linalg.eigvalsh(T)
    return theta.max() + abs(betas[-1])


def cholqr(X):
    """Cholesky-QR: G = X^T X, G = R^T R, Q = X R^-1."""
    G = X.T @ X
    G = 0.5 * (G + G.T)
    R = sla.cholesky(G, lower=False)
    Q = sla.solve_triangular(R, X.T, trans="T", lower=False).T
    return Q, R


def rayleigh_ritz(apply_H, apply_M, Q):
    """Galerkin projection Q^T H Q Psi = eps Q^T M Q Psi (Sec. V), direct dense solve,
    rotation X = Q Psi, and residual norms ||H x_i - eps_i M x_i||_2."""
    HQ = apply_H(Q)
    MQ = apply_M(Q)
    Hp = Q.T @ HQ
    Mp = Q.T @ MQ
    Hp = 0.5 * (Hp + Hp.T)
    Mp = 0.5 * (Mp + Mp.T)
    eps, Psi = sla.eigh(Hp, Mp)
    X = Q @ Psi
    R = HQ @ Psi - (MQ @ Psi) * eps[None, :]
    return eps, X, np.sqrt(np.sum(R * R, axis=0))


def chfsi(disc, X0, m, n_iter_max=100, tol=1e-8, n_lanczos=10, v0=None, scaled=True,
          elemental=True, verbose=False, n_conv=None):
    """Plain ChFSI for a fixed Hamiltonian until the residuals of the lowest
    ``n_conv`` (default: all) Ritz pairs are below tol.

    Order of operations: RR on X0 for a and a0; Lanczos for b; then repeat
    filter -> CholQR -> RR, updating a (largest Ritz value) and a0 (smallest)."""
    apply_Ht = lambda Y: disc.apply_Htilde(Y, elemental=elemental)
    apply_H = disc.apply_H_elemental if elemental else disc.apply_H_assembled
    apply_M = disc.apply_M_assembled
    Q, _ = cholqr(X0)
    eps, X, res = rayleigh_ritz(apply_H, apply_M, Q)
    if v0 is None:
        v0 = np.ones(X0.shape[0])
        v0 = disc.restrict(v0)
    b = lanczos_upper_bound(apply_Ht, apply_M, v0, n_lanczos)
    history = []
    for it in range(n_iter_max):
        a, a0 = eps.max(), eps.min()
        if scaled:
            Y = chebyshev_filter_scaled(apply_Ht, X, m, a, b, a0)
        else:
            Y = chebyshev_filter_plain(apply_Ht, X, m, a, b)
        Q, _ = cholqr(Y)
        eps, X, res = rayleigh_ritz(apply_H, apply_M, Q)
        history.append((eps.copy(), res.copy()))
        if verbose:
            print(it, eps[:4], res.max())
        if res[:n_conv].max() < tol:
            break
    return eps, X, res, b, history


def dense_eigs(disc, k):
    """Lowest k eigenvalues of the assembled generalised problem H^E psi = eps M^E psi."""
    H, M, _ = disc.dense_active()
    return sla.eigh(H, M, eigvals_only=True, subset_by_index=[0, k - 1])
