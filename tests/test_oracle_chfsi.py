"""Oracle pins: Chebyshev filter, CholQR, Rayleigh-Ritz and closed-form spectra (Sec. V)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as ssl
import scipy.sparse as sp

import workloads as W
from oracle.operators import Discretisation
from oracle import chfsi as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


@pytest.fixture(scope="module")
def tiny():
    return Discretisation(W.tiny(seed=11))


def _dense_Ht(d):
    H, M, act = d.dense_active()
    return np.linalg.solve(M, H), act


def test_filter_equals_spectral_closed_form(tiny):
    A, act = _dense_Ht(tiny)
    lam, V = np.linalg.eig(A)
    lam, V = lam.real, V.real
    X = W.random_block(tiny.system, 3, seed=8)
    a, b = np.sort(lam)[6], lam.max() * 1.01
    m = 7
    Y = C.chebyshev_filter_plain(tiny.apply_Htilde, X, m, a, b)
    t = (2 * lam - a - b) / (b - a)
    Tm = np.cos(m * np.arccos(np.clip(t, -1, 1)))
    out = np.abs(t) > 1
    Tm[out] = np.cosh(m * np.arccosh(np.abs(t[out]))) * np.sign(t[out]) ** m
    ref = V @ (Tm[:, None] * np.linalg.solve(V, X[act]))
    np.testing.assert_allclose(Y[act], ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


def test_scaled_filter_equals_plain_over_scale(tiny):
    X = W.random_block(tiny.system, 2, seed=9)
    A, act = _dense_Ht(tiny)
    lam = np.sort(np.linalg.eigvals(A).real)
    a, b, a0 = lam[8], lam[-1] * 1.01, lam[0]
    m = 9
    Yp = C.chebyshev_filter_plain(tiny.apply_Htilde, X, m, a, b)
    Ys = C.chebyshev_filter_scaled(tiny.apply_Htilde, X, m, a, b, a0)
    T = C.chebyshev_scale_factors(m, a, b, a0)
    np.testing.assert_allclose(Ys, Yp / T[m], rtol=1e-9, atol=1e-12 * np.abs(Ys).max())


def test_cholqr():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((300, 12)) @ np.diag(10.0 ** np.linspace(0, 4, 12))
    Q, R = C.cholqr(X)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-8)
    np.testing.assert_allclose(Q @ R, X, rtol=1e-12, atol=1e-10 * np.abs(X).max())
    assert np.allclose(np.tril(R, -1), 0.0)


def test_rayleigh_ritz_full_space_is_exact(tiny):
    H, M, act = tiny.dense_active()
    n = len(act)
    full = np.zeros((tiny.n_nodes + tiny.nE, n))
    full[act, np.arange(n)] = 1.0
    eps, X, res = C.rayleigh_ritz(tiny.apply_H_elemental, tiny.apply_M_assembled, full)
    ref = sla.eigh(H, M, eigvals_only=True)
    np.testing.assert_allclose(eps, ref, rtol=1e-10, atol=1e-10)
    assert res.max() < 1e-8


def test_chfsi_converges_to_dense(tiny):
    N, m = 10, 12
    X0 = W.initial_block(tiny.system, N, seed=1)
    v0 = W.lanczos_start(tiny.system)
    nconv = 7
    eps, X, res, b, hist = C.chfsi(tiny, X0, m, n_iter_max=200, tol=1e-9, v0=v0, n_conv=nconv)
    ref = C.dense_eigs(tiny, N)
    assert res[:nconv].max() < 1e-9
    np.testing.assert_allclose(eps[:nconv], ref[:nconv], atol=1e-9)
    # b is an upper bound of the whole spectrum
    H, M, act = tiny.dense_active()
    assert b >= sla.eigh(H, M, eigvals_only=True).max() * (1 - 1e-12)


def _sparse_lowest(d, k, sigma):
    a = np.nonzero(d.active)[0]
    H = d.H[a][:, a].tocsc()
    M = d.M[a][:, a].tocsc()
    return np.sort(ssl.eigsh(H, k=k, M=M, sigma=sigma, which="LM")[0])


def test_harmonic_oscillator_closed_form_and_rate():
    lv = GOLD["harmonic"]["levels"]
    e_coarse = _sparse_lowest(Discretisation(W.harmonic(cells=3, half=6.0)), 4, 1.0)
    e_fine = _sparse_lowest(Discretisation(W.harmonic(cells=6, half=6.0)), 4, 1.0)
    err_c = abs(e_coarse[0] - lv[0][1])
    err_f = abs(e_fine[0] - lv[0][1])
    assert err_f < 3e-4
    assert abs(e_fine[1:4] - lv[1][1]).max() < 3e-4
    assert np.ptp(e_fine[1:4]) < 1e-9           # three-fold degenerate first excited level
    assert err_c / err_f > 2.0 ** 6             # high-order h-convergence (p = 4)


def test_hydrogen_1s_closed_form():
    """-1/2 lap - 1/r in a 20-bohr box with hydrogenic enrichment: 1s -> -1/2 Ha.

    The box confinement shift is bounded by the hard-sphere (R = 10) value,
    computed here by an independent radial finite-difference solve."""
    n = 20000
    r = np.linspace(0, 10.0, n + 2)[1:-1]
    hh = r[1] - r[0]
    A = sp.diags([np.full(n - 1, -0.5 / hh ** 2), 1 / hh ** 2 - 1 / r, np.full(n - 1, -0.5 / hh ** 2)],
                 [-1, 0, 1]).tocsc()
    sphere = ssl.eigsh(A, k=1, sigma=-0.6, which="LM")[0][0]
    shift = sphere + 0.5
    assert 0 < shift < 2e-6
    d = Discretisation(W.hydrogen(cells=4, half=10.0, tau=1e-8, max_depth=8))
    ev = _sparse_lowest(d, 4, -0.6)
    e1s = GOLD["hydrogen"]["levels"][0][1]
    assert abs(ev[0] - e1s) < 5e-4
    # 2p triplet stays degenerate (cubic symmetry about the nucleus)
    assert np.ptp(ev[1:4]) < 1e-8
