"""Oracle pins: operator blocks and the block-wise overlap inverse (Secs. III, IV.A, IV.D)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle.operators import Discretisation
from oracle.quadrature import gll_rule


@pytest.fixture(scope="module")
def tiny():
    return Discretisation(W.tiny(seed=11))


def test_lumped_mass_sums_to_volume(tiny):
    vol = np.prod([b[-1] - b[0] for b in tiny.breaks])
    assert abs(tiny.D.sum() - vol) < 1e-12 * vol


def test_kinetic_constants_and_linear_energy(tiny):
    for e in [0, 3, tiny.n_cell - 1]:
        K = tiny.kinetic_cell(e)
        np.testing.assert_allclose(K @ np.ones(125), 0.0, atol=1e-12)
        # u = x interpolated at the nodes: 1/2 int |grad x|^2 = vol/2 (exact)
        z, _ = gll_rule(5)
        xa = tiny.lo[e][0] + 0.5 * (z + 1) * tiny.h[e][0]
        u = np.tile(xa, 25)
        assert abs(u @ K @ u - 0.5 * np.prod(tiny.h[e])) < 1e-11


def test_potential_block_of_constant_is_consistent_mass(tiny):
    """int 1 * N_j N_k on a Gauss cell equals |J| M1 (x) M1 (x) M1 (exact 1-D masses)."""
    e = int(np.nonzero(~tiny.enriched)[0][0]) if (~tiny.enriched).any() else 0
    pts, w = tiny.cell_quadrature(e)
    B, _ = tiny.basis_at(e, pts)
    M = B.T @ (w[:, None] * B)
    M1 = tiny.M1
    np.testing.assert_allclose(M, np.prod(tiny.h[e]) / 8 * np.kron(M1, np.kron(M1, M1)), atol=1e-13)


def test_assembled_matrices_symmetric(tiny):
    for A in (tiny.H, tiny.M):
        d = abs(A - A.T).max()
        assert d < 1e-12 * abs(A).max()


def test_elemental_apply_equals_assembled(tiny):
    X = W.random_block(tiny.system, 7, seed=3)
    np.testing.assert_allclose(tiny.apply_H_elemental(X), tiny.apply_H_assembled(X),
                               atol=1e-12 * np.abs(tiny.H).max() * 30)


def test_schur_complement_spd(tiny):
    ev = np.linalg.eigvalsh(tiny.S)
    assert ev.min() > 0


def test_block_inverse_equals_dense_inverse(tiny):
    H, M, act = tiny.dense_active()
    X = W.random_block(tiny.system, 5, seed=4)
    Y = tiny.apply_Minv_block(X)
    ref = np.linalg.solve(M, X[act])
    np.testing.assert_allclose(Y[act], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    # boundary rows stay zero
    assert np.all(Y[:tiny.n_nodes][tiny.boundary] == 0.0)


def test_block_inverse_sign_matters(tiny):
    """A flipped sign in the off-diagonal blocks of the Banachiewicz formula is detected."""
    H, M, act = tiny.dense_active()
    X = W.random_block(tiny.system, 2, seed=6)
    nn = tiny.n_nodes
    Wc, We = X[:nn], X[nn:]
    L = tiny.L
    bad_xe = sla.cho_solve(tiny.S_chol, L @ Wc) + sla.cho_solve(tiny.S_chol, We)
    good = tiny.apply_Minv_block(X)[nn:]
    assert np.abs(bad_xe - good).max() > 1e-3 * np.abs(good).max()


def test_enrichment_blocks_vanish_outside_support(tiny):
    from oracle.enrichment import support_radius
    for e, blk in tiny.Mec.items():
        assert blk.shape == (len(tiny.funcs_of_cell[e]), 125)
    for e in range(tiny.n_cell):
        if not tiny.enriched[e]:
            assert e not in tiny.Hec
