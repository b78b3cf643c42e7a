"""Pins of the learned-initial-density oracle (SAD start, descriptors, MLP, Adam)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import workloads as W
from oracle import learned as L


@pytest.mark.parametrize("n,zeta", [(1, 13.7), (2, 1.625), (3, 1.3833), (2, 4.925)])
def test_slater_radial_normalised(n, zeta):
    val, _ = quad(lambda r: L.slater_radial(n, zeta, np.array([r]))[0] ** 2 * r * r, 0, np.inf, limit=200)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("Z", [1, 6, 8, 14])
def test_sad_shells_hold_Z_electrons(Z):
    sh = W.sad_shells(Z)
    assert abs(sum(s[2] for s in sh) - Z) < 1e-12
    # radial integral of the atom's density
    f = lambda r: 4 * math.pi * r * r * L.sad_density(np.array([[r, 0.0, 0.0]]), np.zeros((1, 3)), [sh])[0]
    val = sum(quad(f, a, b, limit=200)[0] for a, b in [(0, 0.5), (0.5, 3), (3, 60)])
    assert abs(val - Z) < 1e-8


def _geometry(seed=0):
    rng = np.random.default_rng(seed)
    atoms = rng.uniform(-3, 3, size=(5, 3))
    slots = np.array([0, 1, 2, 1, 3])
    pts = rng.uniform(-5, 5, size=(40, 3))
    return atoms, slots, pts


def test_descriptors_invariant_under_rigid_motion_and_permutation():
    atoms, slots, pts = _geometry()
    D = L.descriptors(pts, atoms, slots)
    assert D.shape == (40, L.N_FEAT)
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    t = np.array([0.3, -1.2, 2.0])
    D2 = L.descriptors(pts @ q.T + t, atoms @ q.T + t, slots)
    np.testing.assert_allclose(D2, D, rtol=1e-10, atol=1e-12)
    perm = np.array([3, 0, 4, 2, 1])
    D3 = L.descriptors(pts, atoms[perm], slots[perm])
    np.testing.assert_allclose(D3, D, rtol=1e-12, atol=1e-14)


def test_descriptors_vanish_beyond_cutoff_and_separate_species():
    atoms = np.zeros((1, 3))
    far = np.array([[L.R_CUT + 0.1, 0.0, 0.0]])
    assert np.all(L.descriptors(far, atoms, np.array([2])) == 0.0)
    near = np.array([[1.0, 0.5, 0.0]])
    D = L.descriptors(near, atoms, np.array([2]))
    nr = len(L.RADIAL_MU)
    radial = D[0, :4 * nr].reshape(4, nr)
    assert np.all(radial[[0, 1, 3]] == 0.0) and np.all(radial[2] > 0.0)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    dims = [6, 9, 9, 9, 1]
    P = L.init_params(dims, seed=3)
    for l in range(1, len(P), 2):
        P[l] = rng.standard_normal(P[l].shape) * 0.1
    X = rng.standard_normal((11, 6))
    dy = rng.standard_normal(11)
    y, pre = L.forward(P, X)
    G = L.backward(P, X, pre, dy)
    h = 1e-6
    for k in range(len(P)):
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            yp, _ = L.forward(P, X)
            flat[idx] = old - h
            ym, _ = L.forward(P, X)
            flat[idx] = old
            fd = np.dot(dy, yp - ym) / (2 * h)
            an = G[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_wmse_gradient():
    rng = np.random.default_rng(2)
    yh, y, c = rng.standard_normal(7), rng.standard_normal(7), rng.uniform(0.1, 1, 7)
    l0, g = L.wmse(yh, y, c)
    for i in range(7):
        e = np.zeros(7)
        e[i] = 1e-6
        fd = (L.wmse(yh + e, y, c)[0] - L.wmse(yh - e, y, c)[0]) / 2e-6
        assert abs(fd - g[i]) < 1e-7


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(5)
    p = rng.standard_normal(20)
    g = rng.standard_normal(20)
    p0 = p.copy()
    m, v = np.zeros(20), np.zeros(20)
    L.adam_step(p, g, m, v, 1, lr=1e-2)
    np.testing.assert_allclose(p0 - p, 1e-2 * np.sign(g), rtol=1e-5)


def test_predicted_density_normalised():
    rng = np.random.default_rng(6)
    w = rng.uniform(0.1, 1, 50)
    rho = L.predicted_density(rng.uniform(0, 2, 50), rng.standard_normal(50) * 0.1, w, 7.0)
    assert abs(np.sum(w * rho) - 7.0) < 1e-12 and np.all(rho >= 0)
