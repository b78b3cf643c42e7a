"""Oracle pins: Gauss / GLL rules, Lagrange basis, adaptive rule (Sec. III.B, Sec. IV.C)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.quadrature import gauss_rule, gll_rule, lagrange_values, lagrange_derivs, exact_1d_matrices
from oracle.adaptive import adaptive_rule, gauss_box

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _mono(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("n", [3, 5, 6, 8])
def test_gauss_exact_to_2n_minus_1(n):
    x, w = gauss_rule(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - _mono(k)) < 1e-13
    assert abs(np.sum(w * x ** (2 * n)) - _mono(2 * n)) > 1e-6


@pytest.mark.parametrize("n", [3, 5, 6, 7])
def test_gll_exact_to_2n_minus_3(n):
    x, w = gll_rule(n)
    for k in range(2 * n - 2):
        assert abs(np.sum(w * x ** k) - _mono(k)) < 1e-13
    assert abs(np.sum(w * x ** (2 * n - 2)) - _mono(2 * n - 2)) > 1e-6


def test_gll5_matches_table():
    x, w = gll_rule(5)
    np.testing.assert_allclose(x, GOLD["gll5"]["nodes"], atol=1e-15)
    np.testing.assert_allclose(w, GOLD["gll5"]["weights"], atol=1e-15)


def test_lagrange_cardinal_partition_and_derivative():
    z, _ = gll_rule(5)
    np.testing.assert_allclose(lagrange_values(z, z), np.eye(5), atol=1e-14)
    xs = np.linspace(-1, 1, 17)
    np.testing.assert_allclose(lagrange_values(z, xs).sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(lagrange_derivs(z, xs).sum(axis=1), 0.0, atol=1e-12)
    h = 1e-6
    fd = (lagrange_values(z, xs + h) - lagrange_values(z, xs - h)) / (2 * h)
    np.testing.assert_allclose(lagrange_derivs(z, xs), fd, atol=1e-7)


def test_exact_1d_matrices_vs_gauss():
    z, wl = gll_rule(5)
    M1, K1 = exact_1d_matrices(z)
    x, w = gauss_rule(6)
    L = lagrange_values(z, x)
    dL = lagrange_derivs(z, x)
    np.testing.assert_allclose(M1, L.T @ (w[:, None] * L), atol=1e-14)
    np.testing.assert_allclose(K1, dL.T @ (w[:, None] * dL), atol=1e-12)
    assert abs(M1.sum() - 2.0) < 1e-14
    np.testing.assert_allclose(K1.sum(axis=1), 0.0, atol=1e-12)
    # GLL lumping equals the row sums of the exact mass (p=4 GLL weights)
    np.testing.assert_allclose(M1.sum(axis=1), wl, atol=1e-14)


def _octant_system(kind, zeta=1.0, Z=1.0, n=1, l=0, m=0):
    s = W.hydrogen(cells=1, half=30.0)
    s["atoms"] = np.zeros((1, 3))
    s["Z"] = np.array([Z])
    s["funcs"] = [{"atom": 0, "n": n, "l": l, "m": m, "kind": kind, "zeta": zeta,
                   "r0": 1e3, "t": 1.0}]
    return s


@pytest.mark.parametrize("kind,zeta,Z,n,l,m", [
    ("hydrogenic", 0.0, 1.0, 1, 0, 0), ("hydrogenic", 0.0, 1.0, 2, 1, 1),
    ("slater", 13.7, 14.0, 1, 0, 0), ("slater", 4.9, 14.0, 2, 0, 0)])
def test_adaptive_rule_normalised_density_octant(kind, zeta, Z, n, l, m):
    """A unit-norm orbital with a cusp at a box corner: the octant holds exactly 1/8."""
    s = _octant_system(kind, zeta, Z, n, l, m)
    L = 30.0 if kind == "hydrogenic" else 6.0
    pts, w = adaptive_rule(s, np.zeros(3), np.full(3, L), [0], 1e-9, 12, 6)
    from oracle.enrichment import eval_function
    v, _ = eval_function(s["funcs"][0], s["atoms"][0], Z, pts)
    assert abs(np.sum(w * v * v) - 0.125) < 1e-7
    # the refined rule still integrates polynomials of degree <= 11 per axis exactly
    poly = pts[:, 0] ** 5 * pts[:, 1] ** 3 * pts[:, 2] ** 2
    exact = L ** 6 / 6 * L ** 4 / 4 * L ** 3 / 3
    assert abs(np.sum(w * poly) - exact) < 1e-12 * exact


def test_gauss_box_volume_and_linear():
    P, Wt = gauss_box(np.array([0., 1., 2.]), np.array([1., 3., 5.]), 6)
    assert abs(Wt.sum() - 6.0) < 1e-13
    assert abs(np.sum(Wt * P[:, 1]) - 6.0 * 2.0) < 1e-12
