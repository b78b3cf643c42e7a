"""Oracle pins: smooth cutoff (Eq. Moll1) and enrichment functions (Eqs. KSOrbitalSplit, EnrichedPsi)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.enrichment import cutoff, eval_function, radial_q, solid_harmonic


def _h_of_rt(rt):
    # evaluate h through r for r0 = 1, t = 1:  r~ = 1 - (r - 1)  ->  r = 2 - r~
    return cutoff(2.0 - rt, 1.0, 1.0)[0]


def test_cutoff_partition_identity():
    rt = np.linspace(-0.5, 1.5, 401)
    np.testing.assert_allclose(_h_of_rt(rt) + _h_of_rt(1.0 - rt), 1.0, atol=1e-15)


@pytest.mark.parametrize("r0,t", [(2.0, 1.0), (3.0, 0.5), (1.1, 0.8)])
def test_cutoff_plateau_tail_and_derivative(r0, t):
    r = np.linspace(0.0, r0 * 0.999, 50)
    h, dh = cutoff(r, r0, t)
    assert np.all(h == 1.0) and np.all(dh == 0.0)
    r = np.linspace(r0 + r0 / t + 1e-9, 3 * r0 + r0 / t, 50)
    h, dh = cutoff(r, r0, t)
    assert np.all(h == 0.0) and np.all(dh == 0.0)
    r = np.linspace(r0 * 1.001, (r0 + r0 / t) * 0.999, 200)
    h, dh = cutoff(r, r0, t)
    assert np.all((h >= 0) & (h <= 1)) and np.all(np.diff(h) <= 0) and np.any(np.diff(h) < 0)
    assert abs(cutoff(np.array([r0 + 0.5 * r0 / t]), r0, t)[0][0] - 0.5) < 1e-15
    eps = 1e-6
    fd = (cutoff(r + eps, r0, t)[0] - cutoff(r - eps, r0, t)[0]) / (2 * eps)
    np.testing.assert_allclose(dh, fd, atol=1e-6)


FUNCS = [
    {"n": 1, "l": 0, "m": 0, "kind": "hydrogenic", "zeta": 0.0},
    {"n": 2, "l": 0, "m": 0, "kind": "hydrogenic", "zeta": 0.0},
    {"n": 2, "l": 1, "m": 0, "kind": "hydrogenic", "zeta": 0.0},
    {"n": 1, "l": 0, "m": 0, "kind": "slater", "zeta": 13.7},
    {"n": 2, "l": 0, "m": 0, "kind": "slater", "zeta": 4.925},
    {"n": 2, "l": 1, "m": 1, "kind": "slater", "zeta": 4.925},
]


@pytest.mark.parametrize("f", FUNCS)
@pytest.mark.parametrize("Z", [1.0, 3.0])
def test_radial_unit_norm(f, Z):
    """int_0^inf r^2 R(r)^2 dr = 1 (closed-form normalisation, independent quadrature)."""
    def integrand(r):
        q, _ = radial_q(f, Z, np.array([r]))
        return (r ** f["l"] * q[0]) ** 2 * r * r
    val, _ = integrate.quad(integrand, 0, np.inf, limit=200)
    assert abs(val - 1.0) < 1e-9


@pytest.mark.parametrize("n,l", [(1, 0), (2, 0), (2, 1)])
@pytest.mark.parametrize("Z", [1.0, 2.0])
def test_hydrogenic_radial_equation(n, l, Z):
    """-1/2 (R'' + 2R'/r) + l(l+1)/(2 r^2) R - Z R / r = -Z^2/(2 n^2) R."""
    f = {"n": n, "l": l, "m": 0, "kind": "hydrogenic", "zeta": 0.0}
    r = np.linspace(0.3, 8.0, 40)
    h = 1e-4

    def R(x):
        q, _ = radial_q(f, Z, x)
        return q * x ** l
    Rp = (R(r + h) - R(r - h)) / (2 * h)
    Rpp = (R(r + h) - 2 * R(r) + R(r - h)) / (h * h)
    lhs = -0.5 * (Rpp + 2 * Rp / r) + l * (l + 1) / (2 * r * r) * R(r) - Z * R(r) / r
    np.testing.assert_allclose(lhs, -Z * Z / (2 * n * n) * R(r), atol=2e-6)


def test_real_harmonics_orthonormal_on_sphere():
    ct, wt = np.polynomial.legendre.leggauss(8)
    ph = np.arange(16) * 2 * np.pi / 16
    C, P = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - C ** 2)
    d = np.stack([(st * np.cos(P)).ravel(), (st * np.sin(P)).ravel(), C.ravel()], axis=1)
    w = (wt[:, None] * np.full(16, 2 * np.pi / 16)[None, :]).ravel()
    lm = [(0, 0), (1, -1), (1, 0), (1, 1)]
    Y = np.stack([solid_harmonic(l, m, d)[0] for (l, m) in lm], axis=1)
    np.testing.assert_allclose(Y.T @ (w[:, None] * Y), np.eye(4), atol=1e-14)


@pytest.mark.parametrize("f", FUNCS)
def test_enrichment_gradient_vs_fd(f):
    ff = dict(f, atom=0, r0=1.5, t=0.8)
    R = np.array([0.1, -0.2, 0.3])
    rng = np.random.default_rng(0)
    pts = R + rng.uniform(-3.0, 3.0, size=(30, 3))
    Z = 2.0
    v, g = eval_function(ff, R, Z, pts)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (eval_function(ff, R, Z, pts + e)[0] - eval_function(ff, R, Z, pts - e)[0]) / (2 * h)
        np.testing.assert_allclose(g[:, d], fd, atol=2e-5 * max(1.0, np.abs(v).max()))
