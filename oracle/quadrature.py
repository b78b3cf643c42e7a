"""1-D rules and the spectral (GLL) Lagrange basis -- oracle (test infrastructure only).

Paper, Sec. III.B ("Spectral finite elements"): the classical basis is the
tensor product of Lagrange polynomials through the Gauss-Lobatto-Legendre
(GLL) points; an n-point GLL rule is exact for polynomials of degree 2n-3 and
is used only for the overlap block M^cc (which it makes diagonal), while an
n-point Gauss rule (exact to degree 2n-1) is used for every other integral.

Pins (tests/test_oracle_quadrature.py): exactness of both rules on monomials
up to their stated degree and failure one degree above; Lagrange cardinality;
exact 1-D mass/stiffness matrices compared with the Gauss-rule products.
"""
import functools
import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import Polynomial


def gauss_rule(n):
    """n-point Gauss-Legendre rule on [-1, 1] (Sec. III.B).  Library routine."""
    x, w = _gauss_cached(n)
    return x.copy(), w.copy()


@functools.lru_cache(maxsize=None)
def _gauss_cached(n):
    x, w = npleg.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gll_rule(n):
    """n-point Gauss-Lobatto-Legendre rule on [-1, 1] (Sec. III.B).

    Nodes: the end points and the roots of P'_{n-1}; weights
    2 / (n (n-1) P_{n-1}(x_i)^2) (textbook definition).
    """
    if n < 2:
        raise ValueError("GLL needs n >= 2")
    coef = np.zeros(n)
    coef[-1] = 1.0                       # P_{n-1} in the Legendre basis
    dcoef = npleg.legder(coef)
    inner = np.sort(np.real(npleg.legroots(dcoef))) if n > 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    # polish interior roots with Newton on P'_{n-1}
    d2coef = npleg.legder(dcoef)
    for _ in range(10):
        if n > 2:
            f = npleg.legval(x[1:-1], dcoef)
            fp = npleg.legval(x[1:-1], d2coef)
            x[1:-1] -= f / fp
    pn = npleg.legval(x, coef)
    w = 2.0 / (n * (n - 1) * pn * pn)
    return x, w


def lagrange_values(nodes, x):
    """Values l_a(x) of the Lagrange polynomials through ``nodes``.

    Returns an array of shape (len(x), len(nodes)); plain product formula.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(x), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                out[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return out


def lagrange_derivs(nodes, x):
    """Derivatives l_a'(x): sum over the dropped factor of the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for a in range(n):
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            out[:, a] += term
    return out


def lagrange_polys(nodes):
    """The Lagrange polynomials as numpy Polynomial objects (exact algebra)."""
    polys = []
    for a, xa in enumerate(nodes):
        p = Polynomial([1.0])
        for b, xb in enumerate(nodes):
            if b != a:
                p = p * Polynomial([-xb, 1.0]) / (xa - xb)
        polys.append(p)
    return polys


def exact_1d_matrices(nodes):
    """Exact reference mass M1_ab = int l_a l_b and stiffness K1_ab = int l_a' l_b'
    on [-1, 1], by exact polynomial integration (independent of any rule)."""
    polys = lagrange_polys(nodes)
    n = len(nodes)
    M1 = np.zeros((n, n))
    K1 = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            pm = (polys[a] * polys[b]).integ()
            M1[a, b] = pm(1.0) - pm(-1.0)
            pk = (polys[a].deriv() * polys[b].deriv()).integ()
            K1[a, b] = pk(1.0) - pk(-1.0)
    return M1, K1
