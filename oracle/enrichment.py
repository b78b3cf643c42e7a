"""Atom-centred enrichment functions and the smooth cutoff -- oracle (test infrastructure only).

Paper, Sec. IV.A (Eqs. KSOrbitalSplit, EnrichedPsi): an orbital enrichment
function is a radial function times a real spherical harmonic centred on an
atom, N_alpha(x) = R_nl(|x - R_I|) Y_lm(angles).  Sec. IV.B (Eq. Moll1): the
radial part is multiplied by the smooth cutoff h(r~) = u(r~) / (u(r~) + u(1 - r~)),
u(s) = exp(-1/s) for s > 0 and 0 otherwise, r~ = 1 - t (r - r0) / r0, so that
h = 1 for r < r0, 0 <= h < 1 on the transition and h = 0 beyond r0 + r0/t.

The paper's radial functions come from a 1-D atomic Kohn-Sham solve (out of
scope); here they are closed-form hydrogenic or Slater radials (workload
choice).  Real Y_lm: Y_00 = 1/sqrt(4 pi); l = 1 uses sqrt(3/(4 pi)) * (y, z, x)/r
for m = -1, 0, 1.

Pins (tests/test_oracle_enrichment.py): cutoff identities of Eq. Moll1
(h(r~) + h(1 - r~) = 1, plateau, zero tail, finite-difference derivative),
unit norm of the uncut functions (closed-form radial integrals, orthonormal
Y_lm on the sphere), gradients against finite differences.
"""
import math
import numpy as np


def _u(s):
    out = np.zeros_like(s)
    pos = s > 0
    out[pos] = np.exp(-1.0 / s[pos])
    return out


def _du(s):
    out = np.zeros_like(s)
    pos = s > 0
    out[pos] = np.exp(-1.0 / s[pos]) / (s[pos] * s[pos])
    return out


def cutoff(r, r0, t):
    """h(r~(r)) of Eq. Moll1 and its derivative dh/dr."""
    r = np.asarray(r, dtype=np.float64)
    rt = 1.0 - t * (r - r0) / r0
    a = _u(rt)
    b = _u(1.0 - rt)
    den = a + b
    h = a / den
    dh_drt = (_du(rt) * b + a * _du(1.0 - rt)) / (den * den)
    return h, dh_drt * (-t / r0)


def support_radius(f):
    """Outer end of the cutoff transition, r0 + r0/t (Sec. IV.B)."""
    return f["r0"] + f["r0"] / f["t"]


def radial_q(f, Z, r):
    """q(r) = R_nl(r) / r^l and dq/dr for the closed-form radials.

    hydrogenic (nucleus charge Z):  R_10 = 2 Z^1.5 e^{-Zr},
      R_20 = Z^1.5/(2 sqrt 2) (2 - Zr) e^{-Zr/2},  R_21 = Z^1.5/(2 sqrt 6) Zr e^{-Zr/2};
    slater: R = (2 zeta)^{n+1/2} / sqrt((2n)!) r^{n-1} e^{-zeta r}.
    """
    n, l = f["n"], f["l"]
    r = np.asarray(r, dtype=np.float64)
    if f["kind"] == "hydrogenic":
        if (n, l) == (1, 0):
            q = 2.0 * Z ** 1.5 * np.exp(-Z * r)
            return q, -Z * q
        if (n, l) == (2, 0):
            c = Z ** 1.5 / (2.0 * math.sqrt(2.0))
            e = np.exp(-Z * r / 2.0)
            return c * (2.0 - Z * r) * e, c * e * (Z * Z * r / 2.0 - 2.0 * Z)
        if (n, l) == (2, 1):
            c = Z ** 1.5 / (2.0 * math.sqrt(6.0)) * Z
            q = c * np.exp(-Z * r / 2.0)
            return q, -0.5 * Z * q
        raise ValueError("hydrogenic radial not tabulated")
    if f["kind"] == "slater":
        z = f["zeta"]
        norm = (2.0 * z) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))
        k = n - 1 - l
        if k < 0:
            raise ValueError("slater needs n-1 >= l")
        e = np.exp(-z * r)
        q = norm * r ** k * e
        dq = norm * e * ((k * r ** (k - 1) if k > 0 else 0.0) - z * r ** k)
        return q, dq
    raise ValueError("unknown radial kind")


def solid_harmonic(l, m, d):
    """P_lm(d) = r^l Y_lm(angles) (real form) and its gradient, d = x - R_I."""
    npt = d.shape[0]
    if l == 0:
        return np.full(npt, 1.0 / math.sqrt(4.0 * math.pi)), np.zeros((npt, 3))
    if l == 1:
        c = math.sqrt(3.0 / (4.0 * math.pi))
        axis = {-1: 1, 0: 2, 1: 0}[m]
        g = np.zeros((npt, 3))
        g[:, axis] = c
        return c * d[:, axis], g
    raise ValueError("only l <= 1 enrichment is used")


def eval_function(f, R, Z, pts):
    """Value and gradient of one cut-off enrichment function at points (npt, 3)."""
    d = pts - R[None, :]
    r = np.sqrt(np.sum(d * d, axis=1))
    q, dq = radial_q(f, Z, r)
    h, dh = cutoff(r, f["r0"], f["t"])
    P, dP = solid_harmonic(f["l"], f["m"], d)
    qh = q * h
    dqh = dq * h + q * dh
    val = qh * P
    with np.errstate(invalid="ignore", divide="ignore"):
        rhat = np.where(r[:, None] > 0, d / r[:, None], 0.0)
    grad = (dqh * P)[:, None] * rhat + qh[:, None] * dP
    return val, grad


def eval_all(system, pts, func_ids):
    """Values (npt, k) and gradients (npt, k, 3) of the listed functions."""
    vals = np.zeros((pts.shape[0], len(func_ids)))
    grads = np.zeros((pts.shape[0], len(func_ids), 3))
    for j, fi in enumerate(func_ids):
        f = system["funcs"][fi]
        a = f["atom"]
        v, g = eval_function(f, system["atoms"][a], system["Z"][a], pts)
        vals[:, j] = v
        grads[:, j, :] = g
    return vals, grads
