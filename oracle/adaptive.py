"""Adaptive (divide-and-conquer) quadrature on enriched cells -- oracle (test infrastructure only).

Paper, Sec. IV.C: a cell is the parent box; its integral of each trial
function by an n-point Gauss rule is compared with the sum over its eight
children (bisected in every direction).  If |I^p - sum_i I^c_i| < tau holds for
every trial function the PARENT's Gauss points and weights are appended to the
point list; otherwise each child becomes a parent and the test recurses.

Trial functions (Eq. QuadTrialFunctions): f3 = sum_alpha N_alpha^2 and
f4 = sum_alpha |grad N_alpha|^2.  f1, f2 need electrostatic enrichment, which
these workloads do not use (the external potential is the analytic -sum Z/r).
Because that singular potential enters the integrals directly, one more trial
function is added: f5 = (sum_I Z_I / |x - R_I|) * sum_alpha N_alpha^2.  The
recursion depth is capped at ``max_depth`` (at the cap the box is accepted
without a test).  Children are visited in the order c = cx + 2 cy + 4 cz and
points within a box with x fastest.

Pin (tests/test_oracle_quadrature.py): on a box holding a nucleus the rule
reproduces closed-form integrals of the enrichment densities (hydrogenic and
Slater radials, unit norm) to the tolerance, and polynomials exactly.
"""
import numpy as np

from .quadrature import gauss_rule
from .enrichment import eval_all


def gauss_box(lo, hi, n):
    """Tensor n-point Gauss rule on the box [lo, hi] (points x fastest)."""
    x, w = gauss_rule(n)
    axes = []
    waxes = []
    for d in range(3):
        half = 0.5 * (hi[d] - lo[d])
        axes.append(lo[d] + half * (x + 1.0))
        waxes.append(half * w)
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    WZ, WY, WX = np.meshgrid(waxes[2], waxes[1], waxes[0], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return pts, (WX * WY * WZ).ravel()


def trial_values(system, pts, func_ids):
    """Trial functions f3, f4, f5 at points: array (3, npt)."""
    vals, grads = eval_all(system, pts, func_ids)
    f3 = np.sum(vals * vals, axis=1)
    f4 = np.sum(grads * grads, axis=(1, 2))
    vn = np.zeros(pts.shape[0])
    for R, Z in zip(system["atoms"], system["Z"]):
        vn += Z / np.sqrt(np.sum((pts - R[None, :]) ** 2, axis=1))
    return np.stack([f3, f4, vn * f3])


def children(lo, hi):
    mid = 0.5 * (lo + hi)
    out = []
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        clo = np.array([lo[0] if cx == 0 else mid[0], lo[1] if cy == 0 else mid[1],
                        lo[2] if cz == 0 else mid[2]])
        chi = np.array([mid[0] if cx == 0 else hi[0], mid[1] if cy == 0 else hi[1],
                        mid[2] if cz == 0 else hi[2]])
        out.append((clo, chi))
    return out


def adaptive_rule(system, lo, hi, func_ids, tau, max_depth, n):
    """Point list (npt, 3) and weights of the adaptive rule on one cell box."""
    pts_out, w_out = [], []

    def recurse(blo, bhi, depth):
        P, W = gauss_box(blo, bhi, n)
        if depth >= max_depth:
            pts_out.append(P)
            w_out.append(W)
            return
        kids = children(blo, bhi)
        rules = [(P, W)] + [gauss_box(clo, chi, n) for clo, chi in kids]
        # one evaluation of the trial functions over parent + children points
        F = trial_values(system, np.concatenate([r[0] for r in rules]), func_ids)
        npb = len(W)
        Ip = F[:, :npb] @ W
        Ic = np.zeros_like(Ip)
        for c in range(8):
            Ic += F[:, (c + 1) * npb:(c + 2) * npb] @ rules[c + 1][1]
        if np.all(np.abs(Ip - Ic) < tau):
            pts_out.append(P)
            w_out.append(W)
            return
        for clo, chi in kids:
            recurse(clo, chi, depth + 1)

    recurse(np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64), 0)
    return np.concatenate(pts_out), np.concatenate(w_out)
