"""Learned initial density -- oracle (test infrastructure only).

The SCF of Sec. V starts from an input density rho_in (the paper starts from
single-atom solutions).  The plain start here is the superposition of atomic
densities (SAD) built from Slater-type shells; the learned start multiplies it
by exp(y(x)), y the output of a small MLP on atom-centred descriptors at the
quadrature point x, then rescales to N_e electrons.  Nothing here is in the
paper: the pieces are written from their plain definitions.

  SAD:          rho_0(x) = sum_I sum_shells N_s |R_{n,zeta}(|x - R_I|)|^2 / (4 pi),
                R = C r^(n-1) exp(-zeta r), C^2 = (2 zeta)^(2n+1) / (2n)!
  descriptors:  for each species s (4 slots) and radial centre mu_k (12):
                  G[s,k] = sum_{I of s} exp(-(r_I - mu_k)^2 / (2 sigma^2)) fc(r_I)
                and for 4 broad radial bands g_k:
                  A[s,k] = | sum_{I of s} g_k(r_I) fc(r_I) (x - R_I) / r_I |^2
                with fc(r) = (1 + cos(pi r / r_cut)) / 2 for r < r_cut, else 0
                (64 features: 48 radial + 16 angular);
  MLP:          64 -> 256 -> 256 -> 256 -> 1, SiLU on hidden layers;
  loss:         sum_q c_q (y_hat_q - y_q)^2 / sum_q c_q   (c_q = w_q rho_target(x_q));
  Adam:         Kingma & Ba (2015) with bias correction.

Pins (tests/test_oracle_learned.py): the SAD shells integrate to Z (radial
quadrature, closed form normalisation); descriptors are invariant under a
rigid motion and a permutation of the atoms and vanish beyond the cutoff;
analytic MLP gradients equal central finite differences; one Adam step from
zero moments moves every parameter by lr * sign(g) (up to eps).
"""
import math

import numpy as np

N_SPECIES = 4
RADIAL_MU = np.linspace(0.25, 7.0, 12)
RADIAL_SIGMA = 0.45
ANG_MU = np.array([0.8, 2.0, 3.5, 5.5])
ANG_SIGMA = 0.9
R_CUT = 8.0
N_FEAT = N_SPECIES * (len(RADIAL_MU) + len(ANG_MU))


def slater_radial(n, zeta, r):
    """Normalised Slater radial function: int_0^inf R^2 r^2 dr = 1."""
    c = math.sqrt((2.0 * zeta) ** (2 * n + 1) / math.factorial(2 * n))
    return c * r ** (n - 1) * np.exp(-zeta * r)


def sad_density(pts, atoms, shells):
    """Superposition of atomic densities at pts (n x 3).  shells[I] = [(n, zeta, N_e), ...]."""
    rho = np.zeros(len(pts))
    for R, sh in zip(atoms, shells):
        r = np.sqrt(np.sum((pts - R[None, :]) ** 2, axis=1))
        for n, zeta, ne in sh:
            rho += ne * slater_radial(n, zeta, r) ** 2 / (4.0 * math.pi)
    return rho


def cutoff(r):
    return np.where(r < R_CUT, 0.5 * (1.0 + np.cos(math.pi * r / R_CUT)), 0.0)


def descriptors(pts, atoms, species_slot):
    """64 features per point; species_slot[I] in 0..3 is the atom's species slot."""
    n = len(pts)
    G = np.zeros((n, N_SPECIES, len(RADIAL_MU)))
    Avec = np.zeros((n, N_SPECIES, len(ANG_MU), 3))
    for R, s in zip(atoms, species_slot):
        d = pts - R[None, :]
        r = np.sqrt(np.sum(d * d, axis=1))
        fc = cutoff(r)
        G[:, s, :] += np.exp(-(r[:, None] - RADIAL_MU[None, :]) ** 2 / (2 * RADIAL_SIGMA ** 2)) * fc[:, None]
        u = d / np.maximum(r, 1e-12)[:, None]
        g = np.exp(-(r[:, None] - ANG_MU[None, :]) ** 2 / (2 * ANG_SIGMA ** 2)) * fc[:, None]
        Avec[:, s, :, :] += g[:, :, None] * u[:, None, :]
    A = np.sum(Avec * Avec, axis=3)
    return np.concatenate([G.reshape(n, -1), A.reshape(n, -1)], axis=1)


# ---------------------------------------------------------------------- MLP
def init_params(dims, seed):
    """W_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), b_l = 0; flat list [W0, b0, W1, b1, ...]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = 1.0 / math.sqrt(a)
        out.append(rng.uniform(-lim, lim, size=(b, a)))
        out.append(np.zeros(b))
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X):
    """Returns y (n,) and the pre-activations of every layer."""
    a = X
    pre = []
    nl = len(params) // 2
    for l in range(nl):
        W, b = params[2 * l], params[2 * l + 1]
        z = a @ W.T + b[None, :]
        pre.append(z)
        a = silu(z) if l < nl - 1 else z
    return a[:, 0], pre


def backward(params, X, pre, dy):
    """Gradients of sum_q dy_q y_q with respect to every parameter."""
    nl = len(params) // 2
    grads = [None] * len(params)
    d = dy[:, None]
    for l in range(nl - 1, -1, -1):
        a_prev = X if l == 0 else silu(pre[l - 1])
        grads[2 * l] = d.T @ a_prev
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            d = (d @ params[2 * l]) * silu_grad(pre[l - 1])
    return grads


def wmse(yhat, y, c):
    """Loss and its gradient with respect to yhat."""
    cs = np.sum(c)
    r = yhat - y
    return float(np.sum(c * r * r) / cs), 2.0 * c * r / cs


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on p, m, v (t counts from 1)."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p -= lr * mh / (np.sqrt(vh) + eps)


def target(rho_conv, rho_sad, floor=1e-6):
    """Regression target y = log(rho_conv + floor) - log(rho_sad + floor)."""
    return np.log(rho_conv + floor) - np.log(rho_sad + floor)


def predicted_density(rho_sad, y, w, n_electrons, floor=1e-6):
    """rho = (rho_sad + floor) exp(y) - floor, clipped at 0, scaled to N_e."""
    rho = np.maximum((rho_sad + floor) * np.exp(y) - floor, 0.0)
    return rho * (n_electrons / np.sum(w * rho))
