"""Learned initial density for the SCF: loop control around the library's kernels.

The plain start is the superposition of atomic densities (SAD, efe_sad_density).
The learned start corrects it point by point, rho = (rho_sad + floor) exp(y) -
floor rescaled to N_e, with y predicted by a fully connected network (64 -> 256
-> 256 -> 256 -> 1, SiLU, FP32) from atom-centred descriptors
(efe_descriptors).  Training targets are y = log(rho_conv + floor) -
log(rho_sad + floor) on converged densities the SCF itself produced; the loss
is the squared error weighted by w_q rho_conv(x_q).  Descriptors, network
passes, loss, Adam and the corrected density all run in the library; this
module only sequences the calls and samples training points.
"""
import numpy as np

from ._lib import DescParams, Mlp

FLOOR = 1e-6
SPECIES = (1.0, 6.0, 8.0, 14.0)
RADIAL_MU = np.linspace(0.25, 7.0, 12)
RADIAL_SIGMA = 0.45
ANG_MU = (0.8, 2.0, 3.5, 5.5)
ANG_SIGMA = 0.9
R_CUT = 8.0
N_FEAT = len(SPECIES) * (len(RADIAL_MU) + len(ANG_MU))
DIMS = (N_FEAT, 256, 256, 256, 1)


def desc_params(offset=None, scale=None):
    p = DescParams()
    p.n_species = len(SPECIES)
    for i, z in enumerate(SPECIES):
        p.species_Z[i] = z
    p.n_radial = len(RADIAL_MU)
    for i, m in enumerate(RADIAL_MU):
        p.radial_mu[i] = float(m)
    p.radial_sigma = RADIAL_SIGMA
    p.n_ang = len(ANG_MU)
    for i, m in enumerate(ANG_MU):
        p.ang_mu[i] = float(m)
    p.ang_sigma = ANG_SIGMA
    p.r_cut = R_CUT
    if offset is not None:
        p.standardise = 1
        for i in range(N_FEAT):
            p.offset[i] = float(offset[i])
            p.scale[i] = float(scale[i])
    return p


def scf_to_convergence(G, X, rho_in, n_electrons, m, tol_e=1e-6, tol_rho=1e-4, max_it=100, precision="fp64",
                       fp64_tail=0, passes=1, **scf_kw):
    """Run efe_scf_step until |dE| < tol_e and |rho_out - rho_in| < tol_rho.
    Returns (last result, iterations, rho_out)."""
    import torch
    rho_out = torch.empty_like(rho_in)
    G.scf_init(n_electrons, **scf_kw)
    e_prev, res = None, None
    for it in range(1, max_it + 1):
        res = G.scf_step(X, rho_in, rho_out, m, passes=passes, precision=precision, fp64_tail=fp64_tail)
        if e_prev is not None and abs(res["total"] - e_prev) < tol_e and res["drho"] < tol_rho:
            return res, it, rho_out
        e_prev = res["total"]
    return res, max_it, rho_out


class DensityModel:
    """Descriptor standardisation + network."""

    def __init__(self, seed=0, precision="fp32"):
        self.net = Mlp(DIMS, precision=precision, seed=seed)
        self.offset = None
        self.scale = None

    def set_standardisation(self, D):
        """Per-feature offset / scale from raw training descriptors (n x F tensor)."""
        self.offset = D.double().mean(dim=0).cpu().numpy()
        sd = D.double().std(dim=0).cpu().numpy()
        self.scale = 1.0 / np.maximum(sd, 1e-6)

    def descriptors(self, G):
        return G.descriptors(desc_params(self.offset, self.scale), precision=self.net.prec)

    def fit(self, D, y, c, steps=1500, batch=8192, lr=1e-3, seed=0):
        """Adam on minibatches drawn (seeded) from the training rows; returns the losses."""
        import torch
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        n = D.shape[0]
        losses = []
        for k in range(steps):
            idx = torch.randint(0, n, (min(batch, n),), generator=gen, device="cuda")
            Xb, yb, cb = D[idx].contiguous(), y[idx].contiguous(), c[idx].contiguous()
            yh = self.net.forward(Xb)
            loss, dy = self.net.wmse(yh, yb, cb)
            g = self.net.backward(Xb, dy)
            self.net.adam(g, lr=lr)
            losses.append(loss)
        return losses

    def predict(self, G):
        D = self.descriptors(G)
        return self.net.forward(D.contiguous())

    def start_density(self, G, rho_sad, n_electrons):
        return G.learned_density(rho_sad, self.predict(G), FLOOR, n_electrons)


def training_rows(G, rho_conv, rho_sad, raw_desc, n_rows, seed):
    """Seeded sample of quadrature points of one system: raw descriptors, targets
    and loss weights w_q rho_conv(x_q)."""
    import torch
    y = G.density_log_ratio(rho_conv, rho_sad, FLOOR, precision="fp32")
    w = G.qpoints()[:, 3]
    c = (w * rho_conv).float()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    idx = torch.randint(0, G.n_qpoints, (min(n_rows, G.n_qpoints),), generator=gen, device="cuda")
    return raw_desc[idx].contiguous(), y[idx].contiguous(), c[idx].contiguous()
