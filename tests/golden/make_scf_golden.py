"""Writes the oracle's converged LDA SCF fixtures used by the GPU SCF parity
tests.  Calls only oracle/ and the seeded generators.

    python tests/golden/make_scf_golden.py          # scf_hydrogen_4c.json
    python tests/golden/make_scf_golden.py co       # scf_co.json

scf_hydrogen_4c.json: a hydrogen atom on a 4 x 4 x 4-cell, 20-bohr box
(hydrogenic 1s/2s/2p enrichment).  scf_co.json: the C-O pair of
workloads.carbon_monoxide (14 electrons, Slater enrichment, 49,005 nodes),
started from a sum of atom-centred Gaussian clouds of charge Z.
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import scf as S  # noqa: E402
from oracle.operators import Discretisation  # noqa: E402

SETTINGS = {"cells": 4, "half": 10.0, "tau": 1e-7, "max_depth": 6, "N": 6, "m": 12, "kT_K": 500.0,
            "beta": 0.5, "n_hist": 5, "start_width": 2.0, "block_seed": 1}


def gaussian_start(qc, width):
    """rho_0 = exp(-r^2 / (2 width^2)) normalised to one electron on the quadrature."""
    r = np.sqrt(np.sum(qc.all_pts ** 2, axis=1))
    rho = np.exp(-r * r / (2.0 * width * width))
    return rho / np.sum(qc.all_w * rho)


CO_SETTINGS = {"N": 12, "m": 24, "kT_K": 500.0, "beta": 0.5, "n_hist": 5, "start_width": 1.0, "block_seed": 1}


def gaussian_clouds(qc, atoms, Z, width):
    """rho_0 = sum_I Z_I exp(-|x - R_I|^2 / (2 width^2)) normalised to sum Z on the quadrature."""
    rho = np.zeros(len(qc.all_w))
    for R, z in zip(atoms, Z):
        r2 = np.sum((qc.all_pts - R[None, :]) ** 2, axis=1)
        g = np.exp(-r2 / (2.0 * width * width))
        rho += z * g / np.sum(qc.all_w * g)
    return rho


def main_co():
    c = CO_SETTINGS
    s = W.carbon_monoxide()
    d = Discretisation(s)
    qc = S.QuadCache(d)
    ne = float(np.sum(s["Z"]))
    rho0 = gaussian_clouds(qc, s["atoms"], s["Z"], c["start_width"])
    X0 = W.initial_block(s, c["N"], seed=c["block_seed"])
    out = S.scf(d, qc, s, rho0, X0, c["m"], ne, c["kT_K"] * S.KB_HA_PER_K, beta=c["beta"], n_hist=c["n_hist"],
                tol_e=1e-10, tol_rho=1e-7, max_scf=150, v0=W.lanczos_start(s), verbose=True)
    res = {"settings": c, "energies": {k: float(v) for k, v in out["energies"].items()},
           "eps": [float(x) for x in out["eps"]], "occ": [float(x) for x in out["f"]],
           "mu": float(out["mu"]), "iterations": int(out["iterations"]), "drho": float(out["drho"]),
           "n_qpoints": int(len(qc.all_w)), "int_rho": float(np.sum(qc.all_w * out["rho"]))}
    with open(os.path.join(HERE, "scf_co.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res["energies"]), res["iterations"])


def main():
    c = SETTINGS
    s = W.hydrogen(cells=c["cells"], half=c["half"], tau=c["tau"], max_depth=c["max_depth"])
    d = Discretisation(s)
    qc = S.QuadCache(d)
    rho0 = gaussian_start(qc, c["start_width"])
    X0 = W.initial_block(s, c["N"], seed=c["block_seed"])
    out = S.scf(d, qc, s, rho0, X0, c["m"], 1.0, c["kT_K"] * S.KB_HA_PER_K, beta=c["beta"], n_hist=c["n_hist"],
                tol_e=1e-10, tol_rho=1e-7, max_scf=100, v0=W.lanczos_start(s))
    res = {"settings": c, "energies": {k: float(v) for k, v in out["energies"].items()},
           "eps": [float(x) for x in out["eps"]], "occ": [float(x) for x in out["f"]],
           "mu": float(out["mu"]), "iterations": int(out["iterations"]), "drho": float(out["drho"]),
           "n_qpoints": int(len(qc.all_w)), "int_rho": float(np.sum(qc.all_w * out["rho"]))}
    with open(os.path.join(HERE, "scf_hydrogen_4c.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res["energies"]), res["iterations"])


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "co":
        main_co()
    else:
        main()
