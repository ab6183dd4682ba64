"""Coated-sphere experiment of Sec. 6.2: PCG iterations against grid size and phase contrast.

A centred core (radius r1 = 0.2) with a coating (outer radius r2 = 0.4) in a cubic cell of edge 1,
trilinear hexahedra, macroscopic strain e = [1, 0, 0, 0, 0, 0], stopping tolerance 1e-6.  The core
and coating bulk moduli are balanced for a contrast rho = K2 / K1 so that the coated sphere is
neutral in the surrounding matrix of bulk modulus K_eff = 1; every phase has G / K = 0.6 as in the
printed parameters (K1, K2, K_eff = 0.0013206, 1.3206033, 1.0; G1, G2, G_eff = 0.00079236, 0.7923620,
0.6 at rho = 1e3).  Two reference materials are compared (Sec. 6.2): the symmetrised identity I_s
(the 6 x 6 identity in Mandel form) and the volume mean C_mean.

The balance is the neutral-inclusion condition of a coated sphere (Hashin): with core volume
fraction f = (r1 / r2)^3 inside the coated sphere,
    K_eff = K2 + f (K1 - K2) / (1 + (1 - f)(K1 - K2) / (K2 + 4/3 G2)),
solved for K2 with K1 = K2 / rho and G2 = 0.6 K2.

Usage: ``python -m paper_2203_02962_gb300.coated_sphere --sizes 16 32 64 128`` (needs the GPU
library); prints one JSON line per (grid, contrast, reference) with the PCG iteration count.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs

R1, R2, G_OVER_K, K_EFF = 0.2, 0.4, 0.6, 1.0


def balanced_moduli(rho: float):
    """(K1, G1), (K2, G2), (K_eff, G_eff) of core, coating and matrix for contrast rho = K2 / K1."""
    f = (R1 / R2) ** 3
    # K_eff = K2 * phi(rho) with phi independent of the scale of K2 (all moduli scale together)
    d = 1.0 / rho - 1.0                                  # (K1 - K2) / K2
    phi = 1.0 + f * d / (1.0 + (1.0 - f) * d / (1.0 + 4.0 / 3.0 * G_OVER_K))
    K2 = K_EFF / phi
    K1 = K2 / rho
    return (K1, G_OVER_K * K1), (K2, G_OVER_K * K2), (K_EFF, G_OVER_K * K_EFF)


def phase_moduli(rho: float):
    """Mandel stiffness matrices of core (id 0), coating (id 1) and matrix (id 2)."""
    return np.stack([inputs.bulk_shear_mandel(K, G) for K, G in balanced_moduli(rho)])


def run(sizes, contrasts, tol=1e-6, precision="fp64"):
    from . import fehom
    rows = []
    e = np.array([[1.0, 0, 0, 0, 0, 0]])
    for n in sizes:
        ids = inputs.coated_sphere(n, R1, R2)
        for rho in contrasts:
            mod = phase_moduli(rho)
            for ref_name in ("I_s", "C_mean"):
                ref = np.eye(6) if ref_name == "I_s" else None
                s = fehom.Solver("hex8_3d", "elastic", (n, n, n), ids, mod, ref_material=ref, precision=precision,
                                 max_iter=20000)
                s.precond_build()
                out = s.solve(e, tol=tol, fields=None, raise_on_failure=False)
                info = out["info"][0]
                rows.append(dict(n=n, rho=rho, ref=ref_name, iterations=info["iterations"],
                                 converged=bool(info["converged"]), sigma_11=float(out["mean_flux"][0][0])))
                s.close()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sizes", type=int, nargs="+", default=[16, 32, 64, 128])
    ap.add_argument("--contrasts", type=float, nargs="+", default=[1e-3, 1e-2, 1e-1, 1e1, 1e2, 1e3])
    ap.add_argument("--tol", type=float, default=1e-6)
    args = ap.parse_args()
    for r in run(args.sizes, args.contrasts, args.tol):
        print(json.dumps(r))


if __name__ == "__main__":
    main()
