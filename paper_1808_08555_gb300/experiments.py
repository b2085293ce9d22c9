"""Drivers of the paper's validation experiments on the GPU library.

Each driver sets up one of the paper's test cases from ``workloads``, runs it
with ``lbm3`` (the CUDA path) and reduces the result with ``analysis`` to the
quantity the paper tabulates.
"""
from __future__ import annotations

import math

import numpy as np

from . import analysis as A
from . import lbm3 as L
from . import workloads as W


def young_laplace_compound(R_r: float, force_form: int = L.FORCE_BODY, steps: int = 20000, n: int = 160,
                           sigma: float = 0.01, nu: float = 0.1) -> dict:
    """Sec. 3.2 (Tabs. 1 and 2): a compound droplet -- red core of radius
    R_r inside a green shell of radius R_g = 2 R_r, in blue -- centred in an
    n x n periodic box from the sharp initial condition, all three tensions
    sigma and viscosities nu, relaxed for `steps` steps.

    Returns the Young-Laplace error eps of Eq. 22 (with the equilibrium radii
    taken from the areas of the red and red+green regions), the two pressure
    jumps, and the largest spurious speed |u|max (Tab. 2)."""
    tau = 3.0 * nu + 0.5
    p = L.Params(n, n, tau=(tau, tau, tau), sigma=(sigma, sigma, sigma), force_form=force_form)
    sim = L.Simulation(p)
    sim.init(W.compound_droplet_sharp(n, R_r, 2.0 * R_r))
    sim.step(steps)
    fl = sim.fields()
    sim.close()
    rho = fl["rho"]
    phi = rho / rho.sum(axis=0)
    R_r_eq = math.sqrt(phi[0].sum() / math.pi)
    R_g_eq = math.sqrt((phi[0].sum() + phi[1].sum()) / math.pi)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2.0, y - n / 2.0)
    w = 4.0 * W.XI
    pr = fl["p"]
    p_r = pr[r < R_r_eq - w].mean()
    p_g = pr[(r > R_r_eq + w) & (r < R_g_eq - w)].mean()
    p_b = pr[r > R_g_eq + w].mean()
    dp_rg, dp_gb = p_r - p_g, p_g - p_b
    umax = float(np.hypot(fl["ux"], fl["uy"]).max())
    return {"R_r": R_r, "force_form": force_form, "steps": steps, "R_r_eq": R_r_eq, "R_g_eq": R_g_eq,
            "dp_rg": float(dp_rg), "dp_gb": float(dp_gb),
            "eps": A.laplace_error(dp_gb, R_g_eq, dp_rg, R_r_eq, sigma, sigma), "umax": umax}
