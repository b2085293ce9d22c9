"""Analytic geometry and diagnostics of the paper's test cases (Secs. 3-4).

These are closed forms the paper uses to assess its simulations: Neumann
contact angles, the liquid lens, general and perfect Janus droplets, and the
Young-Laplace error of a compound droplet, plus a pressure-jump helper for
fields read back from the library.  Plain numpy, no part of the time step.
"""
from __future__ import annotations

import math

import numpy as np


def neumann_angles(s12: float, s13: float, s23: float) -> tuple[float, float, float]:
    """Eq. theta_kl: contact angles (phi_12, phi_13, phi_23) in radians; the
    angle phi_kl sits opposite sigma_kl in Neumann's triangle."""
    def ang(skl, smk, sml):
        return math.acos((smk * smk + sml * sml - skl * skl) / (2.0 * smk * sml))
    return ang(s12, s13, s23), ang(s13, s12, s23), ang(s23, s12, s13)


def lens_geometry(area: float, theta1: float, theta2: float) -> tuple[float, float, float]:
    """Eq. 23: length D and heights h1, h2 of a liquid lens of area A with
    contact angles theta1 = phi_rg and theta2 = phi_rb."""
    s = sum((t / math.sin(t) - math.cos(t)) / math.sin(t) for t in (theta1, theta2))
    D = 2.0 * math.sqrt(area / s)
    h = [D / 2.0 * (1.0 - math.cos(t)) / math.sin(t) for t in (theta1, theta2)]
    return D, h[0], h[1]


def gjd_geometry(R_r: float, R_g: float, R_b: float, d_rg: float, sigma_rg: float = 0.01) -> dict:
    """Eqs. gjd_01-06: a general Janus droplet from the radii of its rb, gb
    and rg interfaces (R_r, R_g, R_b) and the centre distance d_rg.  Returns
    the half central angles, d_gb, the junction angles and the two remaining
    tensions (law of sines with the given sigma_rg)."""
    tg = math.acos((R_g * R_g + d_rg * d_rg - R_r * R_r) / (2.0 * R_g * d_rg))   # Eq. gjd_01
    half_chord = R_g * math.sin(tg)                                              # Eq. gjd_02
    tb = math.asin(half_chord / R_b)
    xc = R_g * math.cos(tg)            # chord AB measured from O_g along the centre line
    tr = math.acos(min(1.0, abs(xc - d_rg) / R_r))
    d_gb = xc + R_b * math.cos(tb)     # Eq. gjd_03
    if xc < d_gb and xc >= d_rg:       # Eq. gjd_04
        p_rb = math.pi / 2.0 - tr + tg
        p_gb = math.pi - tr - tb
    else:                              # Eq. gjd_05
        p_rb = tb + tg
        p_gb = tr - tb
    p_rg = math.pi - p_rb - p_gb
    k = sigma_rg / math.sin(p_rg)      # Eq. gjd_06
    return {"theta_g": tg, "theta_r": tr, "theta_b": tb, "d_gb": d_gb, "phi_rb": p_rb, "phi_gb": p_gb,
            "phi_rg": p_rg, "sigma_gb": k * math.sin(p_gb), "sigma_rb": k * math.sin(p_rb)}


def pjd_geometry(R: float, area_fraction: float) -> dict:
    """Eq. pjd: a perfect Janus droplet of radius R = R_g = R_r whose red part
    is the given fraction of its area; solves the area equation for theta_g
    (bisection) and returns theta_g, R_b and d_gb."""
    def frac(t):
        sc = math.sin(t) * math.cos(t)
        return (t - sc + math.tan(t) ** 2 * (math.pi / 2.0 - t - sc)) / math.pi

    lo, hi = 1e-9, math.pi / 2.0 - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if frac(mid) < area_fraction:
            lo = mid
        else:
            hi = mid
    tg = 0.5 * (lo + hi)
    R_b = R * math.tan(tg)
    tb = math.asin(R * math.sin(tg) / R_b)
    return {"theta_g": tg, "R_b": R_b, "theta_b": tb, "d_gb": R * math.cos(tg) + R_b * math.cos(tb)}


def laplace_error(dp_gb: float, R_g: float, dp_rg: float, R_r: float, sigma_gb: float, sigma_rg: float) -> float:
    """Eq. 22: relative error of the two Laplace jumps of a compound droplet."""
    return abs(dp_gb * R_g + dp_rg * R_r - (sigma_gb + sigma_rg)) / (sigma_gb + sigma_rg)


def pressure_jump(p: np.ndarray, centre, r_in: float, r_out: float) -> float:
    """Mean pressure inside radius r_in minus mean pressure beyond r_out."""
    ny, nx = p.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - centre[0], y - centre[1])
    return float(p[r < r_in].mean() - p[r > r_out].mean())
