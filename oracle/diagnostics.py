"""FP64 interface diagnostics of colour-fraction fields: contact angles at the
three-phase junctions (Eq. theta_kl, Sec. 2) and pressure jumps (Eq. 22).

TEST INFRASTRUCTURE.  Only ``tests/``, ``tests/golden/`` scripts and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library, whose own FP64 device diagnostic implements the same
definition independently.

Definition of the measurement (the paper gives none):

* Interface points of the pair (k, l), with m the third colour: on every
  lattice link (x, y)-(x+1, y) and (x, y)-(x, y+1) inside the grid (links
  across the periodic edges are not used) where phi_k, phi_l > 0 at both
  ends, s = ln(phi_k / phi_l) changes sign (s > 0 at one end, s <= 0 at the
  other) and phi_m < third_max at both ends, the point where the linear
  interpolant of s vanishes.  Across the tanh profile of Eq. 21,
  ln(phi_k / phi_l) is linear in the distance to the interface, so the point
  is exact there (interpolating phi_k - phi_l instead is off by up to 0.012
  lattice units).  Coordinates are taken relative to the grid centre
  (nx/2, ny/2).
* Each pair's points are fitted by the circle minimising
  sum (x^2 + y^2 + D x + E y + F)^2 (the algebraic, Kasa, fit): centre
  (-D/2, -E/2), radius sqrt(D^2/4 + E^2/4 - F).
* Junctions: the two intersections of the 1-2 and 1-3 circles; each
  intersection of the 1-2/2-3 and the 1-3/2-3 circles is assigned to the
  nearer of those two, and each junction is the mean of its three points.
* At a junction J every circle gives a line (its tangent at J).  Taking
  one direction r_kl on each line such that no half-plane holds all three
  (the only configuration in which tensions can balance, as in the Neumann
  triangle of Eq. theta_kl), the angle inside fluid m between the interfaces
  k-m and l-m is acos(r_km . r_lm), and the paper's contact angle is
  varphi_kl = pi - (that angle).  The two junctions are averaged.

phi arrays are (3, ny, nx), float64, colours (r, g, b) = fluids (1, 2, 3).
"""
from __future__ import annotations

import math

import numpy as np

PAIRS = ((0, 1), (0, 2), (1, 2))


def interface_points(phi: np.ndarray, k: int, l: int, third_max: float = 1e-3) -> np.ndarray:
    """(n, 2) interface points of the k-l pair (see the module docstring)."""
    m = 3 - k - l
    ny, nx = phi.shape[1:]
    pos = (phi[k] > 0) & (phi[l] > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(pos, np.log(np.where(pos, phi[k], 1.0) / np.where(pos, phi[l], 1.0)), 0.0)
    pts = []
    for axis in (1, 0):  # links along x, then along y
        if axis == 1:
            sa, sb = s[:, :-1], s[:, 1:]
            ma, mb = phi[m][:, :-1], phi[m][:, 1:]
            ok = pos[:, :-1] & pos[:, 1:]
        else:
            sa, sb = s[:-1, :], s[1:, :]
            ma, mb = phi[m][:-1, :], phi[m][1:, :]
            ok = pos[:-1, :] & pos[1:, :]
        cross = ok & ((sa > 0) != (sb > 0)) & (ma < third_max) & (mb < third_max)
        ys, xs = np.nonzero(cross)
        t = sa[ys, xs] / (sa[ys, xs] - sb[ys, xs])
        if axis == 1:
            px, py = xs + t, ys.astype(float)
        else:
            px, py = xs.astype(float), ys + t
        pts.append(np.stack([px - nx / 2.0, py - ny / 2.0], axis=1))
    return np.concatenate(pts, axis=0)


def fit_circle(pts: np.ndarray) -> tuple[float, float, float]:
    """Algebraic least-squares circle (cx, cy, R) through points (n, 2),
    solved as a linear least-squares problem in (D, E, F)."""
    if len(pts) < 3:
        raise ValueError("fewer than three interface points")
    x, y = pts[:, 0], pts[:, 1]
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    b = -(x * x + y * y)
    (D, E, F), *_ = np.linalg.lstsq(A, b, rcond=None)
    cx, cy = -D / 2.0, -E / 2.0
    return float(cx), float(cy), float(math.sqrt(cx * cx + cy * cy - F))


def circle_intersections(c1, c2) -> list[np.ndarray]:
    """Intersection points of two circles (cx, cy, R); empty if none."""
    (x1, y1, r1), (x2, y2, r2) = c1, c2
    d = math.hypot(x2 - x1, y2 - y1)
    if d == 0.0 or d > r1 + r2 or d < abs(r1 - r2):
        return []
    a = (r1 * r1 - r2 * r2 + d * d) / (2.0 * d)
    h = math.sqrt(max(r1 * r1 - a * a, 0.0))
    ux, uy = (x2 - x1) / d, (y2 - y1) / d
    bx, by = x1 + a * ux, y1 + a * uy
    return [np.array([bx - h * uy, by + h * ux]), np.array([bx + h * uy, by - h * ux])]


def _balanced_rays(lines: list[np.ndarray]) -> list[np.ndarray]:
    """One direction on each of three lines through a point such that no
    half-plane contains all three rays."""
    for s2 in (1.0, -1.0):
        for s3 in (1.0, -1.0):
            rays = [lines[0], s2 * lines[1], s3 * lines[2]]
            ang = sorted(math.atan2(r[1], r[0]) for r in rays)
            gaps = [ang[1] - ang[0], ang[2] - ang[1], 2.0 * math.pi - (ang[2] - ang[0])]
            if max(gaps) < math.pi:
                return rays
    raise ValueError("the three interfaces do not surround the junction")


def contact_angles(phi: np.ndarray, third_max: float = 1e-3) -> dict:
    """Contact angles varphi_kl (degrees, pairs 12, 13, 23) of a droplet with
    two three-phase junctions, plus the fitted circles and junctions."""
    ny, nx = phi.shape[1:]
    circ = [fit_circle(interface_points(phi, k, l, third_max)) for (k, l) in PAIRS]
    J = circle_intersections(circ[0], circ[1])
    if len(J) != 2:
        raise ValueError("the 1-2 and 1-3 circles do not intersect")
    groups = [[J[0]], [J[1]]]
    for a, b in ((0, 2), (1, 2)):
        for p in circle_intersections(circ[a], circ[b]):
            j = int(np.argmin([np.hypot(*(p - J[0])), np.hypot(*(p - J[1]))]))
            groups[j].append(p)
    per_junction = []
    junctions = []
    for g in groups:
        Jc = np.mean(g, axis=0)
        junctions.append((float(Jc[0] + nx / 2.0), float(Jc[1] + ny / 2.0)))
        lines = []
        for (cx, cy, _) in circ:
            v = np.array([-(Jc[1] - cy), Jc[0] - cx])
            lines.append(v / np.hypot(*v))
        r12, r13, r23 = _balanced_rays(lines)
        theta = {1: math.acos(np.clip(r12 @ r13, -1, 1)),   # inside fluid 1
                 2: math.acos(np.clip(r12 @ r23, -1, 1)),   # inside fluid 2
                 3: math.acos(np.clip(r13 @ r23, -1, 1))}   # inside fluid 3
        per_junction.append([180.0 - math.degrees(theta[3]),    # varphi_12
                             180.0 - math.degrees(theta[2]),    # varphi_13
                             180.0 - math.degrees(theta[1])])   # varphi_23
    ang = np.mean(per_junction, axis=0)
    return {"varphi": [float(a) for a in ang], "per_junction": per_junction,
            "circles": [(c[0] + nx / 2.0, c[1] + ny / 2.0, c[2]) for c in circ], "junctions": junctions}


def neumann_angles(sigma) -> list[float]:
    """varphi_kl of Eq. theta_kl (degrees, pairs 12, 13, 23)."""
    s12, s13, s23 = sigma
    sig = {(0, 1): s12, (0, 2): s13, (1, 2): s23}
    out = []
    for (k, l) in PAIRS:
        m = 3 - k - l
        smk, sml, skl = sig[tuple(sorted((m, k)))], sig[tuple(sorted((m, l)))], sig[(k, l)]
        out.append(math.degrees(math.acos((smk ** 2 + sml ** 2 - skl ** 2) / (2 * smk * sml))))
    return out


def bulk_pressure(phi: np.ndarray, p: np.ndarray, k: int, bulk_min: float = 0.99) -> float:
    """Mean pressure over the nodes where fluid k is in bulk (phi_k > bulk_min)."""
    sel = phi[k] > bulk_min
    if not sel.any():
        raise ValueError(f"no bulk nodes of fluid {k + 1}")
    return float(p[sel].mean())
