"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only (initial colour-density fields and
parameter sets).  It contains none of the lattice Boltzmann update: both the
CUDA path and the CPU oracle start from the arrays it returns.

All fields are float64 numpy arrays of shape (3, ny, nx) holding the colour
densities (rho_r, rho_g, rho_b) = (fluid 1, fluid 2, fluid 3); node (x, y) has
x fastest.  Diffuse droplet edges follow the tanh profile of Eq. 21 with the
interface width xi = 1.5831 the paper gives for beta^0 = 0.7 (Sec. 3.1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

XI = 1.5831  # Sec. 3.1, xi = 1/(6 k beta^0) with k = 0.1504, beta^0 = 0.7


def _grid(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def _edge(d: np.ndarray, xi: float = XI) -> np.ndarray:
    """0.5 + 0.5 tanh(d / xi): 1 inside (d > 0), 0 outside."""
    return 0.5 + 0.5 * np.tanh(d / xi)


def _stack(p2: np.ndarray, p3: np.ndarray) -> np.ndarray:
    p1 = np.clip(1.0 - p2 - p3, 0.0, None)
    return np.stack([p1, p2, p3]).astype(np.float64)


def two_droplets(nx: int = 64, ny: int = 64, R: float = 12.0, c2=(16.0, 32.0), c3=(48.0, 32.0),
                 xi: float = XI) -> np.ndarray:
    """Two separate static droplets (fluid 2 and fluid 3) in a fluid-1 matrix
    (Sec. 3.1 geometry; 64x64 with R = 12 by default)."""
    x, y = _grid(nx, ny)
    p2 = _edge(R - np.hypot(x - c2[0], y - c2[1]), xi)
    p3 = _edge(R - np.hypot(x - c3[0], y - c3[1]), xi)
    return _stack(p2, p3)


def compound_droplet(nx: int, ny: int, r_core: float, r_shell: float, centre=None,
                     xi: float = XI) -> np.ndarray:
    """Fluid-3 core (r <= r_core) inside a fluid-2 shell (r <= r_shell) in a
    fluid-1 matrix, tanh edges (Sec. 3.2 geometry with diffuse edges)."""
    x, y = _grid(nx, ny)
    cx, cy = centre if centre is not None else (nx / 2.0, ny / 2.0)
    r = np.hypot(x - cx, y - cy)
    core = _edge(r_core - r, xi)
    outer = _edge(r_shell - r, xi)
    return _stack(np.clip(outer - core, 0.0, None), core)


def compound_droplet_sharp(n: int, r_inner: float, r_outer: float, centre=None) -> np.ndarray:
    """Sec. 3.2 initial condition: rho = 1 of exactly one fluid per node.  The
    inner droplet is fluid 1 (r), the shell fluid 2 (g), the matrix fluid 3 (b),
    as in the Young-Laplace test."""
    x, y = _grid(n, n)
    cx, cy = centre if centre is not None else (n / 2.0, n / 2.0)
    d2 = (x - cx) ** 2 + (y - cy) ** 2
    r = (d2 <= r_inner ** 2).astype(np.float64)
    g = ((d2 > r_inner ** 2) & (d2 <= r_outer ** 2)).astype(np.float64)
    b = 1.0 - r - g
    return np.stack([r, g, b])


def touching_droplets(n: int, R: float | None = None, xi: float = XI) -> np.ndarray:
    """Two equal droplets (fluid 2 left, fluid 3 right) of radius n/6 touching
    at the centre of an n x n matrix of fluid 1 (Sec. 4.1 geometry)."""
    R = n / 6.0 if R is None else R
    x, y = _grid(n, n)
    c = n / 2.0
    p2 = _edge(R - np.hypot(x - (c - R), y - c), xi)
    p3 = _edge(R - np.hypot(x - (c + R), y - c), xi)
    return _stack(p2, p3)


def two_discs(n: int, c2, c3, R2: float, R3: float, xi: float = XI) -> np.ndarray:
    """A fluid-2 disc (centre c2, radius R2) and a fluid-3 disc (c3, R3) in
    an n x n matrix of fluid 1, tanh edges (Eq. 21)."""
    x, y = _grid(n, n)
    p2 = _edge(R2 - np.hypot(x - c2[0], y - c2[1]), xi)
    p3 = _edge(R3 - np.hypot(x - c3[0], y - c3[1]), xi)
    return _stack(p2, p3)


def case_adjoint(n: int = 256, seed: int = 1):
    """Gradient workload: the touching discs of radius n/6 (Sec. 4.1
    geometry) as the initial field, and as target the same geometry with
    each centre shifted by U(-4, 4) n/256 per axis and each radius scaled by
    U(0.9, 1.1), drawn from numpy's default_rng(seed).  Returns (rho0,
    rho_target), each (3, n, n)."""
    R = n / 6.0
    c = n / 2.0
    rng = np.random.default_rng(seed)
    d = rng.uniform(-4.0, 4.0, size=4) * (n / 256.0)
    s = rng.uniform(0.9, 1.1, size=2)
    rho0 = two_discs(n, (c - R, c), (c + R, c), R, R)
    tgt = two_discs(n, (c - R + d[0], c + d[1]), (c + R + d[2], c + d[3]), R * s[0], R * s[1])
    return rho0, tgt


def janus_droplet(n: int, R: float, xi: float = XI) -> np.ndarray:
    """One circle of radius R split on the vertical line through its centre:
    fluid 2 on the left, fluid 3 on the right, in a fluid-1 matrix."""
    x, y = _grid(n, n)
    c = n / 2.0
    drop = _edge(R - np.hypot(x - c, y - c), xi)
    left = _edge(c - x, xi)
    return _stack(drop * left, drop * (1.0 - left))


def flat_band(nx: int, ny: int, y0: float, y1: float, sharp: bool = True, xi: float = XI) -> np.ndarray:
    """Two-phase stratified band: fluid 2 for y0 <= y < y1, fluid 1 elsewhere
    (flat interfaces along x; fluid 3 absent)."""
    x, y = _grid(nx, ny)
    if sharp:
        band = ((y >= y0) & (y < y1)).astype(np.float64)
    else:
        band = _edge(np.minimum(y - y0, y1 - y), xi)
    return np.stack([1.0 - band, band, np.zeros_like(band)])


def droplet_field(nx: int, ny: int, seed: int, count: int = 6, rmin: float = 4.0, rmax: float = 10.0,
                  gap: float = 12.0, xi: float = XI) -> np.ndarray:
    """Seeded scatter of up to `count` diffuse droplets of fluid 2 or 3 in a
    fluid-1 matrix, every pair (periodic images included) at least `gap`
    lattice units apart edge to edge, so interfaces never come close.  Used to
    put interfaces across tile seams."""
    rng = np.random.default_rng(seed)
    drops = []
    for _ in range(200 * count):
        if len(drops) == count:
            break
        R = rng.uniform(rmin, rmax)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ok = 2 * R + gap <= min(nx, ny)
        for (dx, dy, dR, _) in drops:
            ddx = min(abs(cx - dx), nx - abs(cx - dx))
            ddy = min(abs(cy - dy), ny - abs(cy - dy))
            if np.hypot(ddx, ddy) < R + dR + gap:
                ok = False
                break
        if ok:
            drops.append((cx, cy, R, 1 + int(rng.integers(0, 2))))
    x, y = _grid(nx, ny)
    p = [np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))]
    for (cx, cy, R, k) in drops:
        ddx = np.minimum(np.abs(x - cx), nx - np.abs(x - cx))
        ddy = np.minimum(np.abs(y - cy), ny - np.abs(y - cy))
        p[k] = p[k] + _edge(R - np.hypot(ddx, ddy), xi)
    return _stack(p[1], p[2])


def random_fields(nx: int, ny: int, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Uniform random positive colour densities (independent per node)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(3, ny, nx))


def random_populations(nx: int, ny: int, seed: int, amp: float = 0.1) -> np.ndarray:
    """Random post-streaming populations (3, 9, ny, nx): rest equilibrium of
    random colour densities times (1 + amp * U(-1, 1)), i.e. a state away from
    equilibrium with non-zero momentum."""
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho = rng.uniform(0.05, 1.0, size=(3, ny, nx))
    f = w[None, :, None, None] * rho[:, None, :, :]
    return f * (1.0 + amp * rng.uniform(-1.0, 1.0, size=f.shape))


# ------------------------------------------------------ three dimensions
# Fields of the D3Q19 path: shape (N, nz, ny, nx), x fastest.

def spheres_3d(nx: int, ny: int, nz: int, spheres, n_fluids: int = 3, xi: float = XI) -> np.ndarray:
    """Spheres ((fluid k >= 1, (cx, cy, cz), R), ...) with tanh edges in a
    fluid-0 matrix (N, nz, ny, nx); overlapping spheres are not intended."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    p = np.zeros((n_fluids, nz, ny, nx))
    for k, (cx, cy, cz), R in spheres:
        p[k] = p[k] + _edge(R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2), xi)
    p[0] = np.clip(1.0 - p[1:].sum(axis=0), 0.0, None)
    return p


def compound_sphere(n: int, r_core: float, r_shell: float, xi: float = XI) -> np.ndarray:
    """Fluid-3 core inside a fluid-2 shell in a fluid-1 matrix on an n^3 grid
    (the compound droplet of Sec. 3.2 in three dimensions), (3, n, n, n)."""
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    r = np.sqrt((x - n / 2.0) ** 2 + (y - n / 2.0) ** 2 + (z - n / 2.0) ** 2)
    core = _edge(r_core - r, xi)
    outer = _edge(r_shell - r, xi)
    return _stack(np.clip(outer - core, 0.0, None), core)


def random_populations_3d(nx: int, ny: int, nz: int, seed: int, n_fluids: int = 3, amp: float = 0.1) -> np.ndarray:
    """Random post-streaming D3Q19 populations (N, 19, nz, ny, nx): rest
    equilibrium of random colour densities times (1 + amp * U(-1, 1))."""
    rng = np.random.default_rng(seed)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rho = rng.uniform(0.05, 1.0, size=(n_fluids, nz, ny, nx))
    f = w[None, :, None, None, None] * rho[:, None]
    return f * (1.0 + amp * rng.uniform(-1.0, 1.0, size=f.shape))


# ----------------------------------------------------------------- configs

@dataclass
class Case:
    """One simulation set-up: grid, per-fluid tau, sigmas and initial field."""

    name: str
    nx: int
    ny: int
    tau: tuple
    sigma: tuple  # (sigma_12, sigma_13, sigma_23)
    beta0: float
    steps: int
    rho: np.ndarray | None = None
    rho0: tuple = (1.0, 1.0, 1.0)


def case_two_droplets_64() -> Case:
    """64x64, two separate droplets of radius 12 whose centres are 32 apart,
    tau = 1 for all fluids, all sigma = 0.01, beta^0 = 0.7, 1000 steps."""
    return Case("two_droplets_64", 64, 64, (1.0, 1.0, 1.0), (0.01, 0.01, 0.01), 0.7, 1000,
                two_droplets(64, 64, 12.0))


# The three relaxation times give kinematic viscosities in the ratio 1:2:4
# (nu_k = (tau_k - 1/2)/3) with every tau inside [0.6, 1.1].
COMPOUND_TAU = (0.6, 0.7, 0.9)
COMPOUND_SIGMA = (0.01, 0.012, 0.005)  # (sigma_12, sigma_13, sigma_23)


def case_compound_2048(build_field: bool = True) -> Case:
    """2048x2048 compound double droplet: fluid-3 core of radius 200 inside a
    fluid-2 shell of radius 400 in a fluid-1 matrix, 20000 steps."""
    rho = compound_droplet(2048, 2048, 200.0, 400.0) if build_field else None
    return Case("compound_2048", 2048, 2048, COMPOUND_TAU, COMPOUND_SIGMA, 0.7, 20000, rho)


def case_compound_scaled(n: int = 256) -> Case:
    """The 2048^2 compound droplet scaled to n^2 (radii scaled by n/2048)."""
    s = n / 2048.0
    return Case(f"compound_{n}", n, n, COMPOUND_TAU, COMPOUND_SIGMA, 0.7, 1000,
                compound_droplet(n, n, 200.0 * s, 400.0 * s))


def sweep_instances(seed: int = 0, count: int = 64):
    """Morphology sweep: grid sizes drawn from {128,192,256,384,512} and the
    tension ratios sigma_12/sigma_23, sigma_13/sigma_23 on an 8x8 grid of
    {0.2,0.4,0.6,0.8,1.0,1.2,1.6,2.0} with sigma_23 = 0.01."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([128, 192, 256, 384, 512], size=count)
    S = [0.2, 0.4, 0.6, 0.8, 1.0, 1.2, 1.6, 2.0]
    out = []
    for j in range(count):
        a, b = S[j // 8 % 8], S[j % 8]
        s23 = 0.01
        out.append(Case(f"sweep_{j}", int(sizes[j]), int(sizes[j]), (1.0, 1.0, 1.0),
                        (a * s23, b * s23, s23), 0.7, 10000, None))
    return out
