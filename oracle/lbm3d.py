"""FP64 D3Q19 restatement of the N-fluid colour-gradient step, in plain numpy
(arXiv 1808.08555: the model of Sec. 2 is written in vector form, Eq. fd1,
Eq. 11 and the recolouring of Eq. 6 hold in any dimension; the paper
simulates two dimensions only, on D2Q9).

TEST INFRASTRUCTURE.  Only ``tests/`` may import this module.  It shares no
code with the CUDA library, with the C oracle or with ``oracle/lbmn.py``: it
is a separate restatement on the D3Q19 lattice, vectorised over the grid
with periodic shifts (np.roll).

Lattice (D3Q19, c_s^2 = 1/3): the rest vector, the six axis vectors (weight
1/18) and the twelve edge diagonals (weight 1/36), rest weight 1/3, ordered
so that directions 2m-1 and 2m are opposite (m = 1 .. 9):
    0 (0,0,0)
    1 (1,0,0)   2 (-1,0,0)   3 (0,1,0)   4 (0,-1,0)   5 (0,0,1)   6 (0,0,-1)
    7 (1,1,0)   8 (-1,-1,0)  9 (1,-1,0) 10 (-1,1,0)
   11 (1,0,1)  12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1)
   15 (0,1,1)  16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)

Per step, in the order of Sec. 2 (collision, recolouring, streaming), the
same steps as the two-dimensional model with three-component vectors:
  rho_k = sum_i f_{i,k}, phi_k = rho_k / rho
  grad phi_k by Eq. fd1, (1/c_s^2) sum_i w_i phi_k(x + e_i) e_i
  G_kl = phi_l grad phi_k - phi_k grad phi_l, C_kl of Eq. 15
  T = sum_k sum_{l != k} (sigma_kl C_kl / 2) |G_kl| (I - n_kl n_kl), I the 3x3 identity (Eq. 11)
  F_a = sum_b d_b T_ab, each derivative by Eq. fd1
  u = (sum_i f_i e_i + F/2) / rho (Eq. uk1); rho/nu = sum_k rho_k/nu_k, tau_f = 3 nu + 1/2
  f^dagger_i = f_i - (f_i - f^eq_i)/tau_f + Phi_i (Eqs. 1-3, Guo's Eq. 5)
  f^ddagger_{i,k} = phi_k f^dagger_i + sum_{l != k} beta_kl w'_i (rho_k rho_l / rho) n_kl . e_i (Eq. 6)
  f_{i,k}(x + e_i) = f^ddagger_{i,k}(x) (Eq. 30)

Readings, those of the two-dimensional oracles where they apply:
  * n_kl = G_kl / max(|G_kl|, normal_delta phi_k phi_l), 0 where |G_kl| <= 1e-15;
  * w'_i = w_i / |e_i| (the cosine form) or w_i (recolor_form 1);
  * beta_kl = beta^0 [1 + sum_{m != k, l} min(35 rho_k rho_l rho_m / rho^3, 1) g(X_kl^m)]
    (Eq. 19 for N = 3), beta_form 1 the constant beta^0 of Eq. fu.

Arrays: f (N, 19, nz, ny, nx); rho (N, nz, ny, nx); sigma (N, N) symmetric
with a zero diagonal; tau, rho0 of length N.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

E = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
])
EX, EY, EZ = E[:, 0], E[:, 1], E[:, 2]
Q = 19
WT = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
CS2 = 1.0 / 3.0
GEPS = 1e-15


@dataclass
class Params3D:
    nx: int
    ny: int
    nz: int
    sigma: np.ndarray            # (N, N), symmetric, zero diagonal
    tau: tuple
    rho0: tuple
    beta0: float = 0.7
    beta_form: int = 0           # 0: Eq. 19 (one junction term per third fluid); 1: Eq. fu
    recolor_form: int = 0        # 0: w_i / |e_i|; 1: w_i
    normal_delta: float = 0.1

    @property
    def n(self) -> int:
        return len(self.tau)


def _at(v, dx, dy, dz):
    """v(x + dx, y + dy, z + dz) on the periodic grid (last three axes z, y, x)."""
    return np.roll(v, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def grad(v):
    """Eq. fd1 on D3Q19: the three components of grad v."""
    out = []
    for a in range(3):
        acc = np.zeros_like(v)
        for i in range(1, Q):
            if E[i, a] != 0:
                acc = acc + WT[i] * E[i, a] * _at(v, EX[i], EY[i], EZ[i])
        out.append(acc / CS2)
    return out


def g_of_X(X: float) -> float:
    """Eq. 20."""
    if X < -1.0:
        return 1.0
    if X < 0.0:
        return 1.0 - math.sin(math.acos(X))
    if X <= 1.0:
        return math.sin(math.acos(X)) - 1.0
    return -1.0


def beta(p: Params3D, rho: np.ndarray, k: int, l: int) -> np.ndarray:
    """beta_kl per node (see the module docstring)."""
    b = np.full(rho.shape[1:], p.beta0)
    if p.beta_form == 1:
        return b
    s = p.sigma
    r = rho.sum(axis=0)
    for m in range(p.n):
        if m in (k, l):
            continue
        X = (s[m, k] ** 2 + s[m, l] ** 2 - s[k, l] ** 2) / (2.0 * s[m, k] * s[m, l])   # Eq. 18
        c = np.minimum(35.0 * rho[k] * rho[l] * rho[m] / r ** 3, 1.0)
        b = b + p.beta0 * c * g_of_X(X)
    return b


def feq(rho, u):
    """Eq. 3 for the nineteen directions: (19, nz, ny, nx)."""
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = []
    for i in range(Q):
        eu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2]
        out.append(WT[i] * rho * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2)))
    return np.stack(out)


def guo(tau, u, F):
    """Eq. 5: w_i (1 - 1/(2 tau)) [(e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4] . F."""
    out = []
    for i in range(Q):
        e = (EX[i], EY[i], EZ[i])
        eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2]
        s = sum(((e[a] - u[a]) / CS2 + eu / (CS2 * CS2) * e[a]) * F[a] for a in range(3))
        out.append(WT[i] * (1.0 - 1.0 / (2.0 * tau)) * s)
    return np.stack(out)


def colour_gradients_and_force(p: Params3D, rho: np.ndarray):
    """G_kl for the ordered pairs and the interfacial force F = div T of
    Eq. 11, from the colour densities rho (N, nz, ny, nx)."""
    N = p.n
    r = rho.sum(axis=0)
    phi = rho / r
    gp = [grad(phi[k]) for k in range(N)]
    G = {}
    for k in range(N):
        for l in range(N):
            if k != l:
                G[k, l] = [phi[l] * gp[k][a] - phi[k] * gp[l][a] for a in range(3)]
    # Eq. 11: the double sum over ordered pairs with the factor 1/2
    T = [[np.zeros_like(r) for _ in range(3)] for _ in range(3)]
    for (k, l), g in G.items():
        mag = np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
        ok = mag > GEPS
        safe = np.where(ok, mag, 1.0)
        n = [g[a] / safe for a in range(3)]
        C = np.minimum(1e6 * rho[k] * rho[l] / (p.rho0[k] * p.rho0[l]), 1.0)
        amp = np.where(ok, p.sigma[k, l] * C / 2.0 * mag, 0.0)
        for a in range(3):
            for b in range(3):
                T[a][b] = T[a][b] + amp * ((1.0 if a == b else 0.0) - n[a] * n[b])
    F = []
    for a in range(3):
        Fa = np.zeros_like(r)
        for b in range(3):
            Fa = Fa + grad(T[a][b])[b]
        F.append(Fa)
    return G, F


def step(p: Params3D, f: np.ndarray) -> np.ndarray:
    """One time step of N colour populations f (N, 19, nz, ny, nx)."""
    N = p.n
    rho = f.sum(axis=1)
    r = rho.sum(axis=0)
    phi = rho / r
    G, F = colour_gradients_and_force(p, rho)
    fi = f.sum(axis=0)
    m = [(fi * E[:, a, None, None, None]).sum(axis=0) for a in range(3)]
    u = [(m[a] + 0.5 * F[a]) / r for a in range(3)]
    nu = [(t - 0.5) * CS2 for t in p.tau]
    tauf = (r / sum(rho[k] / nu[k] for k in range(N))) / CS2 + 0.5
    fdag = fi - (fi - feq(r, u)) / tauf + guo(tauf, u, F)
    norm_e = np.sqrt((E * E).sum(axis=1))
    wrec = np.array([WT[i] if (p.recolor_form == 1 or i == 0) else WT[i] / norm_e[i] for i in range(Q)])
    out = np.empty_like(f)
    for k in range(N):
        v = phi[k][None] * fdag
        for l in range(N):
            if l == k:
                continue
            g = G[k, l]
            mag = np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
            den = np.maximum(mag, p.normal_delta * phi[k] * phi[l])
            ok = mag > GEPS
            safe = np.where(ok, den, 1.0)
            amp = beta(p, rho, min(k, l), max(k, l)) * rho[k] * rho[l] / r
            for i in range(1, Q):
                en = np.where(ok, (g[0] * EX[i] + g[1] * EY[i] + g[2] * EZ[i]) / safe, 0.0)
                v[i] = v[i] + amp * wrec[i] * en
        for i in range(Q):
            out[k, i] = np.roll(v[i], shift=(EZ[i], EY[i], EX[i]), axis=(-3, -2, -1))   # Eq. 30
    return out


def run(p: Params3D, f: np.ndarray, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        f = step(p, f)
    return f


def init(rho: np.ndarray) -> np.ndarray:
    """Rest equilibrium per colour, f_{i,k} = w_i rho_k."""
    return WT[None, :, None, None, None] * rho[:, None]


def pressure(f: np.ndarray) -> np.ndarray:
    """Lattice pressure c_s^2 rho per node."""
    return CS2 * f.sum(axis=(0, 1))


def fields(p: Params3D, f: np.ndarray) -> dict:
    """rho_k (N, nz, ny, nx), u (3, nz, ny, nx) with the F/2 correction of
    Eq. uk1, and p = c_s^2 rho, of the post-streaming populations f."""
    rho = f.sum(axis=1)
    r = rho.sum(axis=0)
    _, F = colour_gradients_and_force(p, rho)
    fi = f.sum(axis=0)
    u = np.stack([((fi * E[:, a, None, None, None]).sum(axis=0) + 0.5 * F[a]) / r for a in range(3)])
    return {"rho": rho, "u": u, "p": CS2 * r}
