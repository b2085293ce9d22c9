"""FP64 N-phase generalisation of the colour-gradient step on D2Q9, in plain
numpy (arXiv 1808.08555: Eq. 11 and the recolouring of Eq. 6 are written for
any number of fluids; Sec. 2 and the conclusions state that the model extends
to N-phase flows, but the paper simulates N = 3 only).

TEST INFRASTRUCTURE.  Only ``tests/`` may import this module.  It shares no
code with the CUDA library or with the C oracle: it is an independent
restatement, vectorised over the grid with periodic shifts (np.roll), so that
for N = 3 it cross-checks the C oracle and for N > 3 it defines the extension.

Per step, in the order of Sec. 2 (collision, recolouring, streaming):
  rho_k = sum_i f_{i,k} (after Eq. 30), phi_k = rho_k / rho
  grad phi_k by Eq. fd1
  G_kl = phi_l grad phi_k - phi_k grad phi_l (after Eq. phi_old),
  C_kl = min(1e6 rho_k rho_l / (rho_k^0 rho_l^0), 1) (Eq. 15)
  T = sum_k sum_{l != k} (sigma_kl C_kl / 2) |G_kl| (I - n_kl n_kl) (Eq. 11)
  F = div T, each component by Eq. fd1
  u = (sum_i f_i e_i + F/2) / rho (Eq. uk1); rho/nu = sum_k rho_k/nu_k,
  tau_f = 3 nu + 1/2 (Eqs. vis_1, tau)
  f^dagger_i = f_i - (f_i - f^eq_i)/tau_f + Phi_i (Eqs. 1-3, Guo's Eq. 5)
  f^ddagger_{i,k} = phi_k f^dagger_i + sum_{l != k} beta_kl w'_i (rho_k rho_l / rho) n_kl . e_i (Eq. 6)
  f_{i,k}(x + e_i) = f^ddagger_{i,k}(x) (Eq. 30)

Readings, the same as the C oracle's (three fluids) where they apply:
  * n_kl = G_kl / max(|G_kl|, normal_delta phi_k phi_l), 0 where |G_kl| <= 1e-15;
  * w'_i = w_i / |e_i| (the cosine form) or w_i (recolor_form 1);
  * beta_kl for N fluids (the paper gives Eqs. 18-20 for three only):
      beta_kl = beta^0 [1 + sum_{m != k, l} min(35 rho_k rho_l rho_m / rho^3, 1) g(X_kl^m)],
      X_kl^m = (sigma_mk^2 + sigma_ml^2 - sigma_kl^2) / (2 sigma_mk sigma_ml),
    which is Eq. 19 exactly for N = 3 (one third fluid m) and adds one
    junction term per third fluid for N > 3.  beta_form 1 is Eq. fu (beta^0).

Arrays: f (N, 9, ny, nx); rho (N, ny, nx); sigma an (N, N) symmetric matrix
with zero diagonal; tau, rho0 length N.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0
GEPS = 1e-15


@dataclass
class NParams:
    nx: int
    ny: int
    sigma: np.ndarray            # (N, N), symmetric, zero diagonal
    tau: tuple
    rho0: tuple
    beta0: float = 0.7
    beta_form: int = 0           # 0: the N-fluid reading of Eqs. 19-20 above; 1: Eq. fu
    recolor_form: int = 0        # 0: w_i / |e_i|; 1: w_i
    normal_delta: float = 0.1

    @property
    def n(self) -> int:
        return len(self.tau)


def sigma_matrix(pairs: dict, n: int) -> np.ndarray:
    """(N, N) tension matrix from {(k, l): sigma_kl} with k < l (0-based)."""
    s = np.zeros((n, n))
    for (k, l), v in pairs.items():
        s[k, l] = s[l, k] = v
    return s


def _at(v, dx, dy):
    """v(x + dx, y + dy) on the periodic grid (last two axes y, x)."""
    return np.roll(v, shift=(-dy, -dx), axis=(-2, -1))


def grad(v):
    """Eq. fd1: d_a v(x) = (1/cs2) sum_i w_i v(x + e_i) e_{i,a}."""
    gx = sum(WT[i] * EX[i] * _at(v, EX[i], EY[i]) for i in range(9)) / CS2
    gy = sum(WT[i] * EY[i] * _at(v, EX[i], EY[i]) for i in range(9)) / CS2
    return gx, gy


def g_of_X(X: float) -> float:
    """Eq. 20."""
    if X < -1.0:
        return 1.0
    if X < 0.0:
        return 1.0 - math.sin(math.acos(X))
    if X <= 1.0:
        return math.sin(math.acos(X)) - 1.0
    return -1.0


def X_of(sig: np.ndarray, k: int, l: int, m: int) -> float:
    """Eq. 18 with m the third fluid."""
    return (sig[m, k] ** 2 + sig[m, l] ** 2 - sig[k, l] ** 2) / (2.0 * sig[m, k] * sig[m, l])


def beta(p: NParams, rho: np.ndarray, k: int, l: int) -> np.ndarray:
    """beta_kl per node (see the module docstring)."""
    b = np.full(rho.shape[1:], p.beta0)
    if p.beta_form == 1:
        return b
    r = rho.sum(axis=0)
    for m in range(p.n):
        if m in (k, l):
            continue
        c = np.minimum(35.0 * rho[k] * rho[l] * rho[m] / r ** 3, 1.0)
        b = b + p.beta0 * c * g_of_X(X_of(p.sigma, k, l, m))
    return b


def feq(rho, ux, uy):
    """Eq. 3, all nine directions: (9, ny, nx)."""
    uu = ux * ux + uy * uy
    out = []
    for i in range(9):
        eu = EX[i] * ux + EY[i] * uy
        out.append(WT[i] * rho * (1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2)))
    return np.stack(out)


def guo(tau, ux, uy, Fx, Fy):
    """Eq. 5, all nine directions."""
    out = []
    for i in range(9):
        eu = EX[i] * ux + EY[i] * uy
        cx = (EX[i] - ux) / CS2 + eu / (CS2 * CS2) * EX[i]
        cy = (EY[i] - uy) / CS2 + eu / (CS2 * CS2) * EY[i]
        out.append(WT[i] * (1.0 - 1.0 / (2.0 * tau)) * (cx * Fx + cy * Fy))
    return np.stack(out)


def gradients_and_force(p: NParams, rho: np.ndarray):
    """G_kl for the ordered pairs and the interfacial force (F_x, F_y) = div T
    of Eq. 11, from the colour densities rho (N, ny, nx)."""
    N = p.n
    r = rho.sum(axis=0)
    phi = rho / r
    gp = [grad(phi[k]) for k in range(N)]
    G = {}
    for k in range(N):
        for l in range(N):
            if k != l:
                G[k, l] = (phi[l] * gp[k][0] - phi[k] * gp[l][0], phi[l] * gp[k][1] - phi[k] * gp[l][1])
    # Eq. 11 as printed: the double sum over ordered pairs with the factor 1/2
    Txx = np.zeros_like(r)
    Txy = np.zeros_like(r)
    Tyy = np.zeros_like(r)
    for (k, l), (gx, gy) in G.items():
        mag = np.sqrt(gx * gx + gy * gy)
        ok = mag > GEPS
        safe = np.where(ok, mag, 1.0)
        nxv, nyv = gx / safe, gy / safe
        C = np.minimum(1e6 * rho[k] * rho[l] / (p.rho0[k] * p.rho0[l]), 1.0)
        a = np.where(ok, p.sigma[k, l] * C / 2.0 * mag, 0.0)
        Txx += a * (1.0 - nxv * nxv)
        Txy += a * (0.0 - nxv * nyv)
        Tyy += a * (1.0 - nyv * nyv)
    dxx, _ = grad(Txx)
    dxy, dyx = grad(Txy)
    _, dyy = grad(Tyy)
    return G, dxx + dyx, dxy + dyy


def step(p: NParams, f: np.ndarray) -> np.ndarray:
    """One time step of N colour populations f (N, 9, ny, nx)."""
    N = p.n
    rho = f.sum(axis=1)
    r = rho.sum(axis=0)
    phi = rho / r
    G, Fx, Fy = gradients_and_force(p, rho)
    fi = f.sum(axis=0)
    mx = (fi * EX[:, None, None]).sum(axis=0)
    my = (fi * EY[:, None, None]).sum(axis=0)
    ux, uy = (mx + 0.5 * Fx) / r, (my + 0.5 * Fy) / r
    nu = [(t - 0.5) * CS2 for t in p.tau]
    tauf = (r / sum(rho[k] / nu[k] for k in range(N))) / CS2 + 0.5
    fdag = fi - (fi - feq(r, ux, uy)) / tauf + guo(tauf, ux, uy, Fx, Fy)
    wrec = np.array([WT[i] if (p.recolor_form == 1 or i == 0) else WT[i] / math.hypot(EX[i], EY[i])
                     for i in range(9)])
    out = np.empty_like(f)
    for k in range(N):
        v = phi[k][None] * fdag
        for l in range(N):
            if l == k:
                continue
            gx, gy = G[k, l]
            mag = np.sqrt(gx * gx + gy * gy)
            den = np.maximum(mag, p.normal_delta * phi[k] * phi[l])
            ok = mag > GEPS
            safe = np.where(ok, den, 1.0)
            amp = beta(p, rho, min(k, l), max(k, l)) * rho[k] * rho[l] / r
            for i in range(1, 9):
                en = np.where(ok, (gx * EX[i] + gy * EY[i]) / safe, 0.0)
                v[i] = v[i] + amp * wrec[i] * en
        for i in range(9):
            out[k, i] = np.roll(v[i], shift=(EY[i], EX[i]), axis=(-2, -1))   # Eq. 30
    return out


def run(p: NParams, f: np.ndarray, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        f = step(p, f)
    return f


def fields(p: NParams, f: np.ndarray) -> dict:
    """rho_k (N, ny, nx), u = (sum_i f_i e_i + F/2) / rho (Eq. uk1) and
    p = rho/3 of the post-streaming populations f."""
    rho = f.sum(axis=1)
    r = rho.sum(axis=0)
    _, Fx, Fy = gradients_and_force(p, rho)
    fi = f.sum(axis=0)
    mx = (fi * EX[:, None, None]).sum(axis=0)
    my = (fi * EY[:, None, None]).sum(axis=0)
    return {"rho": rho, "ux": (mx + 0.5 * Fx) / r, "uy": (my + 0.5 * Fy) / r, "p": r * CS2}


def init(rho: np.ndarray) -> np.ndarray:
    """Rest equilibrium per colour, f_{i,k} = w_i rho_k."""
    return WT[None, :, None, None] * rho[:, None]
