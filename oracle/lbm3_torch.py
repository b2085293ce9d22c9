"""Differentiable FP64 restatement of the ternary colour-gradient step
(arXiv 1808.08555, Sec. 2), in plain PyTorch CPU tensor operations.

TEST INFRASTRUCTURE.  It exists to give exact reference gradients (through
torch.autograd) for the library's hand-written reverse mode; only the tests
may import it.  It shares nothing with the CUDA library.  Its forward is the
same computation as ``lbm3_oracle.c`` -- the same readings of the paper (the
recolouring normal G / max(|G|, normal_delta phi_k phi_l), the 1e-15 tension cutoff, the derivatives of
Eq. fd1 applied twice, the local tau_f in BGK and Guo terms) -- and the tests
pin it to that oracle and its gradients to central differences of that oracle.

Conventions as in ``oracle``: f has shape (3, 9, ny, nx) and holds the
post-streaming populations f_{i,k}(x, t); sigma = (sigma_12, sigma_13,
sigma_23) is a tensor, so gradients with respect to it flow through both the
interfacial force (Eq. 11) and the segregation parameters (Eqs. 18-20).
"""
from __future__ import annotations

import math

import torch
from torch.utils.checkpoint import checkpoint

EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
WT = (4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36)
CS2 = 1.0 / 3.0
GEPS = 1e-15      # |G| at or below which the tension term is 0
PAIRS = ((0, 1), (0, 2), (1, 2))


def _at(v, dx, dy):
    """v(x + dx, y + dy) on the periodic grid (last two axes are y, x)."""
    return torch.roll(v, shifts=(-dy, -dx), dims=(-2, -1))


def grad(v):
    """Eq. fd1: d_a v(x) = (1/cs2) sum_i w_i v(x + e_i) e_{i,a}."""
    gx = sum(WT[i] * EX[i] * _at(v, EX[i], EY[i]) for i in range(9) if EX[i]) / CS2
    gy = sum(WT[i] * EY[i] * _at(v, EX[i], EY[i]) for i in range(9) if EY[i]) / CS2
    return gx, gy


def sig_kl(sigma, k, l):
    a, b = min(k, l), max(k, l)
    return sigma[PAIRS.index((a, b))]


def X_of(sigma):
    """Eq. 18: X_kl = (s_mk^2 + s_ml^2 - s_kl^2) / (2 s_mk s_ml), m the third fluid."""
    out = []
    for k, l in PAIRS:
        m = 3 - k - l
        smk, sml, skl = sig_kl(sigma, m, k), sig_kl(sigma, m, l), sig_kl(sigma, k, l)
        out.append((smk * smk + sml * sml - skl * skl) / (2 * smk * sml))
    return out


def g_of(X):
    """Eq. 20 with sin(arccos X) = sqrt(1 - X^2) on [-1, 1]."""
    one = torch.ones_like(X)
    inside = (X >= -1) & (X <= 1)
    s = torch.sqrt(torch.where(inside, 1 - X * X, one))
    return torch.where(X < -1, one, torch.where(X < 0, 1 - s, torch.where(X <= 1, s - 1, -one)))


def beta(prm, sigma, rk):
    """Segregation parameters of the pairs (12, 13, 23) per node: form 0 =
    Eqs. 19-20, 1 = Eq. fu (constant), 2 = Eq. 16, 3 = Eq. 17; forms 2 and 3
    fall back to beta^0 without a Neumann triangle."""
    b0 = prm["beta0"]
    r = rk[0] + rk[1] + rk[2]
    prod = rk[0] * rk[1] * rk[2] / r ** 3
    X = X_of(sigma)
    tri = all(abs(float(x.detach())) < 1 for x in X)
    form = prm.get("beta_form", 0)
    const = [b0 * torch.ones_like(r)] * 3
    if form == 1 or (form in (2, 3) and not tri):
        return const
    if form == 0:
        c = torch.clamp(35.0 * prod, max=1.0)
        return [b0 + b0 * c * g_of(x) for x in X]
    ang = [torch.acos(x) for x in X]
    if form == 2:
        return [const[0], b0 * (1 + 27.0 * prod * (torch.sin(ang[2]) - 1)),
                b0 * (1 + 27.0 * prod * (torch.sin(ang[1]) - 1))]
    c = torch.clamp(35.0 * prod, max=1.0)
    qm = max(range(3), key=lambda q: float(ang[q].detach()))
    return [const[q] if q == qm else b0 + b0 * c * (torch.sin(math.pi - ang[qm] - ang[q]) - 1) for q in range(3)]


def step(prm, f, sigma):
    """One step (Sec. 2): collision with the Guo force, recolouring (Eq. 6),
    streaming (Eq. 30).  prm: dict with tau, rho0, beta0, beta_form,
    recolor_form and optionally normal_delta (the recolouring normal
    G / max(|G|, normal_delta phi_k phi_l); 0.1 if absent, 0 = G/|G|)."""
    rk = f.sum(dim=1)                                   # rho_k = sum_i f_{i,k}
    r = rk.sum(dim=0)
    phi = rk / r
    gp = [grad(phi[k]) for k in range(3)]
    G = {}
    for k in range(3):
        for l in range(3):
            if k != l:
                G[k, l] = (phi[l] * gp[k][0] - phi[k] * gp[l][0], phi[l] * gp[k][1] - phi[k] * gp[l][1])
    # Eq. 11, double sum over ordered pairs with the factor 1/2; C_kl of Eq. 15
    Txx = Txy = Tyy = torch.zeros_like(r)
    for (k, l), (gx, gy) in G.items():
        g2 = gx * gx + gy * gy
        ok = g2 > GEPS * GEPS
        mag = torch.sqrt(torch.where(ok, g2, torch.ones_like(g2)))
        C = torch.clamp(1e6 * rk[k] * rk[l] / (prm["rho0"][k] * prm["rho0"][l]), max=1.0)
        a = sig_kl(sigma, k, l) * C / 2 * mag
        nxv, nyv = gx / mag, gy / mag
        zero = torch.zeros_like(g2)
        Txx = Txx + torch.where(ok, a * (1 - nxv * nxv), zero)
        Txy = Txy + torch.where(ok, a * (0 - nxv * nyv), zero)
        Tyy = Tyy + torch.where(ok, a * (1 - nyv * nyv), zero)
    dxx, _ = grad(Txx)
    dxy, dyx = grad(Txy)
    _, dyy = grad(Tyy)
    Fx, Fy = dxx + dyx, dxy + dyy
    # Eqs. uk1, vis_1, tau
    fi = f.sum(dim=0)
    mx = sum(EX[i] * fi[i] for i in range(9) if EX[i])
    my = sum(EY[i] * fi[i] for i in range(9) if EY[i])
    ux, uy = (mx + 0.5 * Fx) / r, (my + 0.5 * Fy) / r
    nu = [(t - 0.5) * CS2 for t in prm["tau"]]
    tauf = (r / sum(rk[k] / nu[k] for k in range(3))) / CS2 + 0.5
    uu = ux * ux + uy * uy
    fdag = []
    for i in range(9):
        eu = EX[i] * ux + EY[i] * uy
        feq = WT[i] * r * (1 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2))      # Eq. 3
        cx = (EX[i] - ux) / CS2 + eu / (CS2 * CS2) * EX[i]
        cy = (EY[i] - uy) / CS2 + eu / (CS2 * CS2) * EY[i]
        Phi = WT[i] * (1 - 1 / (2 * tauf)) * (cx * Fx + cy * Fy)                         # Eq. 5
        fdag.append(fi[i] - (fi[i] - feq) / tauf + Phi)                                   # Eqs. 1, 2
    # Eq. 6 with the normal G / max(|G|, normal_delta phi_k phi_l)
    bq = beta(prm, sigma, rk)
    form = prm.get("recolor_form", 0)
    out = []
    for k in range(3):
        row = []
        for i in range(9):
            v = phi[k] * fdag[i]
            for l in range(3):
                if l == k:
                    continue
                gx, gy = G[k, l]
                g2 = gx * gx + gy * gy
                ok = g2 > GEPS * GEPS      # no k-l interface at or below the cutoff: n = 0
                mag = torch.sqrt(torch.where(ok, g2, torch.ones_like(g2)))
                den = torch.maximum(mag, prm.get("normal_delta", 0.1) * phi[k] * phi[l])
                dsafe = torch.where(ok, den, torch.ones_like(den))
                en = (gx * EX[i] + gy * EY[i]) / dsafe
                if form == 0 and i != 0:
                    en = en / math.sqrt(EX[i] ** 2 + EY[i] ** 2)
                q = PAIRS.index((min(k, l), max(k, l)))
                v = v + torch.where(ok, bq[q] * WT[i] * rk[k] * rk[l] / r * en, torch.zeros_like(en))
            row.append(torch.roll(v, shifts=(EY[i], EX[i]), dims=(-2, -1)))   # Eq. 30
        out.append(torch.stack(row))
    return torch.stack(out)


def init(rho):
    """Rest equilibrium f_{i,k} = w_i rho_k (rho: (3, ny, nx))."""
    return torch.stack([torch.stack([WT[i] * rho[k] for i in range(9)]) for k in range(3)])


def phi_of(f):
    """Colour fractions phi_k = rho_k / rho of a post-streaming state."""
    rk = f.sum(dim=1)
    return rk / rk.sum(dim=0)


def run(prm, f, sigma, nsteps, chunk=0):
    """nsteps steps from f; chunk > 0 recomputes chunks of that many steps in
    the backward pass instead of keeping every intermediate."""
    if chunk <= 0:
        for _ in range(nsteps):
            f = step(prm, f, sigma)
        return f

    def seg(f, sigma, n):
        for _ in range(n):
            f = step(prm, f, sigma)
        return f

    done = 0
    while done < nsteps:
        n = min(chunk, nsteps - done)
        f = checkpoint(seg, f, sigma, n, use_reentrant=False)
        done += n
    return f
