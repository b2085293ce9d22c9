"""Pins of the N-phase restatement (oracle.lbmn), CPU only.

Eq. 11 and Eq. 6 are written for any number of fluids; the paper simulates
three.  The restatement is pinned (1) to the C oracle at N = 3, an
independent implementation (numpy with periodic shifts against C loops),
(2) by its exact reduction: an absent fourth fluid changes nothing, bit for
bit, (3) by per-colour mass and total momentum conservation for N = 4 and 5,
and (4) by the Laplace law on every interface of a four-fluid nested
droplet (Eq. laplace), each with its own tension."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lbmn as N
from paper_1808_08555_gb300 import workloads as W

SIG3 = (0.01, 0.013, 0.007)


def _p3(nx, ny, **kw):
    s = N.sigma_matrix({(0, 1): SIG3[0], (0, 2): SIG3[1], (1, 2): SIG3[2]}, 3)
    return N.NParams(nx, ny, sigma=s, tau=(0.6, 0.9, 1.3), rho0=(1.0, 1.0, 1.0), **kw)


@pytest.mark.parametrize("beta_form", [0, 1])
@pytest.mark.parametrize("recolor_form", [0, 1])
@pytest.mark.parametrize("delta", [0.1, 0.0])
def test_three_fluids_equal_c_oracle(beta_form, recolor_form, delta):
    nx, ny = 16, 12
    f = W.random_populations(nx, ny, seed=4)
    op = O.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=SIG3, beta_form=beta_form, recolor_form=recolor_form,
                  normal_delta=delta)
    a = O.step(op, f, 5)
    b = N.run(_p3(nx, ny, beta_form=beta_form, recolor_form=recolor_form, normal_delta=delta), f.copy(), 5)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_absent_fourth_fluid_changes_nothing():
    nx, ny = 16, 12
    f3 = W.random_populations(nx, ny, seed=7)
    f4 = np.concatenate([f3, np.zeros((1,) + f3.shape[1:])])
    s4 = N.sigma_matrix({(0, 1): SIG3[0], (0, 2): SIG3[1], (1, 2): SIG3[2], (0, 3): 0.011, (1, 3): 0.009,
                         (2, 3): 0.012}, 4)
    p4 = N.NParams(nx, ny, sigma=s4, tau=(0.6, 0.9, 1.3, 0.8), rho0=(1.0, 1.0, 1.0, 1.0))
    a = N.run(_p3(nx, ny), f3.copy(), 6)
    b = N.run(p4, f4, 6)
    assert np.array_equal(a, b[:3]) and not b[3].any()


@pytest.mark.parametrize("n_fluids", [4, 5])
def test_mass_and_momentum_conserved(n_fluids):
    nx, ny = 20, 16
    rng = np.random.default_rng(n_fluids)
    rho = rng.uniform(0.05, 1.0, (n_fluids, ny, nx))
    f = N.init(rho) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, (n_fluids, 9, ny, nx)))
    pairs = {(k, l): 0.006 + 0.001 * (k + 2 * l) for k in range(n_fluids) for l in range(k + 1, n_fluids)}
    p = N.NParams(nx, ny, sigma=N.sigma_matrix(pairs, n_fluids), tau=tuple(0.6 + 0.1 * k for k in range(n_fluids)),
                  rho0=(1.0,) * n_fluids)
    g = N.run(p, f, 20)
    m0, m1 = f.sum(axis=(1, 2, 3)), g.sum(axis=(1, 2, 3))
    assert np.allclose(m0, m1, rtol=1e-13)
    mom = lambda h: np.array([(h.sum(axis=0) * N.EX[:, None, None]).sum(), (h.sum(axis=0) * N.EY[:, None, None]).sum()])
    # the Guo force's discrete divergence sums to zero; the recolouring moves no momentum
    assert np.abs(mom(g) - mom(f)).max() <= 1e-12 * m0.sum()


def test_four_fluid_nested_droplet_laplace_jumps():
    """Fluid 4 core R = 8 inside fluid 3 (R = 16) inside fluid 2 (R = 24) in
    fluid 1, 64^2, sigma_12 = 0.01, sigma_23 = 0.008, sigma_34 = 0.006 (the
    non-adjacent pairs 0.012), tau = 1, 3000 steps: each interface's jump of
    the bulk pressures times its radius (from the enclosed area) equals its
    own tension within 6 % (measured 0.99, 1.01 and 1.05, the last for the
    smallest radius)."""
    n = 64
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2, y - n / 2)
    disc = [0.5 + 0.5 * np.tanh((R - r) / W.XI) for R in (24.0, 16.0, 8.0)]
    rho = np.stack([np.clip(1 - disc[0], 0, None), np.clip(disc[0] - disc[1], 0, None),
                    np.clip(disc[1] - disc[2], 0, None), disc[2]])
    s = N.sigma_matrix({(0, 1): 0.01, (1, 2): 0.008, (2, 3): 0.006, (0, 2): 0.012, (0, 3): 0.012, (1, 3): 0.012}, 4)
    p = N.NParams(n, n, sigma=s, tau=(1.0, 1.0, 1.0, 1.0), rho0=(1.0,) * 4)
    f = N.run(p, N.init(rho), 3000)
    rr = f.sum(axis=1)
    ph = rr / rr.sum(axis=0)
    pr = rr.sum(axis=0) / 3.0
    for j in range(3):   # interface between fluid j+1 (outside) and j+2 (inside)
        R = math.sqrt(ph[j + 1:].sum() / math.pi)
        jump = pr[ph[j + 1] > 0.99].mean() - pr[ph[j] > 0.99].mean()
        assert jump * R / s[j, j + 1] == pytest.approx(1.0, abs=0.06), j


def test_three_fluid_fields_equal_c_oracle():
    """rho_k, u with the F/2 correction of Eq. uk1, and p of the N-phase
    restatement equal the C oracle's fields at N = 3."""
    nx, ny = 16, 12
    op = O.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=SIG3)
    f = O.step(op, W.random_populations(nx, ny, seed=6), 3)
    a = O.fields(op, f)
    b = N.fields(_p3(nx, ny), f)
    assert np.allclose(b["rho"], a["rho"], rtol=1e-13, atol=0)
    for k in ("ux", "uy"):
        assert np.abs(b[k] - a[k]).max() <= 1e-15
    assert np.allclose(b["p"], a["p"], rtol=1e-13, atol=0)
