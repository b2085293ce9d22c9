"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each checks a closed form, an
identity, a conservation law, a symmetry or a number the paper prints
(arXiv 1808.08555), chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_08555_gb300 import workloads as W

# D2Q9 lattice as the paper defines it (Sec. 2, after Eq. 3).
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
WGT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX, EY = E[:, 0], E[:, 1]


# ------------------------------------------------------------ lattice pieces

@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.9, 0.03, -0.02), (1.3, -0.07, 0.05)])
def test_feq_moments(rho, ux, uy):
    """Eq. 3: zeroth, first and second moments of f^eq are rho, rho u and
    rho c_s^2 I + rho u u (exact for the D2Q9 weights)."""
    f = O.feq(rho, ux, uy)
    u = np.array([ux, uy])
    assert f.sum() == pytest.approx(rho, abs=1e-15)
    np.testing.assert_allclose(E.T @ f, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, E, E)
    np.testing.assert_allclose(P, rho / 3 * np.eye(2) + rho * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_guo_moments(tau):
    """Eq. 5: sum Phi = 0, sum Phi e = (1 - 1/(2 tau)) F and
    sum Phi e e = (1 - 1/(2 tau)) (u F + F u) (Guo et al.'s design moments)."""
    u = np.array([0.04, -0.03])
    F = np.array([2e-4, 5e-4])
    ph = O.guo(tau, u[0], u[1], F[0], F[1])
    a = 1 - 1 / (2 * tau)
    assert abs(ph.sum()) < 1e-18
    np.testing.assert_allclose(E.T @ ph, a * F, atol=1e-18)
    P = np.einsum("i,ia,ib->ab", ph, E, E)
    np.testing.assert_allclose(P, a * (np.outer(u, F) + np.outer(F, u)), atol=1e-18)


@pytest.mark.parametrize("tauf", [0.6, 0.8, 1.5])
def test_perturbation_operator_moments(tauf):
    """Eqs. phi1 / phi_old with Leclaire's B_i (sum B_i = 1/3): zero mass and
    momentum, and second moment sum_i Phi_i e_i e_i = -sum_{k<l} sigma_kl
    C_kl |G_kl| (I - n n) / tau_f, so that -div(tau_f sum_i Phi_i e_i e_i)
    is the force of Eq. 11 (the Chapman-Enskog link the paper states)."""
    rng = np.random.default_rng(int(tauf * 10))
    G = np.zeros((3, 3, 2))
    C = np.zeros((3, 3))
    sig = (0.01, 0.013, 0.007)
    for q, (k, l) in enumerate([(0, 1), (0, 2), (1, 2)]):
        g = rng.standard_normal(2) * 0.2
        G[k, l], G[l, k] = g, -g
        C[k, l] = C[l, k] = rng.uniform(0.2, 1.0)
    ph = O.perturbation(sig, G, C, tauf)
    assert abs(ph.sum()) < 1e-18
    assert abs((ph * EX).sum()) < 1e-18 and abs((ph * EY).sum()) < 1e-18
    M = np.array([[(ph * EX * EX).sum(), (ph * EX * EY).sum()], [(ph * EY * EX).sum(), (ph * EY * EY).sum()]])
    ref = np.zeros((2, 2))
    for q, (k, l) in enumerate([(0, 1), (0, 2), (1, 2)]):
        m = np.linalg.norm(G[k, l])
        n = G[k, l] / m
        ref -= sig[q] * C[k, l] * m * (np.eye(2) - np.outer(n, n)) / tauf
    np.testing.assert_allclose(M, ref, rtol=1e-13, atol=1e-19)
    # no interface (G = 0): no perturbation
    assert np.abs(O.perturbation(sig, np.zeros((3, 3, 2)), C, tauf)).max() == 0.0


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 2), (3, 1), (2, 5)])
def test_stencil_fourier_closed_form(mx, my):
    """Eq. fd1 on v = sin(kx x + ky y + c): the stencil's exact response is
    cos(.) sin(kx)(2 + cos ky)/3 for d_x and cos(.) sin(ky)(2 + cos kx)/3 for
    d_y (sum over the D2Q9 pairs), which tends to k cos(.) as k -> 0."""
    nx, ny = 24, 20
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    th = kx * x + ky * y + 0.3
    gx, gy = O.grad(np.sin(th))
    np.testing.assert_allclose(gx, np.cos(th) * np.sin(kx) * (2 + np.cos(ky)) / 3, atol=1e-14)
    np.testing.assert_allclose(gy, np.cos(th) * np.sin(ky) * (2 + np.cos(kx)) / 3, atol=1e-14)


def test_stencil_second_order():
    """Error of Eq. fd1 against the exact derivative falls as k^3 (second order)."""
    errs = []
    for n in (32, 64, 128):
        k = 2 * np.pi / n
        y, x = np.mgrid[0:n, 0:n].astype(float)
        gx, _ = O.grad(np.sin(k * x + k * y))
        errs.append(np.abs(gx - k * np.cos(k * x + k * y)).max())
    rates = [math.log2(errs[j] / errs[j + 1]) for j in range(2)]
    assert all(2.8 < r < 3.2 for r in rates), rates


# ------------------------------------------------------- segregation parameter

def test_g_branches():
    """Eq. 20 at points of every branch and at its joints (continuous)."""
    assert O.g(-3.0) == 1.0
    assert O.g(-1.0) == pytest.approx(1.0, abs=1e-12)
    assert O.g(-0.6) == pytest.approx(0.2, abs=1e-12)      # 1 - sqrt(1 - 0.36)
    assert O.g(0.0) == pytest.approx(0.0, abs=1e-12)
    assert O.g(0.6) == pytest.approx(-0.2, abs=1e-12)
    assert O.g(1.0) == pytest.approx(-1.0, abs=1e-12)
    assert O.g(3.0) == -1.0
    for x0 in (-1.0, 0.0, 1.0):
        assert O.g(x0 - 1e-9) == pytest.approx(O.g(x0 + 1e-9), abs=1e-4)


@pytest.mark.parametrize("sig", [(0.01, 0.01, 0.01), (0.010, 0.008, 0.012), (0.01, 0.012, 0.005),
                                 (0.0173, 0.02, 0.01)])
def test_X_is_neumann_triangle(sig):
    """Eqs. theta_kl / 18: when the tensions form a triangle, the angles
    acos(X_kl) are that triangle's angles (sum pi) and obey the law of sines
    sigma_kl / sin(phi_kl) = const (Eq. sin / Eq. gjd_06)."""
    X = O.X_of(sig)
    assert np.all(np.abs(X) < 1)
    ang = np.arccos(X)
    assert ang.sum() == pytest.approx(np.pi, abs=1e-12)
    ratios = np.array(sig) / np.sin(ang)
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)


def test_X_critical_and_equal():
    """Equal tensions give 60 degree angles (X = 1/2); the critical state
    sigma_13 = sigma_12 + sigma_23 gives X_13 = -1 and so g = 1 (Eq. 20)."""
    np.testing.assert_allclose(O.X_of((0.01, 0.01, 0.01)), 0.5, atol=1e-15)
    X = O.X_of((0.004, 0.014, 0.010))
    assert X[1] == pytest.approx(-1.0, abs=1e-12)
    assert O.g(X[1]) == pytest.approx(1.0, abs=1e-6)


def test_beta_forms():
    """beta_kl = beta^0 where one fluid is absent (Eqs. 16, 17, 19); Eq. fu is
    constant; Eq. 17 is Eq. 16 with 27 -> min(35 ., 1) when phi_rg is the
    largest angle (Sec. 2 remark after Eq. 17)."""
    sig = (0.012, 0.01, 0.008)        # phi_rg (opposite the largest sigma) is the largest
    ang = np.arccos(O.X_of(sig))
    assert ang.argmax() == 0
    for form in range(4):
        p = O.Params(8, 8, sigma=sig, beta0=0.7, beta_form=form)
        np.testing.assert_allclose(O.beta(p, [0.6, 0.4, 0.0]), 0.7, atol=1e-15)
    rk = [0.3, 0.2, 0.1]
    prod = 0.3 * 0.2 * 0.1 / 0.6 ** 3
    b1 = O.beta(O.Params(8, 8, sigma=sig, beta_form=1), rk)
    np.testing.assert_allclose(b1, 0.7)
    b2 = O.beta(O.Params(8, 8, sigma=sig, beta_form=2), rk)
    b3 = O.beta(O.Params(8, 8, sigma=sig, beta_form=3), rk)
    assert b2[0] == pytest.approx(0.7) and b3[0] == pytest.approx(0.7)
    np.testing.assert_allclose((b3[1:] - 0.7) / (b2[1:] - 0.7), min(35 * prod, 1) / (27 * prod), rtol=1e-12)
    b0 = O.beta(O.Params(8, 8, sigma=sig, beta_form=0), rk)
    c = min(35 * prod, 1.0)
    X = O.X_of(sig)
    g = np.where(X <= 0, 1 - np.sqrt(1 - X ** 2), np.sqrt(1 - X ** 2) - 1)
    np.testing.assert_allclose(b0, 0.7 * (1 + c * g), rtol=1e-12)


# ----------------------------------------------------------------- the force

def test_two_phase_reduction_of_colour_gradient():
    """With fluid 3 absent, G_12 = grad phi_1 (because phi_2 = 1 - phi_1),
    G_21 = -G_12 and every G involving fluid 3 vanishes."""
    n = 24
    rho = W.compound_droplet(n, n, 0.0, 7.0)
    rho[2] = 0.0
    rho[0] = 1.0 - rho[1]
    rho *= 1.0 + 0.1 * np.sin(2 * np.pi * np.arange(n) / n)[None, None, :]   # rho != 1
    p = O.Params(n, n)
    G, C = O.colour_gradients(p, rho)
    phi1 = rho[0] / rho.sum(0)
    gx, gy = O.grad(phi1)
    np.testing.assert_allclose(G[0, 1, 0], gx, atol=1e-15)
    np.testing.assert_allclose(G[0, 1, 1], gy, atol=1e-15)
    np.testing.assert_allclose(G[1, 0], -G[0, 1], atol=1e-15)
    for k, l in [(0, 2), (2, 0), (1, 2), (2, 1)]:
        assert np.abs(G[k, l]).max() == 0.0
    assert np.all((C >= 0) & (C <= 1))


@pytest.mark.parametrize("pair", [(0, 1), (0, 2), (1, 2)])
def test_force_integrates_to_laplace_jump(pair):
    """Eq. 11 for a two-phase disc of radius R: the radial force integrated
    across the interface equals the Young-Laplace jump -sigma_kl/R (Eq.
    laplace), so each pair picks its own tension."""
    n, R = 96, 20.0
    sig = (0.01, 0.02, 0.03)
    k, l = pair
    disc = W.compound_droplet(n, n, 0.0, R)[1]
    rho = np.zeros((3, n, n))
    rho[l] = disc
    rho[k] = 1.0 - disc
    Fx, Fy, _ = O.force(O.Params(n, n, sigma=sig), rho)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2, y - n / 2)
    Fr = (Fx * (x - n / 2) + Fy * (y - n / 2)) / np.maximum(r, 1e-12)
    band = (r > R - 8) & (r < R + 8)
    s_kl = {(0, 1): 0.01, (0, 2): 0.02, (1, 2): 0.03}[pair]
    assert Fr[band].sum() / (2 * np.pi * R) == pytest.approx(-s_kl / R, rel=0.01)
    assert abs(Fx.sum()) < 1e-15 and abs(Fy.sum()) < 1e-15      # periodic divergence


@pytest.mark.parametrize("force_form", [0, 1])
def test_flat_interface_has_no_force_and_no_flow(force_form):
    """A flat two-phase interface has a tension tensor that depends on y only
    with T_xy = T_yy = 0, so F_s = 0 and the fluid stays at rest (also with
    the perturbation operator, whose stress has the same divergence)."""
    nx, ny = 8, 32
    rho = W.flat_band(nx, ny, 8, 24, sharp=True)
    p = O.Params(nx, ny, tau=(0.8, 1.0, 1.0), force_form=force_form)
    Fx, Fy, _ = O.force(p, rho)
    assert np.abs(Fx).max() < 1e-17 and np.abs(Fy).max() < 1e-17
    f = O.step(p, O.init(p, rho), 300)
    fl = O.fields(p, f)
    assert np.abs(fl["ux"]).max() < 1e-13 and np.abs(fl["uy"]).max() < 1e-13


# ------------------------------------------------------------- the full step

def test_uniform_state_is_fixed_point():
    """A spatially uniform mixture at rest has no gradients, no force and
    f = f^eq, so one step reproduces it (to roundoff)."""
    nx, ny = 10, 7
    rk = np.array([0.3, 0.5, 0.2])
    rho = np.broadcast_to(rk[:, None, None], (3, ny, nx)).copy()
    p = O.Params(nx, ny, tau=(0.7, 0.9, 1.3), sigma=(0.01, 0.02, 0.015))
    f0 = O.init(p, rho)
    f5 = O.step(p, f0, 5)
    np.testing.assert_allclose(f5, f0, rtol=0, atol=1e-15)


def test_random_state_conserves_mass_and_momentum():
    """Per-colour mass (Eq. 6 sums to phi_k rho over i because sum w_i e_i = 0)
    and total momentum (recolouring cancels over colours; sum_x F_s = 0) are
    conserved from any state, here a random non-equilibrium one."""
    nx, ny = 12, 10
    f0 = W.random_populations(nx, ny, seed=3)
    for form, force in ((0, 0), (1, 0), (0, 1)):
        p = O.Params(nx, ny, tau=(0.7, 1.0, 1.4), sigma=(0.01, 0.02, 0.015), recolor_form=form, force_form=force)
        m0, mo0 = O.mass(p, f0)
        f = O.step(p, f0, 20)
        m1, mo1 = O.mass(p, f)
        np.testing.assert_allclose(m1, m0, rtol=1e-13)
        np.testing.assert_allclose(mo1, mo0, atol=1e-13 * m0.sum())


def _rot90(f):
    """Rotate a (3, 9, n, n) population field by +90 degrees about the origin:
    node (x, y) -> (-y, x) and direction e_i -> R e_i."""
    perm = [0, 2, 3, 4, 1, 6, 7, 8, 5]           # i -> index of R e_i
    g = np.empty_like(f)
    for i in range(9):
        src = f[:, i]                            # (3, y, x)
        rot = np.roll(np.swapaxes(src, 1, 2)[:, :, ::-1], 1, axis=2)
        g[:, perm[i]] = rot
    return g


def _mirror_x(f):
    """Mirror x -> -x: node (x, y) -> (-x, y), e_i -> (-e_x, e_y)."""
    perm = [0, 3, 2, 1, 4, 6, 5, 8, 7]
    g = np.empty_like(f)
    for i in range(9):
        g[:, perm[i]] = np.roll(f[:, i, :, ::-1], 1, axis=2)
    return g


@pytest.mark.parametrize("form,force", [(0, 0), (1, 0), (0, 1)])
def test_step_commutes_with_lattice_symmetries(form, force):
    """The update is built from isotropic pieces, so it commutes with the
    square lattice's 90-degree rotation and its mirror (up to roundoff)."""
    n = 10
    f0 = W.random_populations(n, n, seed=11)
    p = O.Params(n, n, tau=(0.7, 1.0, 1.4), sigma=(0.01, 0.02, 0.015), recolor_form=form, force_form=force)
    a = _rot90(O.step(p, f0, 2))
    b = O.step(p, _rot90(f0), 2)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    a = _mirror_x(O.step(p, f0, 2))
    b = O.step(p, _mirror_x(f0), 2)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_two_droplets_64_mass_and_momentum_1000_steps():
    """Two static droplets, 64x64, 1000 steps: per-colour mass drift at most
    1e-12 relative and net momentum zero to roundoff."""
    c = W.case_two_droplets_64()
    p = O.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0)
    f0 = O.init(p, c.rho)
    m0, _ = O.mass(p, f0)
    f = O.step(p, f0, 1000)
    m1, mo = O.mass(p, f)
    assert np.abs(m1 / m0 - 1).max() <= 1e-12
    assert np.abs(mo).max() <= 1e-12 * m0.sum()
    fl = O.fields(p, f)
    # static droplets: spurious currents of the order the paper reports (Tab. 2)
    assert np.hypot(fl["ux"], fl["uy"]).max() < 1e-4


def test_interface_thickness_matches_paper():
    """Sec. 3.1: a relaxed flat two-phase interface follows
    0.5 + 0.5 tanh(d / xi) with xi = 1.5831 for beta^0 = 0.7.  The cosine
    form of the recolouring direction factor reproduces it to 3 %; the
    literal n.e_i of Eq. 6 gives a profile about 7 % thinner."""
    from scipy.optimize import curve_fit

    def xi_fit(form):
        nx, ny = 4, 64
        p = O.Params(nx, ny, recolor_form=form)
        f = O.step(p, O.init(p, W.flat_band(nx, ny, 16, 48, sharp=True)), 3000)
        rho = O.fields(p, f)["rho"]
        phi = rho[1, :, 0] / rho.sum(0)[:, 0]
        y = np.arange(ny, dtype=float)
        sel = (y > 4) & (y < 30)
        popt, _ = curve_fit(lambda yy, y0, xi: 0.5 + 0.5 * np.tanh((yy - y0) / xi), y[sel], phi[sel],
                            p0=(16.0, 1.5))
        return popt[1]

    assert xi_fit(0) == pytest.approx(1.5831, rel=0.03)
    assert abs(xi_fit(1) / 1.5831 - 1) > 0.05


@pytest.mark.parametrize("force_form", [0, 1])
def test_young_laplace_single_droplet(force_form):
    """Eq. laplace: a relaxed two-phase droplet has a pressure jump sigma/R
    (R from the droplet's area).  48x48, R = 10, sigma = 0.01.  With the
    perturbation operator (Eqs. phi1 / phi_old) the same jump follows, as
    its Chapman-Enskog force is Eq. 11."""
    n, R, sig = 48, 10.0, 0.01
    rho = W.compound_droplet(n, n, 0.0, R)
    rho[2] = 0.0
    rho[0] = 1.0 - rho[1]
    p = O.Params(n, n, sigma=(sig, sig, sig), force_form=force_form)
    f = O.step(p, O.init(p, rho), 9000)
    fl = O.fields(p, f)
    phi2 = fl["rho"][1] / fl["rho"].sum(0)
    R_eff = math.sqrt(phi2.sum() / math.pi)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2, y - n / 2)
    dp = fl["p"][r < R - 4 * W.XI].mean() - fl["p"][r > R + 4 * W.XI].mean()
    assert dp * R_eff / sig == pytest.approx(1.0, abs=0.05)


def test_shear_wave_decays_with_harmonic_mean_viscosity():
    """Eqs. vis_1 and tau: a uniform mixture carries a shear wave
    u_x = U sin(k y) that decays as exp(-nu k^2 t) with the harmonic-mean
    viscosity rho/nu = sum_k rho_k/nu_k, nu_k = (tau_k - 1/2)/3.  Recolouring
    is switched off (beta^0 = 0): an immiscible mixture would demix."""
    nx, ny, U = 4, 64, 1e-4
    rk = np.array([0.3, 0.5, 0.2])
    taus = (0.6, 0.8, 1.4)
    k = 2 * np.pi / ny
    y = np.arange(ny, dtype=float)
    f = np.zeros((3, 9, ny, nx))
    for j in range(ny):
        feq = O.feq(1.0, U * np.sin(k * y[j]), 0.0)
        for c in range(3):
            f[c, :, j, :] = (rk[c] * feq)[:, None]
    p = O.Params(nx, ny, tau=taus, beta0=0.0)
    steps = 400
    fl = O.fields(p, O.step(p, f, steps))
    amp = 2 * np.mean(fl["ux"][:, 0] * np.sin(k * y))
    nu_meas = -np.log(amp / U) / (k * k * steps)
    nu_k = (np.array(taus) - 0.5) / 3
    nu_harm = 1.0 / np.sum(rk / nu_k)
    assert nu_meas == pytest.approx(nu_harm, rel=0.01)


def test_concentration_factor_values():
    """Eq. 15 at chosen densities: C_kl = min(1e6 rho_k rho_l/(rho_k^0 rho_l^0), 1)."""
    n = 4
    rho = np.zeros((3, n, n))
    rho[0], rho[1], rho[2] = 1e-4, 1e-3, 0.5
    G, C = O.colour_gradients(O.Params(n, n), rho)
    assert C[0, 1] == pytest.approx(0.1, rel=1e-12) and C[1, 0] == pytest.approx(0.1, rel=1e-12)
    assert np.all(C[0, 2] == 1.0) and np.all(C[1, 2] == 1.0)
    G, C = O.colour_gradients(O.Params(n, n, rho0=(2.0, 2.0, 1.0)), rho)
    assert C[0, 1] == pytest.approx(0.025, rel=1e-12)
    assert C[0, 2] == pytest.approx(min(1e6 * 5e-5 / 2.0, 1.0))
    assert np.all(G == 0.0)


def test_oracle_threads_do_not_change_results():
    """The oracle's node loops run on several host threads (OpenMP) only where
    the iterations write disjoint outputs, each with the same arithmetic in
    the same order: one thread and all threads give bit-identical states."""
    n = 40
    rho = W.droplet_field(n, n, seed=9, count=4, rmin=3.0, rmax=7.0, gap=4.0)
    p = O.Params(n, n, tau=(0.6, 0.9, 1.3), sigma=(0.01, 0.013, 0.007), beta_form=3)
    all_threads = O.threads()
    try:
        O.threads(1)
        one = O.step(p, O.init(p, rho), 20)
        f1 = O.fields(p, one)
        O.threads(max(all_threads, 4))
        many = O.step(p, O.init(p, rho), 20)
        fm = O.fields(p, many)
    finally:
        O.threads(all_threads)
    assert np.array_equal(one, many)
    for k in ("rho", "ux", "uy", "p"):
        assert np.array_equal(f1[k], fm[k])
