"""Pins of the D3Q19 restatement (oracle.lbm3d), CPU only.

The paper writes the model in vector form and simulates two dimensions.  The
three-dimensional restatement is pinned
(1) to the C oracle through an exact projection: a state uniform along one
    axis evolves on D3Q19 as its projection does on D2Q9 (summing the
    populations whose velocities agree in the other two axes), because the
    D3Q19 weights summed that way are the D2Q9 weights.  This holds with the
    weights w_i in the recolouring (recolor_form 1), in each of the three
    planes, both beta forms and both normals;
(2) by the lattice's symmetry: permuting the axes of a state commutes with
    the step;
(3) by the interface thickness of Sec. 3.1, xi = 1 / (6 k beta^0) with the
    geometric constant k = (1/2) sum_i w_i e_i e_i / |e_i| evaluated on
    D3Q19 (k = (1 + sqrt 2) / 18, xi = 1.7752 at beta^0 = 0.7, against
    1.5831 on D2Q9): this fixes the cosine form of the recolouring in 3D;
(4) by the three-dimensional Young-Laplace law, Delta p = 2 sigma / R, for a
    relaxed spherical droplet;
(5) by per-colour mass and total momentum conservation, and by the exact
    reduction that an absent fourth fluid changes nothing."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lbm3d as D
from paper_1808_08555_gb300 import workloads as W

SIG3 = (0.01, 0.013, 0.007)
TAU3 = (0.6, 0.9, 1.3)


def _sig(pairs, n):
    s = np.zeros((n, n))
    for (k, l), v in pairs.items():
        s[k, l] = s[l, k] = v
    return s


def _p3(nx, ny, nz, **kw):
    s = _sig({(0, 1): SIG3[0], (0, 2): SIG3[1], (1, 2): SIG3[2]}, 3)
    return D.Params3D(nx, ny, nz, sigma=s, tau=TAU3, rho0=(1.0, 1.0, 1.0), **kw)


# D2Q9 velocities of the C oracle
EX2 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY2 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
# the plane's two axes (a, b) as indices into (x, y, z), the uniform axis c,
# and the axis of the 3D array (z, y, x) that c is
PLANES = {"xy": (0, 1, 2), "yz": (1, 2, 0), "xz": (0, 2, 1)}


def _d2q9_of(i, a, b):
    """D2Q9 direction whose velocity is D3Q19 direction i's (a, b) components."""
    ea, eb = D.E[i, a], D.E[i, b]
    return int(np.flatnonzero((EX2 == ea) & (EY2 == eb))[0])


def _lift(f2, plane, nc):
    """A 3D state uniform along the plane's third axis whose projection is
    the D2Q9 state f2 (N, 9, n_b, n_a): each 2D population is shared by the
    D3Q19 directions projecting onto it, in proportion to their weights."""
    a, b, c = PLANES[plane]
    N, nb, na = f2.shape[0], f2.shape[2], f2.shape[3]
    wsum = np.zeros(9)
    for i in range(D.Q):
        wsum[_d2q9_of(i, a, b)] += D.WT[i]
    phys = [c, b, a]                                   # physical axes of (uniform, n_b, n_a)
    order = [0] + [phys.index(ax) + 1 for ax in (2, 1, 0)]   # to the array order (z, y, x)
    out = []
    for i in range(D.Q):
        j = _d2q9_of(i, a, b)
        g = np.broadcast_to((f2[:, j] * (D.WT[i] / wsum[j]))[:, None], (N, nc, nb, na))
        out.append(np.transpose(g, order))
    return np.ascontiguousarray(np.stack(out, axis=1))


def _project(f3, plane):
    """Sum the populations of a 3D state uniform along the plane's third axis
    onto D2Q9, taking one slice of the uniform axis: (N, 9, n_b, n_a)."""
    a, b, c = PLANES[plane]
    sl = [slice(None)] * 3
    sl[2 - c] = 0
    g = f3[(slice(None), slice(None)) + tuple(sl)]   # (N, 19, two remaining axes in z, y, x order)
    rem = [ax for ax in (2, 1, 0) if ax != c]        # physical axes of g's last two axes
    if rem != [b, a]:
        g = np.swapaxes(g, -1, -2)
    out = np.zeros((f3.shape[0], 9) + g.shape[2:])
    for i in range(D.Q):
        out[:, _d2q9_of(i, a, b)] += g[:, i]
    return out


def test_lift_and_project_are_inverse():
    f2 = W.random_populations(7, 5, seed=1)
    for plane in PLANES:
        f3 = _lift(f2, plane, 3)
        assert np.allclose(_project(f3, plane), f2, rtol=1e-15, atol=0)
        # uniform along the third axis
        c = PLANES[plane][2]
        assert np.array_equal(np.take(f3, 0, axis=2 + (2 - c)), np.take(f3, 2, axis=2 + (2 - c)))


@pytest.mark.parametrize("plane", sorted(PLANES))
@pytest.mark.parametrize("beta_form", [0, 1])
@pytest.mark.parametrize("delta", [0.1, 0.0])
def test_uniform_state_projects_onto_c_oracle(plane, beta_form, delta):
    na, nb = 14, 10
    f2 = W.random_populations(na, nb, seed=3)
    op = O.Params(na, nb, tau=TAU3, sigma=SIG3, beta_form=beta_form, recolor_form=1, normal_delta=delta)
    ref = O.step(op, f2, 4)
    f3 = _lift(f2, plane, 2)
    nz, ny, nx = f3.shape[2:]
    got = _project(D.run(_p3(nx, ny, nz, beta_form=beta_form, recolor_form=1, normal_delta=delta), f3, 4), plane)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _perm_dirs(perm):
    """Direction map of the axis permutation x' = x_perm: new direction j has
    components E[i][perm]."""
    m = np.empty(D.Q, dtype=int)
    for i in range(D.Q):
        e = D.E[i][list(perm)]
        m[i] = int(np.flatnonzero((D.E == e).all(axis=1))[0])
    return m


def test_axis_permutation_commutes_with_the_step():
    rng = np.random.default_rng(11)
    nx, ny, nz = 9, 8, 7
    rho = rng.uniform(0.05, 1.0, (3, nz, ny, nx))
    f = D.init(rho) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, (3, D.Q, nz, ny, nx)))
    perm = (1, 2, 0)   # new x = old y, new y = old z, new z = old x
    m = _perm_dirs(perm)

    def permute(g):
        # array axes (N, Q, z, y, x); the new axis of physical axis a is the
        # old axis perm[a], so new array axis (z', y', x') reads old axis
        # position 1 + (2 - perm[a]) of a direction's (N, z, y, x) field
        out = np.empty((g.shape[0], D.Q) + tuple(g.shape[2 + (2 - perm[a])] for a in (2, 1, 0)))
        for i in range(D.Q):
            out[:, m[i]] = np.transpose(g[:, i], [0] + [1 + (2 - perm[a]) for a in (2, 1, 0)])
        return out

    p = _p3(nx, ny, nz)
    fp = permute(f)
    q = _p3(fp.shape[4], fp.shape[3], fp.shape[2])
    a = permute(D.run(p, f, 3))
    b = D.run(q, fp, 3)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def _flat_band_xi(axis, recolor_form=0, steps=300):
    """Fitted xi of the relaxed flat band 16 <= c < 48 of fluid 2 in fluid 1
    along the given axis (0: x, 2: z) of a 64 x 1 x 1 column (the profile
    is converged after 250 steps)."""
    from scipy.optimize import curve_fit
    n = 64
    shape = [1, 1, 1]
    shape[2 - axis] = n
    coord = np.arange(n, dtype=float)
    band = ((coord >= 16) & (coord < 48)).astype(float).reshape(shape)
    rho = np.stack([1.0 - band, band])
    p = D.Params3D(shape[2], shape[1], shape[0], sigma=_sig({(0, 1): 0.01}, 2), tau=(1.0, 1.0), rho0=(1.0, 1.0),
                   recolor_form=recolor_form)
    f = D.run(p, D.init(rho), steps)
    r = f.sum(axis=1)
    line = (r[1] / r.sum(axis=0)).reshape(n)
    sel = (coord > 4) & (coord < 30)
    popt, _ = curve_fit(lambda yy, y0, xi: 0.5 + 0.5 * np.tanh((yy - y0) / xi), coord[sel], line[sel],
                        p0=(16.0, 1.5))
    return popt[1]


@pytest.mark.parametrize("axis", [2, 0])
def test_interface_thickness_d3q19(axis):
    """Sec. 3.1: xi = 1 / (6 k beta^0), k = (1/2) sum_i w_i e_ix^2 / |e_i|,
    which on D3Q19 is (1 + sqrt 2) / 18, xi = 1.7752; the cosine form gives
    it to 3 % as on D2Q9 (measured 1.8063, +1.8 %) with the interface normal
    along z and along x.  The weights w_i in place of w_i / |e_i| give a
    profile 19 % thinner (the same formula without |e_i| predicts 1.4286)."""
    k = 0.5 * sum(D.WT[i] * D.E[i, 0] ** 2 / math.sqrt((D.E[i] ** 2).sum()) for i in range(1, D.Q))
    assert k == pytest.approx((1 + math.sqrt(2)) / 18, rel=1e-14)
    xi = 1.0 / (6.0 * k * 0.7)
    assert _flat_band_xi(axis) == pytest.approx(xi, rel=0.03)
    assert _flat_band_xi(axis, recolor_form=1) < 0.9 * xi


def test_sphere_young_laplace():
    """A relaxed two-phase sphere, 24^3, R = 7, sigma = 0.01, tau = 1, 400
    steps: the pressure jump between the bulks is 2 sigma / R (the
    three-dimensional Young-Laplace law; R from the droplet's volume) within
    12 %.  Measured 1.103: the interface (xi = 1.78) is a quarter of the
    radius thick, and the ratio falls towards 1 with the radius (1.063 at
    R = 9 on 32^3).  Tension acting on one curvature direction only would
    give 0.5."""
    n, R0, sig = 24, 7.0, 0.01
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.5) ** 2)
    inside = 0.5 + 0.5 * np.tanh((R0 - r) / W.XI)
    rho = np.stack([1.0 - inside, inside])
    p = D.Params3D(n, n, n, sigma=_sig({(0, 1): sig}, 2), tau=(1.0, 1.0), rho0=(1.0, 1.0))
    f = D.run(p, D.init(rho), 400)
    rr = f.sum(axis=1)
    ph = rr[1] / rr.sum(axis=0)
    pr = D.pressure(f)
    R = (3.0 * ph.sum() / (4.0 * math.pi)) ** (1.0 / 3.0)
    jump = pr[ph > 0.99].mean() - pr[ph < 0.01].mean()
    assert jump * R / (2.0 * sig) == pytest.approx(1.0, abs=0.12)


@pytest.mark.parametrize("n_fluids", [3, 4])
def test_mass_and_momentum_conserved(n_fluids):
    rng = np.random.default_rng(n_fluids + 30)
    nx, ny, nz = 8, 7, 6
    rho = rng.uniform(0.05, 1.0, (n_fluids, nz, ny, nx))
    f = D.init(rho) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, (n_fluids, D.Q, nz, ny, nx)))
    pairs = {(k, l): 0.006 + 0.001 * (k + 2 * l) for k in range(n_fluids) for l in range(k + 1, n_fluids)}
    p = D.Params3D(nx, ny, nz, sigma=_sig(pairs, n_fluids), tau=tuple(0.6 + 0.1 * k for k in range(n_fluids)),
                   rho0=(1.0,) * n_fluids)
    g = D.run(p, f, 10)
    m0, m1 = f.sum(axis=(1, 2, 3, 4)), g.sum(axis=(1, 2, 3, 4))
    assert np.allclose(m0, m1, rtol=1e-13)
    mom = lambda h: np.array([(h.sum(axis=0) * D.E[:, a, None, None, None]).sum() for a in range(3)])
    assert np.abs(mom(g) - mom(f)).max() <= 1e-12 * m0.sum()


def test_absent_fourth_fluid_changes_nothing():
    rng = np.random.default_rng(5)
    nx, ny, nz = 7, 6, 5
    rho = rng.uniform(0.05, 1.0, (3, nz, ny, nx))
    f3 = D.init(rho) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, (3, D.Q, nz, ny, nx)))
    f4 = np.concatenate([f3, np.zeros((1,) + f3.shape[1:])])
    s4 = _sig({(0, 1): SIG3[0], (0, 2): SIG3[1], (1, 2): SIG3[2], (0, 3): 0.011, (1, 3): 0.009, (2, 3): 0.012}, 4)
    p4 = D.Params3D(nx, ny, nz, sigma=s4, tau=TAU3 + (0.8,), rho0=(1.0,) * 4)
    a = D.run(_p3(nx, ny, nz), f3.copy(), 4)
    b = D.run(p4, f4, 4)
    assert np.array_equal(a, b[:3]) and not b[3].any()


@pytest.mark.parametrize("plane", sorted(PLANES))
def test_fields_of_a_uniform_state_project_onto_c_oracle(plane):
    """The fields (rho_k, u with the F/2 correction of Eq. uk1, p) of a state
    uniform along one axis are the C oracle's fields of its projection, with
    no velocity along the uniform axis."""
    na, nb = 14, 10
    f2 = O.step(O.Params(na, nb, tau=TAU3, sigma=SIG3), W.random_populations(na, nb, seed=9), 2)
    ref = O.fields(O.Params(na, nb, tau=TAU3, sigma=SIG3), f2)
    f3 = _lift(f2, plane, 2)
    nz, ny, nx = f3.shape[2:]
    got = D.fields(_p3(nx, ny, nz), f3)
    a, b, c = PLANES[plane]

    def plane_of(v):   # a (z, y, x) field uniform along c, as the D2Q9 (n_b, n_a) field
        g = np.take(v, 0, axis=-3 + (2 - c))
        rem = [ax for ax in (2, 1, 0) if ax != c]
        return g if rem == [b, a] else g.T

    for k in range(3):
        assert np.allclose(plane_of(got["rho"][k]), ref["rho"][k], rtol=1e-13, atol=0)
    assert np.allclose(plane_of(got["u"][a]), ref["ux"], rtol=0, atol=1e-15)
    assert np.allclose(plane_of(got["u"][b]), ref["uy"], rtol=0, atol=1e-15)
    assert np.abs(got["u"][c]).max() <= 1e-15
    assert np.allclose(plane_of(got["p"]), ref["p"], rtol=1e-13, atol=0)
