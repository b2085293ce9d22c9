"""N fluids on the GPU (lbm3n_*, the first CUDA path of the N-fluid step)
against the N-phase FP64 restatement oracle.lbmn, which is itself pinned to
the three-fluid C oracle and to the N-fluid physics (tests/test_oracle_nphase.py).

Bars as for three fluids: relative population error (floor 1e-3 w_i) 1e-5
after one step and 1e-4 after 1000 steps, on inputs whose own FP32-level
sensitivity in the oracle is at most 1e-6."""
import numpy as np
import pytest

from oracle import lbmn as N
from paper_1808_08555_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WGT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def L():
    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3
    lbm3.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm3


def relerr(fg, fo):
    return float(np.max(np.abs(fg - fo) / np.maximum(np.abs(fo), 1e-3 * WGT[None, :, None, None])))


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def sigma_of(n):
    pairs = {(k, l): 0.006 + 0.001 * ((3 * k + 2 * l) % 7) for k in range(n) for l in range(k + 1, n)}
    return N.sigma_matrix(pairs, n)


def sim_of(L, p: N.NParams, storage=0):
    return L.NSimulation(p.nx, p.ny, p.sigma, p.tau, p.rho0, beta0=p.beta0, beta_form=p.beta_form,
                         recolor_form=p.recolor_form, normal_delta=p.normal_delta, storage=storage)


def run_gpu(L, p: N.NParams, f0, steps, storage=0):
    sim = sim_of(L, p, storage)
    sim.set_populations(f0)
    sim.step(steps)
    fg = sim.populations()
    m, _ = sim.mass()
    sim.close()
    return fg, m


def run_both(L, p: N.NParams, f0, steps):
    fg, m = run_gpu(L, p, f0, steps)
    return fg, N.run(p, f0.copy(), steps), m


def sensitivity(p, f0, steps):
    rng = np.random.default_rng(0)
    fp = f0 * (1.0 + 6e-8 * rng.uniform(-1.0, 1.0, f0.shape))
    return relerr(N.run(p, fp, steps), N.run(p, f0.copy(), steps))


def random_state(n, nx, ny, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 1.0, (n, ny, nx))
    f = N.init(rho)
    return f32(f * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, f.shape)))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("beta_form,recolor_form", [(0, 0), (1, 1)])
def test_random_state_one_step(L, n, beta_form, recolor_form):
    p = N.NParams(8, 8, sigma=sigma_of(n), tau=tuple(0.6 + 0.15 * k for k in range(n)), rho0=(1.0,) * n,
                  beta_form=beta_form, recolor_form=recolor_form)
    f0 = random_state(n, 8, 8, seed=n + 20)
    assert sensitivity(p, f0, 1) <= 1e-6
    fg, fo, _ = run_both(L, p, f0, 1)
    assert relerr(fg, fo) <= 1e-5


def _nested(nn, radii):
    y, x = np.mgrid[0:nn, 0:nn].astype(float)
    r = np.hypot(x - nn / 2, y - nn / 2)
    disc = [0.5 + 0.5 * np.tanh((R - r) / W.XI) for R in radii]
    layers = [np.clip(1 - disc[0], 0, None)]
    for j in range(len(radii) - 1):
        layers.append(np.clip(disc[j] - disc[j + 1], 0, None))
    layers.append(disc[-1])
    return np.stack(layers)


def test_four_fluid_nested_droplet_10_steps(L):
    """Four fluids, nested droplet (64^2, radii 24/16/8): 1e-5 after 10
    steps.  (Not run to 1000 steps: the fluid-3 trace at the core's centre,
    4.8e-5, takes its direction from rounding there, and the oracle's own
    response to FP32-level input noise reaches 4.8e-4 by then.)"""
    nn = 64
    rho = _nested(nn, (24.0, 16.0, 8.0))
    s = N.sigma_matrix({(0, 1): 0.01, (1, 2): 0.008, (2, 3): 0.006, (0, 2): 0.012, (0, 3): 0.012, (1, 3): 0.012}, 4)
    p = N.NParams(nn, nn, sigma=s, tau=(1.0, 0.8, 0.9, 1.2), rho0=(1.0,) * 4)
    f0 = f32(N.init(rho))
    assert sensitivity(p, f0, 10) <= 1e-6
    fg, fo, _ = run_both(L, p, f0, 10)
    assert relerr(fg, fo) <= 1e-5


def test_four_fluids_three_droplets_1000_steps(L):
    """Four fluids: droplets of fluids 2, 3 and 4 (R = 10, 12 apart) in
    fluid 1, 96 x 64: 1e-4 after 1000 steps (the oracle's own FP32-level
    sensitivity for this input is 4.1e-7 at 1000 steps), and FP64 per-fluid
    masses of the GPU state within 1e-5 of the start."""
    nx, ny = 96, 64
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    d = lambda cx, R: 0.5 + 0.5 * np.tanh((R - np.hypot(x - cx, y - 32.0)) / W.XI)
    p2, p3, p4 = d(16.0, 10.0), d(48.0, 10.0), d(80.0, 10.0)
    rho = np.stack([np.clip(1 - p2 - p3 - p4, 0, None), p2, p3, p4])
    p = N.NParams(nx, ny, sigma=sigma_of(4), tau=(1.0, 0.8, 0.9, 1.2), rho0=(1.0,) * 4)
    f0 = f32(N.init(rho))
    fg, fo, m = run_both(L, p, f0, 1000)
    assert relerr(fg, fo) <= 1e-4
    m0 = f0.reshape(4, 9, -1).sum(axis=(1, 2))
    assert np.abs(m / m0 - 1).max() <= 1e-5
    # the reduced state runs the same trajectory
    fr, mr = run_gpu(L, p, f0, 1000, storage=L.REDUCED)
    assert np.array_equal(fr, fg) and np.array_equal(mr, m)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("beta_form,recolor_form,delta,nx,ny", [(0, 0, 0.1, 300, 6), (1, 1, 0.0, 300, 6),
                                                                 (0, 0, 0.1, 301, 5)])
def test_reduced_state_is_bit_identical(L, n, beta_form, recolor_form, delta, nx, ny):
    """The reduced state (phi_k, V_k, f^dagger_i per node, by component)
    rebuilds every population from its source node with the operations the
    population form stores it with, so both forms give the same bits:
    populations, masses and fields after 1, 7 and 12 steps of random states
    on a 300 x 6 grid (a ragged last block per row) and a 301 x 5 one (an
    odd node count, so that planes start at odd node offsets), readouts in
    between (which expand the state into the idle buffer) leaving the
    trajectory unchanged.  (Parity of the reduced form with the oracle: the
    1000-step case above.)"""
    p = N.NParams(nx, ny, sigma=sigma_of(n), tau=tuple(0.6 + 0.15 * k for k in range(n)), rho0=(1.0,) * n,
                  beta_form=beta_form, recolor_form=recolor_form, normal_delta=delta)
    f0 = random_state(n, nx, ny, seed=40 + n)
    a, b = sim_of(L, p), sim_of(L, p, storage=L.REDUCED)
    for sim in (a, b):
        sim.set_populations(f0)
    for steps in (1, 6, 5):
        for sim in (a, b):
            sim.step(steps)
        assert np.array_equal(a.populations(), b.populations())
        ma, moa = a.mass()
        mb, mob = b.mass()
        assert np.array_equal(ma, mb) and np.array_equal(moa, mob)
        fa, fb = a.fields(), b.fields()
        for key in ("rho", "ux", "uy", "p"):
            assert np.array_equal(fa[key], fb[key])
    f1 = b.populations()
    b.set_populations(f1)
    assert np.array_equal(b.populations(), f1)
    a.close()
    b.close()


def test_absent_fluid_gives_the_three_fluid_result(L):
    """N = 4 with the fourth fluid absent everywhere equals N = 3 on the GPU,
    bit for bit (every term of the absent fluid is an exact zero)."""
    nx, ny = 40, 24
    f3 = random_state(3, nx, ny, seed=11)
    f4 = np.concatenate([f3, np.zeros((1,) + f3.shape[1:])])
    s4 = sigma_of(4)
    p3 = N.NParams(nx, ny, sigma=s4[:3, :3], tau=(0.6, 0.9, 1.3), rho0=(1.0,) * 3)
    p4 = N.NParams(nx, ny, sigma=s4, tau=(0.6, 0.9, 1.3, 0.8), rho0=(1.0,) * 4)
    g3, _, _ = run_both(L, p3, f3, 5)
    g4, _, _ = run_both(L, p4, f4, 5)
    assert np.array_equal(g3, g4[:3]) and not g4[3].any()


def test_three_fluids_against_the_fused_kernel(L):
    """At N = 3 the N-fluid path and the fused three-fluid kernel compute the
    same method: both within 1e-5 of the C oracle after one step of a random
    state, and within 2e-5 of each other."""
    import oracle as O
    nx, ny = 16, 12
    f0 = f32(W.random_populations(nx, ny, seed=4))
    sig = (0.01, 0.013, 0.007)
    op = O.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=sig)
    ref = O.step(op, f0, 1)
    s = N.sigma_matrix({(0, 1): sig[0], (0, 2): sig[1], (1, 2): sig[2]}, 3)
    gn, _, _ = run_both(L, N.NParams(nx, ny, sigma=s, tau=(0.6, 0.9, 1.3), rho0=(1.0,) * 3), f0, 1)
    sim = L.Simulation(L.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=sig))
    sim.set_populations(f0)
    sim.step(1)
    gf = sim.populations()
    sim.close()
    assert relerr(gn, ref) <= 1e-5 and relerr(gf, ref) <= 1e-5 and relerr(gn, gf) <= 2e-5


def test_invalid_parameters(L):
    with pytest.raises(L.Lbm3Error):
        L.NSimulation(8, 8, sigma_of(7), tau=(1.0,) * 7)           # more than six fluids
    bad = sigma_of(3)
    bad[0, 1] = 0.02                                                # not symmetric
    with pytest.raises(L.Lbm3Error):
        L.NSimulation(8, 8, bad, tau=(1.0,) * 3)
    with pytest.raises(L.Lbm3Error):
        L.NSimulation(8, 8, sigma_of(3), tau=(1.0, 0.5, 1.0))      # tau must exceed 1/2


def test_fields_against_oracle(L):
    """lbm3n_fields after 10 steps of four fluids, against the oracle's fields
    of the same GPU populations (only the readout's own FP32 arithmetic is
    compared): colour densities to 1e-6 relative, the velocity of Eq. uk1 to
    5e-7 absolute, the pressure to 1e-6 relative."""
    n = 4
    p = N.NParams(24, 20, sigma=sigma_of(n), tau=tuple(0.6 + 0.15 * k for k in range(n)), rho0=(1.0,) * n)
    f0 = random_state(n, 24, 20, seed=n + 20)
    sim = L.NSimulation(p.nx, p.ny, p.sigma, p.tau, p.rho0, beta0=p.beta0)
    sim.set_populations(f0)
    sim.step(10)
    got = sim.fields()
    fg = sim.populations()
    sim.close()
    ref = N.fields(p, fg)
    assert np.abs(got["rho"] - ref["rho"]).max() <= 1e-6 * np.abs(ref["rho"]).max()
    for k in ("ux", "uy"):
        assert np.abs(got[k] - ref[k]).max() <= 5e-7, k
    assert np.abs(ref["ux"]).max() > 1e-6
    assert np.abs(got["p"] / ref["p"] - 1).max() <= 1e-6
