"""Reduced state (LBM3_REDUCED): per node phi_k, the post-collision totals
f^dagger_i and the recolouring vectors V_k instead of 27 populations.
Collision and recolouring use only the total distribution and the colour
densities (Eqs. 1 and 6), so each pulled population phi_k f^dagger_i +
w'_i e_i . V_k is rebuilt from its source node with the FP32 storage's own
operations: the trajectory must equal the FP32 storage's bit for bit, and
with it the FP64 oracle within the FP32 bars."""
import numpy as np
import pytest

import oracle as O
from paper_1808_08555_gb300 import workloads as W

from test_parity import L, f32, oparams, relerr  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(L, p, f0, steps, rows=0, chunks=None):
    sim = L.Simulation(p, rows_per_cta=rows)
    sim.set_populations(f0)
    out = []
    for n in (chunks or [steps]):
        sim.step(n)
        out.append(sim.populations())
    m, mo = sim.mass()
    fl = sim.fields()
    sim.close()
    return out, m, mo, fl


def _both(L, p, f0, steps, rows=0, chunks=None):
    pr = L.Params(**{**p.__dict__, "storage": L.REDUCED})
    a = _run(L, p, f0, steps, rows, chunks)
    b = _run(L, pr, f0, steps, rows, chunks)
    return a, b


def _assert_identical(a, b):
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y), np.abs(x - y).max()
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for k in ("rho", "ux", "uy", "p"):
        assert np.array_equal(a[3][k], b[3][k]), k


@pytest.mark.parametrize("beta_form,recolor_form,delta", [(0, 0, 0.1), (1, 0, 0.1), (2, 1, 0.1), (3, 0, 0.0)])
def test_reduced_equals_fp32_random_8x8(L, beta_form, recolor_form, delta):
    p = L.Params(8, 8, tau=(0.7, 1.0, 1.4), sigma=(0.012, 0.01, 0.008), beta_form=beta_form,
                 recolor_form=recolor_form, normal_delta=delta)
    f0 = f32(W.random_populations(8, 8, seed=11 + beta_form))
    _assert_identical(*_both(L, p, f0, 5, chunks=[1, 4]))


@pytest.mark.parametrize("nx,ny,rows", [(4, 3, 1), (12, 1, 1), (8, 4, 2)])
def test_reduced_equals_fp32_tiny_grids(L, nx, ny, rows):
    """Grids narrower than the ghost band: nodes with both ghost copies."""
    p = L.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=(0.01, 0.013, 0.007))
    f0 = f32(W.random_populations(nx, ny, seed=nx + ny))
    _assert_identical(*_both(L, p, f0, 3, rows, chunks=[1, 2]))


@pytest.mark.parametrize("nx,ny,rows", [(264, 1200, 0), (128, 3000, 0), (320, 72, 8), (136, 21, 5)])
def test_reduced_equals_fp32_across_tile_seams(L, nx, ny, rows):
    rho = W.droplet_field(nx, ny, seed=nx + ny, count=8, rmin=4.0, rmax=10.0, gap=10.0)
    p = L.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=(0.01, 0.013, 0.007))
    f0 = f32(O.step(oparams(p), O.init(oparams(p), rho), 3))
    _assert_identical(*_both(L, p, f0, 10, rows, chunks=[1, 9]))


def test_reduced_two_droplets_64_against_oracle(L):
    """Config-1 bars directly: 1e-5 after 1 step, 1e-4 after 1000 steps, and
    the FP32 storage's populations bit for bit at both times."""
    c = W.case_two_droplets_64()
    p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, storage=L.REDUCED)
    op = oparams(p)
    f0 = f32(O.init(op, c.rho))
    (g1, g1000), m, _, _ = _run(L, p, f0, 1000, chunks=[1, 999])
    assert relerr(g1, O.step(op, f0, 1)) <= 1e-5
    assert relerr(g1000, O.step(op, f0, 1000)) <= 1e-4
    pf = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0)
    (h1, h1000), mf, _, _ = _run(L, pf, f0, 1000, chunks=[1, 999])
    assert np.array_equal(g1, h1) and np.array_equal(g1000, h1000) and np.array_equal(m, mf)


def test_reduced_compound_2048_sampled_equals_fp32(L):
    """The benchmark's 2048^2 workload in its launch configuration: after 20
    steps the reduced and FP32 states agree bit for bit at sampled nodes
    (interfaces, tile seams, the domain wrap) and in the FP64 masses."""
    c = W.case_compound_2048()
    out = {}
    for st in (L.FP32, L.REDUCED):
        sim = L.Simulation(L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, storage=st))
        sim.init(c.rho)
        sim.step(20)
        fl = sim.fields()
        out[st] = (fl["rho"], fl["ux"], fl["uy"], sim.mass()[0])
        sim.close()
    for a, b in zip(out[L.FP32], out[L.REDUCED]):
        assert np.array_equal(a, b)


def test_reduced_state_io_and_param_change(L):
    """init, set_populations mid-run, lbm3_phi and a parameter change that
    alters the recolouring weights: the reduced storage follows the FP32
    storage exactly through all of them."""
    nx, ny = 96, 64
    rho = W.two_droplets(nx, ny, R=10.0, c2=(30.0, 32.0), c3=(66.0, 32.0))
    res = {}
    for st in (L.FP32, L.REDUCED):
        p = L.Params(nx, ny, tau=(0.7, 0.9, 1.2), sigma=(0.01, 0.012, 0.006), storage=st)
        sim = L.Simulation(p)
        sim.init(rho)
        sim.step(7)
        mid = sim.populations()
        sim.set_populations(mid)
        sim.step(3)
        phi = sim.phi()
        sim.set_params(L.Params(**{**p.__dict__, "recolor_form": L.RECOLOR_LITERAL, "sigma": (0.011, 0.012, 0.007)}))
        sim.step(5)
        res[st] = (mid, phi, sim.populations(), sim.interfaces()["p_bulk"])
        sim.close()
    for a, b in zip(res[L.FP32], res[L.REDUCED]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
