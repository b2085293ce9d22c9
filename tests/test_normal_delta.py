"""The paper's unit recolouring normal n_kl = G_kl/|G_kl| (Eq. 6; normal_delta
= 0) on the CUDA path, against the FP64 oracle run with the same normal.

The bars are those of the default (regularised) normal: relative population
error 1e-5 after one step and 1e-4 after 1000 steps on inputs whose own
FP32-level sensitivity is small (see test_parity.check_parity).
"""
import numpy as np
import pytest

import oracle as O
from paper_1808_08555_gb300 import workloads as W

from test_parity import L, check_parity, f32, oparams, relerr, run_pair  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("beta_form", [0, 1, 2, 3])
@pytest.mark.parametrize("recolor_form", [0, 1])
def test_unit_normal_random_state_one_step_8x8(L, beta_form, recolor_form):
    p = L.Params(8, 8, tau=(0.7, 1.0, 1.4), sigma=(0.012, 0.01, 0.008), beta_form=beta_form,
                 recolor_form=recolor_form, normal_delta=0.0)
    f0 = f32(W.random_populations(8, 8, seed=5 + beta_form))
    check_parity(L, p, f0, 1)


@pytest.mark.parametrize("nx,ny,R", [(260, 40, (4.0, 8.0)), (264, 1200, (4.0, 10.0))])
def test_unit_normal_droplets_across_tile_seams(L, nx, ny, R):
    rho = W.droplet_field(nx, ny, seed=nx + ny, count=8, rmin=R[0], rmax=R[1], gap=10.0)
    p = L.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=(0.01, 0.013, 0.007), normal_delta=0.0)
    f0 = f32(O.step(oparams(p), O.init(oparams(p), rho), 3))
    check_parity(L, p, f0, 10)


def test_unit_normal_two_droplets_64_1_and_1000_steps(L):
    c = W.case_two_droplets_64()
    p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, normal_delta=0.0)
    op = oparams(p)
    assert op.normal_delta == 0.0
    f0 = f32(O.init(op, c.rho))
    sim = L.Simulation(p)
    sim.set_populations(f0)
    fo, done, errs = f0, 0, {}
    for n in (1, 999):
        sim.step(n)
        fo = O.step(op, fo, n)
        done += n
        errs[done] = relerr(sim.populations(), fo)
    sim.close()
    assert errs[1] <= 1e-5 and errs[1000] <= 1e-4, errs


def test_unit_normal_moving_compound_256(L):
    c = W.case_compound_scaled(256)
    p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, normal_delta=0.0)
    f0 = f32(O.init(oparams(p), c.rho))
    fg, fo = run_pair(L, p, f0, 100)
    assert relerr(fg, fo) <= 1e-4


def test_normal_delta_changes_gpu_state_as_in_oracle(L):
    """The two normals differ on the GPU by what they differ in the oracle
    (two droplets, 200 steps): the GPU difference matches the oracle
    difference to 1e-6 in phi."""
    c = W.case_two_droplets_64()
    phis = {}
    for d in (0.0, 0.1):
        p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, normal_delta=d)
        f0 = f32(O.init(oparams(p), c.rho))
        fg, fo = run_pair(L, p, f0, 200)
        rg, ro = fg.sum(axis=1), fo.sum(axis=1)
        phis[d] = (rg / rg.sum(0), ro / ro.sum(0))
    dg = phis[0.0][0] - phis[0.1][0]
    do = phis[0.0][1] - phis[0.1][1]
    assert np.max(np.abs(dg - do)) <= 1e-6
