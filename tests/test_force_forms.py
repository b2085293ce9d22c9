"""The perturbation-operator force form (Eqs. phi1 / phi_old, Leclaire et
al.), the alternative the paper compares its body-force scheme with (Tab. 2):
GPU parity with the FP64 oracle (which the pins of test_oracle_pins.py tie to
the operator's closed-form moments and to Young-Laplace), and the paper's
Young-Laplace / spurious-velocity experiment (Tabs. 1 and 2) for both forms."""
import numpy as np
import pytest

import oracle as O
from paper_1808_08555_gb300 import workloads as W

from test_parity import check_parity, f32, oparams, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3
    lbm3.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm3


@pytest.mark.parametrize("beta_form,recolor_form", [(0, 0), (1, 0), (3, 1)])
def test_perturbation_one_step_8x8(L, beta_form, recolor_form):
    sig = (0.01, 0.008, 0.012) if beta_form == 3 else (0.012, 0.01, 0.008)
    p = L.Params(8, 8, tau=(0.7, 1.0, 1.4), sigma=sig, beta_form=beta_form, recolor_form=recolor_form,
                 force_form=L.FORCE_PERTURBATION)
    f0 = f32(W.random_populations(8, 8, seed=21 + beta_form))
    check_parity(L, p, f0, 1)


@pytest.mark.parametrize("nx,ny,rows", [(200, 37, 8), (260, 40, 0)])
def test_perturbation_droplets_across_tile_seams(L, nx, ny, rows):
    rho = W.droplet_field(nx, ny, seed=nx + ny, count=8, rmin=4.0, rmax=10.0, gap=10.0)
    p = L.Params(nx, ny, tau=(0.6, 0.9, 1.3), sigma=(0.01, 0.013, 0.007), force_form=L.FORCE_PERTURBATION)
    f0 = f32(O.step(oparams(p), O.init(oparams(p), rho), 3))
    check_parity(L, p, f0, 10, rows)


def test_perturbation_two_droplets_1000_steps_and_fields(L):
    c = W.case_two_droplets_64()
    p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, force_form=L.FORCE_PERTURBATION)
    op = oparams(p)
    f0 = f32(O.init(op, c.rho))
    m0 = f0.reshape(3, 9, -1).sum(axis=(1, 2))
    sim = L.Simulation(p)
    sim.set_populations(f0)
    sim.step(1)
    e1 = relerr(sim.populations(), O.step(op, f0, 1))
    sim.step(999)
    fo = O.step(op, f0, 1000)
    e1000 = relerr(sim.populations(), fo)
    m1, _ = sim.mass()
    fl = sim.fields()
    sim.close()
    assert e1 <= 1e-5 and e1000 <= 1e-4, (e1, e1000)
    assert np.abs(m1 / m0 - 1).max() <= 5e-6, m1 / m0 - 1
    ref = O.fields(op, fo)
    # u = sum_i f_i e_i / rho with this force form (no F/2 term)
    np.testing.assert_allclose(fl["ux"], ref["ux"], rtol=0, atol=2e-7)
    np.testing.assert_allclose(fl["uy"], ref["uy"], rtol=0, atol=2e-7)


def test_tables_1_and_2_young_laplace_and_spurious_velocities(L):
    """Sec. 3.2: compound droplet, R_g = 2 R_r, sigma = 0.01, nu = 0.1, 160^2,
    at equilibrium (40000 steps).  Tab. 1: the Young-Laplace error eps
    (Eq. 22) stays below 1.5 % for R_r = 15..30.  Tab. 2: the body-force
    scheme's spurious speeds are below the perturbation operator's at every
    R_r, the operator's are nearly independent of R_r, and both are of the
    order the paper prints (1.7e-5 and 3.2e-5).  (At equilibrium the
    body-force speeds keep falling with R_r, 1.0e-5 to 0.3e-5; the
    near-constant 1.1-1.4e-5 appears only mid-transient, at 20000 steps.)"""
    from paper_1808_08555_gb300 import experiments as X
    body = [X.young_laplace_compound(R, L.FORCE_BODY) for R in (15, 20, 25, 30)]
    pert = [X.young_laplace_compound(R, L.FORCE_PERTURBATION) for R in (15, 20, 25, 30)]
    for b in body:
        assert b["eps"] < 0.015, b
    ub = np.array([b["umax"] for b in body])
    up = np.array([q["umax"] for q in pert])
    assert np.all(ub < up), (ub, up)
    assert up.max() / up.min() < 1.5, up
    assert np.all((ub > 1e-6) & (ub < 5e-5)) and np.all((up > 1e-5) & (up < 1e-4)), (ub, up)


def test_set_params_switches_force_form_and_validates(L):
    """lbm3_set_params swaps the physical parameters of a live context (here
    the force form and the tensions) and the next steps follow the oracle
    with the new ones; a different grid, storage or an invalid form is
    refused, as is the perturbation operator in a batch."""
    nx, ny = 64, 40
    rho = W.droplet_field(nx, ny, seed=9, count=4, rmin=4.0, rmax=8.0, gap=8.0)
    p0 = L.Params(nx, ny, sigma=(0.01, 0.013, 0.007))
    p1 = L.Params(nx, ny, sigma=(0.012, 0.009, 0.011), force_form=L.FORCE_PERTURBATION)
    f0 = f32(O.step(oparams(p0), O.init(oparams(p0), rho), 3))
    sim = L.Simulation(p0)
    sim.set_populations(f0)
    sim.set_params(p1)
    sim.step(5)
    err = relerr(sim.populations(), O.step(oparams(p1), f0, 5))
    assert err <= 1e-5, err
    for bad in (L.Params(nx + 4, ny), L.Params(nx, ny, storage=L.FP16_DEV), L.Params(nx, ny, force_form=3)):
        with pytest.raises(L.Lbm3Error) as e:
            L.lbm3_set_params(sim.ctx, bad)
        assert e.value.status == L.EINVAL
    sim.close()
    with pytest.raises(L.Lbm3Error):
        L.Batch([L.Params(128, 128, force_form=L.FORCE_PERTURBATION)])


def test_phi_needs_fp32_storage(L):
    sim = L.Simulation(L.Params(32, 32, storage=L.FP16_DEV))
    sim.init(W.two_droplets(32, 32, R=5.0, c2=(8.0, 16.0), c3=(24.0, 16.0)))
    with pytest.raises(L.Lbm3Error) as e:
        sim.phi()
    assert e.value.status == L.EINVAL
    sim.close()
