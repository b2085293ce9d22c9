"""Batched instances (a morphology sweep): every instance of a batch must
evolve exactly as it does alone (same per-node arithmetic, bit for bit), and
one instance is checked against the FP64 oracle as well."""
import numpy as np
import pytest

import oracle as O
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


def _instances(L):
    specs = [  # (nx, ny, tau, sigma, beta_form, recolor_form)
        (128, 128, (1.0, 1.0, 1.0), (0.002, 0.004, 0.01), 0, 0),
        (192, 96, (0.6, 0.7, 0.9), (0.01, 0.012, 0.005), 0, 0),
        (64, 200, (0.8, 0.8, 0.8), (0.01, 0.02, 0.01), 2, 0),     # critical sigma_13 = sigma_12 + sigma_23
        (256, 40, (1.0, 0.9, 1.2), (0.012, 0.01, 0.008), 3, 1),
        (12, 8, (0.7, 1.0, 1.4), (0.01, 0.013, 0.007), 1, 0),
    ]
    params, fields = [], []
    for j, (nx, ny, tau, sig, bf, rf) in enumerate(specs):
        params.append(L.Params(nx, ny, tau=tau, sigma=sig, beta_form=bf, recolor_form=rf))
        n = min(nx, ny)
        if n >= 64:
            rho = W.droplet_field(nx, ny, seed=j, count=5, rmin=5.0, rmax=n / 6, gap=10.0)
        else:
            rho = W.random_fields(nx, ny, seed=j)
        fields.append(rho)
    return params, fields


@pytest.mark.parametrize("steps", [1, 6, 7])
def test_batch_equals_single_instances_bitwise(L, steps):
    params, fields = _instances(L)
    batch = L.Batch(params, rows_per_cta=24)
    for i, rho in enumerate(fields):
        batch.init(i, rho)
    batch.step(steps)
    assert batch.t == steps
    for i, (p, rho) in enumerate(zip(params, fields)):
        sim = L.Simulation(p)
        sim.init(rho)
        sim.step(steps)
        np.testing.assert_array_equal(batch.populations(i), sim.populations(), err_msg=f"instance {i}")
        sim.close()
    batch.close()


def test_batch_instance_against_oracle(L):
    params, fields = _instances(L)
    batch = L.Batch(params[:2])
    op = O.Params(params[1].nx, params[1].ny, tau=params[1].tau, sigma=params[1].sigma)
    f0 = np.asarray(O.init(op, fields[1]), dtype=np.float32).astype(np.float64)
    batch.init(0, fields[0])
    batch.set_populations(1, f0)
    batch.step(4)
    fg = batch.populations(1)
    fo = O.step(op, f0, 4)
    err = np.max(np.abs(fg - fo) / np.maximum(np.abs(fo), 1e-3 * WGT[None, :, None, None]))
    assert err <= 1e-5
    m, _ = batch.mass(1)
    np.testing.assert_allclose(m, fg.reshape(3, 9, -1).sum(axis=(1, 2)), rtol=1e-12)
    batch.close()


def test_batch_errors(L):
    params, fields = _instances(L)
    batch = L.Batch(params[:2])
    batch.init(0, fields[0])
    with pytest.raises(L.Lbm3Error) as e:
        batch.step(1)                      # instance 1 not initialised
    assert e.value.status == L.ESTATE
    with pytest.raises(L.Lbm3Error) as e:
        batch.init(5, fields[0])
    assert e.value.status == L.EINVAL
    batch.close()
    bad = [L.Params(8, 8), L.Params(6, 8)]
    with pytest.raises(L.Lbm3Error):
        L.Batch(bad)


def test_autotune_keeps_state_and_results(L):
    """Empirical tile-height tuning: the timed candidates leave the state and
    the time unchanged, the winner is one of the candidates, and steps after
    tuning (also through the step graphs, which are captured again) equal
    single-instance runs bit for bit."""
    params, fields = _instances(L)
    batch = L.Batch(params)
    for i, rho in enumerate(fields):
        batch.init(i, rho)
    batch.step(3)
    before = [batch.populations(i) for i in range(len(params))]
    res = batch.autotune(candidates=4, steps=3)
    assert batch.t == 3
    assert res["rows"] in [r for r, _ in res["candidates"]]
    assert len(res["candidates"]) >= 4 and all(t > 0 for _, t in res["candidates"])
    assert res["ms_per_step"] == min(t for _, t in res["candidates"])
    for i in range(len(params)):
        np.testing.assert_array_equal(batch.populations(i), before[i])
    batch.step(5)
    for i, (p, rho) in enumerate(zip(params, fields)):
        sim = L.Simulation(p)
        sim.init(rho)
        sim.step(8)
        np.testing.assert_array_equal(batch.populations(i), sim.populations(), err_msg=f"instance {i}")
        sim.close()
    with pytest.raises(L.Lbm3Error):
        batch.autotune(candidates=0)
    batch.close()


def _reduced(L, params):
    return [L.Params(**{**p.__dict__, "storage": L.REDUCED}) for p in params]


@pytest.mark.parametrize("steps", [1, 6, 7])
def test_reduced_batch_equals_single_fp32_instances(L, steps):
    """A batch in the reduced state (the first step from the set
    populations, then reduced steps through the step graphs) gives every
    instance's FP32 single-grid populations bit for bit."""
    params, fields = _instances(L)
    batch = L.Batch(_reduced(L, params), rows_per_cta=24)
    for i, rho in enumerate(fields):
        batch.init(i, rho)
    batch.step(steps)
    for i, (p, rho) in enumerate(zip(params, fields)):
        sim = L.Simulation(p)
        sim.init(rho)
        sim.step(steps)
        np.testing.assert_array_equal(batch.populations(i), sim.populations(), err_msg=f"instance {i}")
        sim.close()
    batch.close()


def test_reduced_batch_one_instance_reset_midway(L):
    """Setting one instance's populations mid-run splits the next step into
    a populations-in launch for it and a reduced launch for the others; the
    instance is set to its own populations, so every trajectory is unchanged.
    Tuning a batch that holds set populations is refused until it steps."""
    params, fields = _instances(L)
    batch = L.Batch(_reduced(L, params))
    for i, rho in enumerate(fields):
        batch.init(i, rho)
    batch.step(3)
    batch.set_populations(1, batch.populations(1))
    with pytest.raises(L.Lbm3Error) as e:
        batch.autotune(candidates=2, steps=1)
    assert e.value.status == L.ESTATE
    batch.step(4)
    res = batch.autotune(candidates=2, steps=2)
    assert res["rows"] > 0
    batch.step(1)
    for i, (p, rho) in enumerate(zip(params, fields)):
        sim = L.Simulation(p)
        sim.init(rho)
        sim.step(8)
        np.testing.assert_array_equal(batch.populations(i), sim.populations(), err_msg=f"instance {i}")
        sim.close()
    batch.close()
