"""Failure detection of the fused step kernel, on the GPU, without a fault.

Every mbarrier wait in the step kernel is bounded (2 s).  The testing hook
lbm3_debug_stall_row makes one CTA announce a population row that is never
copied, so that its consumers' waits run out: the kernel then flags the
error word and returns, and the host reports LBM3_ETIMEOUT at its next
synchronising call.  Nothing traps or hangs, and the context keeps working.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1808_08555_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3
    lbm3.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm3


@pytest.mark.gpu
def test_bounded_wait_times_out_and_context_recovers(L):
    c = W.case_two_droplets_64()
    p = L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0)
    sim = L.Simulation(p)
    sim.init(c.rho)
    m0, _ = sim.mass()
    L.lbm3_debug_stall_row(sim.ctx, 3)
    t0 = time.perf_counter()
    sim.step(1)
    with pytest.raises(L.Lbm3Error) as e:
        sim.mass()
    waited = time.perf_counter() - t0
    assert e.value.status == L.ETIMEOUT, e.value
    assert 1.5 < waited < 30.0, waited          # the 2 s bound, not a hang
    # the error word is cleared and the hook was one-shot: a fresh state steps normally
    sim.init(c.rho)
    sim.step(10)
    m1, _ = sim.mass()
    sim.close()
    assert np.abs(m1 / m0 - 1).max() <= 1e-6


@pytest.mark.gpu
def test_stall_hook_rejects_bad_rows(L):
    c = W.case_two_droplets_64()
    sim = L.Simulation(L.Params(c.nx, c.ny))
    with pytest.raises(L.Lbm3Error) as e:
        L.lbm3_debug_stall_row(sim.ctx, -2)
    assert e.value.status == L.EINVAL
    L.lbm3_debug_stall_row(sim.ctx, -1)
    sim.close()
