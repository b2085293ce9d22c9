"""FP64 interface diagnostics on the device (lbm3_interface_diagnostics):
contact angles (Eq. theta_kl) and bulk pressures (Eq. laplace), against the
oracle's own implementation of the same measurement (oracle.diagnostics,
pinned on constructed fields) applied to the same FP64 fields, and on a
relaxed Janus droplet against the Neumann triangle and the oracle's run."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D
from paper_1808_08555_gb300 import workloads as W

from test_oracle_junctions import NEUMANN_SIGMA, constructed_junctions
from test_parity import L  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _phi(fl):
    return fl["rho"] / fl["rho"].sum(axis=0)


@pytest.mark.parametrize("a23,theta", [(-80.0, (97.18, 138.59, 124.23)), (-70.0, (140.0, 100.0, 120.0))])
def test_device_diagnostic_equals_oracle_measurement(L, a23, theta):
    """Same fields, two implementations: angles to 1e-7 degrees, circles and
    junctions to 1e-7 lattice units, point counts exactly, bulk pressures to
    1e-13 relative."""
    phi, want = constructed_junctions(n=128, a23=a23, theta=theta)
    sim = L.Simulation(L.Params(128, 128))
    sim.init(phi)
    fl = sim.fields()
    got = sim.interfaces()
    sim.close()
    ref = D.contact_angles(_phi(fl))
    assert got["flags"] == 0
    assert np.allclose(got["varphi"], ref["varphi"], rtol=0, atol=1e-7)
    assert np.allclose(got["varphi_junction"], ref["per_junction"], rtol=0, atol=1e-7)
    assert np.allclose(got["circles"], ref["circles"], rtol=0, atol=1e-7)
    assert np.allclose(sorted(got["junctions"]), sorted(ref["junctions"]), rtol=0, atol=1e-7)
    ph = _phi(fl)
    for q, (k, l) in enumerate(D.PAIRS):
        assert got["points"][q] == len(D.interface_points(ph, k, l))
    for k in range(3):
        assert got["n_bulk"][k] == (ph[k] > 0.99).sum()
        assert got["p_bulk"][k] == pytest.approx(D.bulk_pressure(ph, fl["p"], k), rel=1e-13)
    assert np.max(np.abs(np.array(got["varphi"]) - np.array(want))) < 0.3


def test_janus_relaxes_to_neumann_angles_on_gpu(L):
    """The oracle's Janus pin (96^2, R = 24, tensions (0.010, 0.008, 0.012),
    5000 steps) run by the CUDA path: the device diagnostic gives the Neumann
    angles within 1 degree and the oracle run's angles within 0.01 degree."""
    n, R, steps = 96, 24.0, 5000
    rho = W.janus_droplet(n, R)
    sim = L.Simulation(L.Params(n, n, sigma=NEUMANN_SIGMA))
    sim.init(rho)
    sim.step(steps)
    got = sim.interfaces()
    sim.close()
    op = O.Params(n, n, sigma=NEUMANN_SIGMA)
    fo = O.fields(op, O.step(op, O.init(op, rho), steps))
    ref = D.contact_angles(_phi(fo))["varphi"]
    assert np.max(np.abs(np.array(got["varphi"]) - np.array(D.neumann_angles(NEUMANN_SIGMA)))) < 1.0
    assert np.max(np.abs(np.array(got["varphi"]) - np.array(ref))) < 0.01, (got["varphi"], ref)


def test_diagnostics_degenerate_and_invalid(L):
    """A uniform state has no interface: NaN angles with flag bit 0, bulk
    pressure of the one fluid present; bad thresholds are LBM3_EINVAL."""
    sim = L.Simulation(L.Params(64, 32))
    rho = np.zeros((3, 32, 64))
    rho[0] = 1.0
    sim.init(rho)
    got = sim.interfaces()
    assert got["flags"] & 1 and all(np.isnan(got["varphi"]))
    assert got["n_bulk"] == [64 * 32, 0.0, 0.0] and got["p_bulk"][0] == pytest.approx(1 / 3, rel=1e-7)
    assert np.isnan(got["p_bulk"][1])
    for tm, bm in ((0.0, 0.99), (1e-3, 1.0), (2.0, 0.5)):
        with pytest.raises(L.Lbm3Error) as e:
            sim.interfaces(tm, bm)
        assert e.value.status == L.EINVAL
    sim.close()
