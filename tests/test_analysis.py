"""Analytic geometry of the paper's test cases, pinned to its printed tables
(Tab. 3 lens ratios, tab_gjd, tab_pjd) and to Neumann-triangle identities."""
import math

import pytest

from paper_1808_08555_gb300 import analysis as A


def test_neumann_angles_sum_and_sines():
    a = A.neumann_angles(0.010, 0.008, 0.012)
    assert sum(a) == pytest.approx(math.pi)
    assert [math.degrees(t) for t in a] == pytest.approx([55.77, 41.41, 82.82], abs=0.01)


@pytest.mark.parametrize("case,srb,srg,t1,t2,D,h1,h2", [
    ("a", 0.01, 0.01, 60, 60, 55.34, 15.97, 15.97),
    ("b", 0.0087, 0.005, 30, 60, 65.18, 8.73, 18.81),
    ("c", 0.02, 0.0173, 60, 90, 45.84, 13.23, 22.92),   # tensions as in the figure caption (Sec. 3.3)
    ("d", 0.0115, 0.0058, 30, 90, 50.99, 6.83, 25.49),
])
def test_lens_matches_table_3(case, srb, srg, t1, t2, D, h1, h2):
    """Tab. 3 analytic columns (Eq. 23), sigma_gb = 0.01, A = pi 20^2.  The
    printed tension sets are rounded from whole-degree contact angles
    (theta_1, theta_2) = (phi_rg, phi_rb); Eq. theta_kl recovers those to
    0.7 degrees, and Eq. 23 at the whole-degree angles gives the table to
    0.2 %."""
    p12, p13, _ = A.neumann_angles(srg, srb, 0.01)   # fluids r = 1, g = 2, b = 3
    assert math.degrees(p12) == pytest.approx(t1, abs=0.7)
    assert math.degrees(p13) == pytest.approx(t2, abs=0.7)
    Dc, h1c, h2c = A.lens_geometry(math.pi * 20.0 ** 2, math.radians(t1), math.radians(t2))
    assert (Dc, h1c, h2c) == pytest.approx((D, h1, h2), rel=2e-3)


@pytest.mark.parametrize("d_rg,sgb,srb,dgb", [
    (40, 0.01699, 0.01497, 204.08), (60, 0.01182, 0.01261, 201.81), (80, 0.00797, 0.00973, 207.52),
    (100, 0.00583, 0.00812, 216.63), (120, 0.00449, 0.00712, 227.67),
])
def test_gjd_matches_table(d_rg, sgb, srb, dgb):
    """tab_gjd: R_r = 60, R_g = 80, R_b = 160, sigma_rg = 0.01 (Eqs. gjd_01-06)."""
    g = A.gjd_geometry(60.0, 80.0, 160.0, float(d_rg), 0.01)
    assert g["d_gb"] == pytest.approx(dgb, abs=0.006)
    assert g["sigma_gb"] == pytest.approx(sgb, abs=6e-6)
    assert g["sigma_rb"] == pytest.approx(srb, abs=6e-6)


def test_gjd_kissing_limit():
    """tab_gjd's last row (d_rg = 140 = R_r + R_g, touching circles) is the
    limit of Eqs. gjd_01-06."""
    g = A.gjd_geometry(60.0, 80.0, 160.0, 140.0 - 1e-7, 0.01)
    assert g["d_gb"] == pytest.approx(240.00, abs=0.01)
    assert g["sigma_gb"] == pytest.approx(0.00357, abs=6e-6)
    assert g["sigma_rb"] == pytest.approx(0.00643, abs=6e-6)


@pytest.mark.parametrize("frac,Rb,dgb", [(0.1, 48.32, 93.46), (0.2, 88.39, 119.22), (0.3, 154.12, 173.64),
                                          (0.4, 331.92, 341.43)])
def test_pjd_matches_table(frac, Rb, dgb):
    """tab_pjd: R_r = R_g = 80 (Eq. pjd)."""
    g = A.pjd_geometry(80.0, frac)
    assert g["R_b"] == pytest.approx(Rb, abs=0.006)
    assert g["d_gb"] == pytest.approx(dgb, abs=0.006)


def test_laplace_error_definition():
    assert A.laplace_error(0.01 / 40, 40.0, 0.01 / 20, 20.0, 0.01, 0.01) == pytest.approx(0.0)
    assert A.laplace_error(1.013 * 0.01 / 40, 40.0, 1.013 * 0.01 / 20, 20.0, 0.01, 0.01) == pytest.approx(0.013)


def test_pressure_jump_of_a_step():
    import numpy as np
    y, x = np.mgrid[0:64, 0:80].astype(float)
    p = np.where(np.hypot(x - 40, y - 30) < 12, 1.0 + 0.02, 1.0)
    assert A.pressure_jump(p, (40, 30), 8, 16) == pytest.approx(0.02)
