"""The Laplace-law measurement of Sec. III.A (analysis.laplace_measure,
laplace_slope) on synthetic fields whose jump and radius are known."""
import math

import numpy as np
import pytest

from paper_2407_10914_gb300 import analysis as A


def synthetic(n, R, rho_in, rho_out, two_d=False):
    shape = (1, n, n) if two_d else (n, n, n)
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(float)
    c = (n - 1) / 2.0
    r2 = (x - c) ** 2 + (y - c) ** 2 + (0 if two_d else (z - c) ** 2)
    r = np.sqrt(r2)
    phi = -np.tanh((r - R) / 1.5)  # red inside, a diffuse interface
    rho = np.where(r < R, rho_in, rho_out)
    return rho, phi


@pytest.mark.parametrize("two_d", [False, True])
def test_measure_recovers_jump_and_radius(two_d):
    rho, phi = synthetic(64, 14.0, 1.003, 0.999, two_d)
    dp, R = A.laplace_measure(rho, phi)
    assert dp == pytest.approx(0.004 / 3, rel=1e-12)
    assert R == pytest.approx(14.0, rel=0.01)


def test_slope_through_origin():
    gamma = 0.02
    radii = np.array([10.0, 14.0, 20.0, 26.0])
    dps = 2 * gamma / radii
    assert A.laplace_slope(dps, radii) == pytest.approx(gamma, rel=1e-14)
    assert A.laplace_slope(gamma / radii, radii, dims=2) == pytest.approx(
        gamma, rel=1e-14)
