"""The Washburn law of Sec. IV.A (Eqs. 47-51) as washburn.py writes it, and
its interface measurement, pinned against the dimensional form (Eq. 48 in
analysis.py), the implicit law it solves (Eq. 47) and synthetic fields."""
import math

import numpy as np
import pytest

from paper_2407_10914_gb300 import analysis as A
from paper_2407_10914_gb300 import washburn as Wb


def test_eq49_is_eq48_made_dimensionless():
    L, r, gamma = 100.0, 5.0, 1.0 / 45.0
    mu_w, mu_nw = 1.0 / 6.0, 1.0 / 30.0
    m = mu_nw / (mu_w - mu_nw)
    for theta in (30.0, 60.0, 85.0):
        for dP in (0.0, 1e-4):
            t = np.linspace(0.0, 5e4, 11)
            z = A.washburn_z(t, r, L, dP, gamma, theta, mu_w, mu_nw)
            ts = gamma * t / ((mu_w - mu_nw) * L)            # Eq. (51)
            zs = Wb.zstar(ts, theta, m, r / L, dP * r * r / (2 * L * gamma))
            np.testing.assert_allclose(zs, z / L, rtol=1e-12, atol=1e-15)


def test_eq49_solves_eq47():
    """Substituting z(t) back into the implicit Washburn law (Eq. 47)."""
    L, r, gamma, theta = 100.0, 5.0, 1.0 / 45.0, 50.0
    mu_w, mu_nw = 1.0 / 6.0, 1.0 / 30.0
    m = mu_nw / (mu_w - mu_nw)
    ts = np.linspace(0.0, 80.0, 17)
    z = L * Wb.zstar(ts, theta, m, r / L)
    t = ts * (mu_w - mu_nw) * L / gamma
    lhs = z * z * (mu_w - mu_nw) / 2 + mu_nw * L * z
    rhs = r * r / 8 * (2 * gamma / r * math.cos(math.radians(theta))) * t
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-9)


def test_tstar_inverts_zstar():
    for z in (0.03, 0.2, 0.7):
        t = Wb.tstar_of(z, 40.0, 0.25, 0.05)
        assert Wb.zstar(t, 40.0, 0.25, 0.05) == pytest.approx(z, rel=1e-12)


def test_interface_tip_of_a_synthetic_front():
    """A tanh front centred at x = 37.3 in a square tube: the crossing is
    found at 37.3 to interpolation accuracy, from the inlet side."""
    nz = ny = 12
    nx = 101
    x = np.arange(nx, dtype=float)
    phi = np.broadcast_to(np.tanh((x - 37.3) / 2.0), (nz, ny, nx)).copy()
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    solid[:, 0] = solid[:, -1] = 1
    assert Wb.interface_tip(phi, solid) == pytest.approx(37.3, abs=0.02)
    # no crossing: nan
    assert math.isnan(Wb.interface_tip(-np.ones_like(phi), solid))
