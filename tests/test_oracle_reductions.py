"""Pins of the oracle's FP64 diagnostics (orc_reduce), by closed forms:

  - on the state at rest that init_state writes (f^s_i = w_i rho^s with
    rho^r = rho0 (1 + phi0)/2), the colour masses are the sums of those
    densities and S_w (count and smooth, Sec. IV.B) follow from phi0;
  - after one step of a Zou-He tube, the two planes hold exactly the
    prescribed densities (App. B), so Delta P = (rho_in - rho_out)/3
    (Eq. 23);
  - the capillary numbers average u along the flow axis over the nodes of
    one colour with that colour's viscosity, checked against the oracle's
    own velocity and phase fields.

A swapped colour, a missing 1/3 or rho0, the wrong sign of Delta P, a
count over solid nodes or the other colour's viscosity fails one of them."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import workloads as W


def pack_case(rho0=0.9):
    pack = W.sphere_pack((20, 16, 12), 0.4, rmin=2.0, rmax=4.0, seed=3,
                         reservoir=2)
    solid = pack["solid"]
    rng = np.random.default_rng(11)
    phi0 = np.where(rng.random(solid.shape) < 0.4, 1.0, -1.0)
    phi0 = np.where(rng.random(solid.shape) < 0.2,
                    rng.uniform(-0.9, 0.9, solid.shape), phi0)
    o = O.Oracle(19, solid, (True, True, True))
    o.set_params(rho0=rho0, tau_r=1.0, tau_b=0.7)
    o.init_state(phi0)
    return o, solid, phi0


def test_masses_and_saturations_at_rest():
    rho0 = 0.9
    o, solid, phi0 = pack_case(rho0)
    fl = solid == 0
    assert fl.sum() < solid.size  # the solids must be left out
    assert o.reduce(O.MASS_R) == pytest.approx(
        (rho0 * 0.5 * (1.0 + phi0))[fl].sum(), rel=1e-12)
    assert o.reduce(O.MASS_B) == pytest.approx(
        (rho0 * 0.5 * (1.0 - phi0))[fl].sum(), rel=1e-12)
    assert o.reduce(O.SW_COUNT) == pytest.approx((phi0[fl] < 0).mean(),
                                                 abs=1e-15)
    assert o.reduce(O.SW_SMOOTH) == pytest.approx(
        (0.5 * (1.0 - phi0[fl])).mean(), rel=1e-13)


def test_pressure_drop_after_one_zou_he_step():
    case = W.tube_3d(nx=40, red_len=10, rho_in=1.02, rho_out=0.98)
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    o.step(1)
    want = (case.params["rho_in"] - case.params["rho_out"]) / 3.0
    assert o.reduce(O.DP) == pytest.approx(want, rel=1e-12)


def test_capillary_numbers_follow_the_fields():
    o, solid, phi0 = pack_case(1.0)
    p = dict(rho0=1.0, tau_r=1.0, tau_b=0.7, gamma=0.02, g=(2e-4, 0.0, 0.0),
             flow_axis=0)
    o.set_params(**p)
    o.init_state(phi0)
    o.step(5)
    f = o.fields()
    fl = solid == 0
    red = fl & (f["phi"] > 0)
    blue = fl & ~(f["phi"] > 0)
    for kind, sel, tau in ((O.CA_R, red, 1.0), (O.CA_B, blue, 0.7)):
        mu = p["rho0"] * (tau - 0.5) / 3.0
        want = mu * f["u"][0][sel].mean() / p["gamma"]
        assert abs(want) > 0
        assert o.reduce(kind) == pytest.approx(want, rel=1e-12)
