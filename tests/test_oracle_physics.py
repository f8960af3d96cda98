"""Physics pins of the oracle: exact invariants, closed forms and the
validation cases of the paper (Laplace law, Sec. III.A; static contact
angle, Sec. III.B; Washburn flow, Sec. IV.A), at reduced sizes."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import analysis as A
from paper_2407_10914_gb300 import workloads as W


def run(case, steps=None):
    o = O.Oracle(case.lattice, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    o.step(case.steps if steps is None else steps)
    return o


@pytest.mark.parametrize("wetting", [1, 2])
def test_mass_conserved_per_colour(wetting):
    """Streaming with halfway bounce-back, collision and recolouring conserve
    each colour's mass exactly (periodic box, no Zou-He), with wetting,
    unequal viscosities and a body force."""
    pack = W.sphere_pack((24, 20, 18), 0.45, reservoir=0, side_walls=False,
                         seed=3)
    solid = pack["solid"]
    rng = np.random.default_rng(4)
    phi0 = np.where(rng.random(solid.shape) < 0.5, 1.0, -1.0)
    phi0[solid == 1] = 0
    case = W.Case("pack", 19, solid, (True, True, True), phi0,
                  W.base_params(tau_r=1.0, tau_b=0.6, theta_deg=45.0,
                                wetting=wetting, gamma=0.02,
                                g=(2e-5, -1e-5, 0.0)), 600)
    o = O.Oracle(19, solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(phi0)
    m0 = (o.reduce(O.MASS_R), o.reduce(O.MASS_B))
    o.step(600)
    assert abs(o.reduce(O.MASS_R) / m0[0] - 1) < 1e-12
    assert abs(o.reduce(O.MASS_B) / m0[1] - 1) < 1e-12


@pytest.mark.parametrize("wetting", [1, 2])
def test_symmetric_droplet_stays_symmetric(wetting):
    """A half-disc centred on a mirror plane stays mirror-symmetric."""
    case = W.droplet_2d(theta_deg=75.0, wetting=wetting)
    o = run(case, 300)
    phi = o.fields()["phi"][0]
    np.testing.assert_allclose(phi, phi[:, ::-1], atol=1e-11)


def test_laplace_law_2d():
    """Sec. III.A in 2-D: the pressure jump over a drop of radius R is
    gamma / R. Each of three radii within 4 %, and the least-squares slope
    of dP against 1/R through the origin within 3 %."""
    gamma = 0.01
    xs, ys = [], []
    for R0 in (10.0, 14.0, 18.0):
        case = W.laplace_drop(9, 72, R0, gamma=gamma, beta=0.7, steps=3000)
        o = run(case)
        f = o.fields()
        phi, rho = f["phi"][0], f["rho"][0]
        R = math.sqrt(((1 + phi) / 2).sum() / math.pi)
        y, x = np.mgrid[0:72, 0:72]
        r = np.hypot(x - 35.5, y - 35.5)
        dp = (rho[r < R / 2].mean() - rho[r > R + 8].mean()) / 3
        assert abs(dp * R / gamma - 1) < 0.04
        xs.append(1 / R)
        ys.append(dp)
    xs, ys = np.array(xs), np.array(ys)
    slope = (xs * ys).sum() / (xs * xs).sum()
    assert abs(slope / gamma - 1) < 0.03


def test_laplace_law_3d_unequal_viscosity():
    """Sec. III.A in 3-D with the paper's viscosity ratio (tau^r = 1.0,
    tau^b = 0.6): the jump is 2 gamma / R, within 8 % on a 32^3 box."""
    gamma = 0.01
    case = W.laplace_drop(19, 32, 8.0, gamma=gamma, beta=0.95, tau_r=1.0,
                          tau_b=0.6, steps=1200)
    o = run(case)
    f = o.fields()
    phi, rho = f["phi"], f["rho"]
    R = (3 * ((1 + phi) / 2).sum() / (4 * math.pi)) ** (1 / 3)
    z, y, x = np.mgrid[0:32, 0:32, 0:32]
    r = np.sqrt((x - 15.5) ** 2 + (y - 15.5) ** 2 + (z - 15.5) ** 2)
    dp = (rho[r < R / 2].mean() - rho[r > R + 5].mean()) / 3
    assert abs(dp * R / (2 * gamma) - 1) < 0.08


@pytest.mark.parametrize("tau", [1.0, 0.8, 0.5 + math.sqrt(3 / 16)])
def test_poiseuille_closed_form(tau):
    """Body-forced channel between halfway bounce-back walls: the steady
    profile is exactly u(y) = g/(2 nu) (y - y0)(y1 - y) + u_s with the walls
    at y0 = 0.5, y1 = ny - 1.5 and the slip u_s = g (16 L - 3) / (24 nu),
    L = (tau - 1/2)^2 (the single-rate case of the two-relaxation-time
    analysis of bounce-back; zero slip at L = 3/16)."""
    g, ny = 1e-6, 19
    case = W.channel_2d(nx=4, ny=ny, g=g, tau=tau)
    o = run(case, 30000)
    u = o.fields()["u"][0, 0, :, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(ny, dtype=float)[1:-1]
    us = g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
    expect = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y) + us
    np.testing.assert_allclose(u[1:-1], expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("phi0", [0.3, -0.55])
def test_mixture_channel_viscosity(phi0):
    """Eqs. (13)-(14) pinned by a single-phase flow: a uniform mixture phi0
    of fluids with tau^r = 1.0 and tau^b = 0.6 has no colour gradient (C = 0,
    so neither recolouring nor surface tension acts) and flows as one fluid
    of the harmonic-mean viscosity 1/nu = (1 + phi0)/(2 nu^r) +
    (1 - phi0)/(2 nu^b). The body-forced channel then reaches the closed
    form of test_poiseuille_closed_form with tau = 3 nu + 1/2. Swapping
    nu^r and nu^b or taking the arithmetic mean of the viscosities moves
    the centre-line speed by 30-120 %."""
    g, ny = 1e-6, 19
    case = W.channel_2d(nx=4, ny=ny, g=g, tau=1.0)
    phi = np.full(case.solid.shape, float(phi0))
    phi[case.solid == 1] = 0.0
    o = O.Oracle(9, case.solid, case.periodic)
    o.set_params(**dict(case.params, tau_r=1.0, tau_b=0.6))
    o.init_state(phi)
    o.step(30000)
    f = o.fields()
    u = f["u"][0, 0, :, 0]
    fluid = case.solid[0, :, 0] == 0
    assert np.abs(f["phi"][0, :, 0][fluid] - phi0).max() < 1e-12
    nur, nub = 0.5 / 3, 0.1 / 3
    nu = 1.0 / ((1 + phi0) / (2 * nur) + (1 - phi0) / (2 * nub))
    tau = 3 * nu + 0.5
    y = np.arange(ny, dtype=float)[1:-1]

    def profile(nu, tau):
        us = g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
        return g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y) + us

    np.testing.assert_allclose(u[1:-1], profile(nu, tau), rtol=0, atol=1e-12)
    for wrong in (1.0 / ((1 + phi0) / (2 * nub) + (1 - phi0) / (2 * nur)),
                  0.5 * ((1 + phi0) * nur + (1 - phi0) * nub)):
        other = profile(wrong, 3 * wrong + 0.5)
        assert np.abs(other - u[1:-1]).max() > 0.3 * np.abs(u[1:-1]).max()


@pytest.mark.parametrize("wetting,theta,tol", [(2, 60.0, 1.5), (1, 60.0, 1.5),
                                               (2, 120.0, 3.0)])
def test_static_contact_angle(wetting, theta, tol):
    """Sec. III.B: a drop relaxes to the prescribed angle (through fluid b),
    measured from its base and height with Eqs. (45)-(46)."""
    case = W.droplet_2d(theta_deg=theta, wetting=wetting)
    o = run(case, 14000)
    phi = o.fields()["phi"][0]
    th = A.droplet_contact_angle(phi, 0, case.info["centre"][0])
    assert abs(th - theta) < tol, th


@pytest.mark.parametrize("wetting,theta", [(2, 60.0), (1, 120.0)])
def test_static_contact_angle_d3q19(wetting, theta):
    """Sec. III.B in 3-D: a D3Q19 sessile drop (R = 8 on the wall z = 0 of a
    32 x 32 x 20 box) relaxes to the prescribed angle through fluid b,
    measured with the 3-D form of Eqs. (45)-(46) (central sections through
    the drop's axis). At this drop size the diffuse interface biases the
    base measure by 1-4.5 deg (the paper's R = 30 drops: +3.6/-2.2 deg for
    Scheme-I), so the bound is 5 deg; the angle is settled by 4500 steps
    (it moves by less than 0.1 deg from there to 9000)."""
    case = W.droplet_3d(side=32, radius=8.0, theta_deg=theta, wetting=wetting,
                        shape=(20, 32, 32))
    o = run(case, 4500)
    th, ax, ay = A.sessile_angle_3d(o.fields()["phi"], *case.info["centre"][:2])
    assert abs(ax - ay) < 1e-3  # x <-> y symmetric up to summation order
    assert abs(th - theta) < 5.0, th


def test_washburn_equal_viscosity():
    """Sec. IV.A, pressure-driven case with theta = 90 deg (Scheme-I) and
    equal viscosities: Eq. (47) reduces to z(t) = z0 + r^2 dP t/(8 mu L).
    The interface speed must match it within 10 % (the paper's errors in
    this case are about 9 %) on a short tube."""
    nx = 64
    case = W.tube_3d(nx=nx, red_len=16)
    o = O.Oracle(19, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    ts, zs = [], []
    for k in range(6):
        o.step(500)
        ts.append(500.0 * (k + 1))
        zs.append(A.interface_position(o.fields()["phi"], 0, case.solid))
    U = np.polyfit(ts[2:], zs[2:], 1)[0]
    dP = (case.params["rho_in"] - case.params["rho_out"]) / 3
    mu = case.params["rho0"] * (case.params["tau_r"] - 0.5) / 3
    U_ref = case.info["radius"] ** 2 * dP / (8 * mu * (nx - 1))
    assert abs(U / U_ref - 1) < 0.10, (U, U_ref)
