"""Pins of the oracle's MRT collision (Eq. 2 in moment space with the rates
of Eqs. 4, 15 and 16, Appendix A): its M against the printed Eq. (A.3); with
every rate equal it is the single-rate collision (pinned separately against
A.4/A.5); each moment of the printed basis relaxes at its own rate; the
rates of Eq. (16) make the body-forced channel between halfway bounce-back
walls exactly parabolic with no slip (the two-relaxation-time condition
Lambda = 3/16); the step with MRT conserves each colour's mass."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import workloads as W

from test_oracle_lattice import SF_A5, load_M, meq_A4, random_pops


def test_moment_matrix_is_eq_A3():
    """The oracle builds M from the moment polynomials of Eq. (3); it equals
    the printed matrix (with the reading of its garbled rows 13/14), and
    its rows are mutually orthogonal."""
    M = O.moment_matrix()
    np.testing.assert_array_equal(M, load_M())
    G = M @ M.T
    np.testing.assert_array_equal(G, np.diag(np.diag(G)))


def test_equal_rates_give_the_single_rate_collision():
    """S_q = S_m = S_nu turns Eq. (4) into one rate for every non-conserved
    moment: the MRT result equals the velocity-space single-rate form."""
    rng = np.random.default_rng(21)
    for _ in range(40):
        f = random_pops(rng, 19)
        F = 1e-3 * rng.standard_normal(3)
        S = 0.3 + 1.6 * rng.random()
        rho0 = 0.9 + 0.2 * rng.random()
        a, ua = O.collide_mrt(f, F, S, rho0, Sq=S, Sm=S)
        b, ub = O.collide(19, f, F, S, rho0)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
        np.testing.assert_array_equal(ua, ub)


def test_each_moment_relaxes_at_its_rate():
    """Through the printed M: conserved moments keep their value (momentum
    gains F), and every other moment k becomes
    m_k - S_k (m_k - m_k^eq) + (1 - S_k/2) S^F_k with S_k from Eq. (4),
    S_e = S_eps = S_pi = S_nu (Eq. 15) and S_q, S_m chosen independently."""
    rng = np.random.default_rng(22)
    M = load_M()
    for _ in range(40):
        f = random_pops(rng, 19)
        F = 1e-3 * rng.standard_normal(3)
        Snu, Sq, Sm = 0.3 + 1.6 * rng.random(3)
        rho0 = 0.9 + 0.2 * rng.random()
        out, u = O.collide_mrt(f, F, Snu, rho0, Sq=Sq, Sm=Sm)
        m, mo = M @ f, M @ out
        rates = np.full(19, Snu)
        rates[[0, 3, 5, 7]] = 0.0
        rates[[4, 6, 8]] = Sq
        rates[[16, 17, 18]] = Sm
        expect = (m - rates * (m - meq_A4(f.sum(), rho0, u))
                  + (1 - 0.5 * rates) * SF_A5(u, F))
        np.testing.assert_allclose(mo, expect, rtol=2e-15, atol=5e-15)
        # the third-order m_x, m_y, m_z have zero equilibrium and no forcing
        np.testing.assert_allclose(mo[16:], (1 - Sm) * m[16:], atol=1e-16)
        assert abs(out.sum() - f.sum()) < 1e-14
        np.testing.assert_allclose(mo[[3, 5, 7]], m[[3, 5, 7]] + F,
                                   atol=1e-16)


def test_eq16_is_the_magic_combination():
    """Eq. (16) is the rate for which (1/S_nu - 1/2)(1/S_q - 1/2) = 3/16 at
    every S_nu (the two-relaxation-time parameter of exact bounce-back)."""
    S = np.linspace(0.05, 1.95, 39)
    lam = (1 / S - 0.5) * (1 / O.mrt_rate(S) - 0.5)
    np.testing.assert_allclose(lam, 3 / 16, rtol=1e-14)


@pytest.mark.parametrize("tau", [1.0, 0.8, 0.6])
def test_mrt_poiseuille_has_no_slip(tau):
    """D3Q19 channel, body force along x, halfway bounce-back walls at
    y0 = 0.5 and y1 = ny - 1.5: with the MRT rates of Eq. (16) the steady
    profile is the parabola g/(2 nu) (y - y0)(y1 - y) with no slip to
    round-off, for every viscosity. (The single-rate collision has the
    slip g (16 L - 3)/(24 nu), L = (tau - 1/2)^2, as its own pin shows.)"""
    g, ny = 1e-6, 19
    case = W.channel_3d(ny=ny, g=g, tau=tau, collision=1)
    o = O.Oracle(19, case.solid, case.periodic)
    o.set_params(**case.params)
    o.init_state(case.phi0)
    o.step(30000)
    u = o.fields()["u"]
    nu = (tau - 0.5) / 3
    y = np.arange(ny, dtype=float)[1:-1]
    expect = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    for z in range(u.shape[1]):
        for x in range(u.shape[3]):
            np.testing.assert_allclose(u[0, z, 1:-1, x], expect, rtol=0,
                                       atol=1e-14)
    np.testing.assert_allclose(u[1:, :, 1:-1, :], 0.0, atol=1e-15)


def test_mrt_step_conserves_colour_mass():
    """Streaming, MRT collision and recolouring conserve each colour's mass
    exactly (periodic pack, Scheme-II wetting, unequal viscosities, a body
    force)."""
    pack = W.sphere_pack((24, 20, 18), 0.45, reservoir=0, side_walls=False,
                         seed=3)
    solid = pack["solid"]
    rng = np.random.default_rng(5)
    phi0 = np.where(rng.random(solid.shape) < 0.5, 1.0, -1.0)
    phi0[solid == 1] = 0.0
    o = O.Oracle(19, solid, (True, True, True))
    o.set_params(**W.base_params(tau_r=1.0, tau_b=0.6, wetting=2,
                                 theta_deg=50.0, g=(1e-5, 2e-6, 0.0),
                                 collision=1))
    o.init_state(phi0)
    r0, b0 = o.reduce(O.MASS_R), o.reduce(O.MASS_B)
    o.step(60)
    assert o.reduce(O.MASS_R) == pytest.approx(r0, rel=1e-12)
    assert o.reduce(O.MASS_B) == pytest.approx(b0, rel=1e-12)


def test_mrt_refused_on_d2q9():
    case = W.channel_2d(nx=4, ny=9)
    o = O.Oracle(9, case.solid, case.periodic)
    with pytest.raises(ValueError):
        o.set_params(**dict(case.params, collision=1))
    with pytest.raises(ValueError):
        o.set_params(**dict(case.params, collision=2))
