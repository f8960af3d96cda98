"""Pin of the oracle by a symmetry of the method: on a periodic axis the
lattice has no origin, so translating the whole initial state (solid image
and phase field) along that axis and stepping gives the translated result
of stepping the original. The case puts every piece of the step on the
periodic faces: Zou-He ends on x (non-periodic), a solid sphere with
Scheme-I wetting across the y period, and a drop centred on the edge of
the outlet plane and the y faces. Stencils there reach positions off the
box on x and on y at once; the off-box rule (wrap the periodic axis, clamp
the other) keeps the symmetry, a rule that treated the periodic component
any other way, a wrong wrap or a transposed index along y would not."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10914_gb300 import workloads as W


def edge_case(shape=(10, 12, 16)):
    nz, ny, nx = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    dy = np.minimum(y, ny - y)  # distance to y = 0 across the period
    solid = ((x - 6.0) ** 2 + (dy - 1.0) ** 2 + (z - 4.0) ** 2 < 2.6 ** 2)
    solid = solid.astype(np.uint8)
    r = np.sqrt((x - (nx - 1)) ** 2 + dy ** 2 + (z - nz / 2.0) ** 2)
    phi0 = np.tanh((4.5 - r) / 1.5)
    phi0[solid == 1] = 0.0
    p = W.base_params(tau_r=1.0, tau_b=0.8, gamma=0.01, beta=0.95,
                      theta_deg=60.0, wetting=1, zou_he=1, flow_axis=0,
                      rho_in=1.002, rho_out=1.0, zeta_r=1.0)
    return solid, np.ascontiguousarray(phi0), p


def run(solid, phi0, p, steps):
    o = O.Oracle(19, solid, (False, True, True))
    o.set_params(**p)
    o.init_state(phi0)
    o.step(steps)
    return o.pops


@pytest.mark.parametrize("axis,shift", [(1, 1), (1, 5), (0, 3)],
                         ids=["y1", "y5", "z3"])
def test_step_commutes_with_periodic_translation(axis, shift):
    solid, phi0, p = edge_case()
    ref = run(solid, phi0, p, 6)
    got = run(np.ascontiguousarray(np.roll(solid, shift, axis=axis)),
              np.ascontiguousarray(np.roll(phi0, shift, axis=axis)), p, 6)
    want = np.roll(ref, shift, axis=axis + 2)  # pops are [2][Q][nz][ny][nx]
    scale = np.abs(ref).max()
    assert np.abs(got - want).max() <= 1e-13 * scale


def test_translation_along_the_flow_axis_is_not_a_symmetry():
    """The check has teeth: along x the Zou-He planes fix an origin."""
    solid, phi0, p = edge_case()
    ref = run(solid, phi0, p, 6)
    got = run(np.ascontiguousarray(np.roll(solid, 2, axis=2)),
              np.ascontiguousarray(np.roll(phi0, 2, axis=2)), p, 6)
    want = np.roll(ref, 2, axis=4)
    assert np.abs(got - want).max() > 1e-6 * np.abs(ref).max()


def edge_case_2d(nx=40, ny=24):
    """D2Q9: a wetting wall row at y = 0, a clamped top edge, x periodic; a
    red drop centred on the top edge at the x period boundary."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 0, :] = 1
    dx = np.minimum(x, nx - x)  # distance to x = 0 across the period
    r = np.sqrt(dx ** 2 + (y - (ny - 1)) ** 2)
    phi0 = np.tanh((9.0 - r) / 1.5)[None]
    phi0[solid == 1] = 0.0
    p = W.base_params(tau_r=1.0, tau_b=0.7, gamma=0.01, beta=0.9,
                      theta_deg=50.0, wetting=2)
    return solid, np.ascontiguousarray(phi0), p


def run_2d(solid, phi0, p, steps):
    o = O.Oracle(9, solid, (True, False, True))
    o.set_params(**p)
    o.init_state(phi0)
    o.step(steps)
    return o.pops


@pytest.mark.parametrize("shift", [1, 7, 20])
def test_d2q9_step_commutes_with_periodic_translation(shift):
    solid, phi0, p = edge_case_2d()
    ref = run_2d(solid, phi0, p, 8)
    got = run_2d(np.ascontiguousarray(np.roll(solid, shift, axis=2)),
                 np.ascontiguousarray(np.roll(phi0, shift, axis=2)), p, 8)
    want = np.roll(ref, shift, axis=4)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(ref).max()
