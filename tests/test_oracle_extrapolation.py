"""Pins of Eqs. (34)-(35) (Sec. II.B.3): at a solid-boundary node the phase
field and n_c are the lattice-weighted means of the values at its fluid
lattice neighbours inside the box; Eq. (35) is not renormalised.

On a flat wall the fluid neighbours of a wall node are the node just above
it (weight w1: 1/18 in D3Q19, 1/9 in D2Q9) and its diagonal neighbours in
the first fluid layer (weight w2 = 1/36; four in D3Q19, two in D2Q9). For a
field quadratic along the wall, f = a + b x + c x^2 + d y + e y^2, the pair
f(x+1) + f(x-1) is 2 f(x) + 2c, so the weighted mean is exactly

    D3Q19:  f(x, y, z1) + 2 w2 (c + e) / (w1 + 4 w2) = f + (c + e)/3,
    D2Q9:   f(x, y1)    + 2 w2 c / (w1 + 2 w2)       = f + c/3,

with z1 (y1) the first fluid layer. Plausible mistakes give other values:
equal weights f + 2 (c + e)/5 (D3Q19) or f + 2c/3 (D2Q9); letting the solid
in-plane or deeper neighbours into the sum pulls the value towards theirs
(set far off here); renormalising Eq. (35) gives a unit vector, while the
mean of the (non-unit) vectors used here has another length."""
import numpy as np
import pytest

from oracle import oracle as O

TOL = 1e-13


def quad(shape2, coef):
    """a + b x + c x^2 + d y + e y^2 over a (ny, nx) grid."""
    a, b, c, d, e = coef
    y, x = np.mgrid[0:shape2[0], 0:shape2[1]].astype(float)
    return a + b * x + c * x * x + d * y + e * y * y


def test_eq34_eq35_flat_wall_d3q19():
    nz, ny, nx = 7, 9, 11
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:2] = 1                        # wall: z = 0 (pure solid), z = 1
    o = O.Oracle(19, solid, (False, False, False))
    cls, _, _ = o.geometry()
    assert (cls[1] == 1).all() and (cls[0] == 0).all()
    phi_c = (0.11, -0.02, 0.013, 0.05, -0.021)
    nc_c = [(0.6, 0.01, -0.004, 0.02, 0.003), (-0.3, 0.02, 0.006, -0.01, 0.011),
            (0.5, -0.015, 0.002, 0.03, -0.007)]
    phi = np.full(solid.shape, 7.0)     # solid entries: far from the answer
    nc = np.full((3,) + solid.shape, 5.0)
    for z in range(2, nz):
        phi[z] = quad((ny, nx), phi_c) + 0.01 * z
        for a in range(3):
            nc[a, z] = quad((ny, nx), nc_c[a]) - 0.02 * a * z
    po, no = o.extrapolate(phi, nc)
    inner = (slice(1, ny - 1), slice(1, nx - 1))   # all four diagonals in the box
    expect = phi[2][inner] + (phi_c[2] + phi_c[4]) / 3
    np.testing.assert_allclose(po[1][inner], expect, rtol=0, atol=TOL)
    equal_w = phi[2][inner] + 2 * (phi_c[2] + phi_c[4]) / 5
    assert np.abs(equal_w - expect).min() > 1e6 * TOL
    for a in range(3):
        ea = nc[a, 2][inner] + (nc_c[a][2] + nc_c[a][4]) / 3
        np.testing.assert_allclose(no[a, 1][inner], ea, rtol=0, atol=TOL)
    length = np.sqrt((no[:, 1][(slice(None),) + inner] ** 2).sum(0))
    assert np.abs(length - 1).min() > 1e-2        # not renormalised
    # a solid node with no fluid neighbour keeps its value; fluid nodes too
    np.testing.assert_array_equal(po[0], phi[0])
    np.testing.assert_array_equal(po[2:], phi[2:])
    np.testing.assert_array_equal(no[:, 0], nc[:, 0])


def test_eq34_eq35_flat_wall_d2q9():
    ny, nx = 6, 13
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, :2] = 1                     # wall rows y = 0 (pure solid), y = 1
    o = O.Oracle(9, solid, (False, False, True))
    phi_c = (0.2, 0.03, -0.017, 0.0, 0.0)
    phi = np.full(solid.shape, -9.0)
    nc = np.full((3, 1, ny, nx), 4.0)
    x = np.arange(nx, dtype=float)
    for y in range(2, ny):
        phi[0, y] = quad((1, nx), phi_c)[0] + 0.03 * y
        nc[0, 0, y] = 0.5 + 0.02 * x - 0.011 * x * x
        nc[1, 0, y] = -0.4 + 0.01 * x + 0.009 * x * x
        nc[2, 0, y] = 0.0
    po, no = o.extrapolate(phi, nc)
    inner = slice(1, nx - 1)
    expect = phi[0, 2, inner] + phi_c[2] / 3
    np.testing.assert_allclose(po[0, 1, inner], expect, rtol=0, atol=TOL)
    assert np.abs(phi[0, 2, inner] + 2 * phi_c[2] / 3 - expect).min() > 1e6 * TOL
    np.testing.assert_allclose(no[0, 0, 1, inner], nc[0, 0, 2, inner] - 0.011 / 3,
                               rtol=0, atol=TOL)
    np.testing.assert_allclose(no[1, 0, 1, inner], nc[1, 0, 2, inner] + 0.009 / 3,
                               rtol=0, atol=TOL)
    # at the non-periodic x faces the off-box neighbour is left out
    w1, w2 = 1 / 9, 1 / 36
    edge = (w1 * phi[0, 2, 0] + w2 * phi[0, 2, 1]) / (w1 + w2)
    assert abs(po[0, 1, 0] - edge) < TOL


@pytest.mark.parametrize("periodic_x", [True, False])
def test_eq34_wraps_periodic_axes(periodic_x):
    """On a periodic axis the neighbour across the face is in the box (the
    wrapped node) and enters the mean; on a non-periodic one it does not."""
    ny, nx = 5, 8
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 0] = 1
    o = O.Oracle(9, solid, (periodic_x, False, True))
    phi = np.zeros(solid.shape)
    phi[0, 1:] = np.arange(nx, dtype=float)[None, :] * 0.1
    po, _ = o.extrapolate(phi, np.zeros((3,) + solid.shape))
    w1, w2 = 1 / 9, 1 / 36
    if periodic_x:
        expect = (w1 * phi[0, 1, 0] + w2 * (phi[0, 1, 1] + phi[0, 1, nx - 1])) / (w1 + 2 * w2)
    else:
        expect = (w1 * phi[0, 1, 0] + w2 * phi[0, 1, 1]) / (w1 + w2)
    assert abs(po[0, 0, 0] - expect) < TOL
