"""Pins of the stencils of Sec. II.B on prescribed fields.

Eq. (6) (with c = dt = 1) is the isotropic gradient: sum_i w_i e_i e_i =
I/3, so C = 3 sum_i w_i e_i phi(x + e_i) is exactly grad phi for a linear
field, and Eq. (11) gives its direction. Eq. (12) with each d_b n_a taken by
the same stencil is the curvature sum_ab (n_a n_b - delta_ab) d_b n_a; for
the unit field n = -r/|r| (the normal of a red drop, pointing to the red
side) it is 2/r in 3-D and 1/r in 2-D, which the second-order stencil
reaches to 0.37/r^2 (relative). A dropped cross term gives 4/3 of 2/r on
the diagonals; a sign slip in (n_a^2 - 1) or a missing factor 3 is off by
far more."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("lattice", [19, 9])
def test_eq6_exact_on_linear_fields(lattice):
    shape = (20, 22, 24) if lattice == 19 else (1, 22, 24)
    o = O.Oracle(lattice, np.zeros(shape, np.uint8), (True, True, True))
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(float)
    b = np.array([0.02, -0.03, 0.015 if lattice == 19 else 0.0])
    phi = 0.1 + b[0] * x + b[1] * y + b[2] * z
    C, nc, _ = o.stencils(phi, np.zeros((3,) + shape))
    inner = (slice(1, -1) if lattice == 19 else 0, slice(1, -1), slice(1, -1))
    for a in range(3):
        np.testing.assert_allclose(C[(a,) + inner], b[a], rtol=0, atol=1e-15)
        np.testing.assert_allclose(nc[(a,) + inner], b[a] / np.linalg.norm(b),
                                   rtol=0, atol=1e-14)


@pytest.mark.parametrize("lattice", [19, 9])
def test_eq12_curvature_of_a_sphere(lattice):
    n = 40
    shape = (n, n, n) if lattice == 19 else (1, n, n)
    o = O.Oracle(lattice, np.zeros(shape, np.uint8), (True, True, True))
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(float)
    c = 19.3
    dz = (z - c) if lattice == 19 else 0.0 * z
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + dz ** 2) + 1e-300
    nc = -np.stack([(x - c) / r, (y - c) / r, dz / r])
    _, _, kappa = o.stencils(np.zeros(shape), nc)
    dims = 2.0 if lattice == 19 else 1.0
    for R in (6.0, 8.0, 10.0, 14.0):
        m = np.abs(r - R) < 0.5
        rel = kappa[m] * r[m] / dims - 1.0
        assert np.abs(rel).max() < 0.45 / R ** 2, (R, np.abs(rel).max())
        # the diagonal-free sum would be far off on the diagonal shells
        if lattice == 19:
            d = np.stack([nc[a][m] for a in range(3)])
            wrong = ((1 - d ** 2) ** 2).sum(0) / r[m]
            assert np.abs(wrong * r[m] / dims - 1).max() > 0.25
