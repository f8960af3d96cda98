"""Pins of the oracle's geometry preprocessing (node classes, Eq. 25
smoothing, Eq. 26 wall normal) and of the two wetting schemes (Eqs. 28-33)."""
import math

import numpy as np
import pytest
from scipy import ndimage, optimize

from oracle import oracle as O
from tests.test_oracle_lattice import E_A1


def brute_classes(solid, periodic, q):
    """Node classes by direct enumeration of lattice neighbours."""
    nz, ny, nx = solid.shape
    sub = [0, 1, 2, 3, 4, 7, 8, 9, 10] if q == 9 else list(range(19))
    E = E_A1[sub]
    cls = np.zeros_like(solid)
    dims = (nx, ny, nz)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                bnd = False
                for e in E[1:]:
                    c = [x + e[0], y + e[1], z + e[2]]
                    ok = True
                    for a in range(3):
                        if not 0 <= c[a] < dims[a]:
                            if periodic[a]:
                                c[a] %= dims[a]
                            else:
                                ok = False
                    if not ok:
                        continue
                    if solid[z, y, x] != solid[c[2], c[1], c[0]]:
                        bnd = True
                s = solid[z, y, x]
                cls[z, y, x] = (0 if s else 2) + (1 if bnd else 0)
    return cls


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_classes_brute_force(periodic):
    rng = np.random.default_rng(5)
    solid = (rng.random((5, 6, 7)) < 0.35).astype(np.uint8)
    o = O.Oracle(19, solid, periodic)
    cls, _, _ = o.geometry()
    np.testing.assert_array_equal(cls, brute_classes(solid, periodic, 19))
    s2 = (rng.random((1, 9, 11)) < 0.3).astype(np.uint8)
    o2 = O.Oracle(9, s2, periodic)
    np.testing.assert_array_equal(o2.geometry()[0],
                                  brute_classes(s2, periodic, 9))


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_smoothing_is_separable_eq25(periodic):
    """Eq. (25)'s 27-point weights 8/27, 2/27, 1/54, 1/216 are the tensor
    product of (1/6, 2/3, 1/6): three passes of that 1-D kernel along each
    axis (wrap on periodic axes, edge replication otherwise) must agree."""
    rng = np.random.default_rng(6)
    solid = (rng.random((7, 8, 9)) < 0.4).astype(np.uint8)
    o = O.Oracle(19, solid, periodic)
    _, gsm, _ = o.geometry()
    g = 1.0 - solid.astype(float)
    k = np.array([1 / 6, 2 / 3, 1 / 6])
    for _ in range(3):
        for ax_xyz in range(3):
            mode = "wrap" if periodic[ax_xyz] else "nearest"
            g = ndimage.correlate1d(g, k, axis=2 - ax_xyz, mode=mode)
    np.testing.assert_allclose(gsm, g, atol=1e-14)


def test_wall_normal_flat_plate():
    solid = np.zeros((6, 10, 5), np.uint8)
    solid[:, 0, :] = 1
    solid[:, 9, :] = 1
    o = O.Oracle(19, solid, (True, True, True))
    cls, _, nw = o.geometry()
    np.testing.assert_allclose(nw[:, :, 1, :], np.array([0, 1, 0])[:, None, None]
                               * np.ones((3, 6, 5)), atol=1e-15)
    np.testing.assert_allclose(nw[:, :, 8, :], np.array([0, -1, 0])[:, None, None]
                               * np.ones((3, 6, 5)), atol=1e-15)
    assert (cls[:, 1, :] == 3).all() and (cls[:, 2, :] == 2).all()


def test_wall_normal_sphere_is_radial():
    n = 28
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    c = (n - 1) / 2
    solid = (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) < 8.0 ** 2).astype(np.uint8)
    o = O.Oracle(19, solid, (True, True, True))
    cls, _, nw = o.geometry()
    sel = cls == 3
    radial = np.stack([x - c, y - c, z - c])[:, sel]
    radial /= np.linalg.norm(radial, axis=0)
    cosang = (nw[:, sel] * radial).sum(0)
    assert np.degrees(np.arccos(np.clip(cosang, -1, 1))).max() < 12.0
    assert np.degrees(np.arccos(np.clip(cosang, -1, 1))).mean() < 4.0


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def test_scheme2_against_gram_schmidt():
    """Eqs. (32)-(33): the chosen n lies in the plane of n_c and n_w, makes
    the angle theta with n_w and is the nearer of the two such unit vectors
    to n_c, i.e. cos(theta) n_w + sin(theta) t with t the unit component of
    n_c normal to n_w."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        nc, nw = unit(rng.standard_normal(3)), unit(rng.standard_normal(3))
        th = rng.uniform(0.05, math.pi - 0.05)
        out = O.scheme2(nc, nw, th)
        t = unit(nc - (nc @ nw) * nw)
        expect = math.cos(th) * nw + math.sin(th) * t
        np.testing.assert_allclose(out, expect, atol=1e-12)
        assert abs(out @ nw - math.cos(th)) < 1e-12
        other = math.cos(th) * nw - math.sin(th) * t
        assert np.linalg.norm(out - nc) <= np.linalg.norm(other - nc) + 1e-12


def test_scheme2_parallel_is_unchanged():
    nw = np.array([0, 0, 1.0])
    for nc in (nw, -nw):
        np.testing.assert_array_equal(O.scheme2(nc, nw, 1.0), nc)


def test_scheme1_secant_on_its_line():
    """Eqs. (28)-(31): every secant iterate is an affine combination of the
    previous two, so v4 lies on the line v(s) = n_c - s (n_c + n_w) through
    v0 = n_c and v1 (lambda = 1/2). That line reaches the angles
    (theta'/2, 180 deg) to n_w, theta' being the angle of n_c. Where the
    requested theta is within 20 deg of theta', the result must be the
    line's root of f(v) = v.n_w - |v| cos(theta) (found here by bracketing),
    normalised, to the accuracy that three secant steps reach: 1e-3 within
    2 deg, 0.1 up to 20 deg."""
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(400):
        nw = unit(rng.standard_normal(3))
        nc = unit(rng.standard_normal(3))
        thp = math.acos(np.clip(nc @ nw, -1, 1))
        th = thp + math.radians(rng.uniform(-20, 20))
        if not (math.radians(5) < th < math.radians(175)) or th < thp / 2 + 0.05:
            continue
        out = O.scheme1(nc, nw, th)
        assert abs(np.linalg.norm(out) - 1) < 1e-12
        d = nc + nw
        line_normal = np.cross(nc, d)
        assert abs(out @ line_normal) < 1e-9 * max(1.0, np.linalg.norm(line_normal))

        def fres(s):
            v = nc - s * d
            return v @ nw - np.linalg.norm(v) * math.cos(th)
        ss = np.linspace(-60, 1, 24401)
        V = nc[None, :] - ss[:, None] * d[None, :]
        vals = V @ nw - np.linalg.norm(V, axis=1) * math.cos(th)
        ks = np.where(np.sign(vals[:-1]) != np.sign(vals[1:]))[0]
        if len(ks) == 0:
            continue
        roots = [optimize.brentq(fres, ss[k], ss[k + 1], xtol=1e-15) for k in ks]
        dist = min(np.linalg.norm(out - unit(nc - r * d)) for r in roots)
        tol = 1e-3 if abs(th - thp) < math.radians(2) else 0.1
        assert dist < tol, (dist, math.degrees(thp), math.degrees(th))
        assert abs(out @ nw - math.cos(th)) < tol
        checked += 1
    assert checked > 200


def test_scheme1_converged_input_unchanged():
    nw = np.array([0, 1.0, 0])
    th = math.radians(70)
    nc = np.array([math.sin(th), math.cos(th), 0])
    np.testing.assert_allclose(O.scheme1(nc, nw, th), nc, atol=1e-12)
