"""Post-processing of phase fields: the measurements the paper makes on its
results (Sec. III and Sec. IV.A), done headless with numpy.

These functions read a phase field phi (or densities) and return numbers; they
take no part in the time step.
"""
from __future__ import annotations

import math

import numpy as np


def _crossing(values: np.ndarray, coords: np.ndarray) -> float:
    """Coordinate where ``values`` first changes sign (linear interpolation),
    scanning from the start; nan if it never does."""
    for k in range(len(values) - 1):
        a, b = values[k], values[k + 1]
        if a == 0.0:
            return float(coords[k])
        if (a > 0) != (b > 0):
            t = a / (a - b)
            return float(coords[k] + t * (coords[k + 1] - coords[k]))
    return float("nan")


def contact_angle_from_cap(b: float, h: float) -> float:
    """Eqs. (45)-(46): the angle (degrees) of a spherical/circular cap of base
    b and height h, measured inside the cap. r = (4h^2 + b^2)/(8h) and
    theta = arctan((b/2)/(r - h)), taken with atan2 so that caps higher than
    their radius (r < h) give angles above 90 degrees."""
    r = (4.0 * h * h + b * b) / (8.0 * h)
    return math.degrees(math.atan2(b / 2.0, r - h))


def droplet_base_height(phi_slice: np.ndarray, wall_row: int, axis_col: float):
    """Base width and height of a red cap (phi > 0) sitting on a wall.

    ``phi_slice`` is a 2-D array indexed [normal, tangential], whose row
    ``wall_row`` is the last solid row; the wall plane lies halfway between it
    and the first fluid row. The base is the distance between the two phi = 0
    crossings on the first fluid row; the height is the distance from the wall
    plane to the phi = 0 crossing on the drop's axis column ``axis_col``
    (interpolated between the two nearest columns)."""
    row = phi_slice[wall_row + 1]
    ncol = row.shape[0]
    c0 = int(math.floor(axis_col))
    cols = np.arange(ncol, dtype=np.float64)
    right = _crossing(row[c0:], cols[c0:])
    left = _crossing(row[:c0 + 1][::-1], cols[:c0 + 1][::-1])
    base = right - left
    t = axis_col - c0
    column = (1 - t) * phi_slice[:, c0] + t * phi_slice[:, min(c0 + 1, ncol - 1)]
    rows = np.arange(phi_slice.shape[0], dtype=np.float64)
    top = _crossing(column[wall_row + 1:], rows[wall_row + 1:])
    height = top - (wall_row + 0.5)
    return base, height


def droplet_contact_angle(phi_slice, wall_row, axis_col):
    """Contact angle of the red cap measured through fluid b (the paper's
    convention, Sec. III.B): 180 deg minus the angle inside the red cap."""
    b, h = droplet_base_height(phi_slice, wall_row, axis_col)
    return 180.0 - contact_angle_from_cap(b, h)


def sessile_angle_3d(phi: np.ndarray, cx: float, cy: float,
                     wall_layer: int = 0):
    """Contact angle (degrees, through fluid b) of a red sessile drop on the
    wall z = ``wall_layer`` of a 3-D phase field phi[z, y, x], with Eqs.
    (45)-(46) applied to the two central sections through the drop's axis
    (x, y) = (cx, cy): the x-z section (interpolated between the two rows
    nearest cy) and the y-z section (between the two columns nearest cx).
    Returns (mean, x-z angle, y-z angle)."""
    y0 = int(math.floor(cy))
    ty = cy - y0
    sxz = (1 - ty) * phi[:, y0, :] + ty * phi[:, min(y0 + 1, phi.shape[1] - 1), :]
    x0 = int(math.floor(cx))
    tx = cx - x0
    syz = (1 - tx) * phi[:, :, x0] + tx * phi[:, :, min(x0 + 1, phi.shape[2] - 1)]
    ax = droplet_contact_angle(sxz, wall_layer, cx)
    ay = droplet_contact_angle(syz, wall_layer, cy)
    return 0.5 * (ax + ay), ax, ay


def interface_position(phi: np.ndarray, axis: int = 0, solid=None) -> float:
    """Volume-equivalent position of a red slug entering along ``axis`` from
    coordinate 0: the number of red-filled cross-sections, i.e. the red
    volume sum (1+phi)/2 over fluid nodes divided by the fluid nodes of one
    cross-section (mean over the tube)."""
    red = 0.5 * (1.0 + phi)
    if solid is not None:
        red = np.where(solid == 0, red, 0.0)
        fl = (solid == 0)
    else:
        fl = np.ones_like(phi, bool)
    ax = {0: 2, 1: 1, 2: 0}[axis]
    per_slice = fl.sum(axis=tuple(a for a in range(3) if a != ax))
    return float(red.sum() / per_slice.mean())


def washburn_linear(t, z0, r, dP, mu, L):
    """Eq. (47) for equal viscosities (mu_w = mu_nw = mu) and cos(theta) = 0:
    z(t) = z0 + r^2 dP t / (8 mu L)."""
    return z0 + r * r * dP * np.asarray(t, dtype=np.float64) / (8.0 * mu * L)


def washburn_z(t, r, L, dP, gamma, theta_deg, mu_w, mu_nw):
    """Eq. (48): interface tip position for unequal viscosities."""
    a = L * mu_nw / (mu_w - mu_nw)
    src = (dP * r * r / 2.0 + r * gamma * math.cos(math.radians(theta_deg)))
    return -a + np.sqrt(a * a + src * np.asarray(t, np.float64)
                        / (2.0 * (mu_w - mu_nw)))


def area_error(z_sim, z_ref, t) -> float:
    """Relative difference of the areas under two z(t) curves, the error
    metric of Sec. IV.A.1."""
    a_sim = np.trapezoid(z_sim, t)
    a_ref = np.trapezoid(z_ref, t)
    return abs(a_sim - a_ref) / a_ref


def laplace_measure(rho: np.ndarray, phi: np.ndarray, inner: float = 0.5,
                    gap: float = 5.0):
    """Pressure jump and radius of a red drop centred in a periodic box
    (Sec. III.A). R is the radius of the sphere (disc in 2-D, shape
    (1, ny, nx)) with the drop's red volume sum (1 + phi)/2; the pressures
    p = rho/3 are averaged inside r < inner R and outside r > R + gap, r
    measured from the box centre. Returns (dP, R)."""
    two_d = phi.shape[0] == 1
    red = ((1.0 + phi) / 2.0).sum()
    R = math.sqrt(red / math.pi) if two_d else (3 * red / (4 * math.pi)) ** (1 / 3)
    nz, ny, nx = phi.shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    r2 = (x - (nx - 1) / 2.0) ** 2 + (y - (ny - 1) / 2.0) ** 2
    if not two_d:
        r2 = r2 + (z - (nz - 1) / 2.0) ** 2
    r = np.sqrt(r2)
    dp = (rho[r < inner * R].mean() - rho[r > R + gap].mean()) / 3.0
    return float(dp), float(R)


def laplace_slope(dps, radii, dims: int = 3) -> float:
    """Least-squares slope through the origin of dP against (dims - 1)/R:
    the interfacial tension of Laplace's law dP = (dims - 1) gamma / R."""
    xs = (dims - 1) / np.asarray(radii, np.float64)
    ys = np.asarray(dps, np.float64)
    return float((xs * ys).sum() / (xs * xs).sum())
