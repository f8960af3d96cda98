"""Seeded synthetic inputs: solid images, initial phase fields and run
parameters for the workloads of the paper's experiments.

This module holds no lattice-Boltzmann arithmetic. It is the one module that
both the CUDA path's tests/bench and the oracle side use, so that both run on
the same inputs.

Every field is a numpy array of shape ``(nz, ny, nx)`` (x fastest); a solid
image holds 1 for solid, 0 for fluid; ``phi0`` is +1 for red, -1 for blue.

Stand-ins for the paper's inputs:
  * the static droplet of Sec. III.B (102x201x201, R = 30) is reduced to a
    2-D D2Q9 half-disc on a wall (128x64, R = 24) and to 3-D sessile drops of
    48^3..128^3 (the batched sweep);
  * the capillary tube of Sec. IV.A (12x12x101, r = 5) becomes a 20x20x256
    tube of radius 8 along x;
  * the Bentheimer sandstone of Sec. IV.B (Digital Rocks, 300x300x500 +
    2x10 reservoir layers, porosity 21.3 %) is not available; a Boolean
    model of overlapping solid spheres (radii uniform in [4, 10]) with the
    same reservoir layers and solid side walls, porosity 0.22, and isolated
    pores removed (the paper's bwareaopen step) stands in for it.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

AXES = ("x", "y", "z")


@dataclasses.dataclass
class Case:
    """A fully specified run: lattice, solid image, periodicity, phi0 and the
    parameter dictionary (keys of the C-ABI parameter block)."""
    name: str
    lattice: int
    solid: np.ndarray
    periodic: tuple
    phi0: np.ndarray
    params: dict
    steps: int = 1
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def shape(self):
        return self.solid.shape

    @property
    def n_nodes(self) -> int:
        return int(self.solid.size)

    @property
    def n_fluid(self) -> int:
        return int((self.solid == 0).sum())


def base_params(**kw) -> dict:
    p = dict(tau_r=1.0, tau_b=1.0, gamma=0.01, beta=0.95, rho0=1.0,
             theta_deg=90.0, wetting=0, zou_he=0, flow_axis=0,
             rho_in=1.0, rho_out=1.0, zeta_r=1.0, g=(0.0, 0.0, 0.0),
             collision=0)
    p.update(kw)
    return p


# --------------------------------------------------------------- droplets
def droplet_2d(nx=128, ny=64, radius=24.0, theta_deg=60.0, wetting=2,
               gamma=0.01, beta=0.7, tau=1.0, steps=2000) -> Case:
    """D2Q9 red half-disc on a flat wall in blue fluid: solid row y = 0,
    periodic in x; y is not periodic, so the top edge is a plain bounce-back
    boundary without wetting (a periodic y would make the single solid row
    average phi over both of its faces in Eq. 34). The disc centre lies on
    the halfway wall plane at (nx/2 - 0.5, 0.5)."""
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 0, :] = 1
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy = nx / 2 - 0.5, 0.5
    inside = (x - cx) ** 2 + (y - cy) ** 2 < radius ** 2
    phi0 = np.where(inside, 1.0, -1.0)[None]
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau, tau_b=tau, gamma=gamma, beta=beta,
                    theta_deg=theta_deg, wetting=wetting)
    return Case("droplet2d", 9, solid, (True, False, True), phi0, p, steps,
                dict(radius=radius, centre=(cx, cy)))


def droplet_3d(side=48, radius=12.0, theta_deg=60.0, wetting=2, gamma=0.01,
               beta=0.95, tau=1.0, steps=5000, shape=None) -> Case:
    """D3Q19 red hemisphere on a flat solid wall at z = 0 in blue fluid,
    periodic in x and y; z is not periodic (plain bounce-back at the top)."""
    nz, ny, nx = shape if shape is not None else (side, side, side)
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0] = 1
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    cx, cy, cz = nx / 2 - 0.5, ny / 2 - 0.5, 0.5
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 < radius ** 2
    phi0 = np.where(inside, 1.0, -1.0)
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau, tau_b=tau, gamma=gamma, beta=beta,
                    theta_deg=theta_deg, wetting=wetting)
    return Case(f"droplet3d_{nx}x{ny}x{nz}", 19, solid, (True, True, False),
                phi0, p, steps, dict(radius=radius, centre=(cx, cy, cz)))


def laplace_drop(lattice=9, n=64, radius=12.0, gamma=0.01, beta=0.7,
                 tau_r=1.0, tau_b=1.0, steps=3000) -> Case:
    """Red disc (D2Q9) or sphere (D3Q19) in blue fluid, fully periodic, no
    walls (Sec. III.A)."""
    if lattice == 9:
        shape = (1, n, n)
    else:
        shape = (n, n, n)
    solid = np.zeros(shape, np.uint8)
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(np.float64)
    c = (n - 1) / 2.0
    r2 = (x - c) ** 2 + (y - c) ** 2
    if lattice == 19:
        r2 = r2 + (z - c) ** 2
    phi0 = np.where(r2 < radius ** 2, 1.0, -1.0)
    p = base_params(tau_r=tau_r, tau_b=tau_b, gamma=gamma, beta=beta)
    return Case(f"laplace{lattice}_{n}_R{radius:g}", lattice, solid,
                (True, True, True), phi0, p, steps, dict(radius=radius))


# ---------------------------------------------------------- channels/tubes
def channel_2d(nx=4, ny=33, g=1e-6, tau=1.0, steps=4000) -> Case:
    """Single-phase (all red) D2Q9 channel between solid rows y = 0 and
    y = ny - 1, periodic in x, driven by a body acceleration along x."""
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, 0, :] = 1
    solid[0, ny - 1, :] = 1
    phi0 = np.ones((1, ny, nx))
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau, tau_b=tau, g=(g, 0.0, 0.0))
    return Case("channel2d", 9, solid, (True, False, True), phi0, p, steps)


def channel_3d(nx=4, ny=19, nz=4, g=1e-6, tau=1.0, collision=0,
               steps=4000) -> Case:
    """Single-phase (all red) D3Q19 channel between solid planes y = 0 and
    y = ny - 1, periodic in x and z, driven by a body acceleration along x."""
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    phi0 = np.ones((nz, ny, nx))
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau, tau_b=tau, g=(g, 0.0, 0.0),
                    collision=collision)
    return Case("channel3d", 19, solid, (True, False, True), phi0, p, steps)


def tube_3d(nx=256, ny=20, nz=20, radius=8.0, red_len=32, theta_deg=90.0,
            wetting=1, rho_in=1.01, rho_out=0.99, tau=1.0, gamma=0.01,
            beta=0.95, zou_he=True, g_x=0.0, steps=20000) -> Case:
    """D3Q19 capillary tube along x (Sec. IV.A): solid where the distance from
    the axis (y, z) = ((ny-1)/2, (nz-1)/2) exceeds the radius; red fills the
    first ``red_len`` layers, blue the rest; Zou-He ends on x (Type-I) with
    red injected, or a body force (Type-II)."""
    z, y = np.mgrid[0:nz, 0:ny].astype(np.float64)
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    out = ((y - cy) ** 2 + (z - cz) ** 2) > radius ** 2
    solid = np.broadcast_to(out[:, :, None], (nz, ny, nx)).astype(np.uint8)
    solid = np.ascontiguousarray(solid)
    x = np.arange(nx)[None, None, :]
    phi0 = np.where(np.broadcast_to(x < red_len, solid.shape), 1.0, -1.0)
    phi0 = np.ascontiguousarray(phi0)
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau, tau_b=tau, gamma=gamma, beta=beta,
                    theta_deg=theta_deg, wetting=wetting,
                    zou_he=int(zou_he), flow_axis=0, rho_in=rho_in,
                    rho_out=rho_out, zeta_r=1.0, g=(g_x, 0.0, 0.0))
    periodic = (not zou_he, True, True)
    return Case(f"tube_{nx}x{ny}x{nz}_r{radius:g}", 19, solid, periodic,
                phi0, p, steps, dict(radius=radius, red_len=red_len))


def washburn_tube(theta_deg=60.0, wetting=1, nx=101, ny=12, nz=12,
                  radius=5.0, tau_w=1.0, tau_nw=0.6, gamma=1.0 / 45.0,
                  beta=0.95, rho=1.0, b_layers=1) -> Case:
    """Spontaneous imbibition in a capillary tube (Sec. IV.A, Case-I): the
    paper's 12 x 12 x 101 tube of radius 5 along x, the wetting fluid b
    (tau^b = 1.0) in the first ``b_layers`` layers, the non-wetting fluid r
    (tau^r = 0.6, viscosity ratio 1/5) in the rest, equal Zou-He densities
    at both ends (Delta P = 0) with b injected (zeta^r = 0), and the lattice
    tension 1/45 of the paper's unit system (0.02 N/m at a_o = 1e-6 m)."""
    c = tube_3d(nx=nx, ny=ny, nz=nz, radius=radius, red_len=0,
                theta_deg=theta_deg, wetting=wetting, rho_in=rho, rho_out=rho,
                tau=1.0, gamma=gamma, beta=beta)
    x = np.arange(nx)[None, None, :]
    phi0 = np.where(np.broadcast_to(x < b_layers, c.solid.shape), -1.0, 1.0)
    phi0 = np.ascontiguousarray(phi0)
    phi0[c.solid == 1] = 0.0
    p = dict(c.params, tau_r=tau_nw, tau_b=tau_w, zeta_r=0.0)
    return Case(f"washburn_{nx}x{ny}x{nz}_r{radius:g}_th{theta_deg:g}", 19,
                c.solid, c.periodic, phi0, p, 0,
                dict(radius=radius, length=nx - 1))


# ------------------------------------------------------------ porous rock
def sphere_pack(n=(256, 256, 256), porosity=0.22, rmin=4.0, rmax=10.0,
                seed=240710914, reservoir=10, side_walls=True,
                max_spheres: Optional[int] = None) -> dict:
    """Boolean model of overlapping solid spheres in the rock region
    ``reservoir <= x < nx - reservoir``: centres uniform over the region,
    radii uniform in [rmin, rmax], spheres added in a fixed seeded order until
    the porosity of the rock region first drops to ``porosity`` or below.
    Then solid side walls on the y and z faces, and every pore not connected
    (18-neighbour lattice connectivity) to the inlet plane x = 0 is filled
    (the paper's isolated-pore removal). Returns the solid image and facts
    about it."""
    from scipy import ndimage

    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    x0, x1 = reservoir, nx - reservoir
    rock = np.zeros((nz, ny, x1 - x0), bool)
    total = rock.size
    target_solid = (1.0 - porosity) * total
    covered = 0
    count = 0
    batch = 4096
    done = False
    while not done:
        cx = rng.uniform(0, x1 - x0, batch)
        cy = rng.uniform(0, ny, batch)
        cz = rng.uniform(0, nz, batch)
        rr = rng.uniform(rmin, rmax, batch)
        for k in range(batch):
            r = rr[k]
            lo = [int(np.floor(c - r)) for c in (cz[k], cy[k], cx[k])]
            hi = [int(np.ceil(c + r)) + 1 for c in (cz[k], cy[k], cx[k])]
            dims = rock.shape
            lo = [max(0, v) for v in lo]
            hi = [min(d, v) for d, v in zip(dims, hi)]
            if any(h <= l for l, h in zip(lo, hi)):
                continue
            zz, yy, xx = np.ogrid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
            ball = ((xx + 0.5 - cx[k]) ** 2 + (yy + 0.5 - cy[k]) ** 2
                    + (zz + 0.5 - cz[k]) ** 2) <= r * r
            sub = rock[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
            new = ball & ~sub
            covered += int(new.sum())
            sub |= ball
            count += 1
            if covered >= target_solid:
                done = True
                break
            if max_spheres is not None and count >= max_spheres:
                done = True
                break
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, :, x0:x1] = rock
    if side_walls:
        solid[0, :, :] = 1
        solid[-1, :, :] = 1
        solid[:, 0, :] = 1
        solid[:, -1, :] = 1
    fluid = solid == 0
    struct = ndimage.generate_binary_structure(3, 2)
    lab, nlab = ndimage.label(fluid, structure=struct)
    inlet_labels = np.unique(lab[:, :, 0])
    inlet_labels = inlet_labels[inlet_labels > 0]
    keep = np.isin(lab, inlet_labels)
    outlet_labels = np.unique(lab[:, :, nx - 1])
    percolates = bool(np.intersect1d(inlet_labels, outlet_labels).size)
    solid = np.where(keep, 0, 1).astype(np.uint8)
    rock_fluid = (solid[:, :, x0:x1] == 0).sum()
    return dict(solid=solid, spheres=count, percolates=percolates,
                rock_porosity=float(rock_fluid) / total,
                porosity_before_cleanup=1.0 - covered / total)


def porous_3d(n=(256, 256, 256), porosity=0.22, seed=240710914,
              reservoir=10, drive="typeII", theta_deg=45.0, wetting=1,
              tau_r=1.0, tau_b=0.6, gamma=0.01, beta=0.95, g_x=1e-5,
              rho_in=1.005, rho_out=0.995, invading="r", steps=10000,
              pack: Optional[dict] = None) -> Case:
    """D3Q19 drainage in the synthetic rock (stand-in for Sec. IV.B).

    Initially the pore space holds the defending fluid; the invading fluid is
    injected through the Zou-He inlet (zeta = 1 for it). ``drive`` "typeI":
    Zou-He densities rho_in/rho_out; "typeII": body acceleration g_x with
    equal Zou-He densities at both ends. ``invading`` "r" (drainage: red
    displaces blue) or "b" (imbibition: the defending red is everywhere except
    a blue inlet reservoir)."""
    if pack is None:
        pack = sphere_pack(n, porosity, seed=seed, reservoir=reservoir)
    solid = pack["solid"]
    nz, ny, nx = solid.shape
    x = np.arange(nx)[None, None, :]
    if invading == "r":
        phi0 = np.full(solid.shape, -1.0)
        zeta_r = 1.0
    else:
        phi0 = np.where(np.broadcast_to(x < reservoir, solid.shape), -1.0, 1.0)
        phi0 = np.ascontiguousarray(phi0)
        zeta_r = 0.0
    phi0[solid == 1] = 0.0
    if drive == "typeI":
        p = base_params(tau_r=tau_r, tau_b=tau_b, gamma=gamma, beta=beta,
                        theta_deg=theta_deg, wetting=wetting, zou_he=1,
                        flow_axis=0, rho_in=rho_in, rho_out=rho_out,
                        zeta_r=zeta_r)
    else:
        p = base_params(tau_r=tau_r, tau_b=tau_b, gamma=gamma, beta=beta,
                        theta_deg=theta_deg, wetting=wetting, zou_he=1,
                        flow_axis=0, rho_in=1.0, rho_out=1.0, zeta_r=zeta_r,
                        g=(g_x, 0.0, 0.0))
    info = {k: v for k, v in pack.items() if k != "solid"}
    return Case(f"porous_{nx}x{ny}x{nz}_{drive}", 19, solid,
                (False, True, True), phi0, p, steps, info)


def batched_droplets(count=96, smin=48, smax=128, seed=7, steps=5000,
                     scale: float = 1.0):
    """The contact-angle sweep: ``count`` sessile drops on flat walls with box
    sides side_k = smin + round((smax-smin) k/(count-1)), shuffled; radius
    8..24 with the side; theta from 30 to 150 deg over an independent
    shuffle; Scheme-I for even k and Scheme-II for odd k. ``scale`` < 1
    shrinks every box (for tests)."""
    rng = np.random.default_rng(seed)
    ks = np.arange(count)
    sides = smin + np.round((smax - smin) * ks / max(count - 1, 1)).astype(int)
    order = rng.permutation(count)
    korder = rng.permutation(count)
    cases = []
    for j in range(count):
        k = int(order[j])
        side = int(sides[k])
        radius = 8 + round(16 * (side - smin) / max(smax - smin, 1))
        theta = 30.0 + 120.0 * int(korder[j]) / max(count - 1, 1)
        if scale != 1.0:
            side = max(12, int(round(side * scale)))
            radius = max(3, int(round(radius * scale)))
        wetting = 1 if k % 2 == 0 else 2
        c = droplet_3d(side=side, radius=float(radius), theta_deg=theta,
                       wetting=wetting, steps=steps)
        c.name = f"drop{j}_s{side}_th{theta:.0f}_w{wetting}"
        cases.append(c)
    return cases


# ------------------------------------------------------------ adjoint pack
def adjoint_pack(n=(128, 128, 128), porosity=0.25, seed=2025, theta_deg=40.0,
                 g_x=5e-6, slab: Optional[int] = None, steps=2000,
                 tau_r=1.0, tau_b=1.0, gamma=0.01, beta=0.95) -> Case:
    """The gradient workload: a D3Q19 sphere pack (Boolean model as in
    sphere_pack, no reservoirs or side walls) periodic on every axis, filled
    with red (non-wetting) fluid except a blue (wetting, theta < 90 deg
    through fluid b) slab x < slab; Scheme-II; the body acceleration g_x
    drives the flow (Type-II, Eq. 36). Periodic ends stand in for the
    paper's reservoirs so that no Zou-He plane enters the adjoint."""
    nx, ny, nz = n
    pack = sphere_pack((nx, ny, nz), porosity, seed=seed, reservoir=0,
                       side_walls=False)
    solid = pack["solid"]
    s = slab if slab is not None else max(2, nx // 8)
    phi0 = np.ones((nz, ny, nx))
    phi0[:, :, :s] = -1.0
    phi0[solid == 1] = 0.0
    p = base_params(tau_r=tau_r, tau_b=tau_b, gamma=gamma, beta=beta,
                    theta_deg=theta_deg, wetting=2, g=(g_x, 0.0, 0.0))
    return Case(f"adjoint_pack{nx}x{ny}x{nz}", 19, solid, (True, True, True),
                phi0, p, steps,
                dict(rock_porosity=pack["rock_porosity"], slab=s))
