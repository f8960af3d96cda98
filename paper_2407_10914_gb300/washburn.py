"""Washburn tests of Sec. IV.A: the wetting fluid b entering a capillary
tube filled with the non-wetting fluid r, against the Washburn law with
unequal viscosities (Eqs. 47-51) and the paper's area error. Case-I:
spontaneous imbibition (theta < 90 deg, equal end pressures). Case-II:
neutral wetting (theta = 90 deg) and a pressure difference, imposed by the
Zou-He densities (Type-I) or a body force (Type-II).

In non-dimensional form (Eqs. 49-51), with m = mu_nw / (mu_w - mu_nw),
    z*(t*) = -m + sqrt(m^2 + (Delta P r^2 / (2 L gamma) + (r/L) cos(theta))
                            t* / 2),
    z* = z / L,   t* = gamma t / ((mu_w - mu_nw) L),
and the error is |int z_lbm dt - int z_analytical dt| / int z_analytical dt.

Procedure (as the paper runs it): b occupies the first layer and the tube
is run at theta = 90 deg (neutral, no capillary drive) until the interface
is steady; its position z*_init fixes the start time t*_init = Eq. (49)
solved for t*. Then the contact angle is set and the interface position
is sampled as it advances. Host logic over an engine with set_params /
step / macros (the GPU session)."""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np

from .analysis import area_error  # the paper's error metric (Sec. IV.A.1)


def zstar(tstar, theta_deg: float, m: float, r_over_L: float,
          dp_term: float = 0.0):
    """Eq. (49). dp_term = Delta P r^2 / (2 L gamma) (0 in Case-I)."""
    k = dp_term + r_over_L * math.cos(math.radians(theta_deg))
    return -m + np.sqrt(m * m + 0.5 * k * np.asarray(tstar, np.float64))


def tstar_of(z, theta_deg: float, m: float, r_over_L: float,
             dp_term: float = 0.0) -> float:
    """Eq. (49) solved for t*: the time at which the interface is at z*."""
    k = dp_term + r_over_L * math.cos(math.radians(theta_deg))
    return ((z + m) ** 2 - m * m) / (0.5 * k)


def interface_tip(phi: np.ndarray, solid: np.ndarray) -> float:
    """Interface position along x: the phi = 0 crossing (b -> r, searched
    from the inlet) on the lines parallel to the tube axis that are nearest
    to it, averaged; linear interpolation between nodes. phi and solid
    have shape (nz, ny, nx)."""
    nz, ny, nx = phi.shape
    cz, cy = (nz - 1) / 2.0, (ny - 1) / 2.0
    zs = sorted({int(math.floor(cz)), int(math.ceil(cz))})
    ys = sorted({int(math.floor(cy)), int(math.ceil(cy))})
    out = []
    for z in zs:
        for y in ys:
            if solid[z, y, 0]:
                continue
            line = phi[z, y, :]
            pos = None
            for x in range(nx - 1):
                if line[x] < 0.0 <= line[x + 1]:
                    pos = x + line[x] / (line[x] - line[x + 1])
                    break
            if pos is not None:
                out.append(pos)
    return float(np.mean(out)) if out else float("nan")


def run_case1(make_session: Callable[[dict], object], case,
              theta_deg: float, wetting: int, tstar_end: float = 60.0,
              sample_every: int = 500, init_tol: float = 0.01,
              init_max_steps: int = 40000) -> dict:
    """Case-I (Sec. IV.A.1): spontaneous imbibition at contact angle
    theta_deg, equal end pressures."""
    return run(make_session, case, theta_deg, wetting, 0.0, "typeI",
               tstar_end, sample_every, init_tol, init_max_steps)


def run_case2(make_session: Callable[[dict], object], case, dp_lbm: float,
              drive: str, wetting: int = 1, tstar_end: float = 60.0,
              sample_every: int = 500, init_tol: float = 0.01,
              init_max_steps: int = 40000) -> dict:
    """Case-II (Sec. IV.A.2): neutral wetting (theta = 90 deg), the fluids
    driven by a lattice pressure difference dp_lbm, imposed by the Zou-He
    densities (Type-I, rho_in - rho_out = 3 dp) or by a body force with
    equal end densities (Type-II, g = dp / (rho0 L))."""
    return run(make_session, case, 90.0, wetting, dp_lbm, drive,
               tstar_end, sample_every, init_tol, init_max_steps)


def run(make_session, case, theta_deg: float, wetting: int, dp_lbm: float,
        drive: str, tstar_end: float, sample_every: int, init_tol: float,
        init_max_steps: int) -> dict:
    """One run: the settled neutral start, then the contact angle and the
    drive; the sampled curve beside Eq. (49) and the area error.

    make_session(params) returns an engine holding `case`'s geometry with
    those parameters and the initial phase field loaded (e.g. a GPU
    Session)."""
    if drive not in ("typeI", "typeII"):
        raise ValueError("drive must be typeI or typeII")
    p = dict(case.params)
    L = float(case.info["length"])
    r = float(case.info["radius"])
    rho0 = p["rho0"]
    mu_w = rho0 * (p["tau_b"] - 0.5) / 3.0   # b is the wetting fluid
    mu_nw = rho0 * (p["tau_r"] - 0.5) / 3.0
    m = mu_nw / (mu_w - mu_nw)
    gamma = p["gamma"]
    steps_per_tstar = (mu_w - mu_nw) * L / gamma  # Eq. (51)
    dp_term = dp_lbm * r * r / (2.0 * L * gamma)
    # 1) neutral initial run without drive until the interface stops
    s = make_session(dict(p, theta_deg=90.0, wetting=wetting))
    z_prev, steps = None, 0
    while steps < init_max_steps:
        s.step(sample_every)
        steps += sample_every
        z = interface_tip(s.macros()["phi"].cpu().numpy(), case.solid)
        if z_prev is not None and abs(z - z_prev) < init_tol:
            break
        z_prev = z
    z_init = z / L
    # 2) contact angle and drive; t* starts at Eq. (49)'s time of z*_init
    q = dict(p, theta_deg=theta_deg, wetting=wetting)
    if dp_lbm != 0.0:
        rho = p["rho_out"]
        if drive == "typeI":
            q.update(rho_in=rho + 1.5 * dp_lbm, rho_out=rho - 1.5 * dp_lbm)
        else:
            q.update(g=(dp_lbm / (rho0 * L), 0.0, 0.0))
    s.set_params(**q)
    t0 = tstar_of(z_init, theta_deg, m, r / L, dp_term)
    n_steps = int(math.ceil((tstar_end - t0) * steps_per_tstar))
    ts, zs = [t0], [z_init]
    done = 0
    while done < n_steps:
        k = min(sample_every, n_steps - done)
        s.step(k)
        done += k
        zz = interface_tip(s.macros()["phi"].cpu().numpy(), case.solid) / L
        if not np.isfinite(zz) or zz >= 0.95:
            break  # the interface reached the outlet end
        ts.append(t0 + done / steps_per_tstar)
        zs.append(zz)
    ts = np.asarray(ts)
    zs = np.asarray(zs)
    ref = zstar(ts, theta_deg, m, r / L, dp_term)
    return dict(theta_deg=theta_deg, wetting=wetting, dp_lbm=dp_lbm,
                drive=drive, z_init=z_init, tstar_init=t0, init_steps=steps,
                tstar=ts, zstar=zs, zstar_eq49=ref,
                area_error=area_error(zs, ref, ts),
                steps_per_tstar=steps_per_tstar)
