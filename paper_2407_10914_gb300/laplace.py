"""The Laplace-law test of Sec. III.A at the paper's scale: red drops of
several radii in blue fluid, fully periodic box, the paper's viscosity
ratio (tau^r = 1.0, tau^b = 0.6) and lattice tension; the slope of the
pressure jump against 2/R is the simulated interfacial tension, converted
to N/m with the unit system of Sec. III.A (Eqs. 40-44).

The jump is averaged over the second half of each run: the drop's initial
relaxation leaves pressure waves in the periodic box that oscillate about
the steady value (single readings at 8000 and 12000 steps of a 128^3 box
differ by 4 %). Host logic over an engine with set_params / init_state /
step / macros (the GPU session)."""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from . import analysis as A
from . import workloads as W
from .units import Units

# Sec. III.A's unit system: a_o = 1 um, rho = 1000 kg/m^3, fluid r with
# nu_phys = 5e-6 m^2/s at tau^r = 1.0
PAPER_UNITS = Units.from_tau(1e-6, 1000.0, 5e-6, 1.0)


def run_drop(make_session: Callable[[object], object], n: int, radius: float,
             gamma: float, steps: int, sample_every: int = 250,
             beta: float = 0.95, collision: int = 0):
    """One drop: the time-averaged (dP, R) over steps/2..steps.
    collision 0: single-rate Eq. 2; 1: MRT (the paper's operator)."""
    case = W.laplace_drop(19, n, float(radius), gamma=gamma, beta=beta,
                          tau_r=1.0, tau_b=0.6)
    case.params["collision"] = collision
    s = make_session(case)
    half = steps // 2
    s.step(half)
    dps, rs = [], []
    done = half
    while done < steps:
        k = min(sample_every, steps - done)
        s.step(k)
        done += k
        m = s.macros()
        dp, R = A.laplace_measure(m["rho"].cpu().numpy(),
                                  m["phi"].cpu().numpy())
        dps.append(dp)
        rs.append(R)
    return float(np.mean(dps)), float(np.mean(rs))


def sweep(make_session, n: int, radii: Sequence[float], steps: int,
          gamma_phys: float = 0.02, units: Units = PAPER_UNITS,
          collision: int = 0) -> dict:
    """The sweep of Sec. III.A; returns the per-drop results, the slope in
    lattice units and in N/m, and its error against the input tension."""
    g = units.gamma_lbm(gamma_phys)
    drops = [run_drop(make_session, n, R0, g, steps, collision=collision)
             for R0 in radii]
    dps = [d for d, _ in drops]
    rs = [r for _, r in drops]
    slope = A.laplace_slope(dps, rs)
    return {"gamma_lbm_input": g, "radii": rs, "dp_lbm": dps,
            "dp_phys": [units.pressure_phys(d) for d in dps],
            "gamma_lbm_sim": slope, "gamma_phys_sim": units.gamma_phys(slope),
            "error": abs(slope - g) / g}
