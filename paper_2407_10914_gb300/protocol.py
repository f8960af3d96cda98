"""The displacement protocol of Sec. IV.B: primary drainage, spontaneous
imbibition and forced imbibition in a porous sample, recorded as a
capillary-pressure / water-saturation (P_c - S_w) curve.

The experiment it reproduces (a SCAL laboratory test):

* the sample starts full of the wetting fluid ("b", water; the contact
  angle is measured through it, so theta < 90 deg makes it wetting);
* primary drainage: the non-wetting fluid ("r", oil) is injected at the
  inlet (zeta^r = 1) and the pressure difference is raised level by level,
  each level held until S_w settles; drainage stops when a further increase
  barely lowers S_w (the irreducible saturation);
* spontaneous imbibition: the pressure difference is lowered level by level
  to zero with oil still at the inlet;
* forced imbibition: water replaces oil at the inlet (Eqs. 37-38 on the
  inlet plane, zeta^r = 0) and the pressure difference is raised again; it
  is reported as a negative capillary pressure; the stage stops when a
  further increase barely raises S_w.

S_w is the fraction of fluid nodes with phi < 0 (LBM_SW_COUNT, as the paper
defines it in Sec. IV.B); its smooth form (LBM_SW_SMOOTH) is recorded
beside it. P_c is the imposed pressure difference (the paper's reading:
P_c = P_nw - P_w).

Drive (Sec. II.C): Type-I sets the Zou-He densities, rho_in = rho_out +
3 Delta P; Type-II keeps rho_in = rho_out and applies the body acceleration
g = Delta P / (rho0 L) along the flow axis, L the distance between the
Zou-He planes, so both impose the same mean gradient.

The runner is host logic only. Its `engine` is any object with
``set_params(**params)``, ``step(n)``, ``reduce(kind) -> float`` and
``swap_inlet(colour)``: the GPU session (:class:`lbm.Session`) for runs.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

from .units import Units

SW_COUNT, SW_SMOOTH = 2, 3  # lbm_reduce kinds (LBM_SW_COUNT, LBM_SW_SMOOTH)
RED, BLUE = 0, 1


@dataclasses.dataclass
class Level:
    """One held pressure level of the protocol."""
    stage: str          # "drainage", "spontaneous", "forced"
    dp_lbm: float       # imposed lattice pressure difference (>= 0)
    pc_lbm: float       # capillary pressure: +dp (oil injected), -dp (water)
    pc_phys: Optional[float]  # P_c in Pa (Eq. 43), if units were given
    sw: float           # S_w, fraction of fluid nodes with phi < 0
    sw_smooth: float    # mean of (1 - phi)/2 over fluid nodes
    steps: int          # steps spent at this level
    settled: bool       # S_w changed by < sw_tol over the last check


class Displacement:
    """Runs the protocol on `engine` from its current state.

    params      full parameter dict of the run (the C-ABI's keys); zou_he
                must be 1 (the inlet plane is where the fluids enter)
    drive       "typeI" or "typeII"
    length      lattice distance between the inlet and outlet planes
                (n_axis - 1)
    units       optional unit system for P_c in Pa
    check_every steps between two S_w readings at a level
    sw_tol      a level is settled when S_w moves by less than this between
                two readings
    max_steps   cap on the steps of one level
    stop_dsw    a stage ends when one level changes S_w by less than this
                (after S_w has started to move)
    """

    def __init__(self, engine, params: dict, drive: str = "typeI",
                 length: float = 1.0, units: Optional[Units] = None,
                 check_every: int = 500, sw_tol: float = 1e-3,
                 max_steps: int = 20000, stop_dsw: float = 0.01):
        if drive not in ("typeI", "typeII"):
            raise ValueError("drive must be typeI or typeII")
        if not params.get("zou_he"):
            raise ValueError("the protocol injects through a Zou-He inlet")
        self.engine = engine
        self.params = dict(params)
        self.drive = drive
        self.length = float(length)
        self.units = units
        self.check_every = int(check_every)
        self.sw_tol = float(sw_tol)
        self.max_steps = int(max_steps)
        self.stop_dsw = float(stop_dsw)
        self.curve: List[Level] = []

    # ------------------------------------------------------------ drive
    def drive_params(self, dp: float) -> dict:
        """The parameter dict that imposes the lattice pressure difference
        dp between inlet and outlet with the chosen drive."""
        p = dict(self.params)
        a = int(p.get("flow_axis", 0))
        rho_out = float(p.get("rho_out", 1.0))
        g = [0.0, 0.0, 0.0]
        if self.drive == "typeI":
            p["rho_in"] = rho_out + 3.0 * dp
        else:
            p["rho_in"] = rho_out
            g[a] = dp / (float(p.get("rho0", 1.0)) * self.length)
        p["g"] = tuple(g)
        return p

    def _set(self, dp: float):
        self.engine.set_params(**self.drive_params(dp))

    # ------------------------------------------------------------ levels
    def hold(self, stage: str, dp: float, sign: float) -> Level:
        """Impose dp and step until S_w settles (or max_steps)."""
        self._set(dp)
        e = self.engine
        prev = e.reduce(SW_COUNT)
        steps, settled = 0, False
        while steps < self.max_steps:
            n = min(self.check_every, self.max_steps - steps)
            e.step(n)
            steps += n
            sw = e.reduce(SW_COUNT)
            if abs(sw - prev) < self.sw_tol:
                settled = True
                break
            prev = sw
        sw = e.reduce(SW_COUNT)
        pc = sign * dp
        lev = Level(stage, dp, pc,
                    self.units.pressure_phys(pc) if self.units else None,
                    sw, e.reduce(SW_SMOOTH), steps, settled)
        self.curve.append(lev)
        return lev

    def _stage(self, stage: str, levels: Sequence[float], sign: float,
               until_flat: bool) -> List[Level]:
        out: List[Level] = []
        moved = False
        for dp in levels:
            before = out[-1].sw if out else self.engine.reduce(SW_COUNT)
            lev = self.hold(stage, dp, sign)
            out.append(lev)
            change = abs(lev.sw - before)
            if change >= self.stop_dsw:
                moved = True
            elif until_flat and moved:
                break  # a further increase barely changed S_w
        return out

    # ------------------------------------------------------------ stages
    def primary_drainage(self, levels: Sequence[float]) -> List[Level]:
        """Oil (r) injected; dp raised over `levels` until S_w stops
        falling."""
        self.params["zeta_r"] = 1.0
        return self._stage("drainage", sorted(levels), +1.0, True)

    def spontaneous_imbibition(self, levels: Sequence[float]) -> List[Level]:
        """Oil still at the inlet; dp lowered over `levels` (to zero)."""
        self.params["zeta_r"] = 1.0
        return self._stage("spontaneous", sorted(levels, reverse=True), +1.0,
                           False)

    def forced_imbibition(self, levels: Sequence[float]) -> List[Level]:
        """Water (b) replaces oil at the inlet (Eqs. 37-38), then dp is
        raised over `levels` until S_w stops rising; P_c = -dp."""
        self.params["zeta_r"] = 0.0
        self.engine.swap_inlet(BLUE)
        return self._stage("forced", sorted(levels), -1.0, True)

    def run(self, drainage: Sequence[float], spontaneous: Sequence[float],
            forced: Sequence[float]) -> List[Level]:
        """The three stages in turn; returns the whole curve."""
        self.primary_drainage(drainage)
        self.spontaneous_imbibition(spontaneous)
        self.forced_imbibition(forced)
        return self.curve
