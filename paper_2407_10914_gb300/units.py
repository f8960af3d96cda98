"""Conversion between lattice units and physical units, Sec. II.E.

The lattice results are scaled by a length unit a_o, a mass unit m_o and a
time unit t_o (Eqs. 40-42):

    a_o = l_phys / x_lbm                 (m per lattice length)
    m_o = rho_phys a_o^3 / rho_lbm       (kg per lattice mass)
    t_o = nu_lbm a_o^2 / nu_phys         (s per lattice time step)

and pressures and interfacial tensions convert as (Eqs. 43-44)

    P_phys     = P_lbm m_o / (a_o t_o^2)      (Pa)
    gamma_phys = gamma_lbm m_o / t_o^2        (N/m).

The lattice viscosity of a fluid is nu_lbm = (tau - 1/2)/3 (Eq. 13). A
lattice pressure difference is Delta rho / 3 (p = rho c_s^2, c_s^2 = 1/3).
Host-side arithmetic only; nothing here touches the device.
"""
from __future__ import annotations

import dataclasses


def nu_lattice(tau: float) -> float:
    """Eq. (13): lattice kinematic viscosity of relaxation time tau."""
    return (tau - 0.5) / 3.0


@dataclasses.dataclass(frozen=True)
class Units:
    """Unit system of Eqs. (40)-(42). `nu_lbm` and `nu_phys` belong to the
    same fluid (any fluid of the run gives the same t_o when the lattice
    viscosities were chosen to match the physical ones)."""
    a0: float            # m per lattice length unit, Eq. (40) with x_lbm = 1
    rho_phys: float      # kg/m^3
    nu_phys: float       # m^2/s
    nu_lbm: float        # lattice length^2 per time step
    rho_lbm: float = 1.0  # lattice mass per lattice length^3

    @classmethod
    def from_tau(cls, a0: float, rho_phys: float, nu_phys: float, tau: float,
                 rho_lbm: float = 1.0) -> "Units":
        return cls(a0, rho_phys, nu_phys, nu_lattice(tau), rho_lbm)

    @property
    def m0(self) -> float:
        """Eq. (41)."""
        return self.rho_phys * self.a0 ** 3 / self.rho_lbm

    @property
    def t0(self) -> float:
        """Eq. (42)."""
        return self.nu_lbm * self.a0 ** 2 / self.nu_phys

    def pressure_phys(self, p_lbm: float) -> float:
        """Eq. (43): lattice pressure to Pa."""
        return p_lbm * self.m0 / (self.a0 * self.t0 ** 2)

    def pressure_lbm(self, p_phys: float) -> float:
        """Eq. (43) solved for the lattice pressure."""
        return p_phys * self.a0 * self.t0 ** 2 / self.m0

    def gamma_phys(self, gamma_lbm: float) -> float:
        """Eq. (44): lattice interfacial tension to N/m."""
        return gamma_lbm * self.m0 / self.t0 ** 2

    def gamma_lbm(self, gamma_phys: float) -> float:
        """Eq. (44) solved for the lattice interfacial tension."""
        return gamma_phys * self.t0 ** 2 / self.m0

    def density_difference(self, p_phys: float) -> float:
        """Lattice density difference Delta rho = 3 P_lbm that carries the
        physical pressure difference p_phys (the Zou-He rho_in - rho_out of
        a Type-I run)."""
        return 3.0 * self.pressure_lbm(p_phys)
