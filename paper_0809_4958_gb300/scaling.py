"""Reduced-unit matching between the DNS sub-volume and the LB box (Sec. 3).

The LB box resolves the DNS sub-volume z = Delta / a times finer (zoom), so
the Kolmogorov length in LB sites is eta~ = (eta / Delta) z; with the LB
viscosity nu~ = (tau - 1/2) / 3 the Kolmogorov time in LB steps is
tau~_eta = eta~^2 / nu~.  Eq. (1) matches velocities in Kolmogorov units,
w~ tau~_eta / eta~ = w tau_eta / eta, and the times t~ / tau~_eta =
t / tau_eta; lengths scale with eta~ / eta.  Accelerations (the co-moving
frame force -dv/dt) follow as length / time^2.  The Mach number of the LB run
is Ma = eta~ / (tau~_eta c_s) (Sec. 3).  Host-side arithmetic only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

CS = 1.0 / math.sqrt(3.0)  # lattice speed of sound


def kolmogorov(nu: float, eps: float) -> tuple[float, float]:
    """Kolmogorov length eta = nu^(3/4) eps^(-1/4) and time tau_eta = sqrt(nu / eps)."""
    return nu ** 0.75 * eps ** -0.25, math.sqrt(nu / eps)


@dataclass
class UnitMap:
    """DNS scales (eta, tau_eta, grid spacing delta, all in DNS units), the
    zoom z and the LB relaxation time tau."""
    eta: float
    tau_eta: float
    delta: float
    z: float
    tau: float

    @property
    def nu_lb(self) -> float:
        return (self.tau - 0.5) / 3.0

    @property
    def eta_lb(self) -> float:
        """Kolmogorov length in LB sites."""
        return self.eta / self.delta * self.z

    @property
    def tau_eta_lb(self) -> float:
        """Kolmogorov time in LB steps."""
        return self.eta_lb ** 2 / self.nu_lb

    @property
    def length(self) -> float:
        """LB sites per DNS length unit."""
        return self.eta_lb / self.eta

    @property
    def time(self) -> float:
        """LB steps per DNS time unit."""
        return self.tau_eta_lb / self.tau_eta

    @property
    def velocity(self) -> float:
        """LB velocity per DNS velocity (Eq. 1)."""
        return self.length / self.time

    @property
    def acceleration(self) -> float:
        """LB acceleration per DNS acceleration."""
        return self.length / self.time ** 2

    @property
    def mach(self) -> float:
        return self.eta_lb / (self.tau_eta_lb * CS)

    def steps(self, dt: float) -> float:
        """LB steps spanned by a DNS time interval dt."""
        return dt * self.time
