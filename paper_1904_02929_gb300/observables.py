"""Derived observables of the paper, computed on the host from what the
library returns (time-averaged stress tensors, moduli).  No method arithmetic
of the step lives here.

* ``stress_anisotropy``: Delta lambda = sigma_1 - sigma_3 (largest minus
  smallest eigenvalue of the stress tensor) and P = -(sigma_1 + sigma_2 +
  sigma_3) / 3, with their ratio (Sec. 3.3); ``stress_anisotropy_2d`` the
  monolayer's in-plane form sigma_1 - sigma_2 and P = -(sigma_1 + sigma_2) / 2
  from the x-y block (Sec. 4.4).
* ``reduced_shear_rate``: gamma_dot* = 6 pi eta0 a_min^2 gamma_dot / F0
  (Sec. 3.2).
* ``relative_viscosity``: eta / eta0 = sigma_xy / (eta0 gamma_dot) under a
  constant rate.
* ``dimensionless_moduli``: G'* = G' / kn, G''* = G'' / kn and
  eta* = G''* / (omega tau_c) (Sec. 4.1).
* ``strain_window``: the lattice steps over which a constant-rate run is
  averaged, strains gamma = 5 to 11 (Sec. 3.1); ``wall_shear_rate``: the
  nominal rate U / (y_top - y_bottom) of bumpy walls moving apart at U
  (Sec. 3).
"""
from __future__ import annotations

import math

import numpy as np


def solvent_viscosity(tau: float, rho0: float = 1.0) -> float:
    """Lattice-Boltzmann shear viscosity eta0 = rho0 (tau - 1/2) / 3."""
    return rho0 * (tau - 0.5) / 3.0


def stress_anisotropy(sigma) -> tuple[float, float, float]:
    """(Delta lambda, P, Delta lambda / P) of a 3 x 3 stress tensor (its
    symmetric part; eigenvalues sorted sigma_1 >= sigma_2 >= sigma_3)."""
    s = np.asarray(sigma, dtype=float).reshape(3, 3)
    ev = np.linalg.eigvalsh(0.5 * (s + s.T))[::-1]
    dl = float(ev[0] - ev[2])
    p = float(-ev.sum() / 3.0)
    return dl, p, (dl / p if p != 0.0 else math.inf)


def stress_anisotropy_2d(sigma) -> tuple[float, float, float]:
    """(Delta lambda, P, Delta lambda / P) of the monolayer: eigenvalues
    sigma_1 >= sigma_2 of the symmetric x-y block of the stress tensor,
    Delta lambda = sigma_1 - sigma_2, P = -(sigma_1 + sigma_2) / 2."""
    s = np.asarray(sigma, dtype=float).reshape(3, 3)[:2, :2]
    ev = np.linalg.eigvalsh(0.5 * (s + s.T))[::-1]
    dl = float(ev[0] - ev[1])
    p = float(-ev.sum() / 2.0)
    return dl, p, (dl / p if p != 0.0 else math.inf)


def reduced_shear_rate(rate: float, eta0: float, a_min: float, F0: float) -> float:
    """gamma_dot* = 6 pi eta0 a_min^2 gamma_dot / F0."""
    return 6.0 * math.pi * eta0 * a_min * a_min * rate / F0


def relative_viscosity(sigma_xy: float, rate: float, eta0: float) -> float:
    """Apparent viscosity over the solvent's, eta / eta0 = sigma_xy / (eta0 gamma_dot)."""
    return sigma_xy / (eta0 * rate)


def dimensionless_moduli(Gp: float, Gpp: float, kn: float, omega: float,
                         tau_c: float) -> tuple[float, float, float]:
    """(G'*, G''*, eta*) = (G' / kn, G'' / kn, (G'' / kn) / (omega tau_c))."""
    gps, gpps = Gp / kn, Gpp / kn
    return gps, gpps, gpps / (omega * tau_c)


def strain_window(rate: float, gamma_start: float = 5.0, gamma_end: float = 11.0) -> tuple[int, int]:
    """(first, last) lattice step of the averaging window gamma_start <=
    rate t <= gamma_end: step ``box.step(first)``, ``box.stress_reset()``,
    then ``box.step(last - first)`` and read the time-averaged stress."""
    if not rate > 0.0 or not gamma_end > gamma_start >= 0.0:
        raise ValueError("need rate > 0 and 0 <= gamma_start < gamma_end")
    return math.ceil(gamma_start / rate - 1e-9), math.floor(gamma_end / rate + 1e-9)


def wall_shear_rate(wall_speed: float, y_bottom: float, y_top: float) -> float:
    """Nominal shear rate of two bumpy walls whose relative speed is
    ``wall_speed``, from the distance between their centre planes."""
    return wall_speed / (y_top - y_bottom)
