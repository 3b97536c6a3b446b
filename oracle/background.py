"""Background cosmology in the paper's time variable (test infrastructure only).

Units: lengths in Mpc/h, time in 1/H0 (so H0 = 1 and H(a) = E(a)).

* Super-comoving time: d tau = dt / a^2 (Sec. 1, conventions paragraph), so
  da/dtau = a^3 E(a) and Delta tau(a1, a2) = int_{a1}^{a2} da / (a^3 E(a)).
* kappa(a) = 4 pi G rho_bar a^4 = (3/2) Omega_m H0^2 a (Sec. 1; Sec. 3, Eq. geodesicdispfield).
* Flat LCDM expansion E(a)^2 = Omega_m a^-3 + 1 - Omega_m (App. B: the fiducial background).

Pins: Delta tau against the Einstein-de Sitter closed form; E and its
logarithmic derivative against finite differences (tests/test_oracle_basics.py).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate

# Speed of light in units of (Mpc/h) * H0, i.e. c / (100 km/s).
C_LIGHT = 2997.92458


def E(a, Om):
    """H(a)/H0 for flat LCDM."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(Om * a**-3 + 1.0 - Om)


def dlnE_da(a, Om):
    """d ln E / da."""
    a = np.asarray(a, dtype=np.float64)
    return -1.5 * Om * a**-4 / E(a, Om) ** 2


def Omega_m_a(a, Om):
    """Omega_m(a) = Omega_m a^-3 / E(a)^2."""
    a = np.asarray(a, dtype=np.float64)
    return Om * a**-3 / E(a, Om) ** 2


def kappa(a, Om):
    """kappa = (3/2) Omega_m a in H0 = 1 units."""
    return 1.5 * Om * np.asarray(a, dtype=np.float64)


def dadtau(a, Om):
    """da/dtau = a^3 E(a)  (d tau = dt/a^2 and da/dt = a H)."""
    a = np.asarray(a, dtype=np.float64)
    return a**3 * E(a, Om)


def dtau(a1: float, a2: float, Om: float) -> float:
    """Delta tau = int_{a1}^{a2} da / (a^3 E(a)), adaptive Gauss-Kronrod."""
    if a1 == a2:
        return 0.0
    val, _ = integrate.quad(lambda a: 1.0 / (a**3 * float(E(a, Om))), a1, a2,
                            epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def a_nodes(a_ini: float, a_final: float, nsteps: int) -> np.ndarray:
    """Time grid uniform in a: a_i = a_ini + i (a_final - a_ini) / nsteps."""
    i = np.arange(nsteps + 1, dtype=np.float64)
    a = a_ini + i * (a_final - a_ini) / nsteps
    a[-1] = a_final
    return a
