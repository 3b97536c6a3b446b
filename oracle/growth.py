"""Scale-dependent 1LPT/2LPT growth factors (test infrastructure only).

Sec. 4.1: per Fourier mode, d^2 D1/dtau^2 = kappa mu(k,a) D1, with D1(tau_ini) = 1 and
dD1/dtau = (1/a) da/dtau = a^2 E at tau_ini.

Sec. 4.2, Eq. fofrapprox (and App. B): the approximate second-order factor
d^2 D2/dtau^2 - kappa mu D2 = -kappa mu D1^2 (1 + 2 a^4 H^2 gamma_2(k, k/sqrt2, k/sqrt2, a)/(kappa mu)),
with D2(tau_ini) = -3/7 and dD2/dtau = -(6/7) a^2 E at tau_ini (Sec. 3.2).

The ODEs are integrated in ln a with an explicit Runge-Kutta 8(5,3) scheme
(SciPy DOP853, rtol 1e-12) for all k columns at once.  The result is a table
on nk log-spaced wavenumbers between k_F/2 and 1.01 sqrt(3) k_Nyq(N_p), read
per mode by linear interpolation in ln k; the table is the discretisation
of the growth factors used by both the oracle and the CUDA path.

Pins (tests/test_oracle_growth.py): Einstein-de Sitter D1 = a/a_ini and
D2 = -3/7 D1^2; EdS with constant mu against the power-law solution; EdS with
constant mu and a constant gamma_2 against the closed-form D2 (power-law
particular solutions of the gamma_2 source term); LCDM
against the growing-mode integral E(a) int da/(a E)^3; f(R) columns reduce to
LCDM at k -> 0 and to mu = 4/3 at k -> infinity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import integrate

from . import models
from .background import E, kappa


def k_table_nodes(Np: int, Lbox: float, nk: int):
    """(ln k0, dlnk, k) of the log-k table: k0 = k_F/2, k_max = 1.01 sqrt(3) k_Nyq."""
    kF = 2.0 * np.pi / Lbox
    kmin = 0.5 * kF
    kmax = 1.01 * np.sqrt(3.0) * np.pi * Np / Lbox
    lnk0, lnk1 = np.log(kmin), np.log(kmax)
    dlnk = (lnk1 - lnk0) / (nk - 1)
    return lnk0, dlnk, np.exp(lnk0 + dlnk * np.arange(nk))


def _rhs_factory(model, Om, k, lcdm_growth: bool):
    def rhs(t, y):
        a = np.exp(t)
        nk = k.size
        D1, dD1, D2, dD2 = y[:nk], y[nk:2 * nk], y[2 * nk:3 * nk], y[3 * nk:]
        if lcdm_growth:
            mu = np.ones_like(k)
            g2 = np.zeros_like(k)
        else:
            mu = models.mu(model, k, a, Om)
            g2 = models.gamma2_orth(model, k, a, Om)
        kap = kappa(a, Om)
        Ea = E(a, Om)
        dtau_dlna = 1.0 / (a**2 * Ea)          # dtau/dln a = a dtau/da = 1/(a^2 E)
        ddD1 = kap * mu * D1
        ddD2 = kap * mu * (D2 - D1 * D1) - 2.0 * a**4 * Ea**2 * g2 * D1 * D1
        return np.concatenate([dD1, ddD1, dD2, ddD2]) * dtau_dlna
    return rhs


@dataclass
class GrowthTable:
    a: np.ndarray        # a-nodes, shape (na,)
    lnk0: float
    dlnk: float
    k: np.ndarray        # table wavenumbers, shape (nk,)
    D1: np.ndarray       # shape (na, nk)
    dD1: np.ndarray      # dD1/dtau
    ddD1: np.ndarray     # d^2D1/dtau^2
    D2: np.ndarray
    dD2: np.ndarray
    ddD2: np.ndarray

    def interp(self, arr_row: np.ndarray, kmag: np.ndarray) -> np.ndarray:
        """Linear interpolation in ln k of one table row at wavenumbers kmag (k = 0 -> node 0)."""
        nk = self.k.size
        kk = np.where(kmag > 0, kmag, np.exp(self.lnk0))
        u = (np.log(kk) - self.lnk0) / self.dlnk
        i = np.clip(np.floor(u).astype(np.int64), 0, nk - 2)
        f = u - i
        return arr_row[i] * (1.0 - f) + arr_row[i + 1] * f


def solve_growth(model, Om: float, a_nodes: np.ndarray, k: np.ndarray,
                 lcdm_growth: bool = False, rtol: float = 1e-12) -> dict:
    """Integrate the 1LPT/2LPT growth ODEs from a_nodes[0]; values at every node."""
    a0 = float(a_nodes[0])
    nk = k.size
    E0 = float(E(a0, Om))
    y0 = np.concatenate([np.ones(nk), np.full(nk, a0**2 * E0),
                         np.full(nk, -3.0 / 7.0), np.full(nk, -6.0 / 7.0 * a0**2 * E0)])
    rhs = _rhs_factory(model, Om, k, lcdm_growth)
    t_eval = np.log(np.asarray(a_nodes, dtype=np.float64))
    if t_eval.size == 1:
        Y = y0[:, None]
    else:
        sol = integrate.solve_ivp(rhs, (t_eval[0], t_eval[-1]), y0, method="DOP853",
                                  t_eval=t_eval, rtol=rtol, atol=1e-14)
        if not sol.success:
            raise RuntimeError(sol.message)
        Y = sol.y
        Y[:, 0] = y0
    out = {"D1": Y[:nk].T.copy(), "dD1": Y[nk:2 * nk].T.copy(),
           "D2": Y[2 * nk:3 * nk].T.copy(), "dD2": Y[3 * nk:].T.copy()}
    ddD1 = np.empty_like(out["D1"])
    ddD2 = np.empty_like(out["D2"])
    for n, a in enumerate(a_nodes):
        if lcdm_growth:
            mu = np.ones_like(k)
            g2 = np.zeros_like(k)
        else:
            mu = models.mu(model, k, a, Om)
            g2 = models.gamma2_orth(model, k, a, Om)
        kap = kappa(a, Om)
        Ea = float(E(a, Om))
        D1n, D2n = out["D1"][n], out["D2"][n]
        ddD1[n] = kap * mu * D1n
        ddD2[n] = kap * mu * (D2n - D1n * D1n) - 2.0 * a**4 * Ea**2 * g2 * D1n * D1n
    out["ddD1"] = ddD1
    out["ddD2"] = ddD2
    return out


def growth_table(model, Om: float, a_nodes: np.ndarray, Np: int, Lbox: float,
                 nk: int = 1024) -> GrowthTable:
    """Per-k growth table on the log-k nodes; LCDM growth if model.scale_dependent == 0."""
    lnk0, dlnk, k = k_table_nodes(Np, Lbox, nk)
    lcdm = (model.kind == models.LCDM) or (not model.scale_dependent)
    g = solve_growth(model, Om, a_nodes, k, lcdm_growth=lcdm)
    return GrowthTable(a=np.asarray(a_nodes, dtype=np.float64), lnk0=lnk0, dlnk=dlnk, k=k, **g)


def lcdm_D1(Om: float, a_ini: float, a_eval) -> np.ndarray:
    """LCDM D1(a) with the paper's normalisation D1(a_ini) = 1 (mu = 1 column)."""
    a_eval = np.atleast_1d(np.asarray(a_eval, dtype=np.float64))
    nodes = np.concatenate([[a_ini], a_eval])
    g = solve_growth(None, Om, nodes, np.array([1.0]), lcdm_growth=True)
    return g["D1"][1:, 0]


def d2_exact(model, Om: float, a_ini: float, a_end: float, k: float, k1: float, k2: float,
             rtol: float = 1e-11) -> float:
    """D2(k, k1, k2) at a_end from the exact second-order equation of Sec. 4 (Eq. fofrexact).

    With cos(theta) = k1.k2/(k1 k2) fixed by the triangle k^2 = k1^2 + k2^2 + 2 k1 k2 cos(theta):
      D2'' - kappa mu(k) D2 = -kappa mu(k) D1(k1) D1(k2) [1 - (2 mu(k1) - mu(k))/mu(k) cos^2
                              + 2 a^4 H^2 gamma_2(k, k1, k2) / (kappa mu(k))],
      gamma_2 = gamma_2^E(k, k1, k2) + (3/2) Omega_m(a) [mu(k) - mu(k1)] k1.k2 / k2^2,
    D2 = -(3/7)(1 - cos^2), D2' = -(6/7)(1 - cos^2) a^2 E at a_ini (' = d/dtau, H in units of
    H0).  gamma_2^E: Sec. 5.1 for f(R), Sec. 5.2 (prop. to 1 - cos^2) for nDGP.  Used only to check
    the orthogonal-configuration approximation of Eq. fofrapprox (Fig. 1).
    """
    c = (k * k - k1 * k1 - k2 * k2) / (2.0 * k1 * k2)
    if not -1.0 - 1e-12 <= c <= 1.0 + 1e-12:
        raise ValueError("(k, k1, k2) is not a triangle")
    c2 = min(c * c, 1.0)
    kk = np.array([k, k1, k2], dtype=np.float64)

    def rhs(t, y):
        a = np.exp(t)
        Ea = float(E(a, Om))
        dt = 1.0 / (a * a * Ea)
        kap = kappa(a, Om)
        mu_k, mu_1, mu_2 = models.mu(model, kk, a, Om)
        Om_a = Om / (a**3 * Ea * Ea)
        if model.kind == models.FOFR:
            g2E = float(models.fr_gamma2E(k, k1, k2, a, Om, model.fR0))
        elif model.kind == models.NDGP:
            g2E = float(models.dgp_gamma2E(a, Om, model.rcH0, c2))
        else:
            raise ValueError("exact D2: f(R) or nDGP")
        g2 = g2E + 1.5 * Om_a * (mu_k - mu_1) * k1 * k2 * c / (k2 * k2)
        D1a, dD1a, D1b, dD1b, D2, dD2 = y
        src = 1.0 - (2.0 * mu_1 - mu_k) / mu_k * c2 + 2.0 * a**4 * Ea * Ea * g2 / (kap * mu_k)
        return [dD1a * dt, kap * mu_1 * D1a * dt, dD1b * dt, kap * mu_2 * D1b * dt,
                dD2 * dt, (kap * mu_k * D2 - kap * mu_k * D1a * D1b * src) * dt]

    E0 = float(E(a_ini, Om))
    y0 = [1.0, a_ini**2 * E0, 1.0, a_ini**2 * E0, -3.0 / 7.0 * (1 - c2), -6.0 / 7.0 * (1 - c2) * a_ini**2 * E0]
    sol = integrate.solve_ivp(rhs, (np.log(a_ini), np.log(a_end)), y0, method="DOP853", rtol=rtol, atol=1e-14)
    if not sol.success:
        raise RuntimeError(sol.message)
    return float(sol.y[4, -1])
