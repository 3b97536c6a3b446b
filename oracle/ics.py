"""Gaussian initial field and the 2LPT potentials (test infrastructure only).

Conventions (unnormalised forward DFT, e^{+ikx} synthesis with 1/N^3):

* delta_hat(k) = DFT[g](k) sqrt(P_ini(k) N^3 / L^3), delta_hat(0) = 0, where g is the
  Philox white noise and P_ini(k) = P(k, z=0) [D_LCDM(a_ini)/D_LCDM(1)]^2 (LCDM ICs
  for every model, as in the paper's MG runs).
* 1LPT (Sec. 3.1): div Psi1 = -delta, Psi1 = grad phi1, so phi1(k) = delta_hat(k)/k^2.
* 2LPT (Sec. 3.2, Eq. lcdm2lpt): lap phi2 = 1/2[(lap phi1)^2 - (phi1_ij)^2]
  = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2), so phi2(k) = -DFT[src](k)/k^2.
* Derivatives are spectral: d_i <-> i k_i with k_i = 2 pi n_i / L.  A first
  derivative along an axis is zero on that axis' Nyquist plane; a mixed second
  derivative phi_ij (i != j) is zero if either index sits on its Nyquist plane;
  a pure second derivative phi_ii uses -k_i^2 everywhere.

Arrays are indexed [z][y][x] and the half spectrum keeps kx = 0..N/2 (numpy rfftn).

Pins (tests/test_oracle_pm.py): one cosine mode gives phi2 = 0; two
perpendicular modes give phi2 = -A B k1^2 k2^2 cos(k1 x) cos(k2 y)/(k1^2 + k2^2);
the IC power spectrum matches P_ini within cosmic variance; the DFT
conventions against a direct sum on an 8^3 grid.
"""
from __future__ import annotations

import numpy as np
from scipy import fft as sfft

from . import philox
from .power import linear_pk_z0
from .growth import lcdm_D1

WORKERS = -1  # scipy.fft: all host cores


def kgrid(N: int, L: float):
    """(kx, ky, kz, nyq_x, nyq_y, nyq_z) broadcastable to the [z][y][x/2+1] half spectrum."""
    kf = 2.0 * np.pi / L
    n_full = np.fft.fftfreq(N, d=1.0 / N)            # 0..N/2-1, -N/2..-1
    n_half = np.arange(N // 2 + 1, dtype=np.float64)
    kz = (kf * n_full)[:, None, None]
    ky = (kf * n_full)[None, :, None]
    kx = (kf * n_half)[None, None, :]
    nyz = (np.abs(n_full) == N // 2)[:, None, None]
    nyy = (np.abs(n_full) == N // 2)[None, :, None]
    nyx = (n_half == N // 2)[None, None, :]
    return kx, ky, kz, nyx, nyy, nyz


def grad_factor(N: int, L: float):
    """(i kx, i ky, i kz), each zero on its own Nyquist plane."""
    kx, ky, kz, nyx, nyy, nyz = kgrid(N, L)
    return (1j * np.where(nyx, 0.0, kx), 1j * np.where(nyy, 0.0, ky), 1j * np.where(nyz, 0.0, kz))


def k2_grid(N: int, L: float):
    kx, ky, kz, *_ = kgrid(N, L)
    return kx**2 + ky**2 + kz**2


def rfft3(x):
    return sfft.rfftn(x, workers=WORKERS)


def irfft3(X, N):
    return sfft.irfftn(X, s=(N, N, N), workers=WORKERS)


def delta_k(cosmo, N: int, L: float, seed: int, a_ini: float) -> np.ndarray:
    """Gaussian density contrast at a_ini in the unnormalised half spectrum."""
    g = philox.white_noise(N, seed)
    G = rfft3(g)
    k2 = k2_grid(N, L)
    kmag = np.sqrt(k2)
    pk0 = linear_pk_z0(cosmo)
    Dratio = 1.0 / lcdm_D1(cosmo.Omega_m, a_ini, [1.0])[0]   # D(a_ini)/D(1), D(a_ini) = 1
    amp = np.zeros_like(kmag)
    nz = kmag > 0
    amp[nz] = np.sqrt(pk0(kmag[nz]) * Dratio**2 * N**3 / L**3)
    d = G * amp
    d[0, 0, 0] = 0.0
    return d


def potentials_from_delta(dk: np.ndarray, N: int, L: float):
    """(phi1(k), phi2(k)) from delta(k) by Sec. 3.1 and Eq. lcdm2lpt."""
    kx, ky, kz, nyx, nyy, nyz = kgrid(N, L)
    k2 = kx**2 + ky**2 + kz**2
    inv_k2 = np.zeros_like(k2)
    inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
    phi1 = dk * inv_k2
    kk = (kx, ky, kz)
    nyq = (nyx, nyy, nyz)

    def hess(i, j):
        f = -kk[i] * kk[j]
        if i != j:
            f = np.where(nyq[i] | nyq[j], 0.0, f)
        return irfft3(phi1 * f, N)

    h = {(i, j): hess(i, j) for i in range(3) for j in range(i, 3)}
    src = (h[0, 0] * h[1, 1] - h[0, 1] ** 2
           + h[0, 0] * h[2, 2] - h[0, 2] ** 2
           + h[1, 1] * h[2, 2] - h[1, 2] ** 2)
    phi2 = -rfft3(src) * inv_k2
    phi2[0, 0, 0] = 0.0
    return phi1, phi2


def initial_potentials(cosmo, N: int, L: float, seed: int, a_ini: float):
    return potentials_from_delta(delta_k(cosmo, N, L, seed, a_ini), N, L)
