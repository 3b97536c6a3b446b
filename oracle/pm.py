"""Particle-mesh pieces: CIC assignment, the (screened) field solve, forces, P(k).

Test infrastructure only.  Follows:

* Sec. 2 (Eq. nbody): lap Phi_N = kappa delta, delta = rho/rho_bar - 1 from the
  particle positions; force = -grad Phi.
* App. B: the fifth force solves lap phi = m^2 a^2 phi + C(a) kappa delta eps_screen,
  and the total force is -grad(Phi_N + phi).  In Fourier space
  Phi_tot(k) = -kappa [delta(k) + C S(k) k^2/(k^2 + a^2 m^2)] / k^2 with
  S = FFT[delta eps].  f(R) (Sec. 6.1): C = 1/3, m = m(a), eps from Phi_N.
  Symmetron (App. C): C = 2 beta(a)^2, m = m(a), eps from Phi_N with the App. C Phi_crit.
  nDGP (Sec. 6.2 and App. B): C = 1/(3 beta), m = 0, eps from the smoothed density,
  with App. B's three windows of x = kR: Gaussian exp(-x^2/2), top-hat
  3 (sin x - x cos x)/x^3, sharp-k Theta(1 - x).  Screening off: S = delta (so G_eff = mu).
* Readings (silent in the paper): cloud-in-cell assignment with mesh points at
  integer multiples of the cell size; continuous Green's function -1/k^2;
  spectral gradient i k with the Nyquist plane of that axis zeroed; no CIC
  deconvolution in the force; delta(0) = S(0) = Phi(0) = 0.

Power spectrum (this build's estimator): CIC deposit, P = |delta(k)|^2 L^3/N^6 divided by
prod_i sinc^4(pi n_i/N), linear bins [ (b+1/2) k_F, (b+3/2) k_F ), modes weighted
once on the kx = 0 and kx = N/2 planes and twice elsewhere, no shot-noise
subtraction.

Readings: the top-hat window below x = 1/2 uses its Taylor series (the closed
form cancels there); the sharp-k cut keeps the modes with (kR)^2 <= 1, decided
in double precision.  A single-precision kernel can decide a mode whose (kR)^2
lies within float rounding of 1 either way; the parity tests list such modes
for their radius and box (there are none at the radii they use).

Pins (tests/test_oracle_pm.py): CIC mass conservation and hand-computed
weights; a single Fourier mode of density gives F = -kappa A k sin(k.x)/|k|^2;
the top-hat window equals the Fourier transform of a uniform sphere by radial
quadrature, its series meets the closed form at x = 1/2, and W(pi) = 3/pi^2;
the sharp-k window keeps exactly the modes with kR <= 1;
screening off multiplies the single-mode force by mu(k, a); zero net force;
the P(k) of a single mode lands in its bin with amplitude A^2 L^3/4 after deconvolution.
"""
from __future__ import annotations

import numpy as np

from . import models
from .background import C_LIGHT, kappa
from .ics import grad_factor, irfft3, k2_grid, kgrid, rfft3


def _cic_setup(pos: np.ndarray, N: int, L: float):
    u = np.mod(np.asarray(pos, dtype=np.float64), L) * (N / L)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    i0 %= N
    i1 = (i0 + 1) % N
    return i0, i1, f


def cic_deposit(pos: np.ndarray, N: int, L: float, mass: float = 1.0) -> np.ndarray:
    """Cloud-in-cell density (mass per cell) on an N^3 mesh indexed [z][y][x]; pos is (P, 3) = (x, y, z)."""
    i0, i1, f = _cic_setup(pos, N, L)
    rho = np.zeros(N**3, dtype=np.float64)
    for cz in (0, 1):
        iz = i1[:, 2] if cz else i0[:, 2]
        wz = f[:, 2] if cz else 1.0 - f[:, 2]
        for cy in (0, 1):
            iy = i1[:, 1] if cy else i0[:, 1]
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            for cx in (0, 1):
                ix = i1[:, 0] if cx else i0[:, 0]
                wx = f[:, 0] if cx else 1.0 - f[:, 0]
                rho += np.bincount((iz * N + iy) * N + ix, weights=mass * wx * wy * wz,
                                   minlength=N**3)
    return rho.reshape(N, N, N)


def cic_gather(field: np.ndarray, pos: np.ndarray, N: int, L: float) -> np.ndarray:
    """Cloud-in-cell interpolation of a [z][y][x] mesh field to positions (P, 3)."""
    i0, i1, f = _cic_setup(pos, N, L)
    flat = field.reshape(-1)
    out = np.zeros(pos.shape[0], dtype=np.float64)
    for cz in (0, 1):
        iz = i1[:, 2] if cz else i0[:, 2]
        wz = f[:, 2] if cz else 1.0 - f[:, 2]
        for cy in (0, 1):
            iy = i1[:, 1] if cy else i0[:, 1]
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            for cx in (0, 1):
                ix = i1[:, 0] if cx else i0[:, 0]
                wx = f[:, 0] if cx else 1.0 - f[:, 0]
                out += flat[(iz * N + iy) * N + ix] * wx * wy * wz
    return out


def fifth_force_coupling(model, a: float, Om: float):
    """(C, a^2 m^2) of the App. B field equation for the model (C = 0 for LCDM)."""
    if model.kind == models.FOFR:
        return 1.0 / 3.0, a * a * float(models.fr_m2(a, Om, model.fR0))
    if model.kind == models.NDGP:
        return 1.0 / (3.0 * float(models.dgp_beta(a, Om, model.rcH0))), 0.0
    if model.kind == models.SYMM:
        m2_fn, beta_fn = models.symm_fns(model)
        return 2.0 * float(beta_fn(a)) ** 2, a * a * float(m2_fn(a))
    if model.kind == models.MB:
        b, m2, _ = models.table_mb(model, a)
        return 2.0 * b * b, a * a * m2
    return 0.0, 0.0


def tophat_window(x):
    """Fourier transform of a normalised uniform sphere, W(x) = 3 (sin x - x cos x)/x^3, x = kR;
    the Taylor series 1 - x^2/10 + x^4/280 - x^6/15120 + x^8/1330560 below x = 1/2."""
    x = np.asarray(x, dtype=np.float64)
    xs = np.where(x < 0.5, 1.0, x)
    closed = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs**3
    x2 = x * x
    series = 1.0 - x2 / 10.0 + x2**2 / 280.0 - x2**3 / 15120.0 + x2**4 / 1330560.0
    return np.where(x < 0.5, series, closed)


def smoothing_window(N: int, L: float, R: float, kind: int):
    """W(k) on the [z][y][x/2+1] half spectrum for the Vainshtein density (App. B):
    0 Gaussian exp(-k^2 R^2/2), 1 top-hat, 2 sharp-k (1 for kR <= 1, else 0)."""
    k2 = k2_grid(N, L)
    if kind == 0:
        return np.exp(-0.5 * k2 * R * R)
    if kind == 1:
        return tophat_window(np.sqrt(k2) * R)
    if kind == 2:
        return (k2 * R * R <= 1.0).astype(np.float64)
    raise ValueError("smoothing window: 0 Gaussian, 1 top-hat, 2 sharp-k")


def screening_factor(model, delta_k: np.ndarray, N: int, L: float, a: float, Om: float):
    """eps(x) on the mesh: chameleon from Phi_N (Sec. 6.1) or Vainshtein from delta_R (Sec. 6.2)."""
    k2 = k2_grid(N, L)
    if model.kind in (models.FOFR, models.SYMM, models.MB):
        inv_k2 = np.zeros_like(k2)
        inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
        PhiN = irfft3(-kappa(a, Om) * delta_k * inv_k2, N)          # code potential
        PhiN_metric = PhiN / (a * a * C_LIGHT**2)
        return models.eps_chameleon(PhiN_metric, models.phi_crit(model, a, Om))
    if model.kind == models.NDGP:
        W = smoothing_window(N, L, model.R_smooth, getattr(model, "filter", 0))
        deltaR = irfft3(W * delta_k, N)
        return models.eps_vainshtein(models.vainshtein_x(1.0 + deltaR, a, Om, model.rcH0))
    raise ValueError("no screening for this model")


def potential_k(rho: np.ndarray, rho_bar: float, N: int, L: float, a: float, Om: float, model):
    """Phi_tot(k) of App. B (Newtonian plus the screened fifth force) from the mesh density."""
    delta = rho / rho_bar - 1.0
    dk = rfft3(delta)
    dk[0, 0, 0] = 0.0
    C, am2 = fifth_force_coupling(model, a, Om)
    k2 = k2_grid(N, L)
    inv_k2 = np.zeros_like(k2)
    inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
    if C != 0.0 and model.screening:
        eps = screening_factor(model, dk, N, L, a, Om)
        Sk = rfft3(delta * eps)
        Sk[0, 0, 0] = 0.0
    else:
        Sk = dk
    yuk = np.zeros_like(k2)
    yuk[k2 > 0] = k2[k2 > 0] / (k2[k2 > 0] + am2)
    return -kappa(a, Om) * (dk + C * Sk * yuk) * inv_k2


def force_mesh(rho: np.ndarray, rho_bar: float, N: int, L: float, a: float, Om: float, model):
    """(Fx, Fy, Fz) = -grad Phi_tot on the mesh, each [z][y][x]."""
    Phik = potential_k(rho, rho_bar, N, L, a, Om, model)
    gx, gy, gz = grad_factor(N, L)
    return tuple(irfft3(-g * Phik, N) for g in (gx, gy, gz))


def power_spectrum(pos: np.ndarray, N: int, L: float, nbins: int | None = None):
    """(k_mean, P(k), n_modes) of the CIC density of unit-mass particles."""
    rho = cic_deposit(pos, N, L)
    rho_bar = pos.shape[0] / N**3
    return power_spectrum_mesh(rho / rho_bar - 1.0, N, L, nbins)


def power_spectrum_mesh(delta: np.ndarray, N: int, L: float, nbins: int | None = None):
    if nbins is None:
        nbins = N // 2
    dk = rfft3(delta)
    kx, ky, kz, *_ = kgrid(N, L)
    kf = 2.0 * np.pi / L
    nx, ny, nz = kx / kf, ky / kf, kz / kf
    nmag = np.sqrt(nx**2 + ny**2 + nz**2)

    def sinc(x):
        return np.sinc(x / np.pi)          # sin(x)/x

    W2 = (sinc(np.pi * nx / N) * sinc(np.pi * ny / N) * sinc(np.pi * nz / N)) ** 4
    P = np.abs(dk) ** 2 * L**3 / N**6 / W2
    wt = np.where((nx == 0) | (nx == N // 2), 1.0, 2.0) * np.ones_like(nmag)
    b = np.floor(nmag - 0.5).astype(np.int64)
    ok = (nmag >= 0.5) & (b < nbins)
    cnt = np.bincount(b[ok], weights=wt[ok], minlength=nbins)
    psum = np.bincount(b[ok], weights=(wt * P)[ok], minlength=nbins)
    ksum = np.bincount(b[ok], weights=(wt * nmag * kf)[ok], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt
