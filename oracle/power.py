"""Linear matter power spectrum for the initial conditions (test infrastructure only).

The paper does not fix an initial power spectrum; this build uses the
Eisenstein & Hu (1998, ApJ 496, 605) "no-wiggle" transfer function
(their Eqs. 26, 28-31), written from that publication:

    s        = 44.5 ln(9.83/w_m) / sqrt(1 + 10 w_b^(3/4))          [Mpc]
    alpha_G  = 1 - 0.328 ln(431 w_m) f_b + 0.38 ln(22.3 w_m) f_b^2
    Gamma    = Omega_m h (alpha_G + (1 - alpha_G)/(1 + (0.43 k s)^4))  (k in 1/Mpc)
    q        = k Theta_2.7^2 / Gamma                                (k in h/Mpc)
    T0(q)    = L0/(L0 + C0 q^2),  L0 = ln(2e + 1.8 q),  C0 = 14.2 + 731/(1 + 62.5 q)

with w_m = Omega_m h^2, w_b = Omega_b h^2, f_b = Omega_b/Omega_m and
T_CMB = 2.7255 K.  P(k, z=0) = A k^n_s T0(k)^2 with A fixed by sigma_8 in a
real-space top-hat of radius 8 Mpc/h.

Pins (tests/test_oracle_basics.py): T0 -> 1 as k -> 0; the sigma_8
normalisation reproduces sigma_8 by an independent quadrature; the
small-scale slope T0 ~ ln(q)/q^2.  The fit's interior coefficients (s,
alpha_G, C0) have no printed value to check them against here: parity
unpinned for the shape of T0 between those limits.  It only generates the
initial conditions; the GPU library evaluates its own restatement of the fit,
and the IC parity tests compare the two through the initial potentials.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate

T_CMB = 2.7255


def eh_nowiggle_T(k, Om, Ob, h):
    """Eisenstein-Hu no-wiggle transfer function, k in h/Mpc."""
    k = np.asarray(k, dtype=np.float64)
    wm, wb = Om * h * h, Ob * h * h
    fb = Ob / Om
    theta = T_CMB / 2.7
    s = 44.5 * np.log(9.83 / wm) / np.sqrt(1.0 + 10.0 * wb**0.75)
    alpha = 1.0 - 0.328 * np.log(431.0 * wm) * fb + 0.38 * np.log(22.3 * wm) * fb * fb
    kmpc = k * h
    gamma = Om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * kmpc * s) ** 4))
    q = k * theta * theta / gamma
    L0 = np.log(2.0 * np.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def tophat_W(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = 1.0 - xs * xs / 10.0
    xl = x[~small]
    out[~small] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl**3
    return out


def sigma_R(pk_fn, R: float) -> float:
    """sigma(R)^2 = 1/(2 pi^2) int k^2 P(k) W(kR)^2 dk, integrated in ln k."""
    def integrand(lnk):
        k = np.exp(lnk)
        return k**3 * pk_fn(k) * float(tophat_W(np.array([k * R]))[0]) ** 2 / (2.0 * np.pi**2)
    val, _ = integrate.quad(integrand, np.log(1e-6), np.log(1e3), epsabs=0.0, epsrel=1e-11,
                            limit=1000)
    return float(np.sqrt(val))


def linear_pk_z0(cosmo):
    """P(k, z=0) [(Mpc/h)^3], sigma_8-normalised; returns a callable of k [h/Mpc]."""
    Om, Ob, h, ns, s8 = cosmo.Omega_m, cosmo.Omega_b, cosmo.h, cosmo.n_s, cosmo.sigma8

    def shape(k):
        return np.asarray(k, dtype=np.float64) ** ns * eh_nowiggle_T(k, Om, Ob, h) ** 2

    amp = (s8 / sigma_R(shape, 8.0)) ** 2

    def pk(k):
        return amp * shape(k)
    return pk
