"""Modified-gravity model functions (test infrastructure only).

Follows the paper:

* f(R) Hu-Sawicky n=1 (Sec. 5.1): mu(k,a) = 1 + (1/3) k^2/(k^2 + a^2 m^2(a)),
  m^2(a) from Eq. mofahus, background field f_R(a), gamma_2^E with Pi(k,a).
* nDGP (Sec. 5.2): mu(a) = 1 + 1/(3 beta(a)),
  beta(a) = 1 + 2 r_c H (1 + Hdot/(3 H^2)), gamma_2^E proportional to (1 - cos^2 theta).
* gamma_2 = gamma_2^E + (3/2) Omega_m(a) [mu(k) - mu(k1)] (k1.k2)/k2^2 (Sec. 4),
  evaluated at the orthogonal configuration k1 = k2 = k/sqrt(2) used by the
  approximate second-order growth (Eq. fofrapprox); the second term vanishes there.
* General {m(a), beta(a)} chameleon (App. C): mu, gamma_2^E and Phi_crit, used
  here to pin the f(R) special case, and the symmetron model of App. C:
  beta = beta_* sqrt(u), m^2 = m_*^2 u, u = 1 - (a_*/a)^3, both 0 before a_*.
* Screening factors (Sec. 6): chameleon eps = min(1, |3 f_R(a) / (2 Phi_N)|);
  Vainshtein eps = 2 (sqrt(1+x) - 1)/x with x = 8 (r_c H0)^2 Omega_m (rho/rho_bar) / (9 beta^2).

Readings of the paper taken here, where it is silent, garbled or inconsistent:
* The printed Vainshtein factor 2 sqrt(1+x)/x diverges as x -> 0; the factor
  used is 2 (sqrt(1+x) - 1)/x, the positive root of the spherical solution of
  the nDGP field equation (eps -> 1 as x -> 0).
* x takes rho/rho_bar = 1 + delta_R of the smoothed density literally (clamped
  at 0), without an a^-3 factor.
* Phi_N in the chameleon factor is the metric potential: the code potential
  (a^2 times it, in (Mpc/h)^2 H0^2) divided by a^2 c^2.
* (k/(aH))^2 in the f(R) gamma_2^E uses H = H(a).
* A general {m(a), beta(a)} model is given by tables of beta and m/H0 at ascending
  scale factors; beta and m^2 are linear in a between nodes, dm^2/da is the
  slope of the segment, and Phi_crit(a) is the App. C integral from the first
  node plus the given Phi_crit there.
* Symmetron Phi_crit is the App. C integral from a_* with Phi_crit(a_*) = 0; it
  equals 3 Omega_m H0^2/(a_*^3 m_*^2), twice the printed closed form (the same
  integral gives Sec. 6.1's 3 |f_R(a)|/2 for f(R), so the integral is taken).

Units: k in h/Mpc; m^2 in (h/Mpc)^2, using H0/c = 1/C_LIGHT h/Mpc.

Pins (tests/test_oracle_basics.py): mu limits k->0, k->inf and k = a m;
f(R) mu and gamma_2^E against the App. C {m, beta} forms with beta = 1/sqrt(6);
Phi_crit quadrature against the closed form, for f(R) and the symmetron; symmetron
mu limits and gamma_2^E with the analytic dm^2/da; a tabulated model with constant
beta and m against the closed-form integral, and one sampled from f(R) against
Sec. 5.1 and Sec. 6.1; nDGP beta(1) closed form; the
Vainshtein factor against a numerical solution of the spherical field equation;
nDGP gamma_2 coefficient against the Vainshtein coefficient through the same
spherical reduction.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate

from .background import C_LIGHT, E, dlnE_da

LCDM, FOFR, NDGP, SYMM, MB = 0, 1, 2, 3, 4
H0_OVER_C = 1.0 / C_LIGHT   # h/Mpc


# ---------------------------------------------------------------- f(R), Sec. 5.1
def fr_X(a, Om):
    """(Omega_m a^-3 + 4 Omega_L) / (Omega_m + 4 Omega_L)."""
    OL = 1.0 - Om
    return (Om * np.asarray(a, dtype=np.float64) ** -3 + 4.0 * OL) / (Om + 4.0 * OL)


def fr_m2(a, Om, fR0):
    """m^2(a) of Eq. mofahus in (h/Mpc)^2."""
    OL = 1.0 - Om
    return H0_OVER_C**2 * (Om + 4.0 * OL) / (2.0 * fR0) * fr_X(a, Om) ** 3


def fr_fR(a, Om, fR0):
    """|f_R(a)| = |f_R0| ((Om + 4 OL)/(Om a^-3 + 4 OL))^2."""
    return fR0 / fr_X(a, Om) ** 2


def fr_mu(k, a, Om, fR0):
    k2 = np.asarray(k, dtype=np.float64) ** 2
    return 1.0 + k2 / (3.0 * (k2 + a * a * fr_m2(a, Om, fR0)))


def fr_Pi(k, a, Om, fR0):
    """Pi(k,a) = (k/(a H0))^2 + (Om a^-3 + 4 OL)^3 / (2 |f_R0| (Om + 4 OL)^2)."""
    OL = 1.0 - Om
    kk = np.asarray(k, dtype=np.float64) / H0_OVER_C
    return (kk / a) ** 2 + (Om * a**-3 + 4.0 * OL) ** 3 / (2.0 * fR0 * (Om + 4.0 * OL) ** 2)


def fr_gamma2E(k, k1, k2, a, Om, fR0):
    """gamma_2^E of Sec. 5.1 (dimensionless), H = H(a)."""
    OL = 1.0 - Om
    H = H0_OVER_C * E(a, Om)
    kk = np.asarray(k, dtype=np.float64)
    pref = -9.0 * Om**2 / (48.0 * a**6 * fR0**2) * (kk / (a * H)) ** 2
    pref = pref * (Om * a**-3 + 4.0 * OL) ** 5 / (Om + 4.0 * OL) ** 4
    return pref / (fr_Pi(k, a, Om, fR0) * fr_Pi(k1, a, Om, fR0) * fr_Pi(k2, a, Om, fR0))


# ---------------------------------------------------------------- nDGP, Sec. 5.2
def dgp_beta(a, Om, rcH0):
    """beta(a) = 1 + 2 r_c H (1 + Hdot/(3H^2)); Hdot/H^2 = a dlnE/da."""
    a = np.asarray(a, dtype=np.float64)
    return 1.0 + 2.0 * rcH0 * E(a, Om) * (1.0 + a * dlnE_da(a, Om) / 3.0)


def dgp_mu(a, Om, rcH0):
    return 1.0 + 1.0 / (3.0 * dgp_beta(a, Om, rcH0))


def dgp_gamma2E(a, Om, rcH0, cos2=0.0):
    """gamma_2^E = -(H0/H)^2 (r_c H0)^2 Omega_m^2 / (6 beta^3 a^6) (1 - cos^2 theta)."""
    b = dgp_beta(a, Om, rcH0)
    return -(1.0 / E(a, Om) ** 2) * rcH0**2 * Om**2 / (6.0 * b**3 * a**6) * (1.0 - cos2)


# ---------------------------------------------------------------- model dispatch
def mu(model, k, a, Om):
    """mu(k,a) for a workloads.Model-like record (kind, fR0, rcH0, beta_star, m_star, a_star)."""
    k = np.asarray(k, dtype=np.float64)
    if model.kind == FOFR:
        return fr_mu(k, a, Om, model.fR0)
    if model.kind == NDGP:
        return np.full_like(k, dgp_mu(a, Om, model.rcH0))
    if model.kind == SYMM:
        m2_fn, beta_fn = symm_fns(model)
        return mb_mu(k, a, m2_fn(a), beta_fn(a))
    if model.kind == MB:
        b, m2, _ = table_mb(model, a)
        return mb_mu(k, a, m2, b)
    return np.ones_like(k)


def gamma2_orth(model, k, a, Om):
    """gamma_2(k, k/sqrt2, k/sqrt2, a): the value used in Eq. fofrapprox.

    At k1 = k2 = k/sqrt(2) with k = k1 + k2, k1.k2 = 0, so the Lagrangian
    correction term of gamma_2 (Sec. 4) vanishes and cos^2 theta = 0.
    """
    k = np.asarray(k, dtype=np.float64)
    if model.kind == FOFR:
        q = k / np.sqrt(2.0)
        return fr_gamma2E(k, q, q, a, Om, model.fR0)
    if model.kind == NDGP:
        return np.full_like(k, dgp_gamma2E(a, Om, model.rcH0, 0.0))
    if model.kind == SYMM:
        q = k / np.sqrt(2.0)
        m2_fn, beta_fn = symm_fns(model)
        return mb_gamma2E(k, q, q, a, Om, m2_fn, beta_fn)
    if model.kind == MB:
        b, m2, dm2 = table_mb(model, a)
        h0 = H0_OVER_C
        H = h0 * E(a, Om)
        Pk = (k / (a * h0)) ** 2 + m2 / h0**2
        Pq = 0.5 * (k / (a * h0)) ** 2 + m2 / h0**2
        return m2 * dm2 * b**2 * Om * k**2 / (2.0 * h0**4 * Pk * Pq * Pq * a**4 * H**2)
    return np.zeros_like(k)


# ---------------------------------------------------------------- screening, Sec. 6
def phi_crit_fr(a, Om, fR0):
    """Critical potential of the chameleon factor: 3 |f_R(a)| / 2 (Sec. 6.1)."""
    return 1.5 * fr_fR(a, Om, fR0)


def eps_chameleon(PhiN_metric, phicrit):
    """eps = min(1, |Phi_crit / Phi_N|), with eps = 1 where Phi_N = 0."""
    P = np.abs(np.asarray(PhiN_metric, dtype=np.float64))
    out = np.ones_like(P)
    m = P > phicrit
    out[m] = phicrit / P[m]
    return out


def vainshtein_x(one_plus_delta, a, Om, rcH0):
    """x = 8 (r_c H0)^2 Omega_m / (9 beta^2) * rho/rho_bar, rho/rho_bar clamped >= 0."""
    b = dgp_beta(a, Om, rcH0)
    r = np.maximum(np.asarray(one_plus_delta, dtype=np.float64), 0.0)
    return 8.0 * rcH0**2 * Om / (9.0 * b * b) * r


def eps_vainshtein(x):
    """eps = 2 (sqrt(1+x) - 1)/x, eps(0) = 1 (written as 2/(sqrt(1+x)+1) to avoid 0/0)."""
    x = np.asarray(x, dtype=np.float64)
    return 2.0 / (np.sqrt(1.0 + x) + 1.0)


# ---------------------------------------------------------------- App. C {m, beta}
def mb_mu(k, a, m2, beta):
    """mu = 1 + 2 beta^2 k^2/(k^2 + a^2 m^2) (App. C)."""
    k2 = np.asarray(k, dtype=np.float64) ** 2
    return 1.0 + 2.0 * beta**2 * k2 / (k2 + a * a * m2)


def mb_gamma2E(k, k1, k2, a, Om, m2_fn, beta_fn, da=1e-6):
    """gamma_2^E = m^2 (dm^2/da) beta^2 Omega_m k^2 / (2 H0^4 Pi Pi Pi a^4 H^2) (App. C).

    Pi(k) = (k/(a H0))^2 + m^2/H0^2.  m2_fn returns m^2 in (h/Mpc)^2; dm^2/da by
    a centred difference.
    """
    m2 = m2_fn(a)
    dm2 = (m2_fn(a + da) - m2_fn(a - da)) / (2 * da)
    h0 = H0_OVER_C
    H = h0 * E(a, Om)

    def Pi(q):
        return (np.asarray(q, dtype=np.float64) / (a * h0)) ** 2 + m2 / h0**2

    kk = np.asarray(k, dtype=np.float64)
    return (m2 * dm2 * beta_fn(a) ** 2 * Om * kk**2
            / (2.0 * h0**4 * Pi(k) * Pi(k1) * Pi(k2) * a**4 * H**2))


def mb_phi_crit(a, a_ini, phicrit_ini, Om, m2_fn, beta_fn):
    """Phi_crit(a) = Phi_crit(a_ini) + 9 Om/(2 beta(a)) int_{a_ini}^a beta/(m^2/H0^2 a^4) da' (App. C)."""
    h0 = H0_OVER_C
    val, _ = integrate.quad(lambda x: beta_fn(x) / (m2_fn(x) / h0**2 * x**4), a_ini, a,
                            epsabs=0.0, epsrel=1e-13, limit=400)
    return phicrit_ini + 9.0 * Om / (2.0 * beta_fn(a)) * val


# ---------------------------------------------------------------- symmetron (App. C)
def symm_u(a, a_star):
    """1 - (a_*/a)^3, and 0 before a_* (no fifth force there)."""
    a = np.asarray(a, dtype=np.float64)
    return np.where(a > a_star, 1.0 - (a_star / a) ** 3, 0.0)


def symm_beta(a, beta_star, a_star):
    """beta(a) = beta_* sqrt(1 - (a_*/a)^3)."""
    return beta_star * np.sqrt(symm_u(a, a_star))


def symm_m2(a, m_star, a_star):
    """m^2(a) = m_*^2 (1 - (a_*/a)^3) in (h/Mpc)^2; m_star is m_*/H0."""
    return (m_star * H0_OVER_C) ** 2 * symm_u(a, a_star)


def symm_fns(model):
    """(m^2(a), beta(a)) of a symmetron record (beta_star, m_star = m_*/H0, a_star)."""
    return (lambda a: symm_m2(a, model.m_star, model.a_star),
            lambda a: symm_beta(a, model.beta_star, model.a_star))


def phi_crit(model, a, Om):
    """Critical metric potential of the chameleon-type factor at a.

    f(R): 3 |f_R(a)| / 2 (Sec. 6.1).  Symmetron: the App. C integral from a_* (where
    Phi_crit starts at 0), by quadrature after a' = a_* + t^2; 0 before a_*.
    """
    if model.kind == FOFR:
        return float(phi_crit_fr(a, Om, model.fR0))
    if model.kind == SYMM:
        if a <= model.a_star:
            return 0.0
        # integrand beta/(m^2/H0^2 a'^4) = beta_* /(m_*^2/H0^2 sqrt(u) a'^4), u = 1 - (a_*/a')^3, which
        # goes as (a' - a_*)^(-1/2); with a' = a_* + t^2, u = t^2 (a'^2 + a' a_* + a_*^2)/a'^3 and
        # 2 t dt / sqrt(u) is smooth
        s = model.a_star

        def f(t):
            x = s + t * t
            return 2.0 * model.beta_star / (model.m_star**2 * x**4 * np.sqrt((x * x + x * s + s * s) / x**3))

        val, _ = integrate.quad(f, 0.0, np.sqrt(a - s), epsabs=0.0, epsrel=1e-13, limit=400)
        return float(9.0 * Om / (2.0 * symm_beta(a, model.beta_star, s)) * val)
    if model.kind == MB:
        # adaptive quadrature segment by segment (beta and m^2 are linear on each)
        ta = np.asarray(model.mb_a, dtype=np.float64)
        tb = np.asarray(model.mb_beta, dtype=np.float64)
        tM2 = np.asarray(model.mb_m, dtype=np.float64) ** 2          # m^2 / H0^2
        val = 0.0
        for i in range(len(ta) - 1):
            lo, hi = ta[i], min(ta[i + 1], a) if i < len(ta) - 2 else a
            if hi <= lo:
                break
            w = ta[i + 1] - ta[i]

            def f(x, i=i, w=w):
                t = (x - ta[i]) / w
                return (tb[i] + t * (tb[i + 1] - tb[i])) / ((tM2[i] + t * (tM2[i + 1] - tM2[i])) * x**4)

            val += integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1e-13)[0]
        return float(model.mb_phicrit0 + 9.0 * Om / (2.0 * table_mb(model, a)[0]) * val)
    raise ValueError("no chameleon-type screening for this model")


# ---------------------------------------------------------------- tabulated {m(a), beta(a)} (App. C)
def table_mb(model, a):
    """(beta, m^2 [(h/Mpc)^2], dm^2/da) of a tabulated {m, beta} record at a: beta and m^2 linear
    in a between the nodes mb_a (m^2 from the node values of m/H0), dm^2/da the slope of the
    segment [a_i, a_i+1) holding a (the last segment at and beyond the last node)."""
    ta = np.asarray(model.mb_a, dtype=np.float64)
    tb = np.asarray(model.mb_beta, dtype=np.float64)
    tm2 = (np.asarray(model.mb_m, dtype=np.float64) * H0_OVER_C) ** 2
    i = int(np.clip(np.searchsorted(ta, a, side="right") - 1, 0, len(ta) - 2))
    t = (a - ta[i]) / (ta[i + 1] - ta[i])
    slope = (tm2[i + 1] - tm2[i]) / (ta[i + 1] - ta[i])
    return (float(tb[i] + t * (tb[i + 1] - tb[i])), float(tm2[i] + t * (tm2[i + 1] - tm2[i])), float(slope))
