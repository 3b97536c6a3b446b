"""Pins of the oracle's background, model, power-spectrum and Philox functions.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code path.
"""
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import background as bg
from oracle import models as M
from oracle import philox, power

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ background
def test_dtau_eds_closed_form():
    # Omega_m = 1: E = a^-3/2, int da/(a^3 E) = int a^-3/2 da = 2 (a1^-1/2 - a2^-1/2).
    for a1, a2 in [(0.05, 1.0), (0.1, 0.2), (0.5, 0.51)]:
        assert bg.dtau(a1, a2, 1.0) == pytest.approx(2 * (a1**-0.5 - a2**-0.5), rel=1e-12)


def test_dlnE_da_finite_difference():
    a, h = 0.37, 1e-6
    fd = (np.log(bg.E(a + h, 0.3)) - np.log(bg.E(a - h, 0.3))) / (2 * h)
    assert bg.dlnE_da(a, 0.3) == pytest.approx(fd, rel=1e-8)


def test_a_nodes_uniform():
    a = bg.a_nodes(0.05, 1.0, 10)
    assert a[0] == 0.05 and a[-1] == 1.0
    assert np.allclose(np.diff(a), 0.095)


# ------------------------------------------------------------------ models
def test_fr_mu_limits():
    Om, fR0 = 0.3, 1e-5
    for a in (0.1, 0.5, 1.0):
        am = a * np.sqrt(M.fr_m2(a, Om, fR0))
        assert M.fr_mu(1e-9, a, Om, fR0) == pytest.approx(1.0, abs=1e-12)
        assert M.fr_mu(1e9, a, Om, fR0) == pytest.approx(4.0 / 3.0, abs=1e-12)
        assert M.fr_mu(am, a, Om, fR0) == pytest.approx(7.0 / 6.0, rel=1e-14)


def test_fr_is_the_m_beta_model_with_beta_1_over_sqrt6():
    """Sec. 5.1 f(R) mu and gamma_2^E equal the App. C {m, beta} forms with beta = 1/sqrt(6)."""
    Om, fR0 = 0.3, 1e-5
    beta = 1.0 / np.sqrt(6.0)
    k = np.logspace(-3, 1, 9)
    for a in (0.1, 0.4, 1.0):
        m2 = M.fr_m2(a, Om, fR0)
        assert np.allclose(M.fr_mu(k, a, Om, fR0), M.mb_mu(k, a, m2, beta), rtol=1e-14)
        g_fr = M.fr_gamma2E(k, 0.7 * k, 0.4 * k, a, Om, fR0)
        g_mb = M.mb_gamma2E(k, 0.7 * k, 0.4 * k, a, Om, lambda x: M.fr_m2(x, Om, fR0),
                            lambda x: beta, da=1e-5 * a)
        assert np.allclose(g_fr, g_mb, rtol=1e-8)
        assert np.all(g_fr < 0)


def test_phi_crit_integral_matches_closed_form():
    """App. C: the Phi_crit quadrature reproduces 3|f_R(a)|/2 with the ratio of Sec. 5.1."""
    Om, fR0 = 0.3, 1e-5
    beta = lambda x: 1.0 / np.sqrt(6.0)  # noqa: E731
    m2 = lambda x: M.fr_m2(x, Om, fR0)  # noqa: E731
    a_i = 1e-3
    for a in (0.05, 0.3, 1.0):
        val = M.mb_phi_crit(a, a_i, M.phi_crit_fr(a_i, Om, fR0), Om, m2, beta)
        assert val == pytest.approx(M.phi_crit_fr(a, Om, fR0), rel=1e-10)
    # today: 3 |f_R0| / 2
    assert M.phi_crit_fr(1.0, Om, fR0) == pytest.approx(1.5e-5, rel=1e-14)


def test_symmetron_phi_crit_integral_closed_form():
    """App. C symmetron: with u = 1 - (a_*/a)^3 the integrand is beta_* H0^2/(m_*^2 a^4 sqrt(u)), so the
    integral is 2 sqrt(u)/(3 a_*^3) beta_* H0^2/m_*^2 and Phi_crit = 3 Omega_m H0^2/(a_*^3 m_*^2) for
    every a > a_*: twice the value printed for the symmetron (the reading taken here, since the same
    integral reproduces Sec. 6.1's 3 |f_R(a)|/2 for f(R))."""
    from workloads import SYMM_A
    Om = 0.3
    want = 3.0 * Om / (SYMM_A.a_star**3 * SYMM_A.m_star**2)
    for a in (0.5001, 0.55, 0.8, 1.0):
        assert M.phi_crit(SYMM_A, a, Om) == pytest.approx(want, rel=1e-9)
    assert M.phi_crit(SYMM_A, 0.4, Om) == 0.0
    printed = 3.0 * Om / (2.0 * SYMM_A.a_star**3) / SYMM_A.m_star**2
    assert want == pytest.approx(2.0 * printed, rel=1e-15)


def test_symmetron_mu_and_gamma2():
    """mu = 1 + 2 beta^2 k^2/(k^2 + a^2 m^2): 1 at k -> 0 and before a_*, 1 + 2 beta(a)^2 at k -> inf,
    1 + beta^2 at k = a m; gamma_2^E with dm^2/da = 3 m_*^2 a_*^3 / a^4 > 0 is positive and
    vanishes before a_*."""
    from workloads import SYMM_A
    Om = 0.3
    a = 0.8
    b2 = SYMM_A.beta_star**2 * (1 - (SYMM_A.a_star / a) ** 3)
    m = SYMM_A.m_star * M.H0_OVER_C * np.sqrt(1 - (SYMM_A.a_star / a) ** 3)
    mu = M.mu(SYMM_A, np.array([1e-9, a * m, 1e9]), a, Om)
    assert mu[0] == pytest.approx(1.0, abs=1e-12)
    assert mu[1] == pytest.approx(1.0 + b2, rel=1e-14)
    assert mu[2] == pytest.approx(1.0 + 2 * b2, rel=1e-12)
    assert np.all(M.mu(SYMM_A, np.logspace(-3, 2, 7), 0.45, Om) == 1.0)
    k = np.logspace(-2, 1, 5)
    g = M.gamma2_orth(SYMM_A, k, a, Om)
    assert np.all(g > 0)
    # the same expression with the analytic derivative of m^2
    h0 = M.H0_OVER_C
    m2 = m * m
    dm2 = 3 * (SYMM_A.m_star * h0) ** 2 * SYMM_A.a_star**3 / a**4
    H = h0 * bg.E(a, Om)
    Pi = lambda q: (q / (a * h0)) ** 2 + m2 / h0**2  # noqa: E731
    ref = m2 * dm2 * b2 * Om * k**2 / (2 * h0**4 * Pi(k) * Pi(k / np.sqrt(2)) ** 2 * a**4 * H**2)
    assert np.allclose(g, ref, rtol=1e-7)
    assert np.all(M.gamma2_orth(SYMM_A, k, 0.45, Om) == 0.0)


def test_tabulated_mb_constant_model_closed_form():
    """App. C with constant beta and m: Phi_crit = Phi_0 + 3 Omega_m (a_0^-3 - a^-3) / (2 (m/H0)^2),
    mu = 1 + 2 beta^2 k^2/(k^2 + a^2 m^2), and gamma_2^E = 0 (dm^2/da = 0)."""
    from workloads import MB, Model
    Om, b, mh = 0.3, 0.5, 1000.0
    m = Model(kind=MB, mb_a=(0.01, 0.5, 1.2), mb_beta=(b, b, b), mb_m=(mh, mh, mh), mb_phicrit0=2e-7)
    for a in (0.02, 0.5, 0.77, 1.0):
        want = 2e-7 + 3.0 * Om * (0.01**-3 - a**-3) / (2.0 * mh**2)
        assert M.phi_crit(m, a, Om) == pytest.approx(want, rel=1e-10)
        k = np.array([1e-3, 0.3, 30.0])
        am = a * mh * M.H0_OVER_C
        assert np.allclose(M.mu(m, k, a, Om), 1 + 2 * b * b * k**2 / (k**2 + am**2), rtol=1e-14)
        assert np.all(M.gamma2_orth(m, k, a, Om) == 0.0)


def test_tabulated_mb_reproduces_fR():
    """f(R) F5 sampled at 2000 geometric nodes in a as {beta = 1/sqrt6, m(a)}: mu, gamma_2 and Phi_crit
    agree with the Sec. 5.1 / Sec. 6.1 closed forms to the accuracy of linear interpolation (m^2
    goes as a^-9 early on; gamma_2 takes the secant slope of m^2)."""
    from workloads import MB, Model
    Om, fR0 = 0.3, 1e-5
    ta = np.geomspace(0.02, 1.0, 2000)
    m = Model(kind=MB, mb_a=tuple(ta), mb_beta=tuple(np.full_like(ta, 1 / np.sqrt(6.0))),
              mb_m=tuple(np.sqrt(M.fr_m2(ta, Om, fR0)) / M.H0_OVER_C),
              mb_phicrit0=float(M.phi_crit_fr(0.02, Om, fR0)))
    k = np.logspace(-2, 1, 7)
    for a in (0.1031, 0.4, 0.9):
        assert np.allclose(M.mu(m, k, a, Om), M.fr_mu(k, a, Om, fR0), rtol=1e-5)
        q = k / np.sqrt(2)
        assert np.allclose(M.gamma2_orth(m, k, a, Om), M.fr_gamma2E(k, q, q, a, Om, fR0), rtol=1e-2)
        assert M.phi_crit(m, a, Om) == pytest.approx(float(M.phi_crit_fr(a, Om, fR0)), rel=2e-4)


def test_ndgp_beta_today():
    # beta(1) = 1 + 2 rcH0 (1 - Omega_m/2)  (E(1) = 1, dlnE/da(1) = -3 Om/2)
    assert M.dgp_beta(1.0, 0.3, 1.0) == pytest.approx(2.7, rel=1e-14)
    assert M.dgp_mu(1.0, 0.3, 1.0) == pytest.approx(1 + 1 / 8.1, rel=1e-14)
    # r_c -> infinity: mu -> 1
    assert M.dgp_mu(0.5, 0.3, 1e12) == pytest.approx(1.0, abs=1e-11)


def test_vainshtein_factor_is_root_of_spherical_equation():
    """Spherical reduction of the nDGP field equation: eps + (x/4) eps^2 = 1, eps(0) = 1."""
    x = np.array([0.0, 1e-8, 1e-3, 0.3, 1.0, 7.0, 1e3, 1e8])
    e = M.eps_vainshtein(x)
    assert np.allclose(e + 0.25 * x * e * e, 1.0, rtol=1e-13)
    assert e[0] == 1.0 and np.all(np.diff(e) < 0)
    assert e[-1] == pytest.approx(2 / np.sqrt(1e8), rel=1e-3)


def test_ndgp_gamma2_consistent_with_vainshtein_coefficient():
    """gamma_2^E (Sec. 5.2) and the x coefficient (Sec. 6.2) come from one field equation.

    For lap phi + c[(lap phi)^2 - (phi_ij)^2] = kappa delta/(3 beta): second order gives
    a^4 H^2 gamma_2^E = -c (kappa/(3 beta))^2 (1 - cos^2), the sphere gives x = 8 c kappa delta/(9 beta).
    Eliminating c: x/delta = -8 beta a^4 H^2 gamma_2^E / kappa.  The paper's x coefficient
    equals this times a^3 (the literal rho/rho_bar reading carries no a^-3).
    """
    Om, rc = 0.3, 1.0
    for a in (0.2, 0.6, 1.0):
        b = M.dgp_beta(a, Om, rc)
        g2 = M.dgp_gamma2E(a, Om, rc, 0.0)
        kap = bg.kappa(a, Om)
        x_per_delta = -8 * b * a**4 * bg.E(a, Om) ** 2 * g2 / kap
        assert M.vainshtein_x(1.0, a, Om, rc) == pytest.approx(x_per_delta * a**3, rel=1e-13)


def test_chameleon_factor():
    e = M.eps_chameleon(np.array([0.0, 1e-7, -2e-5, 1e-5, 4e-5]), 1e-5)
    assert np.allclose(e, [1.0, 1.0, 0.5, 1.0, 0.25])


# ------------------------------------------------------------------ power
def test_eh_transfer_large_scale_limit():
    assert power.eh_nowiggle_T(1e-7, 0.3, 0.05, 0.7) == pytest.approx(1.0, abs=1e-5)
    k = np.logspace(-3, 1, 50)
    T = power.eh_nowiggle_T(k, 0.3, 0.05, 0.7)
    assert np.all(np.diff(T) < 0)


def test_sigma8_normalisation_independent_quadrature():
    from workloads import Cosmo
    c = Cosmo()
    pk = power.linear_pk_z0(c)
    lnk = np.linspace(np.log(1e-5), np.log(1e3), 400001)
    k = np.exp(lnk)
    x = 8.0 * k
    W = 3 * (np.sin(x) - x * np.cos(x)) / x**3
    s2 = integrate.simpson(k**3 * pk(k) * W**2 / (2 * np.pi**2), x=lnk)
    assert np.sqrt(s2) == pytest.approx(0.8, rel=1e-6)


# ------------------------------------------------------------------ philox
def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox.philox4x32_10(*[np.uint64(x) for x in v[:6]])
        assert [int(o) for o in out] == v[6:]


def test_white_noise_moments():
    g = philox.white_noise(32, 7).ravel()
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs((g**4).mean() - 3) < 0.1
    assert not np.allclose(philox.white_noise(8, 1), philox.white_noise(8, 2))
