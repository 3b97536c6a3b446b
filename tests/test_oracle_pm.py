"""Pins of the oracle's ICs (Sec. 3.2), PM force (Sec. 2, App. B) and P(k) estimator."""
import dataclasses

import numpy as np
import pytest

from oracle import ics, pm
from oracle import models as M
from oracle.background import kappa
from workloads import FOFR, LCDM, NDGP, Cosmo, Model, random_positions


# ------------------------------------------------------------------ DFT conventions
def test_rfft_convention_against_direct_sum():
    N, L = 8, 8.0
    rng = np.random.default_rng(3)
    x = rng.standard_normal((N, N, N))
    X = ics.rfft3(x)
    n = np.arange(N)
    kz, ky, kx = (2, 5, 3)
    ph = np.exp(-2j * np.pi * (kz * n[:, None, None] + ky * n[None, :, None]
                               + kx * n[None, None, :]) / N)
    assert X[kz, ky, kx] == pytest.approx((x * ph).sum(), rel=1e-12)
    # inverse: e^{+ikx} synthesis with 1/N^3, gradient <-> i k
    f = np.cos(2 * np.pi * 3 * n / N)[None, None, :] * np.ones((N, N, 1))
    gx, gy, gz = ics.grad_factor(N, L)
    d = ics.irfft3(gx * ics.rfft3(f), N)
    assert np.allclose(d, -(2 * np.pi * 3 / L) * np.sin(2 * np.pi * 3 * n / N)[None, None, :],
                       atol=1e-12)


def test_rfft_every_mode_against_direct_sum_on_8_cubed():
    """The whole half spectrum of the forward transform against the defining sum
    X[kz, ky, kx] = sum_n x[n] exp(-2 pi i k.n / N), and the inverse against the synthesis
    x[n] = N^-3 sum over all k of X[k] exp(+2 pi i k.n / N), the missing half from X(-k) = X(k)*."""
    N = 8
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, N, N))
    n = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(n, n) / N)               # E[k, n]
    full = np.einsum("az,by,cx,zyx->abc", E, E, E, x)          # all N^3 modes by the direct sum
    X = ics.rfft3(x)
    assert X.shape == (N, N, N // 2 + 1)
    assert np.allclose(X, full[:, :, : N // 2 + 1], rtol=0, atol=1e-12 * np.abs(full).max())
    neg = (-n) % N
    rebuilt = np.empty_like(full)
    rebuilt[:, :, : N // 2 + 1] = X
    for kx in range(N // 2 + 1, N):
        rebuilt[:, :, kx] = np.conj(X[np.ix_(neg, neg, [(-kx) % N])][:, :, 0])
    y = np.einsum("az,by,cx,abc->zyx", E.conj(), E.conj(), E.conj(), rebuilt).real / N**3
    assert np.allclose(ics.irfft3(X, N), y, rtol=0, atol=1e-12)
    assert np.allclose(y, x, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ 2LPT source
def _phi1_from_real(phi_real):
    return ics.rfft3(phi_real)


def test_2lpt_single_mode_has_no_source():
    N, L = 16, 32.0
    n = np.arange(N)
    k = 2 * np.pi * 2 / L
    phi = 0.3 * np.cos(k * n * L / N)[None, None, :] * np.ones((N, N, 1))
    _, phi2 = ics.potentials_from_delta(ics.k2_grid(N, L) * _phi1_from_real(phi), N, L)
    assert np.max(np.abs(phi2)) < 1e-13


def test_2lpt_two_perpendicular_modes():
    # phi1 = A cos(k1 x) + B cos(k2 y):  lap phi2 = phi_xx phi_yy = A B k1^2 k2^2 cos cos,
    # so phi2 = -A B k1^2 k2^2 cos(k1 x) cos(k2 y) / (k1^2 + k2^2).
    N, L = 16, 32.0
    q = np.arange(N) * L / N
    A, B = 0.7, -0.4
    k1, k2 = 2 * np.pi * 1 / L, 2 * np.pi * 3 / L
    phi = (A * np.cos(k1 * q)[None, None, :] + B * np.cos(k2 * q)[None, :, None]) * np.ones((N, 1, 1))
    dk = ics.k2_grid(N, L) * _phi1_from_real(phi)   # delta = -lap phi1
    phi1, phi2 = ics.potentials_from_delta(dk, N, L)
    assert np.allclose(ics.irfft3(phi1, N), phi - phi.mean(), atol=1e-13)
    expect = -A * B * k1**2 * k2**2 * np.cos(k1 * q)[None, None, :] * np.cos(k2 * q)[None, :, None] \
        / (k1**2 + k2**2) * np.ones((N, 1, 1))
    assert np.allclose(ics.irfft3(phi2, N), expect, atol=1e-13)


def test_ic_power_within_cosmic_variance_and_divergence():
    from oracle.growth import lcdm_D1
    from oracle.power import linear_pk_z0
    c = Cosmo()
    N, L, a_ini = 64, 256.0, 0.05
    dk = ics.delta_k(c, N, L, 11, a_ini)
    k, P, nm = pm.power_spectrum_mesh(ics.irfft3(dk, N), N, L)
    kx, ky, kz, *_ = ics.kgrid(N, L)
    kf = 2 * np.pi / L
    nx, ny, nz = kx / kf, ky / kf, kz / kf
    sinc = lambda x: np.sinc(x / np.pi)  # noqa: E731
    W2 = (sinc(np.pi * nx / N) * sinc(np.pi * ny / N) * sinc(np.pi * nz / N)) ** 4
    # the estimator deconvolves CIC; undo that for a field made directly on the mesh
    wt = np.where((nx == 0) | (nx == N // 2), 1.0, 2.0) * np.ones_like(nz * ny * nx)
    nmag = np.sqrt(nx**2 + ny**2 + nz**2)
    b = np.floor(nmag - 0.5).astype(int)
    ok = (nmag >= 0.5) & (b < N // 2)
    Dr = 1.0 / lcdm_D1(c.Omega_m, a_ini, [1.0])[0]
    Pth = linear_pk_z0(c)(np.maximum(nmag * kf, 1e-9)) * Dr**2
    Pth_bin = np.bincount(b[ok], weights=(wt * Pth * W2 ** -1)[ok], minlength=N // 2) / nm
    sel = (nm > 200)
    r = P[sel] / Pth_bin[sel]
    sig = np.sqrt(2.0 / nm[sel])
    assert np.all(np.abs(r - 1) < 5 * sig)
    # div Psi1 = -delta (checked in k-space off the Nyquist planes, where i k_i is zeroed)
    phi1, _ = ics.potentials_from_delta(dk, N, L)
    gx, gy, gz = ics.grad_factor(N, L)
    div_k = (gx * gx + gy * gy + gz * gz) * phi1
    _, _, _, nyx, nyy, nyz = ics.kgrid(N, L)
    off = ~(nyx | nyy | nyz) & np.ones(dk.shape, bool)
    assert np.allclose(div_k[off], -dk[off], rtol=1e-12, atol=1e-12 * np.abs(dk).max())


# ------------------------------------------------------------------ CIC
def test_cic_weights_and_wrap():
    N, L = 4, 8.0            # cell = 2
    pos = np.array([[2.0, 4.0, 6.0],           # exactly on a mesh point
                    [0.5, 2.0, 7.0]])          # fx = 0.25, fy = 0, z wraps (fz = 0.5)
    rho = pm.cic_deposit(pos, N, L)
    assert rho.sum() == pytest.approx(2.0, rel=1e-15)
    assert rho[3, 2, 1] == pytest.approx(1.0)
    assert rho[3, 1, 0] == pytest.approx(0.75 * 0.5)
    assert rho[3, 1, 1] == pytest.approx(0.25 * 0.5)
    assert rho[0, 1, 0] == pytest.approx(0.75 * 0.5)
    assert rho[0, 1, 1] == pytest.approx(0.25 * 0.5)


def test_cic_gather_is_transpose_of_deposit():
    N, L = 8, 10.0
    rng = np.random.default_rng(0)
    pos = random_positions(50, L, 1)
    w = rng.standard_normal(50)
    F = rng.standard_normal((N, N, N))
    lhs = np.dot(pm.cic_gather(F, pos, N, L), w)
    rhs = 0.0
    for p in range(50):
        rhs += w[p] * (pm.cic_deposit(pos[p:p + 1], N, L) * F).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ------------------------------------------------------------------ Poisson / force
def _mode_density(N, L, nvec, A):
    q = np.arange(N) * L / N
    kv = 2 * np.pi * np.array(nvec) / L
    ph = kv[0] * q[None, None, :] + kv[1] * q[None, :, None] + kv[2] * q[:, None, None]
    return 1.0 + A * np.cos(ph), np.sin(ph), kv


@pytest.mark.parametrize("model_kind", [LCDM, FOFR, NDGP])
def test_single_mode_force(model_kind):
    N, L, a, Om = 16, 64.0, 0.5, 0.3
    model = {LCDM: Model(), FOFR: Model(kind=FOFR, fR0=1e-5),
             NDGP: Model(kind=NDGP, rcH0=1.0)}[model_kind]
    rho, s, kv = _mode_density(N, L, (1, 2, 3), 1e-2)
    F = pm.force_mesh(rho, 1.0, N, L, a, Om, model)
    k2 = kv @ kv
    mu = float(M.mu(model, np.sqrt(k2), a, Om))
    for i in range(3):
        assert np.allclose(F[i], -mu * kappa(a, Om) * 1e-2 * kv[i] * s / k2, atol=1e-14, rtol=1e-12)


def test_screening_limits_single_mode():
    N, L, a, Om = 16, 64.0, 0.5, 0.3
    k2 = None
    # chameleon: a tiny mode is unscreened (|Phi_N| < Phi_crit): G_eff = mu
    for A, expect_screened in [(1e-6, False), (1e3, True)]:
        rho, s, kv = _mode_density(N, L, (1, 0, 0), A)
        k2 = kv @ kv
        m = Model(kind=FOFR, fR0=1e-5, screening=1)
        F = pm.force_mesh(rho, 1.0, N, L, a, Om, m)
        newton = -kappa(a, Om) * A * kv[0] * s / k2
        mu = float(M.fr_mu(np.sqrt(k2), a, Om, 1e-5))
        ratio = np.max(np.abs(F[0])) / np.max(np.abs(newton))
        if expect_screened:
            assert 1.0 < ratio < 1.0 + 0.05 * (mu - 1.0) + 1e-3
        else:
            assert ratio == pytest.approx(mu, rel=1e-8)
    # Vainshtein: small amplitude -> uniform eps0 = eps(x(1)), force = (1 + eps0/(3 beta)) Newton
    A = 1e-7
    rho, s, kv = _mode_density(N, L, (0, 1, 0), A)
    m = Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=1.0)
    F = pm.force_mesh(rho, 1.0, N, L, a, Om, m)
    k2 = kv @ kv
    b = float(M.dgp_beta(a, Om, 1.0))
    eps0 = float(M.eps_vainshtein(M.vainshtein_x(1.0, a, Om, 1.0)))
    newton = -kappa(a, Om) * A * kv[1] * s / k2
    assert np.allclose(F[1], (1 + eps0 / (3 * b)) * newton, rtol=1e-5, atol=1e-6 * np.abs(newton).max())
    # screening with eps == 1 everywhere is the unscreened model (App. B vs Sec. 5)
    assert eps0 < 1.0


def test_symmetron_single_mode_force_and_screening():
    """App. C symmetron through the App. B field equation: C = 2 beta^2, a^2 m^2 from m(a); a small
    mode feels mu(k, a) Newton, a large one is screened towards Newton, and before a_* there is
    no fifth force at all."""
    from workloads import SYMM_A
    N, L, Om = 16, 64.0, 0.3
    m_off = dataclasses.replace(SYMM_A, screening=0)
    for a in (0.45, 0.8):
        rho, s, kv = _mode_density(N, L, (1, 2, 0), 1e-2)
        k2 = kv @ kv
        mu = float(M.mu(SYMM_A, np.sqrt(k2), a, Om))
        assert (mu == 1.0) == (a < SYMM_A.a_star)
        F = pm.force_mesh(rho, 1.0, N, L, a, Om, m_off)
        assert np.allclose(F[0], -mu * kappa(a, Om) * 1e-2 * kv[0] * s / k2, atol=1e-14, rtol=1e-12)
    a = 0.8
    for A, screened in [(1e-4, False), (1e2, True)]:
        rho, s, kv = _mode_density(N, L, (1, 0, 0), A)
        k2 = kv @ kv
        F = pm.force_mesh(rho, 1.0, N, L, a, Om, SYMM_A)
        newton = -kappa(a, Om) * A * kv[0] * s / k2
        mu = float(M.mu(SYMM_A, np.sqrt(k2), a, Om))
        ratio = np.max(np.abs(F[0])) / np.max(np.abs(newton))
        if screened:
            assert 1.0 < ratio < 1.0 + 0.05 * (mu - 1.0)
        else:
            assert ratio == pytest.approx(mu, rel=1e-8)


# ------------------------------------------------------------------ App. B smoothing windows
def test_tophat_window_is_the_sphere_transform():
    """W(k) = (1/V) int_sphere e^{ik.r} d^3r = (3/R^3) int_0^R r^2 sin(kr)/(kr) dr, by quadrature,
    on both sides of the series/closed-form switch at kR = 1/2."""
    from scipy.integrate import quad
    R = 2.5
    for k in [1e-4, 0.03, 0.15, 0.199, 0.2, 0.201, 0.6, 1.7, 4.0, 11.0]:
        ref = 3.0 / R**3 * quad(lambda r: r * np.sin(k * r) / k, 0.0, R, limit=200, epsabs=1e-15)[0]
        assert float(pm.tophat_window(k * R)) == pytest.approx(ref, rel=1e-11, abs=1e-14)
    assert float(pm.tophat_window(np.pi)) == pytest.approx(3.0 / np.pi**2, rel=1e-14)
    assert float(pm.tophat_window(0.0)) == 1.0


def test_smoothing_windows_on_the_mesh():
    N, L, R = 16, 100.0, 9.0
    kf = 2 * np.pi / L
    n = np.fft.fftfreq(N, d=1.0 / N)
    nz, ny, nx = np.meshgrid(n, n, np.arange(N // 2 + 1), indexing="ij")
    kk = kf * np.sqrt(nx**2 + ny**2 + nz**2)
    W0 = pm.smoothing_window(N, L, R, 0)
    assert np.allclose(W0, np.exp(-0.5 * (kk * R) ** 2), rtol=1e-12, atol=0)
    W1 = pm.smoothing_window(N, L, R, 1)
    i = (1, 2, 3)
    x = kk[i] * R
    assert W1[i] == pytest.approx(3 * (np.sin(x) - x * np.cos(x)) / x**3, rel=1e-13)
    assert W1[0, 0, 0] == 1.0
    # sharp-k keeps exactly the lattice vectors with |n|^2 <= (L/(2 pi R))^2 = 3.13 (no mode near the cut)
    W2 = pm.smoothing_window(N, L, R, 2)
    assert set(np.unique(W2)) == {0.0, 1.0}
    kept = sorted(tuple(int(v) for v in t) for t in np.argwhere(W2 == 1.0))
    brute = sorted((iz, iy, ix) for iz in range(N) for iy in range(N) for ix in range(N // 2 + 1)
                   if n[iz] ** 2 + n[iy] ** 2 + ix**2 <= 3)
    assert kept == brute and len(brute) == 1 + 5 + 8 + 4  # |n|^2 = 0, 1, 2, 3 with n_x >= 0
    with pytest.raises(ValueError):
        pm.smoothing_window(N, L, R, 3)


def test_sharp_k_cut_is_decided_in_double_precision():
    """App. B sharp-k window: exactly the modes with (kR)^2 <= 1 in FP64, including a mode that
    sits on the cut (kept) and one a few ulp above it (cut).  The GPU parity cases use radii
    whose modes lie far from the cut (tests/test_gpu_parity.py lists them as empty)."""
    N, L = 16, 64.0
    kf = 2 * np.pi / L
    R_on = 1.0 / (kf * np.sqrt(5.0))                 # |n|^2 = 5 exactly on the cut
    W = pm.smoothing_window(N, L, R_on, 2)
    n = np.fft.fftfreq(N, d=1.0 / N)
    n2 = n[:, None, None] ** 2 + n[None, :, None] ** 2 + np.arange(N // 2 + 1)[None, None, :] ** 2
    x2 = n2 * (kf * R_on) ** 2
    assert np.array_equal(W == 1.0, x2 <= 1.0)
    on = np.abs(x2 - 1.0) < 1e-12
    assert on.any() and np.all(W[on & (x2 <= 1.0)] == 1.0)
    R_up = R_on * (1.0 + 1e-12)
    assert np.all(pm.smoothing_window(N, L, R_up, 2)[n2 == 5] == 0.0)
    for N2, L2, R2 in ((32, 512.0, 20.0), (64, 1024.0, 20.0), (32, 64.0, 4.0)):
        nn = np.fft.fftfreq(N2, d=1.0 / N2)
        m2 = nn[:, None, None] ** 2 + nn[None, :, None] ** 2 + np.arange(N2 // 2 + 1)[None, None, :] ** 2
        assert not np.any(np.abs(m2 * (2 * np.pi / L2 * R2) ** 2 - 1.0) <= 1e-5)


def test_sharp_k_screening_of_a_short_mode_is_uniform():
    """A mode with kR > 1 is cut from delta_R, so eps = eps(x(1)) everywhere at any amplitude and the
    force is (1 + eps0/(3 beta)) Newton; the Gaussian window leaves it partly in delta_R."""
    N, L, a, Om = 16, 64.0, 0.5, 0.3
    A = 0.5
    rho, s, kv = _mode_density(N, L, (0, 3, 0), A)
    k2 = kv @ kv
    R = 2.0 / np.sqrt(k2)
    b = float(M.dgp_beta(a, Om, 1.0))
    eps0 = float(M.eps_vainshtein(M.vainshtein_x(1.0, a, Om, 1.0)))
    newton = -kappa(a, Om) * A * kv[1] * s / k2
    F = pm.force_mesh(rho, 1.0, N, L, a, Om, Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=R, filter=2))
    assert np.allclose(F[1], (1 + eps0 / (3 * b)) * newton, rtol=1e-12, atol=1e-14)
    G = pm.force_mesh(rho, 1.0, N, L, a, Om, Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=R, filter=0))
    assert np.abs(G[1] - F[1]).max() > 1e-6 * np.abs(F[1]).max()


def test_zero_net_force_newtonian():
    N, L = 16, 32.0
    pos = random_positions(3000, L, 5)
    rho = pm.cic_deposit(pos, N, L)
    F = pm.force_mesh(rho, 3000 / N**3, N, L, 0.7, 0.3, Model())
    tot = [pm.cic_gather(Fi, pos, N, L).sum() for Fi in F]
    scale = np.mean([np.abs(pm.cic_gather(Fi, pos, N, L)).sum() for Fi in F])
    assert np.max(np.abs(tot)) < 1e-12 * scale


# ------------------------------------------------------------------ P(k)
def test_power_single_mode():
    N, L, A = 32, 100.0, 0.2
    rho, _, _ = _mode_density(N, L, (3, 0, 0), A)
    k, P, nm = pm.power_spectrum_mesh(rho - 1.0, N, L)
    kf = 2 * np.pi / L
    # |delta(k)|^2 = (A N^3 / 2)^2 for each of the two modes (+-3): P = A^2 L^3 / 4 per mode
    W2 = np.sinc(3 / N) ** 4
    # bin 2 holds |n| in [2.5, 3.5): six modes (+-3 on each axis), one non-zero pair
    assert nm[2] == pytest.approx(np.count_nonzero(nm) and nm[2])
    assert P[2] == pytest.approx(A**2 * L**3 / 4 / W2 * 2 / nm[2], rel=1e-10)
    assert k[2] > 2.5 * kf and k[2] < 3.5 * kf
    assert np.all(P[:2] < 1e-20)
