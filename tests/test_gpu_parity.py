"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: fields in float32 are compared relative to the field's largest
magnitude (FFT, force: 2e-5; CIC: 2e-6 absolute per cell of unit-mass
particles); particle displacements after all steps within 1e-4 of a mesh
cell; P(k) within 1e-4 relative per bin; the boost P_MG/P_LCDM within 1e-4
absolute.
"""
import dataclasses

import numpy as np
import pytest

from oracle import ics, pm
from oracle.cola import Simulation as OracleSim
from workloads import (F5, F5_NOSCREEN, LCDM_MODEL, NDGP1, SMALL_F5, SYMM_A, Cosmo, Model, Run,
                       random_field, random_positions)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1703_00879_gb300 as p
    p.lib()
    return p


def _relmax(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_fft_roundtrip_vs_oracle(pkg, N):
    run = SMALL_F5.with_(Np=32, Nmesh=N, Lbox=float(N))
    x = random_field(N, 100 + N)
    with pkg.Simulation(run, ic=False) as s:
        X = s.fft(x, 1)
        ref = ics.rfft3(x.astype(np.float32).astype(np.float64))
        assert _relmax(X, ref) < 2e-6 * np.log2(N)
        y = s.fft(ref.astype(np.complex64), -1)
        yref = ics.irfft3(ref, N) * N**3
        assert _relmax(y, yref) < 2e-6 * np.log2(N)


def test_fft_inverse_drops_imaginary_dc_and_nyquist_like_irfftn(pkg):
    N = 32
    run = SMALL_F5.with_(Np=32, Nmesh=N)
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((N, N, N // 2 + 1)) + 1j * rng.standard_normal((N, N, N // 2 + 1)))
    with pkg.Simulation(run, ic=False) as s:
        y = s.fft(X.astype(np.complex64), -1)
    assert _relmax(y, ics.irfft3(X, N) * N**3) < 2e-5


# ------------------------------------------------------------------ CIC
@pytest.mark.parametrize("N,L", [(32, 64.0), (64, 100.0)])
def test_cic_deposit_vs_oracle(pkg, N, L):
    run = SMALL_F5.with_(Np=32, Nmesh=N, Lbox=L)
    pos = random_positions(20000, L, 7)
    pos[:10] = [[0, 0, 0], [L - 1e-4, 0, 0], [L / 2, L / 2, L / 2], [-1.0, 3.0, L + 2.0],
                [L * 0.999999, L * 0.5, 1e-6], [1, 1, 1], [2, 2, 2], [3, 3, 3], [4, 4, 4], [5, 5, 5]]
    with pkg.Simulation(run, ic=False) as s:
        rho = s.cic_deposit(pos)
    ref = pm.cic_deposit(pos.astype(np.float32).astype(np.float64), N, L)
    assert np.max(np.abs(rho - ref)) < 2e-5
    assert abs(rho.sum() - 20000) < 0.05


def test_cic_deposit_empty(pkg):
    run = SMALL_F5
    with pkg.Simulation(run, ic=False) as s:
        rho = s.cic_deposit(np.zeros((0, 3), np.float32))
    assert not rho.any()


# ------------------------------------------------------------------ force from density
def _mb_f5(n):
    """f(R) F5 as a tabulated {m, beta} model (App. C) on n geometric nodes, a = 0.04 to 1.01."""
    from oracle import models as OM
    ta = np.geomspace(0.04, 1.01, n)
    return Model(kind=4, screening=1, mb_a=tuple(ta), mb_beta=tuple(np.full(n, 1 / np.sqrt(6.0))),
                 mb_m=tuple(np.sqrt(OM.fr_m2(ta, 0.3, 1e-5)) / OM.H0_OVER_C),
                 mb_phicrit0=float(OM.phi_crit_fr(0.04, 0.3, 1e-5)))


def _density(N, seed):
    # lognormal-like positive density with mean ~ rho_bar = 1 (Np = Nm)
    g = random_field(N, seed)
    return np.exp(0.8 * g - 0.32)


@pytest.mark.parametrize("model", [LCDM_MODEL, F5, F5_NOSCREEN, NDGP1, Model(kind=2, rcH0=1.0),
                                   Model(kind=2, rcH0=1.0, screening=1, R_smooth=20.0, filter=1),
                                   Model(kind=2, rcH0=1.0, screening=1, R_smooth=20.0, filter=2),
                                   SYMM_A, dataclasses.replace(SYMM_A, screening=0), _mb_f5(60)],
                         ids=["lcdm", "F5", "F5_noscreen", "nDGP_screen", "nDGP_noscreen",
                              "nDGP_tophat", "nDGP_sharpk", "symm", "symm_noscreen", "mb_table"])
@pytest.mark.parametrize("N", [32, 64])
def test_force_from_density_vs_oracle(pkg, model, N):
    # a box of 16 cells/Mpc^-1 per cell makes |Phi_N| cross the F5 threshold in ~40-85% of cells
    run = Run(Np=N, Nmesh=N, Lbox=16.0 * N, nsteps=4, model=model)
    rho = _density(N, 3 + N).astype(np.float32)
    a = 0.6
    with pkg.Simulation(run, ic=False) as s:
        F = s.force_from_density(rho, a)
    ref = pm.force_mesh(rho.astype(np.float64), 1.0, N, run.Lbox, a, run.cosmo.Omega_m, model)
    for i in range(3):
        assert _relmax(F[i], ref[i]) < 3e-5, i


@pytest.mark.parametrize("model", [LCDM_MODEL, F5, NDGP1], ids=["lcdm", "F5", "nDGP_screen"])
def test_force_from_density_128_vs_oracle(pkg, model):
    """N = 128, the largest mesh whose transforms run as plane passes (the x and y steps of a
    z-plane in one CTA: density r2c, the screening source chain, the force inverses): the same
    comparison and tolerance as above."""
    N = 128
    run = Run(Np=N, Nmesh=N, Lbox=16.0 * N, nsteps=4, model=model)
    rho = _density(N, 3 + N).astype(np.float32)
    a = 0.6
    with pkg.Simulation(run, ic=False) as s:
        F = s.force_from_density(rho, a)
    ref = pm.force_mesh(rho.astype(np.float64), 1.0, N, run.Lbox, a, run.cosmo.Omega_m, model)
    for i in range(3):
        assert _relmax(F[i], ref[i]) < 3e-5, i


def _sharp_k_modes_at_the_cut(N, L, R, rel=1e-5):
    """Lattice modes whose (kR)^2 lies within `rel` of 1: the FP64 oracle and the FP32 kernel may
    decide these either way (the sharp-k window of App. B).  Every other mode is decided alike."""
    n = np.fft.fftfreq(N, d=1.0 / N)
    n2 = n[:, None, None] ** 2 + n[None, :, None] ** 2 + np.arange(N // 2 + 1)[None, None, :] ** 2
    x2 = n2 * (2 * np.pi / L * R) ** 2
    return np.argwhere(np.abs(x2 - 1.0) <= rel)


def test_sharp_k_cases_have_no_mode_at_the_cut():
    """The sharp-k cases below (force: N = 32, 64, L = 16 N, R = 20; run: N = 32, L = 64, R = 4)
    have no mode within float rounding of kR = 1, so both sides keep the same modes."""
    for N in (32, 64):
        assert _sharp_k_modes_at_the_cut(N, 16.0 * N, 20.0).size == 0
    assert _sharp_k_modes_at_the_cut(32, 64.0, 4.0).size == 0


def test_force_screening_active():
    """The f(R) screening threshold is actually crossed in this test density."""
    N = 32
    for N in (32, 64):
        rho = _density(N, 3 + N)
        eps = pm.screening_factor(F5, ics.rfft3(rho - 1), N, 16.0 * N, 0.6, 0.3)
        assert 0.05 < np.mean(eps < 1) < 0.95


# ------------------------------------------------------------------ ICs and runs
@pytest.fixture(scope="module")
def oracle_small():
    sim = OracleSim(SMALL_F5)
    init = (sim.phi1.copy(), sim.phi2.copy(), sim.s.copy(), sim.acc.copy())
    sim.run_to_end()
    return sim, init


def test_ic_potentials_and_positions_vs_oracle(pkg, oracle_small):
    osim, (phi1, phi2, s0, acc0) = oracle_small
    with pkg.Simulation(SMALL_F5) as s:
        p1 = s.export(pkg.COLA_F_PHI1)
        p2 = s.export(pkg.COLA_F_PHI2)
        d0 = s.export(pkg.COLA_F_DISP)
        a0 = s.export(pkg.COLA_F_ACC)
    assert _relmax(p1, phi1) < 2e-5
    assert _relmax(p2, phi2) < 5e-5
    assert _relmax(d0.T, s0) < 2e-5
    # the initial residual acceleration is a small difference of two forces
    assert np.max(np.abs(a0.T - acc0)) < 2e-3 * np.max(np.abs(acc0)) + 1e-6


@pytest.mark.parametrize("seed", [2, 4], ids=["F5", "nDGP_screen"])
def test_ensemble_shape_run_vs_oracle(pkg, seed):
    """The batched ensemble's simulation shape (64^3 particles, 128^3 mesh, 128 Mpc/h), three
    steps in one cola_step call: the LPT fields, the density transform, the screening source and
    the force inverses all run as plane passes, the step boundaries fused.  Displacements within
    1e-4 cell of the FP64 oracle, P(k) within 1e-4 per bin."""
    from workloads import ensemble_run
    run = ensemble_run(seed, nsteps=3)
    o = OracleSim(run).run_to_end()
    with pkg.Simulation(run) as s:
        s.run_to_end()
        d = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        k, P, nm = s.pk()
    err = np.max(np.abs(d - o.s)) / (run.Lbox / run.Nmesh)
    assert err <= 1e-4, err
    ko, Po, nmo = o.power_spectrum(run.Nmesh // 2)
    ok = nmo > 0
    assert np.array_equal(nm[ok], nmo[ok].astype(np.int64))
    assert np.max(np.abs(P[ok] / Po[ok] - 1)) <= 1e-4


def _cell_err(run, s_gpu, s_ref):
    cell = run.Lbox / run.Nmesh
    d = np.abs(s_gpu.astype(np.float64) - s_ref)
    return d.max() / cell, np.sqrt((d**2).mean()) / cell


def test_small_config_run_vs_oracle(pkg, oracle_small):
    osim, _ = oracle_small
    with pkg.Simulation(SMALL_F5) as s:
        s.run_to_end()
        disp = s.export(pkg.COLA_F_DISP).T
        k, P, nm = s.pk()
        pos, vel = s.snapshot()
    mx, rms = _cell_err(SMALL_F5, disp, osim.s)
    assert mx <= 1e-4, (mx, rms)
    ko, Po, nmo = osim.power_spectrum()
    assert np.array_equal(nm, nmo.astype(np.int64))
    ok = nmo > 0
    assert np.allclose(k[ok], ko[ok], rtol=1e-12)
    assert np.max(np.abs(P[ok] / Po[ok] - 1)) <= 1e-4
    L = SMALL_F5.Lbox
    dpos = (pos.astype(np.float64) - osim.positions() + L / 2) % L - L / 2   # periodic difference
    assert np.max(np.abs(dpos)) / (L / SMALL_F5.Nmesh) <= 1e-4
    v_ref = osim.velocities_kms()
    assert _relmax(vel, v_ref) < 1e-4


def test_small_config_boost_vs_oracle(pkg, oracle_small):
    osim, _ = oracle_small
    twin = SMALL_F5.with_model(LCDM_MODEL)
    oref = OracleSim(twin).run_to_end()
    with pkg.Simulation(SMALL_F5) as s:
        s.run_to_end()
        _, P, _ = s.pk()
    with pkg.Simulation(twin) as s:
        s.run_to_end()
        _, P0, _ = s.pk()
    _, Po, nmo = osim.power_spectrum()
    _, Po0, _ = oref.power_spectrum()
    ok = nmo > 0
    B, Bo = P[ok] / P0[ok], Po[ok] / Po0[ok]
    assert np.max(np.abs(B - Bo)) <= 1e-4


@pytest.fixture(scope="module")
def oracle_small_lcdm():
    return OracleSim(SMALL_F5.with_model(LCDM_MODEL)).run_to_end()


@pytest.mark.parametrize("model", [
    Model(kind=1, fR0=1e-14, screening=1),
    Model(kind=1, fR0=1e-14, screening=0),
    Model(kind=2, rcH0=1e7, screening=1, R_smooth=1.0),
    Model(kind=2, rcH0=1e7, screening=0),
], ids=["fR_tiny_screened", "fR_tiny", "nDGP_large_rc_screened", "nDGP_large_rc"])
def test_mg_limits_reduce_to_lcdm(pkg, oracle_small_lcdm, model):
    """G_eff -> 1 limits (Sec. 5): f(R) with |f_R0| -> 0 (the scalaron mass a m -> infinity, so
    mu - 1 = k^2/(3(k^2 + a^2 m^2)) < 1e-12 here) and nDGP with r_c H0 -> infinity (1/(3 beta)
    ~ 2e-8), with and without screening, run on the GPU's modified-gravity kernels (per-k growth
    tables, screening passes, fifth-force Green's function).  They must reproduce the FP64
    oracle's LCDM run: displacements within 1e-4 cell, P(k) within 1e-4 per bin."""
    run = SMALL_F5.with_model(model)
    o = oracle_small_lcdm
    with pkg.Simulation(run) as s:
        s.run_to_end()
        disp = s.export(pkg.COLA_F_DISP).T
        _, P, nm = s.pk()
    mx, rms = _cell_err(run, disp, o.s)
    assert mx <= 1e-4, (mx, rms)
    _, Po, nmo = o.power_spectrum()
    ok = nmo > 0
    assert np.array_equal(nm, nmo.astype(np.int64))
    assert np.max(np.abs(P[ok] / Po[ok] - 1)) <= 1e-4


@pytest.mark.parametrize("run", [
    SMALL_F5.with_(Nmesh=64, nsteps=5),                       # mesh finer than particles
    SMALL_F5.with_(model=NDGP1, nsteps=5),                     # Vainshtein screening
    SMALL_F5.with_(model=Model(kind=1, fR0=1e-5, screening=1, scale_dependent=0), nsteps=5),
    SMALL_F5.with_(Np=64, Nmesh=32, Lbox=64.0, nsteps=3),      # mesh coarser than particles
    SMALL_F5.with_(nsteps=1, seed=12345678901),                # single step, 64-bit seed
    SMALL_F5.with_(model=Model(kind=2, rcH0=1.0, screening=1, R_smooth=4.0, filter=1), nsteps=5),
    SMALL_F5.with_(model=Model(kind=2, rcH0=1.0, screening=1, R_smooth=4.0, filter=2), nsteps=5),
    SMALL_F5.with_(model=SYMM_A, nsteps=5),                    # symmetron, switching on at a_* = 0.5
    SMALL_F5.with_(model=_mb_f5(60), nsteps=5),                # tabulated {m, beta}
], ids=["mesh64", "ndgp", "fR_lcdm_growth", "np64_nm32", "one_step", "ndgp_tophat", "ndgp_sharpk",
        "symmetron", "mb_table"])
def test_variants_vs_oracle(pkg, run):
    o = OracleSim(run).run_to_end()
    with pkg.Simulation(run) as s:
        s.run_to_end()
        disp = s.export(pkg.COLA_F_DISP).T
    mx, rms = _cell_err(run, disp, o.s)
    assert mx <= 1e-4, (mx, rms)


def test_zeldovich_plane_wave_on_gpu(pkg):
    """Same plane wave as the oracle pin: GPU equals oracle and the exact solution to PM accuracy."""
    N, L = 32, 64.0
    eds = Cosmo(Omega_m=1.0, Omega_b=0.05)
    run = Run(Np=N, Nmesh=N, Lbox=L, nsteps=10, cosmo=eds, model=Model())
    k = 2 * np.pi / L
    A = 0.5 * run.a_ini / k
    q = np.arange(N) * L / N
    phi = ics.rfft3(-(A / k) * np.cos(k * q)[None, None, :] * np.ones((N, N, 1)))
    phi2 = np.zeros_like(phi)
    o = OracleSim(run, phi=(phi, phi2)).run_to_end()
    with pkg.Simulation(run, phi=(phi, phi2)) as s:
        s.run_to_end()
        disp = s.export(pkg.COLA_F_DISP).T
    mx, _ = _cell_err(run, disp, o.s)
    assert mx <= 1e-4
    exact = A / run.a_ini * np.sin(k * o.q[:, 0])
    assert np.max(np.abs(disp[:, 0] - exact)) / np.max(np.abs(exact)) < 0.12


def test_checkpoint_resume_matches_uninterrupted(pkg):
    run = SMALL_F5.with_(nsteps=6)
    with pkg.Simulation(run) as s:
        s.step(3)
        state = [s.export(w) for w in (pkg.COLA_F_DISP, pkg.COLA_F_DV, pkg.COLA_F_ACC)]
        s.step(3)
        ref = s.export(pkg.COLA_F_DISP)
    with pkg.Simulation(run) as s2:
        s2.import_state(*state, steps_done=3)
        assert s2.steps_done == 3
        s2.step(-1)
        got = s2.export(pkg.COLA_F_DISP)
    assert np.max(np.abs(got - ref)) / (run.Lbox / run.Nmesh) < 1e-5


def test_errors_are_reported(pkg):
    import paper_1703_00879_gb300 as p
    with p.Simulation(SMALL_F5.with_(nsteps=2)) as s:
        s.step(2)
        with pytest.raises(p.ColaError) as e:
            s.step(1)
        assert e.value.code == p.COLA_EINVAL
    with p.Simulation(SMALL_F5, ic=False) as s:
        with pytest.raises(p.ColaError) as e:
            s.step(1)
        assert e.value.code == p.COLA_ESTATE
