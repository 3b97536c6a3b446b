"""Pins of the oracle's COLA stepper (Sec. 2, Sec. 4.1, App. A)."""
import numpy as np
import pytest

from oracle import ics
from oracle.cola import Simulation
from workloads import Cosmo, Model, Run, SMALL_F5

EDS = Cosmo(Omega_m=1.0, Omega_b=0.05)


def _plane_wave_run(N, nsteps=10, L=64.0, amp_final=0.5):
    """Zel'dovich plane wave along x in EdS: Psi1_x = A sin(k q_x), A k D1(a=1) = amp_final."""
    run = Run(Np=N, Nmesh=N, Lbox=L, nsteps=nsteps, cosmo=EDS, model=Model(), z_ini=19.0)
    k = 2 * np.pi / L
    A = amp_final * run.a_ini / k               # D1 = a / a_ini in EdS
    q = np.arange(N) * L / N
    phi = -(A / k) * np.cos(k * q)[None, None, :] * np.ones((N, N, 1))
    phi1 = ics.rfft3(phi)
    return run, (phi1, np.zeros_like(phi1)), A, k


def _plane_wave_error(N):
    run, phi, A, k = _plane_wave_run(N)
    sim = Simulation(run, phi=phi).run_to_end()
    qx = sim.q[:, 0]
    exact = (1.0 / run.a_ini) * A * np.sin(k * qx)
    assert np.max(np.abs(sim.s[:, 1:])) < 1e-12
    return np.max(np.abs(sim.s[:, 0] - exact)) / np.max(np.abs(exact))


def test_zeldovich_plane_wave_converges_with_mesh():
    """Exact Zel'dovich solution x = q + (a/a_ini) Psi1 (EdS, before shell crossing).

    With N_mesh = N_p the CIC density of a cold lattice displaced by less than a
    cell is a one-sided difference of the displacement (half a cell off, on the
    side the particles moved to), so the PM force error is first order in the
    cell size: the error halves when the mesh doubles.  A wrong kappa, sign or
    time integral would not converge at all.
    """
    e16, e32 = _plane_wave_error(16), _plane_wave_error(32)
    assert e32 < 0.12
    assert 1.8 < e16 / e32 < 2.2


def test_lpt_only_limit_is_exact():
    """Replacing the PM force by A_LPT leaves delta_v = 0 and s = Psi_LPT(a) exactly."""
    run = SMALL_F5.with_(Np=16, Nmesh=16, Lbox=32.0, nsteps=4)

    def lpt_force(sim, a):
        n = int(np.argmin(np.abs(sim.a - a)))
        return sim.lpt_field(sim.table.ddD1[n], sim.table.ddD2[n])

    sim = Simulation(run, force_fn=lpt_force).run_to_end()
    t = sim.table
    expect = sim.lpt_field(t.D1[-1], t.D2[-1])
    assert np.max(np.abs(sim.dv)) < 1e-13
    assert np.allclose(sim.s, expect, rtol=0, atol=1e-11 * np.abs(expect).max())


def test_lcdm_kspace_reweight_equals_real_space_growth():
    """mu = 1: the per-k reweight path equals D1(a) Psi1(q) + D2(a) Psi2(q) (Sec. 3 vs Sec. 4.1)."""
    run = SMALL_F5.with_(Np=16, Nmesh=16, Lbox=32.0, nsteps=3, model=Model())
    sim = Simulation(run)
    t = sim.table
    one = np.ones_like(t.D1[0])
    psi1 = sim.lpt_field(one, 0 * one)
    psi2 = sim.lpt_field(0 * one, one)
    for n in range(len(t.a)):
        assert np.allclose(t.D1[n], t.D1[n][0]) and np.allclose(t.D2[n], t.D2[n][0])
        got = sim.lpt_field(t.D1[n], t.D2[n])
        assert np.allclose(got, t.D1[n][0] * psi1 + t.D2[n][0] * psi2, atol=1e-13)
    assert t.D2[0][0] == -3.0 / 7.0 and t.D1[0][0] == 1.0


def test_fr_with_tiny_fR0_equals_lcdm_run():
    """G_eff -> 1 and growth -> LCDM as |f_R0| -> 0 (screening off): same trajectory."""
    base = SMALL_F5.with_(Np=16, Nmesh=16, Lbox=32.0, nsteps=3)
    a = Simulation(base.with_model(Model())).run_to_end()
    b = Simulation(base.with_model(Model(kind=1, fR0=1e-20, screening=0))).run_to_end()
    assert np.allclose(a.s, b.s, rtol=0, atol=1e-9 * np.abs(a.s).max())


@pytest.mark.parametrize("model", [
    Model(kind=1, fR0=1e-14, screening=1),
    Model(kind=2, rcH0=1e7, screening=0),
    Model(kind=2, rcH0=1e7, screening=1, R_smooth=1.0),
], ids=["fR_screened", "nDGP", "nDGP_screened"])
def test_mg_limits_with_and_without_screening_equal_lcdm_run(model):
    """Sec. 5 limits with the screening passes in the path: chameleon screening with |f_R0| -> 0
    (threshold and fifth-force range both -> 0) and nDGP with r_c H0 -> infinity (the fifth-force
    coefficient 1/(3 beta) -> 0, eps finite) leave the LCDM trajectory; mu - 1 < 1e-7 here, so
    the displacements agree to 1e-6 of their largest value."""
    base = SMALL_F5.with_(Np=16, Nmesh=16, Lbox=32.0, nsteps=3)
    a = Simulation(base.with_model(Model())).run_to_end()
    b = Simulation(base.with_model(model)).run_to_end()
    assert np.allclose(a.s, b.s, rtol=0, atol=1e-6 * np.abs(a.s).max())


def test_small_config_runs_and_boost_positive():
    """F5 boost B(k) = P_MG/P_LCDM > 1 and growing with k at the small scales of config 1."""
    sim = Simulation(SMALL_F5).run_to_end()
    ref = Simulation(SMALL_F5.with_model(Model())).run_to_end()
    k, P, _ = sim.power_spectrum()
    _, P0, _ = ref.power_spectrum()
    B = P / P0
    assert np.all(np.isfinite(B[:10]))
    assert B[10] > 1.0 and B[10] > B[1]
    # largest scale: linear theory B ~ [D1_MG(k)/D1_LCDM]^2 to a few per cent
    Dmg = sim.table.interp(sim.table.D1[-1], np.array([k[0]]))[0]
    Dl = ref.table.D1[-1][0]
    assert B[0] == pytest.approx((Dmg / Dl) ** 2, rel=0.05)
