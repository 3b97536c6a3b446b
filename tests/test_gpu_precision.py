"""Reduced precision (variant a.S1): the seed fields phi1, phi2 (Sec. 4.1
reweighting reads them every step) and the six per-step LPT drift and kick
fields (App. A: the displacement-derivative fields) in BF16 or FP16 storage with
one FP32 scale per field, arithmetic in FP32, against the FP64 oracle run with
exact fields.

The bound.  Rounding a complex mode to a format of unit roundoff u (BF16 8
significant bits, u = 2^-8; FP16 11 bits, u = 2^-11) moves each component by
at most u times its magnitude, so the mode moves by at most u |phi_k|.  The
LPT displacement Psi(a) = grad(c1(k,a) phi1 + c2(k,a) phi2) is linear in the
seeds mode by mode, so by Parseval the RMS of its error over the lattice is at
most u (RMS|grad c1 phi1| + RMS|grad c2 phi2|).  At a_ini (c1 = 1, c2 = -3/7)
that bounds the initial displacements; the FP32 parity slack is added on top.
At the end of a run the residual displacement also carries the error through
the nonlinear forces; the asserted end-of-run bounds are the initial bound
scaled by the growth of the RMS displacement, with a factor 2 for that
nonlinear part.  The 16-bit LPT fields add, per step, at most u |dPsi_n| to the
drift and u |A_n| dtau to the kick: the drift part sums to at most u times the
LPT displacement accumulated over the run (the per-step increments grow
coherently), and the kick part is of the same order, so 2 u RMS|s(z=0)| is
added to the end-of-run bound.  P(k) per bin within 6u (|delta_k|^2 moves by
2u + u^2 at linear order per source of displacement error: seeds and fields).
The measured errors are printed.
"""
import numpy as np
import pytest

from oracle import ics
from oracle.cola import Simulation as OracleSim
from workloads import SMALL_F5

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -8, 2: 2.0 ** -11}
NAME = {1: "bf16", 2: "fp16"}


@pytest.fixture(scope="module")
def oracle_run():
    sim = OracleSim(SMALL_F5)
    s0 = sim.s.copy()
    N, L = SMALL_F5.Np, SMALL_F5.Lbox
    rms = []
    for phi in (sim.phi1, sim.phi2):
        g = np.stack([ics.irfft3(f * phi, N).ravel() for f in ics.grad_factor(N, L)], axis=1)
        rms.append(float(np.sqrt((g ** 2).sum(axis=1).mean())))
    sim.run_to_end()
    return sim, s0, rms


def _rms(x):
    return float(np.sqrt((np.asarray(x, np.float64) ** 2).sum(axis=1).mean()))


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_seed_precision_error_vs_fp64_oracle(prec, oracle_run):
    import paper_1703_00879_gb300 as pkg
    osim, s0_ref, (rms1, rms2) = oracle_run
    run = SMALL_F5
    cell = run.Lbox / run.Nmesh
    u = U[prec]
    with pkg.Simulation(run, seed_precision=prec) as s:
        d0 = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        s.run_to_end()
        d = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        k, P, nm = s.pk()
    # a_ini: the Parseval bound plus the FP32 parity slack (2e-5 of the largest displacement)
    e0 = _rms(d0 - s0_ref)
    bound0 = u * (rms1 + 3.0 / 7.0 * rms2) + 2e-5 * np.max(np.abs(s0_ref))
    # end of run: scaled by the displacement growth, factor 2 for the nonlinear part,
    # plus the 16-bit LPT fields (drift and kick) of every step
    e1 = _rms(d - osim.s)
    bound1 = 2.0 * bound0 * _rms(osim.s) / _rms(s0_ref) + 2.0 * u * _rms(osim.s)
    _, Po, nmo = osim.power_spectrum()
    ok = nmo > 0
    perr = float(np.max(np.abs(P[ok] / Po[ok] - 1)))
    mx1 = float(np.max(np.abs(d - osim.s))) / cell
    print(f"\n{NAME[prec]}: a_ini RMS err {e0 / cell:.3e} cell (bound {bound0 / cell:.3e}); "
          f"z=0 RMS err {e1 / cell:.3e} cell, max {mx1:.3e} cell (bound {bound1 / cell:.3e}); "
          f"P(k) max rel err {perr:.3e} (bound {6 * u:.3e})")
    assert e0 <= bound0
    assert e1 <= bound1
    assert perr <= 6 * u


def test_reduced_seeds_are_used_and_stay_within_bound():
    """The library keeps the FP32 potentials (for export) beside the 16-bit
    copies the steps read, and a BF16 run of the same seed differs from the
    FP32 one (the reduced seeds and LPT fields are really used) by no more than
    the bound (seeds u, LPT fields 2u, of the RMS displacement)."""
    import paper_1703_00879_gb300 as pkg
    run = SMALL_F5.with_(nsteps=2)
    assert pkg.cola_device_bytes(run, 1) > pkg.cola_device_bytes(run, 0)
    with pkg.Simulation(run) as s:
        s.run_to_end()
        d32 = s.export(pkg.COLA_F_DISP).astype(np.float64)
    with pkg.Simulation(run, seed_precision=1) as s:
        s.run_to_end()
        d16 = s.export(pkg.COLA_F_DISP).astype(np.float64)
    assert not np.array_equal(d32, d16)
    e = float(np.sqrt(((d16 - d32) ** 2).sum(axis=0).mean()))
    assert e <= 4 * U[1] * float(np.sqrt((d32 ** 2).sum(axis=0).mean()))


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
def test_sixteen_bit_lpt_fields_are_exported_dequantised(prec):
    """After a step the exported LPT drift / kick fields are the 16-bit ones times their field
    scale: within u (relative to the field's largest value) of the FP32 run's fields."""
    import paper_1703_00879_gb300 as pkg
    run = SMALL_F5.with_(nsteps=3)
    out = {}
    for p in (0, prec):
        with pkg.Simulation(run, seed_precision=p) as s:
            s.step(2)
            out[p] = [s.export(w).astype(np.float64) for w in (pkg.COLA_F_LPT_DISP, pkg.COLA_F_LPT_ACC)]
    for a, b in zip(out[0], out[prec]):
        for c in range(3):
            # seeds (u) and the field itself (u of the scale, which holds the field's largest value
            # with up to 4x headroom for fp16)
            assert np.max(np.abs(b[c] - a[c])) <= 6 * U[prec] * np.max(np.abs(a[c]))
            assert not np.array_equal(a[c], b[c])
