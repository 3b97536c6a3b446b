"""Scale-independent LPT fast path (cola_set_lpt_fast): with growth that does
not depend on k, the step's LPT fields are c1 Psi1 + c2 Psi2 of the real-space
2LPT displacements (Sec. 4.1 with D(k, a) = D(a)).  Runs on the fast path match
the FP64 oracle within 1e-4 of a mesh cell and the default GPU path to FP32
rounding; models whose growth depends on k are refused."""
import numpy as np
import pytest

from oracle.cola import Simulation as OracleSim
from workloads import LCDM_MODEL, NDGP1, SMALL_F5

pytestmark = pytest.mark.gpu


def _periodic(d, L):
    return (d + 0.5 * L) % L - 0.5 * L


@pytest.mark.parametrize("model", [LCDM_MODEL, NDGP1], ids=["lcdm", "ndgp_screened"])
def test_fast_lpt_matches_oracle_and_default_path(model):
    import paper_1703_00879_gb300 as pkg
    run = SMALL_F5.with_(model=model)
    cell = run.Lbox / run.Nmesh
    osim = OracleSim(run)
    osim.run_to_end()
    _, Po, nmo = osim.power_spectrum()
    with pkg.Simulation(run) as s:
        s.run_to_end()
        d_def = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        pos_def, vel_def = s.snapshot()
    with pkg.Simulation(run, lpt_fast=True) as s:
        s.run_to_end()
        d = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        pos, vel = s.snapshot()
        _, P, nm = s.pk()
        lpt_disp = s.export(pkg.COLA_F_LPT_DISP)
    err = np.abs(_periodic(d - osim.s, run.Lbox)).max() / cell
    err_def = np.abs(_periodic(d - d_def, run.Lbox)).max() / cell
    ok = nmo > 0
    perr = float(np.max(np.abs(P[ok] / Po[ok] - 1)))
    print(f"\nkind {model.kind}: fast vs oracle {err:.2e} cell, fast vs default {err_def:.2e} cell, "
          f"P(k) {perr:.2e}")
    assert err <= 1e-4
    assert err_def <= 1e-5
    assert perr <= 1e-4
    assert np.abs(_periodic(pos - pos_def, run.Lbox)).max() / cell <= 1e-5
    assert np.allclose(vel, vel_def, rtol=1e-4, atol=1e-4 * np.abs(vel_def).max())
    assert np.all(np.isfinite(lpt_disp)) and np.abs(lpt_disp).max() > 0


def test_fast_lpt_refused_for_scale_dependent_growth():
    import paper_1703_00879_gb300 as pkg
    with pytest.raises(pkg.ColaError, match="depends on k"):
        pkg.Simulation(SMALL_F5, lpt_fast=True)


def test_fast_lpt_batch_matches_solo():
    """A batch of fast-path contexts (one multi-simulation launch sequence per
    step) reproduces the same runs advanced one at a time."""
    import paper_1703_00879_gb300 as pkg
    runs = [SMALL_F5.with_(model=m, seed=sd) for m, sd in ((LCDM_MODEL, 3), (NDGP1, 4), (LCDM_MODEL, 5))]
    solo = []
    for r in runs:
        with pkg.Simulation(r, lpt_fast=True) as s:
            s.run_to_end()
            solo.append(s.export(pkg.COLA_F_DISP))
    sims = [pkg.Simulation(r, lpt_fast=True) for r in runs]
    try:
        b = pkg.Batch(sims)
        b.step(runs[0].nsteps)
        b.close()
        for s, ref, r in zip(sims, solo, runs):
            d = s.export(pkg.COLA_F_DISP)
            assert np.abs(_periodic(d - ref, r.Lbox)).max() / (r.Lbox / r.Nmesh) <= 1e-4
    finally:
        for s in sims:
            s.close()
