"""Multi-step cola_step joins the kick of each step but the last with the drift and
deposit of the next (one pass over the particles, Sec. 2), forming the next step's
LPT fields first.  The arithmetic per particle is that of separate steps; only the
order of the float additions in the CIC deposit differs, so K steps in one call and
K calls of one step agree to FP32 rounding, and both agree with the FP64 oracle."""
import numpy as np
import pytest

from workloads import SMALL_F5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1703_00879_gb300 as p
    return p


def _run(pkg, run, calls):
    with pkg.Simulation(run) as s:
        for k in calls:
            s.step(k)
        out = {w: s.export(w).astype(np.float64) for w in (pkg.COLA_F_DISP, pkg.COLA_F_DV, pkg.COLA_F_ACC,
                                                              pkg.COLA_F_LPT_DISP, pkg.COLA_F_LPT_ACC)}
        _, P, _ = s.pk()
    return out, P


@pytest.mark.parametrize("split", [[10], [2, 3, 5], [7, 1, 2]], ids=["one_call", "three_calls", "mixed"])
def test_fused_steps_equal_single_steps(pkg, split):
    run = SMALL_F5
    ref, Pref = _run(pkg, run, [1] * 10)
    got, P = _run(pkg, run, split)
    cell = run.Lbox / run.Nmesh
    for w in (pkg.COLA_F_DISP, pkg.COLA_F_DV, pkg.COLA_F_ACC):
        scale = np.max(np.abs(ref[w])) or 1.0
        err = np.max(np.abs(got[w] - ref[w]))
        assert err <= 1e-4 * (cell if w == pkg.COLA_F_DISP else scale), (w, err)
    # the last step's LPT fields (kick fields from whichever slot the last call left them in)
    for w in (pkg.COLA_F_LPT_DISP, pkg.COLA_F_LPT_ACC):
        np.testing.assert_allclose(got[w], ref[w], rtol=0, atol=1e-6 * np.max(np.abs(ref[w])))
    assert np.max(np.abs(P / Pref - 1)) <= 1e-5


def test_fused_steps_then_batch_step_use_the_right_kick_fields(pkg):
    """A context stepped by a fused call (kick fields left in the second slot) and then by a
    cola_step_many step exports the kick fields of its last step."""
    run = SMALL_F5.with_(nsteps=4)
    a, _ = _run(pkg, run, [1, 1, 1])
    with pkg.Simulation(run) as s:
        s.step(2)
        pkg.step_many([s])
        b = s.export(pkg.COLA_F_LPT_ACC).astype(np.float64)
    np.testing.assert_allclose(b, a[pkg.COLA_F_LPT_ACC], rtol=0, atol=1e-6 * np.max(np.abs(b)))


def _batch_run(pkg, runs, calls):
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims) as b:
        for k in calls:
            b.step(k)
        k, P, nm = b.pk()
    out = []
    for s in sims:
        out.append({w: s.export(w).astype(np.float64) for w in (pkg.COLA_F_DISP, pkg.COLA_F_DV,
                                                                pkg.COLA_F_LPT_ACC)})
        s.close()
    return out, P


@pytest.mark.parametrize("split", [[6], [2, 1, 3]], ids=["one_call", "three_calls"])
def test_fused_batch_steps_equal_single_batch_steps(pkg, split):
    """A batch of the ensemble's model set stepped K at a time (fused boundaries, kick fields in
    alternating slots) against the same batch stepped once per call: every member's state and
    last kick fields agree to FP32 rounding, P(k) within 1e-5."""
    from workloads import ENSEMBLE_MODELS, ensemble_run
    runs = [ensemble_run(seed, Np=32, Nmesh=64, Lbox=64.0, nsteps=6) for seed in range(len(ENSEMBLE_MODELS))]
    ref, Pref = _batch_run(pkg, runs, [1] * 6)
    got, P = _batch_run(pkg, runs, split)
    for r, a, b in zip(runs, ref, got):
        cell = r.Lbox / r.Nmesh
        assert np.max(np.abs(b[pkg.COLA_F_DISP] - a[pkg.COLA_F_DISP])) <= 1e-4 * cell
        assert np.max(np.abs(b[pkg.COLA_F_DV] - a[pkg.COLA_F_DV])) <= 1e-4 * np.max(np.abs(a[pkg.COLA_F_DV]))
        np.testing.assert_allclose(b[pkg.COLA_F_LPT_ACC], a[pkg.COLA_F_LPT_ACC], rtol=0,
                                   atol=1e-6 * np.max(np.abs(a[pkg.COLA_F_LPT_ACC])))
    ok = Pref > 0
    assert np.max(np.abs(P[ok] / Pref[ok] - 1)) <= 1e-5


def test_fused_batch_steps_eager_equal_graph(pkg):
    """With stage timing on, batch steps launch eagerly (no graph) through the same launch
    sequences, fused boundaries included: the state and the stage record agree with the graph
    run (the fused particle pass appears in the record)."""
    from workloads import ENSEMBLE_MODELS, ensemble_run
    runs = [ensemble_run(seed, Np=32, Nmesh=64, Lbox=64.0, nsteps=4) for seed in range(len(ENSEMBLE_MODELS))]
    ref, _ = _batch_run(pkg, runs, [4])
    sims = [pkg.Simulation(r) for r in runs]
    sims[0].profile(True)
    with pkg.Batch(sims) as b:
        b.step(4)
    st = sims[0].profile_read()
    assert st["kick_drift_deposit"][1] == 3 and st["drift_deposit"][1] == 1 and st["gather_kick"][1] == 1
    for r, s, a in zip(runs, sims, ref):
        d = s.export(pkg.COLA_F_DISP).astype(np.float64)
        assert np.max(np.abs(d - a[pkg.COLA_F_DISP])) <= 1e-4 * r.Lbox / r.Nmesh
        s.close()
