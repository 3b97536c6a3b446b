"""Batched ensembles (one CUDA graph launch per step) and the serving loop on the GPU.

A simulation's result must not depend on whether it runs alone, in a batch,
or in the serving mix: displacements within 1e-4 of a mesh cell of the solo
run (the parity tolerance; only the order of the float atomics differs) and
P(k) within 1e-4.
"""
import numpy as np
import pytest

from workloads import ENSEMBLE_MODELS, ensemble_run

pytestmark = pytest.mark.gpu


def _runs(n, Np=32, Nmesh=64, steps=4):
    return [ensemble_run(seed, Np=Np, Nmesh=Nmesh, Lbox=2.0 * Np, nsteps=steps) for seed in range(n)]


def _solo(pkg, run):
    with pkg.Simulation(run) as s:
        s.run_to_end()
        return s.export(pkg.COLA_F_DISP), s.pk()


@pytest.mark.parametrize("plan", [None, (2, 1, 0), (4, 2, 0), (3, 2, 76), (1, 3, 0), (6, 1, 0, 16384, 8192),
                                  (6, 1, 0, 64, 64), (2, 2, 0, 4096, 0)],
                         ids=["one_group", "pairs", "quads_2chains", "triples_capped", "singles_3chains",
                              "shared_boxes", "tiny_boxes_fall_back", "pairs_deposit_bins"])
def test_batch_equals_solo(plan):
    """Every model of the ensemble set (LCDM, f(R) x3, nDGP x2) in one batch:
    the model-dependent force stages run per model subset of each group."""
    import paper_1703_00879_gb300 as pkg
    runs = _runs(len(ENSEMBLE_MODELS))
    solo = [_solo(pkg, r) for r in runs]
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims, plan=plan) as b:
        b.step(-1)
        assert b.steps_done == runs[0].nsteps
        k, P, nm = b.pk()
    for i, (r, s, (d0, (k0, P0, nm0))) in enumerate(zip(runs, sims, solo)):
        d = s.export(pkg.COLA_F_DISP)
        assert s.steps_done == r.nsteps
        assert np.max(np.abs(d - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        ok = nm0 > 0
        assert np.array_equal(nm[i], nm0)
        assert np.allclose(k[i][ok], k0[ok], rtol=1e-12)
        assert np.max(np.abs(P[i][ok] / P0[ok] - 1)) <= 1e-4
        s.close()


def test_batch_with_boxes_on_paired_force_mesh_equals_solo():
    """Meshes above 128 points keep F_x and F_y as interleaved pairs: the shared-memory box
    gather stages and interpolates the pairs.  Two F5 / nDGP members (32^3 particles on a 256^3
    mesh) with deposit bins and gather boxes against their solo runs."""
    import paper_1703_00879_gb300 as pkg
    runs = [ensemble_run(seed, Np=32, Nmesh=256, Lbox=64.0, nsteps=3) for seed in (2, 4)]
    solo = [_solo(pkg, r) for r in runs]
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims, plan=(2, 1, 0, 16384, 8192)) as b:
        b.step(-1)
        k, P, nm = b.pk()
    for i, (r, s, (d0, (k0, P0, nm0))) in enumerate(zip(runs, sims, solo)):
        d = s.export(pkg.COLA_F_DISP)
        assert np.max(np.abs(d - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        ok = nm0 > 0
        assert np.max(np.abs(P[i][ok] / P0[ok] - 1)) <= 1e-4
        s.close()


def test_batch_members_vs_oracle():
    """One member of every model class of the ensemble (LCDM, f(R) 1e-6/1e-5/1e-4, nDGP r_c H0 = 1
    and 5, each screened) advanced together in one batch, against the FP64 oracle run of the same
    record: displacements within 1e-4 cell, every P(k) bin within 1e-4 (Sec. 2, Sec. 6, App. B)."""
    import paper_1703_00879_gb300 as pkg
    from oracle.cola import Simulation as OracleSim
    runs = _runs(len(ENSEMBLE_MODELS))
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims) as b:
        b.step(-1)
        k, P, nm = b.pk()
    for i, (r, s) in enumerate(zip(runs, sims)):
        o = OracleSim(r).run_to_end()
        d = s.export(pkg.COLA_F_DISP).T.astype(np.float64)
        err = np.max(np.abs(d - o.s)) / (r.Lbox / r.Nmesh)
        ko, Po, nmo = o.power_spectrum(r.Nmesh // 2)
        ok = nmo > 0
        print(f"\nbatch member {i} (model kind {r.model.kind}): {err:.2e} cell, "
              f"P(k) {np.max(np.abs(P[i][ok] / Po[ok] - 1)):.2e}")
        assert err <= 1e-4
        assert np.array_equal(nm[i][ok], nmo[ok].astype(np.int64))
        assert np.max(np.abs(P[i][ok] / Po[ok] - 1)) <= 1e-4
        s.close()


def test_batch_of_mixed_shapes_runs_one_context_per_group():
    import paper_1703_00879_gb300 as pkg
    runs = [ensemble_run(0, Np=32, Nmesh=64, Lbox=64.0, nsteps=3),
            ensemble_run(1, Np=64, Nmesh=64, Lbox=64.0, nsteps=3),
            ensemble_run(2, Np=32, Nmesh=32, Lbox=64.0, nsteps=3)]
    solo = [_solo(pkg, r) for r in runs]
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims, plan=(3, 1, 0)) as b:
        assert b.plan[0] == 1
        b.step(-1)
        _, P, _ = b.pk(16)
    for i, (r, s, (d0, _)) in enumerate(zip(runs, sims, solo)):
        assert np.max(np.abs(s.export(pkg.COLA_F_DISP) - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        _, P0, nm0 = s.pk(16)
        ok = nm0 > 0
        assert np.max(np.abs(P[i][ok] / P0[ok] - 1)) <= 1e-4
        s.close()


def test_batch_of_reduced_precision_seeds_equals_solo():
    import paper_1703_00879_gb300 as pkg
    runs = _runs(4, steps=3)
    solo = []
    for r in runs:
        with pkg.Simulation(r, seed_precision=1) as s:
            s.run_to_end()
            solo.append(s.export(pkg.COLA_F_DISP))
    sims = [pkg.Simulation(r, seed_precision=1) for r in runs]
    with pkg.Batch(sims) as b:
        b.step(-1)
    for r, s, d0 in zip(runs, sims, solo):
        assert np.max(np.abs(s.export(pkg.COLA_F_DISP) - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        s.close()


def test_batch_autotune_keeps_results():
    import paper_1703_00879_gb300 as pkg
    runs = _runs(8, steps=10)
    solo = [_solo(pkg, r) for r in runs]
    sims = [pkg.Simulation(r) for r in runs]
    with pkg.Batch(sims) as b:
        group, chains, cap, dep, gk = b.autotune(max_steps=8)
        assert 1 <= group <= 8 and 1 <= chains <= 8 and cap >= 0
        assert dep in (0, 4096, 16384) and gk in (0, 4096, 8192)
        assert b.plan == (group, chains, cap, dep, gk)
        b.step(-1)
    for r, s, (d0, _) in zip(runs, sims, solo):
        assert np.max(np.abs(s.export(pkg.COLA_F_DISP) - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        s.close()


def test_batch_rejects_mismatched_steps():
    import paper_1703_00879_gb300 as pkg
    runs = _runs(2)
    a, b = pkg.Simulation(runs[0]), pkg.Simulation(runs[1])
    a.step(1)
    with pytest.raises(pkg.ColaError):
        pkg.Batch([a, b])
    a.close()
    b.close()


def test_step_many_mixes_shapes_models_step_counts_and_progress():
    """cola_step_many over runs of two shapes, every model, different step
    counts, started at different times: each run ends where its solo run does."""
    import paper_1703_00879_gb300 as pkg
    runs = [ensemble_run(seed, Np=32, Nmesh=64, Lbox=64.0, nsteps=3 + seed % 3) for seed in range(6)]
    runs += [ensemble_run(10 + seed, Np=32, Nmesh=32, Lbox=64.0, nsteps=4) for seed in range(2)]
    solo = [_solo(pkg, r) for r in runs]
    sims = [pkg.Simulation(r) for r in runs]
    sims[1].step(2)                      # ahead of the others
    sims[4].step(1)
    while True:
        live = [s for s in sims if s.steps_done < s.run.nsteps]
        if not live:
            break
        pkg.step_many(live)
    for r, s, (d0, (k0, P0, nm0)) in zip(runs, sims, solo):
        assert s.steps_done == r.nsteps
        assert np.max(np.abs(s.export(pkg.COLA_F_DISP) - d0)) / (r.Lbox / r.Nmesh) <= 1e-4
        _, P, nm = s.pk()
        ok = nm0 > 0
        assert np.max(np.abs(P[ok] / P0[ok] - 1)) <= 1e-4
        s.close()


def test_ic_many_equals_cola_ic():
    """Initial conditions of many contexts in one launch sequence: the same
    displacements, bit for bit, as cola_ic per context (no atomics on that
    path), and runs that end where the solo runs end; two shapes, every model,
    reduced-precision seeds in one of them."""
    import paper_1703_00879_gb300 as pkg
    runs = [ensemble_run(seed, Np=32, Nmesh=64, Lbox=64.0, nsteps=3) for seed in range(6)]
    runs += [ensemble_run(20 + seed, Np=32, Nmesh=32, Lbox=64.0, nsteps=3) for seed in range(3)]
    precs = [0] * 6 + [1] * 3
    solo = []
    for r, pr in zip(runs, precs):
        with pkg.Simulation(r, seed_precision=pr) as s:
            d0 = s.export(pkg.COLA_F_DISP)
            s.run_to_end()
            solo.append((d0, s.export(pkg.COLA_F_DISP)))
    sims = [pkg.Simulation(r, seed_precision=pr, ic=False) for r, pr in zip(runs, precs)]
    pkg.ic_many(sims)
    for s, (d0, _) in zip(sims, solo):
        assert np.array_equal(s.export(pkg.COLA_F_DISP), d0)
    while any(s.steps_done < s.run.nsteps for s in sims):
        pkg.step_many([s for s in sims if s.steps_done < s.run.nsteps])
    for r, s, (_, d1) in zip(runs, sims, solo):
        assert np.max(np.abs(s.export(pkg.COLA_F_DISP) - d1)) / (r.Lbox / r.Nmesh) <= 1e-4
        s.close()


def test_step_many_rejects_finished_and_duplicate_contexts():
    import paper_1703_00879_gb300 as pkg
    r = ensemble_run(0, Np=32, Nmesh=32, Lbox=64.0, nsteps=1)
    with pkg.Simulation(r) as a, pkg.Simulation(r.with_(seed=5)) as b:
        with pytest.raises(pkg.ColaError):
            pkg.step_many([a, a])
        pkg.step_many([a, b])
        with pytest.raises(pkg.ColaError):
            pkg.step_many([a])


def test_serving_results_equal_solo_runs():
    import paper_1703_00879_gb300 as pkg
    from paper_1703_00879_gb300.serve import Server
    from workloads import serving_requests
    reqs = serving_requests(10, rate_hz=200.0, seed=3, sizes=(32, 64), steps=(3, 5))
    budget = 3 * max(pkg.cola_device_bytes(r) for _, r in reqs)   # forces staggered admission
    st = Server(budget, max_slots=4).run(reqs, realtime=True)
    assert len(st.results) == 10 and st.peak_bytes <= budget and st.peak_active >= 2
    for res in st.results:
        _, (k, P, nm) = _solo(pkg, res.run)
        ok = nm > 0
        assert np.array_equal(res.nmodes, nm)
        assert np.max(np.abs(res.pk[ok] / P[ok] - 1)) <= 1e-4
    s = st.summary()
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    # two served requests (one of each size) against the FP64 oracle run of the same record
    from oracle.cola import Simulation as OracleSim
    picked = {}
    for res in st.results:
        picked.setdefault(res.run.Np, res)
    for res in picked.values():
        ko, Po, nmo = OracleSim(res.run).run_to_end().power_spectrum(len(res.pk))
        ok = nmo > 0
        assert np.array_equal(res.nmodes[ok], nmo[ok].astype(np.int64))
        assert np.max(np.abs(res.pk[ok] / Po[ok] - 1)) <= 1e-4, res.run
