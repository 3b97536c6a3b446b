"""The allocation-free power spectrum entry point, cola_pk_noalloc.

It serves callers that cannot allocate device memory when they need a P(k)
(a latency-bound serving loop that must not let cudaFree synchronise the
device, a process whose device memory is held by another allocator, a
diagnostic that must not fail on an allocation in the middle of a run).  Its
scratch is a fixed static device array, so it is checked here against the
regular entry point cola_pk on the same particles, on two calls in a row
(the second call must not see leftovers of the first), and for the size
limit of that array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from workloads import SMALL_F5

pytestmark = pytest.mark.gpu


def _device_positions(pkg, sim, run):
    import torch
    pos = torch.empty((run.Np ** 3, 3), dtype=torch.float32, device="cuda")
    sim.snapshot_device(pos, None)
    torch.cuda.synchronize()
    return pos


@pytest.mark.parametrize("nmesh", [32, 64, 128])
def test_pk_noalloc_matches_cola_pk_on_two_calls(nmesh):
    import torch

    import paper_1703_00879_gb300 as pkg
    run = SMALL_F5.with_(Nmesh=nmesh, nsteps=3)
    with pkg.Simulation(run) as sim:
        sim.step(3)
        k0, p0, n0 = sim.pk()
        pos = _device_positions(pkg, sim, run)
        stream = torch.cuda.current_stream().cuda_stream
        ok = n0 > 0
        free_before = None
        for call in range(2):
            k, p, n = pkg.cola_pk_noalloc(pos.data_ptr(), pos.shape[0], nmesh, run.Lbox, nmesh // 2, stream)
            torch.cuda.synchronize()
            if call == 0:
                free_before = torch.cuda.mem_get_info()[0]
            else:
                # the second call allocated nothing: the device's free memory is unchanged
                assert torch.cuda.mem_get_info()[0] == free_before
            assert np.array_equal(n, n0)
            assert np.allclose(k[ok], k0[ok], rtol=1e-12)
            assert np.max(np.abs(p[ok] / p0[ok] - 1.0)) <= 1e-4


def test_pk_noalloc_matches_the_oracle():
    """The same entry point against the FP64 oracle's estimator (CIC deposit, deconvolved
    |delta(k)|^2, the same bins) on the same positions: every bin within 1e-4."""
    import torch

    import paper_1703_00879_gb300 as pkg
    from oracle import pm
    run = SMALL_F5.with_(Nmesh=64, nsteps=3)
    with pkg.Simulation(run) as sim:
        sim.step(3)
        pos = _device_positions(pkg, sim, run)
    k, p, n = pkg.cola_pk_noalloc(pos.data_ptr(), pos.shape[0], 64, run.Lbox, 32,
                                  torch.cuda.current_stream().cuda_stream)
    ko, po, no = pm.power_spectrum(pos.double().cpu().numpy(), 64, run.Lbox, 32)
    ok = no > 0
    assert np.array_equal(n[ok], no[ok].astype(np.int64))
    assert np.allclose(k[ok], ko[ok], rtol=1e-12)
    assert np.max(np.abs(p[ok] / po[ok] - 1.0)) <= 1e-4


def test_pk_noalloc_rejects_meshes_beyond_its_static_scratch():
    import torch

    import paper_1703_00879_gb300 as pkg
    pos = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    too_big = pkg.COLA_PK_NOALLOC_MAX_NMESH * 2
    with pytest.raises(pkg.ColaError) as e:
        pkg.cola_pk_noalloc(pos.data_ptr(), 8, too_big, 64.0, 16)
    assert e.value.code == pkg.COLA_EINVAL
    assert "static scratch" in str(e.value)
