"""The C ABI's memory and waiting rules, on the GPU.

* Every device byte a context, a batch or a multi-context call uses comes through the caller's
  alloc/free callbacks, and all of it is released by cola_free / cola_batch_free.
* Creating, set-up and freeing of many contexts with distinct growth tables (more keys than any
  cache of device tables would hold) never synchronises the device: work queued on another stream
  is still running afterwards.
* Bounded host waits: with a wait limit, a call that waits for queued work returns COLA_ETIMEOUT and
  leaves the work queued; the context stays usable.
"""
import ctypes
import math
import time

import numpy as np
import pytest

from workloads import BIG_NDGP, F5, SMALL_F5, Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1703_00879_gb300 as p
    p.lib()
    return p


class _Counting:
    """alloc/free callbacks into PyTorch's caching allocator that record every live pointer."""

    def __init__(self, pkg):
        import torch
        dev = torch.cuda.current_device()
        self.live, self.calls = {}, []

        def _alloc(nbytes, stream, user):
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            self.live[int(p)] = int(nbytes)
            self.calls.append(int(nbytes))
            return p

        def _free(ptr, stream, user):
            assert int(ptr) in self.live, "free of a pointer the callbacks did not hand out"
            del self.live[int(ptr)]
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (pkg.ALLOC_FN(_alloc), pkg.FREE_FN(_free))


def _ctx(pkg, run, cb, stream):
    L = pkg.lib()
    cfg = pkg.make_config(run)
    h = ctypes.c_void_p()
    pkg._check(L.cola_init(ctypes.byref(cfg), cb.cbs[0], cb.cbs[1], None, ctypes.c_void_p(stream.cuda_stream),
                           ctypes.byref(h)))
    pkg._check(L.cola_set_model(h, ctypes.byref(pkg.make_model(run.model))), h)
    return h


def test_all_device_memory_through_the_callbacks(pkg):
    import torch
    L = pkg.lib()
    cb = _Counting(pkg)
    st = torch.cuda.current_stream()
    run = SMALL_F5.with_(nsteps=4)
    ctxs = [_ctx(pkg, run.with_(seed=i), cb, st) for i in range(3)]
    # cola_init makes one allocation of cola_device_bytes (tables and twiddles included)
    assert cb.calls == [pkg.cola_device_bytes(run)] * 3
    for h in ctxs:
        pkg._check(L.cola_ic(h), h)
    pkg._check(L.cola_step(ctxs[0], 1), ctxs[0])
    arr = (ctypes.c_void_p * 3)(*[h.value for h in ctxs])
    pkg._check(L.cola_step_many(arr, 3, ctypes.c_void_p(st.cuda_stream)))     # shift array via callbacks
    b = ctypes.c_void_p()
    pkg._check(L.cola_step(ctxs[1], 1), ctxs[1])
    pkg._check(L.cola_step(ctxs[2], 1), ctxs[2])
    pkg._check(L.cola_batch_create(arr, 3, None, ctypes.c_void_p(st.cuda_stream), ctypes.byref(b)))
    pkg._check(L.cola_batch_step(b, 1))
    nb = 16
    k, P, nm = np.empty(3 * nb), np.empty(3 * nb), np.empty(3 * nb, np.int64)
    pkg._check(L.cola_batch_pk(b, nb, k.ctypes.data, P.ctypes.data, nm.ctypes.data))
    pos = np.empty((run.Np ** 3, 3), np.float32)
    pkg._check(L.cola_snapshot(ctxs[0], pos.ctypes.data, None, pkg.COLA_HOST), ctxs[0])
    assert len(cb.calls) > 3          # shift arrays, batch P(k) sums and snapshot staging came through too
    L.cola_batch_free(b)
    for h in ctxs:
        L.cola_free(h)
    torch.cuda.synchronize()
    assert cb.live == {}, f"{len(cb.live)} allocations left after the frees"


def test_many_distinct_models_never_synchronise_the_device(pkg):
    """600 contexts with distinct f(R) amplitudes (600 distinct growth-table keys) are created, set
    up and freed on one stream while a long run is queued on another: the long run is still in
    flight afterwards, so nothing synchronised the device."""
    import torch
    L = pkg.lib()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    small = SMALL_F5.with_(nsteps=3, nk_table=16)

    def churn(i):
        m = Model(kind=1, fR0=1e-5 * (1.0 + 1e-3 * i), screening=1)
        with torch.cuda.stream(sb):
            s = pkg.Simulation(small.with_model(m), ic=False, stream=sb)
            s.close()

    for i in range(20):          # warm the allocator and the upload ring
        churn(100000 + i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(20):
        churn(200000 + i)
    torch.cuda.synchronize()
    t_ctx = (time.perf_counter() - t0) / 20
    nctx = 600
    long_run = BIG_NDGP.with_(Np=64, nsteps=400, model=F5)
    with torch.cuda.stream(sa):
        s = pkg.Simulation(long_run, stream=sa)
        s.step(2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.step(2)
        torch.cuda.synchronize()
        t_step = (time.perf_counter() - t1) / 2
        nsteps = min(long_run.nsteps - 4, max(20, math.ceil(3.0 * nctx * t_ctx / t_step)))
        s.step(nsteps)
        done = torch.cuda.Event()
        done.record(sa)
    t2 = time.perf_counter()
    for i in range(nctx):
        churn(i)
    t_churn = time.perf_counter() - t2
    still_running = not done.query()
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t2
    s.close()
    print(f"\n{nctx} contexts in {t_churn:.2f} s while {nsteps} queued steps ran {t_all:.2f} s")
    assert still_running, (t_churn, t_all)


def test_wait_limit_returns_etimeout_and_keeps_the_context_usable(pkg):
    import torch
    run = BIG_NDGP.with_(Np=64, Nmesh=256, Lbox=256.0, nsteps=40)
    with pkg.Simulation(run) as s:
        s.step(30)                                   # queued, not waited for
        s.set_wait_limit(1e-6)
        with pytest.raises(pkg.ColaError) as e:
            s.pk()
        assert e.value.code == pkg.COLA_ETIMEOUT
        s.pk_async()
        with pytest.raises(pkg.ColaError) as e:
            s.pk_result()
        assert e.value.code == pkg.COLA_ETIMEOUT
        s.set_wait_limit(0)
        k, P, nm = s.pk_result()                     # the pending request is still there
        assert np.all(np.isfinite(P[nm > 0]))
        s.wait()
        assert s.steps_done == 30
        s.step(1)
        k2, P2, _ = s.pk()
        assert np.all(np.isfinite(P2[nm > 0])) and not np.array_equal(P, P2)
    torch.cuda.synchronize()


class _Failing(_Counting):
    """Counting callbacks that return NULL once `budget` allocations have been handed out."""

    def __init__(self, pkg, budget):
        import torch
        dev = torch.cuda.current_device()
        self.live, self.calls, self.budget = {}, [], budget

        def _alloc(nbytes, stream, user):
            if len(self.calls) >= self.budget:
                self.calls.append(-int(nbytes))
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            self.live[int(p)] = int(nbytes)
            self.calls.append(int(nbytes))
            return p

        def _free(ptr, stream, user):
            assert int(ptr) in self.live
            del self.live[int(ptr)]
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (pkg.ALLOC_FN(_alloc), pkg.FREE_FN(_free))


def test_failing_allocator_gives_enomem_and_leaks_nothing(pkg):
    """Fault injection on the host: an allocator that refuses.  cola_init returns COLA_ENOMEM with
    nothing allocated; a batch whose shift array cannot be allocated fails its step with
    COLA_ENOMEM and the contexts stay usable."""
    import torch
    L = pkg.lib()
    st = torch.cuda.current_stream()
    run = SMALL_F5.with_(nsteps=3)
    cb = _Failing(pkg, 0)
    cfg = pkg.make_config(run)
    h = ctypes.c_void_p()
    rc = L.cola_init(ctypes.byref(cfg), cb.cbs[0], cb.cbs[1], None, ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
    assert rc == pkg.COLA_ENOMEM and not h.value and cb.live == {}
    cb = _Failing(pkg, 2)                                  # the two contexts, then nothing
    ctxs = [_ctx(pkg, run.with_(seed=i), cb, st) for i in range(2)]
    for c in ctxs:
        pkg._check(L.cola_ic(c), c)
    arr = (ctypes.c_void_p * 2)(*[c.value for c in ctxs])
    b = ctypes.c_void_p()
    pkg._check(L.cola_batch_create(arr, 2, None, ctypes.c_void_p(st.cuda_stream), ctypes.byref(b)))
    assert L.cola_batch_step(b, 1) == pkg.COLA_ENOMEM     # the graph's shift array
    L.cola_batch_free(b)
    pkg._check(L.cola_step(ctxs[0], 1), ctxs[0])           # the contexts are still usable
    for c in ctxs:
        L.cola_free(c)
    torch.cuda.synchronize()
    assert cb.live == {}


def test_misaligned_allocator_block_is_refused(pkg):
    """An allocator whose block is not on a 256-byte boundary: cola_init releases it and fails
    with COLA_EINVAL before any kernel touches it (the kernels' vector accesses need the
    alignment)."""
    import torch
    L = pkg.lib()
    st = torch.cuda.current_stream()
    dev = torch.cuda.current_device()
    live = {}

    def _alloc(nbytes, stream, user):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 256, dev, int(stream or 0))
        live[int(base) + 16] = int(base)
        return int(base) + 16

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(live.pop(int(ptr)))

    cbs = (pkg.ALLOC_FN(_alloc), pkg.FREE_FN(_free))
    cfg = pkg.make_config(SMALL_F5.with_(nsteps=3))
    h = ctypes.c_void_p()
    rc = L.cola_init(ctypes.byref(cfg), cbs[0], cbs[1], None, ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
    torch.cuda.synchronize()
    assert rc == pkg.COLA_EINVAL and not h.value and live == {}


def test_check_state_counts_non_finite_values(pkg):
    """cola_check_state: 0 for a healthy run; a NaN and an Inf planted in the imported state are
    counted, and the next step's residual acceleration is checked as well."""
    run = SMALL_F5.with_(nsteps=4)
    with pkg.Simulation(run) as s:
        s.step(2)
        assert s.check_state() == 0
        d, v, a = (s.export(w) for w in (pkg.COLA_F_DISP, pkg.COLA_F_DV, pkg.COLA_F_ACC))
        d[0, 5] = np.nan
        v[2, 7] = np.inf
        s.import_state(d, v, a, steps_done=2)
        assert s.check_state() == 2


def test_snapshot_into_page_locked_buffers(pkg):
    """A snapshot into caller-owned page-locked buffers (direct DMA) equals the pageable one
    (staged through the download ring above 64 MB, plain copy below), at a size on each side."""
    import torch
    for run in (SMALL_F5.with_(nsteps=2), SMALL_F5.with_(Np=256, Nmesh=256, Lbox=256.0, nsteps=2)):
        with pkg.Simulation(run) as s:
            s.step(1)
            p0, v0 = s.snapshot()
            P = run.Np ** 3
            out = tuple(torch.empty((P, 3), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2))
            p1, v1 = s.snapshot(out=out)
            assert p1 is out[0] and v1 is out[1]
            np.testing.assert_array_equal(p1, p0)
            np.testing.assert_array_equal(v1, v0)
            with pytest.raises(ValueError):
                s.snapshot(out=(np.empty((P, 3), np.float64), None))


def test_device_wait_gives_up_at_its_limit(pkg):
    """The one wait on the device (a TMA-staged transform's mbarrier wait for its tile) is bounded:
    on a barrier phase that no copy completes it gives up after its limit and reports it, and the
    device stays usable (a step runs afterwards)."""
    t0 = time.perf_counter()
    assert pkg.selftest_wait(0.02) is True
    dt = time.perf_counter() - t0
    assert 0.02 <= dt < 5.0
    with pytest.raises(pkg.ColaError):
        pkg.selftest_wait(0.0)
    with pkg.Simulation(SMALL_F5.with_(nsteps=2)) as s:
        s.step(1)
        assert s.check_state() == 0
