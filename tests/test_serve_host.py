"""Host logic of the continuous-batching server, with a fake device backend (no GPU).

Checks: the HBM budget is never exceeded, admission is FIFO, runs that arrive
while others are active join mid-flight, every request completes, and a request
larger than the whole budget is refused up front.
"""
import numpy as np
import pytest

from paper_1703_00879_gb300.serve import Server
from workloads import Run


class FakeSim:
    def __init__(self, run, log):
        self.run, self.log, self.closed, self.steps = run, log, False, 0

    def close(self):
        self.closed = True


class FakeEvent:
    def __init__(self, sim):
        self.sim = sim

    def query(self):
        return True


class FakeBackend:
    def __init__(self):
        self.log = []          # (event, rid-name)
        self.active = 0
        self.max_active = 0

    def stream(self):
        return object()

    def event(self, stream):
        return FakeEvent(None)

    def simulation(self, run, stream):
        self.active += 1
        self.max_active = max(self.max_active, self.active)
        self.log.append(("admit", run.name))
        return FakeSim(run, self.log)

    def step(self, sim, stream):
        sim.steps += 1

    def pk(self, sim, stream, nbins):
        assert sim.steps == sim.run.nsteps
        self.active -= 1
        self.log.append(("done", sim.run.name))
        n = nbins or 4
        return np.arange(n) + 1.0, np.ones(n) * sim.run.Np, np.ones(n, np.int64)

    def synchronize(self):
        pass


def _req(i, Np, steps, t):
    return (t, Run(Np=Np, Nmesh=2 * Np, Lbox=2.0 * Np, nsteps=steps, name=f"r{i}"))


def test_budget_fifo_and_completion():
    reqs = [_req(i, [32, 64, 128][i % 3], 3 + i % 4, 0.0) for i in range(12)]
    size = {32: 1, 64: 3, 128: 5}
    be = FakeBackend()
    srv = Server(hbm_budget_bytes=8, max_slots=8, backend=be, bytes_for=lambda r: size[r.Np])
    st = srv.run(reqs, realtime=False)
    assert len(st.results) == 12 and [r.rid for r in st.results] == list(range(12))
    assert st.peak_bytes <= 8
    admits = [n for e, n in be.log if e == "admit"]
    assert admits == [f"r{i}" for i in range(12)]                 # FIFO
    # continuous: some run is admitted while others are still active
    first_done = [i for i, (e, _) in enumerate(be.log) if e == "done"][0]
    later_admits = [i for i, (e, _) in enumerate(be.log) if e == "admit" and i > first_done]
    assert later_admits and be.max_active >= 2
    for r in st.results:
        assert r.pk[0] == r.run.Np and r.latency >= 0


def test_request_larger_than_budget_is_refused():
    srv = Server(hbm_budget_bytes=2, backend=FakeBackend(), bytes_for=lambda r: 5)
    with pytest.raises(ValueError):
        srv.run([_req(0, 32, 2, 0.0)], realtime=False)


def test_realtime_arrivals_respect_order():
    t = [0.0, 0.001, 0.002, 0.02]
    reqs = [_req(i, 32, 2, t[i]) for i in range(4)]
    be = FakeBackend()
    srv = Server(hbm_budget_bytes=100, backend=be, bytes_for=lambda r: 1)
    st = srv.run(reqs, realtime=True)
    assert [r.rid for r in st.results] == [0, 1, 2, 3]
    assert all(r.admitted >= r.arrival - 1e-9 for r in st.results)
