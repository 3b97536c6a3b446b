"""Host logic of the continuous-batching server, with a fake device backend (no GPU).

Checks: the HBM budget is never exceeded, admission is FIFO, runs that arrive
while others are active join mid-flight, every request completes, a request
larger than the whole budget is refused up front, each tick advances only runs
of one shape bucket (at different steps, with different step counts), and a
bucket never has more than `ticks_ahead` ticks in flight.
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
    """Completes after `delay` queries (a tick the device has not reached yet)."""

    def __init__(self, delay=0):
        self.left = delay

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True


class FakeBackend:
    def __init__(self, event_delay=0):
        self.log = []          # (event, rid-name)
        self.active = 0
        self.max_active = 0
        self.ticks = []        # (stream, [(name, step before the tick)])
        self.event_delay = event_delay
        self.pending = {}      # stream -> events not yet complete

    def stream(self):
        return object()

    def event(self, stream):
        e = FakeEvent(self.event_delay)
        self.pending.setdefault(stream, []).append(e)
        return e

    def step_many(self, sims, stream):
        assert all(getattr(s, "stream", None) is stream for s in sims)   # joined their bucket
        inflight = [e for e in self.pending.get(stream, []) if e.left > 0]
        self.ticks.append((stream, [(s.run.name, s.steps) for s in sims], len(inflight)))
        for s in sims:
            s.steps += 1

    def simulations(self, runs, stream):
        out = []
        for run in runs:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.log.append(("admit", run.name))
            out.append(FakeSim(run, self.log))
        return out

    def move(self, sim, stream):
        sim.stream = stream

    def pk_start(self, sim, nbins):
        assert sim.steps == sim.run.nsteps
        sim.nbins = nbins

    def pk_poll(self, sim):
        self.active -= 1
        self.log.append(("done", sim.run.name))
        n = sim.nbins or 4
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


@pytest.mark.parametrize("one_stream", [False, True])
def test_ticks_batch_runs_of_one_shape_at_different_steps(one_stream):
    reqs = [_req(0, 32, 6, 0.0), _req(1, 64, 4, 0.0), _req(2, 32, 3, 0.0), _req(3, 32, 5, 0.0)]
    be = FakeBackend()
    # only three fit at first: r3 is admitted when one finishes and joins mid-flight
    srv = Server(hbm_budget_bytes=3, max_slots=8, backend=be, bytes_for=lambda r: 1, one_stream=one_stream)
    st = srv.run(reqs, realtime=False)
    assert len(st.results) == 4
    by_shape, streams = {}, set()
    for stream, members, _ in be.ticks:
        names = [n for n, _ in members]
        shapes = {reqs[int(n[1:])][1].Np for n in names}
        assert len(shapes) == 1                                   # one bucket per tick
        by_shape.setdefault(shapes.pop(), set()).update(names)
        streams.add(id(stream))
    assert by_shape == {32: {"r0", "r2", "r3"}, 64: {"r1"}}
    assert len(streams) == (1 if one_stream else 2)
    # r3 joined while r0 was mid-run: some tick holds both at different steps
    mixed = [m for _, m, _ in be.ticks if {"r0", "r3"} <= {n for n, _ in m}]
    assert any(len({s for _, s in m}) > 1 for m in mixed)
    # every run got exactly its own number of steps
    steps = {}
    for _, m, _ in be.ticks:
        for n, _ in m:
            steps[n] = steps.get(n, 0) + 1
    assert steps == {"r0": 6, "r1": 4, "r2": 3, "r3": 5}


def test_ticks_in_flight_are_bounded():
    reqs = [_req(i, 32, 8, 0.0) for i in range(3)]
    be = FakeBackend(event_delay=3)
    srv = Server(hbm_budget_bytes=100, backend=be, bytes_for=lambda r: 1, ticks_ahead=2)
    st = srv.run(reqs, realtime=False)
    assert len(st.results) == 3
    assert max(n for _, _, n in be.ticks) <= 1      # at most one earlier tick still in flight
