"""Continuous-batching request loop for COLA simulations on one GPU.

Requests (workloads.Run records, mixed sizes, models and step counts) arrive
over time.  A request is admitted as soon as a slot is free and its device
memory (cola_device_bytes) fits in the HBM budget.  Admitted runs are grouped
into shape buckets (equal particles, mesh, box, table size and seed
precision); each bucket has its own CUDA stream, so buckets overlap on the
device.  Every tick advances all in-flight runs of a bucket by one step with
ONE multi-simulation launch sequence (cola_step_many): runs at different
steps, with different models and different total step counts share each
kernel launch.  A run whose last step has been enqueued is finished when its
bucket's stream reaches that tick; it returns its P(k) and releases its
memory, which lets waiting requests in.  Requests that arrive while others
run join their bucket at its next tick (continuous batching, not a queue
drained in waves).  At most `ticks_ahead` ticks per bucket are in flight, so
late arrivals join early instead of queueing behind work enqueued long ago.
With one_stream, the ICs and all buckets share one stream: the persistent
kernels then never compete for SMs with another bucket's kernels.

Nothing in the loop waits for the device: the initial conditions of the runs
admitted together run on a side stream as one multi-simulation sequence
(cola_ic_many), a run joins its bucket's ticks once they are done (its context
then moves to the bucket stream), results are fetched with a non-blocking
P(k), and finished contexts are freed when their bucket has no tick in flight.

The loop is host logic on top of the C ABI (cola_init, cola_ic_many,
cola_set_stream, cola_step_many, cola_pk_async, cola_free); every step of the
method runs in the library's kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import Simulation, cola_device_bytes, ic_many, step_many


@dataclass
class Result:
    rid: int
    run: object
    k: np.ndarray
    pk: np.ndarray
    nmodes: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Slot:
    rid: int
    run: object
    sim: Simulation
    bucket: tuple
    arrival: float
    admitted: float
    bytes: int
    ic_event: object = None      # ICs done on the side stream
    joined: bool = False         # on the bucket stream, part of its ticks
    steps_enqueued: int = 0
    done_event: object = None    # the tick of its last step
    pk_started: bool = False


@dataclass
class _Bucket:
    stream: object
    inflight: deque = field(default_factory=deque)   # events of enqueued ticks
    to_free: list = field(default_factory=list)      # finished slots, freed when no tick is in flight


@dataclass
class ServerStats:
    results: list = field(default_factory=list)
    peak_bytes: int = 0
    peak_active: int = 0
    ticks: int = 0
    wall_s: float = 0.0

    def latencies(self):
        return np.array([r.latency for r in self.results])

    def summary(self):
        lat = self.latencies()
        n = len(self.results)
        return {"completed": n, "wall_s": self.wall_s,
                "sims_per_hour": n / self.wall_s * 3600.0 if self.wall_s > 0 else None,
                "p50_latency_s": float(np.percentile(lat, 50)) if n else None,
                "p99_latency_s": float(np.percentile(lat, 99)) if n else None,
                "peak_active": self.peak_active, "peak_bytes": self.peak_bytes, "ticks": self.ticks}


def shape_key(run, seed_precision: int = 0) -> tuple:
    """Runs with equal keys can share multi-simulation launches."""
    return (run.Np, run.Nmesh, float(run.Lbox), int(getattr(run, "nk_table", 1024)), int(seed_precision))


class _TorchBackend:
    """CUDA streams/events from PyTorch and libcola Simulations."""

    def __init__(self):
        import torch
        self.torch = torch

    def stream(self):
        return self.torch.cuda.Stream()

    def event(self, stream):
        e = self.torch.cuda.Event()
        e.record(stream)
        return e

    def simulations(self, runs, stream):
        """Contexts for runs, their initial conditions in one multi-simulation launch sequence."""
        with self.torch.cuda.stream(stream):
            sims = [Simulation(r, stream=stream, ic=False) for r in runs]
            ic_many(sims, stream)
        return sims

    def move(self, sim, stream):
        sim.set_stream(stream)

    def step_many(self, sims, stream):
        step_many(sims, stream)

    def pk_start(self, sim, nbins):
        sim.pk_async(nbins)

    def pk_poll(self, sim):
        """(k, P, nmodes) once the P(k) started by pk_start has landed, else None."""
        return sim.pk_result() if sim.pk_ready() else None

    def synchronize(self):
        self.torch.cuda.synchronize()


class Server:
    """Admits runs by device-memory budget and advances every admitted run of a
    shape bucket with one multi-simulation launch sequence per tick."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, nbins: Optional[int] = None,
                 clock: Callable[[], float] = time.perf_counter, backend=None,
                 bytes_for: Optional[Callable] = None, ticks_ahead: int = 2, one_stream: bool = True):
        self.one_stream = bool(one_stream)
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.nbins = nbins
        self.clock = clock
        self.backend = backend
        self.ticks_ahead = max(1, int(ticks_ahead))
        self._bytes_for = bytes_for or cola_device_bytes

    def bytes_for(self, run) -> int:
        return int(self._bytes_for(run))

    def run(self, requests, realtime: bool = True) -> ServerStats:
        """Serve (arrival_time_s, Run) requests; arrival times are relative to the start."""
        be = self.backend or _TorchBackend()
        pending = deque(sorted(((float(t), i, r) for i, (t, r) in enumerate(requests)), key=lambda x: x[0]))
        for _, _, r in pending:
            if self.bytes_for(r) > self.budget:
                raise ValueError(f"request {r.name} needs more than the whole HBM budget")
        waiting: deque = deque()
        active: list[_Slot] = []
        buckets: dict = {}
        ic_stream = be.stream()
        shared = ic_stream if self.one_stream else None   # one stream: ICs and every bucket in order
        used = 0
        stats = ServerStats()
        t0 = self.clock()
        while pending or waiting or active or any(bk.to_free for bk in buckets.values()):
            now = self.clock() - t0
            while pending and (pending[0][0] <= now or not realtime):
                waiting.append(pending.popleft())
            # admission: FIFO, by memory budget and free slots; the ICs of everything
            # admitted now run on the side stream as one multi-simulation sequence
            admitted = []
            while waiting and len(active) + len(admitted) < self.max_slots:
                t_arr, rid, run = waiting[0]
                need = self.bytes_for(run)
                if used + need > self.budget:
                    break
                waiting.popleft()
                key = shape_key(run)
                if key not in buckets:
                    buckets[key] = _Bucket(shared or be.stream())
                used += need
                admitted.append((rid, run, key, t_arr, need))
            if admitted:
                sims = be.simulations([a[1] for a in admitted], ic_stream)
                ev = be.event(ic_stream)
                now_adm = self.clock() - t0
                for (rid, run, key, t_arr, need), sim in zip(admitted, sims):
                    active.append(_Slot(rid, run, sim, key, t_arr, now_adm, need, ic_event=ev))
            stats.peak_bytes = max(stats.peak_bytes, used)
            stats.peak_active = max(stats.peak_active, len(active))
            progressed = False
            # runs whose ICs are done join their bucket
            for sl in active:
                if not sl.joined and sl.ic_event.query():
                    be.move(sl.sim, buckets[sl.bucket].stream)
                    sl.joined = True
                    progressed = True
            # one tick per bucket with room in its pipeline: every joined run with steps left, one step
            for key, bk in buckets.items():
                while bk.inflight and bk.inflight[0].query():
                    bk.inflight.popleft()
                if not bk.inflight and bk.to_free:
                    for sl in bk.to_free:
                        sl.sim.close()
                        used -= sl.bytes
                    bk.to_free = []
                    progressed = True
                if len(bk.inflight) >= self.ticks_ahead:
                    continue
                members = [sl for sl in active
                           if sl.bucket == key and sl.joined and sl.steps_enqueued < sl.run.nsteps]
                if not members:
                    continue
                be.step_many([sl.sim for sl in members], bk.stream)
                ev = be.event(bk.stream)
                bk.inflight.append(ev)
                stats.ticks += 1
                progressed = True
                for sl in members:
                    sl.steps_enqueued += 1
                    if sl.steps_enqueued == sl.run.nsteps:
                        sl.done_event = ev
            # finished runs: start their P(k) without waiting, collect it when it lands
            still = []
            for sl in active:
                if sl.done_event is not None and not sl.pk_started and sl.done_event.query():
                    be.pk_start(sl.sim, self.nbins)
                    sl.pk_started = True
                    progressed = True
                if sl.pk_started:
                    res = be.pk_poll(sl.sim)
                    if res is not None:
                        k, pk, nm = res
                        stats.results.append(Result(sl.rid, sl.run, k, pk, nm, sl.arrival, sl.admitted,
                                                    self.clock() - t0))
                        buckets[sl.bucket].to_free.append(sl)
                        progressed = True
                        continue
                still.append(sl)
            active = still
            if not progressed:
                if active or any(bk.to_free for bk in buckets.values()):
                    time.sleep(5e-5)      # the device is behind: let it catch up
                elif not waiting and pending and realtime:
                    time.sleep(max(0.0, min(0.01, pending[0][0] - (self.clock() - t0))))
        be.synchronize()
        stats.wall_s = self.clock() - t0
        stats.results.sort(key=lambda r: r.rid)
        return stats
