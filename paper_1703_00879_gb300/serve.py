"""Continuous-batching request loop for COLA simulations on one GPU.

Requests (workloads.Run records, mixed sizes and models) arrive over time.  A
request is admitted as soon as a slot is free and its device memory
(cola_device_bytes) fits in the HBM budget; admitted runs get their own CUDA
stream, so the work of every active run overlaps on the device.  Each pass of
the loop enqueues up to `steps_per_pass` steps of every active run (0: all
its remaining steps at once, so the host never throttles small runs); a run
that has enqueued its last step is finished when its stream reaches it,
returns its P(k) and releases its memory, which lets waiting requests in.  Requests that arrive
while others are running join mid-flight (continuous batching, not a queue
drained in waves).

The loop is host logic on top of the C ABI (cola_init, cola_ic, cola_step,
cola_pk, cola_free); every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import Simulation, cola_device_bytes


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
    stream: object
    arrival: float
    admitted: float
    bytes: int
    steps_enqueued: int = 0
    done_event: object = None


@dataclass
class ServerStats:
    results: list = field(default_factory=list)
    peak_bytes: int = 0
    peak_active: int = 0
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
                "peak_active": self.peak_active, "peak_bytes": self.peak_bytes}


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

    def simulation(self, run, stream):
        with self.torch.cuda.stream(stream):
            return Simulation(run, stream=stream)

    def step(self, sim, stream):
        with self.torch.cuda.stream(stream):
            sim.step(1)

    def pk(self, sim, stream, nbins):
        with self.torch.cuda.stream(stream):
            return sim.pk(nbins)

    def synchronize(self):
        self.torch.cuda.synchronize()


class Server:
    """Admits runs by device-memory budget and advances all admitted runs together.

    Slot streams come from a fixed pool (one per slot), so device memory freed
    by a finished run is reused by the next run on that stream.
    """

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, nbins: Optional[int] = None,
                 clock: Callable[[], float] = time.perf_counter, backend=None,
                 bytes_for: Optional[Callable] = None, steps_per_pass: int = 0):
        self.steps_per_pass = int(steps_per_pass)
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.nbins = nbins
        self.clock = clock
        self.backend = backend
        self._bytes_for = bytes_for or cola_device_bytes

    def bytes_for(self, run) -> int:
        return int(self._bytes_for(run))

    def run(self, requests, realtime: bool = True) -> ServerStats:
        """Serve (arrival_time_s, Run) requests; arrival times are relative to the start."""
        be = self.backend or _TorchBackend()
        free_streams = [be.stream() for _ in range(self.max_slots)]
        pending = deque(sorted(((float(t), i, r) for i, (t, r) in enumerate(requests)), key=lambda x: x[0]))
        for _, _, r in pending:
            if self.bytes_for(r) > self.budget:
                raise ValueError(f"request {r.name} needs more than the whole HBM budget")
        waiting: deque = deque()
        active: list[_Slot] = []
        used = 0
        stats = ServerStats()
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and (pending[0][0] <= now or not realtime):
                waiting.append(pending.popleft())
            # admission: FIFO, by memory budget and free slots
            while waiting and len(active) < self.max_slots:
                t_arr, rid, run = waiting[0]
                need = self.bytes_for(run)
                if used + need > self.budget:
                    break
                waiting.popleft()
                stream = free_streams.pop()
                sim = be.simulation(run, stream)
                used += need
                active.append(_Slot(rid, run, sim, stream, t_arr, self.clock() - t0, need))
            stats.peak_bytes = max(stats.peak_bytes, used)
            stats.peak_active = max(stats.peak_active, len(active))
            # enqueue steps of every active run that still has steps to enqueue
            for sl in active:
                left = sl.run.nsteps - sl.steps_enqueued
                todo = left if self.steps_per_pass <= 0 else min(left, self.steps_per_pass)
                for _ in range(todo):
                    be.step(sl.sim, sl.stream)
                    sl.steps_enqueued += 1
                if todo and sl.steps_enqueued == sl.run.nsteps:
                    sl.done_event = be.event(sl.stream)
            # retire finished runs
            still = []
            for sl in active:
                if sl.done_event is not None and sl.done_event.query():
                    k, pk, nm = be.pk(sl.sim, sl.stream, self.nbins)
                    sl.sim.close()
                    free_streams.append(sl.stream)
                    used -= sl.bytes
                    stats.results.append(Result(sl.rid, sl.run, k, pk, nm, sl.arrival, sl.admitted,
                                                self.clock() - t0))
                else:
                    still.append(sl)
            active = still
            if not active and waiting == deque() and pending and realtime:
                time.sleep(max(0.0, min(0.01, pending[0][0] - (self.clock() - t0))))
        be.synchronize()
        stats.wall_s = self.clock() - t0
        stats.results.sort(key=lambda r: r.rid)
        return stats
