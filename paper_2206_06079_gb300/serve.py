"""A request loop that serves scans from many robots into resident maps.

Scans arrive over time (each robot has its own map).  The loop keeps one
FIFO queue per map and runs continuous batching: whenever the device is free
it launches one batched step (ohm.Batch, one kernel launch per stage for all
maps, replayed from a CUDA graph) with the oldest waiting scan of every map
that has one, so scans that arrived while the previous step was running join
the next step and the work of different robots overlaps on the device.  Per
map the scans are integrated one at a time in arrival order, so every map ends
exactly as if its robot's scans had been integrated alone, in order.

Memory admission: each map may keep at most `budget_regions` regions resident;
before a step, a map above its budget moves its least recently used regions to
pinned host memory (ohm.Map.evict).  A scan that reaches evicted regions makes
its map's step a no-op (OHM_ERR_EVICTED); the loop restores those regions and
integrates that scan again before the map's next scan.

Latency of a scan = completion of the step that integrated it (observed on the
host) minus its arrival time.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ohm


@dataclass
class Request:
    map_index: int
    arrival: float                 # seconds since the start of the run
    rays: tuple                    # (origins, endpoints, flags) CUDA tensors
    kind: str = ""
    done: float = float("nan")     # completion time, seconds since the start

    @property
    def n(self) -> int:
        return int(self.rays[1].shape[0])


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    rays: int = 0
    steps: int = 0
    evicted_regions: int = 0
    restored_regions: int = 0
    faults: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": len(self.latencies_ms), "rays": self.rays, "steps": self.steps,
                "rays_per_s": self.rays / self.wall_s if self.wall_s else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "max": float(lat.max()), "mean": float(lat.mean())},
                "evicted_regions": self.evicted_regions, "restored_regions": self.restored_regions,
                "faults": self.faults, "wall_s": self.wall_s}


class ServeLoop:
    def __init__(self, maps, budget_regions=None, stream=None, graph=True):
        self.maps = list(maps)
        self.batch = ohm.Batch(self.maps)
        self.stream = stream or torch.cuda.Stream()
        self.graph = graph
        self.budget = budget_regions
        self.queues = [collections.deque() for _ in self.maps]
        self.stats = ServeStats()
        self._visible = {}

    def _admit_memory(self):
        if self.budget is None:
            return
        for m in self.maps:
            resident, _ = m.residency(self.stream)
            if resident > self.budget:
                self.stats.evicted_regions += m.evict(int(self.budget * 0.75), self.stream)

    def _step(self, t0):
        heads = [q[0] if q else None for q in self.queues]
        sets = [r.rays if r is not None else None for r in heads]
        self._admit_memory()
        with torch.cuda.stream(self.stream):
            self.batch.integrate(sets, graph=self.graph)
        self.stream.synchronize()
        faulted = []
        for i, m in enumerate(self.maps):
            if heads[i] is None:
                continue
            try:
                m.sync(self.stream)
            except ohm.OhmError as err:
                if err.code != ohm.ERR_EVICTED:
                    raise
                faulted.append(i)
        for i in faulted:
            # bring the regions back and integrate the scan again (synchronous path)
            self.stats.faults += 1
            self.stats.restored_regions += self.maps[i].restore_pending(self.stream)
            with torch.cuda.stream(self.stream):
                self.maps[i].integrate(*heads[i].rays, stream=self.stream, sync=True)
        now = time.perf_counter() - t0
        for i, r in enumerate(heads):
            if r is None:
                continue
            self.queues[i].popleft()
            r.done = now
            self.stats.latencies_ms.append(1e3 * (r.done - self._visible.get(id(r), r.arrival)))
            self.stats.rays += r.n
        self.stats.steps += 1

    def run(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival).  realtime: requests become
        visible at their arrival times on the wall clock; otherwise all are
        visible at once (arrival 0) and the loop runs as fast as it can."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        visible = [r.arrival if realtime else 0.0 for r in reqs]
        t0 = time.perf_counter()
        k = 0
        pending = 0
        while k < len(reqs) or pending:
            now = time.perf_counter() - t0
            while k < len(reqs) and visible[k] <= now:
                self._visible[id(reqs[k])] = visible[k]
                self.queues[reqs[k].map_index].append(reqs[k])
                k += 1
                pending += 1
            if pending:
                n_before = len(self.stats.latencies_ms)
                self._step(t0)
                pending -= len(self.stats.latencies_ms) - n_before
            elif k < len(reqs):
                time.sleep(max(0.0, min(0.0005, visible[k] - now)))
        self.stats.wall_s = time.perf_counter() - t0
        return self.stats


def poisson_times(rate_hz: float, duration_s: float, rng) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate on [0, duration)."""
    n = rng.poisson(rate_hz * duration_s * 1.2 + 10)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    return t[t < duration_s]
