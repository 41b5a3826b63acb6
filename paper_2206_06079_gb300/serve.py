"""A request loop that serves scans from many robots into resident maps.

Scans arrive over time (each robot has its own map).  The loop keeps one
FIFO queue per map and runs continuous batching: it launches one batched step
(ohm.Batch, one kernel launch per stage for all maps, replayed from a CUDA
graph) with the oldest waiting scan of every map that has one, and it keeps
`depth` steps in flight: step k + 1 is enqueued before the host waits for
step k, so the device never idles on host bookkeeping, and scans that arrive
while steps run join the next step.  Per map the scans are integrated one at
a time in arrival order, so every map ends exactly as if its robot's scans had
been integrated alone, in order.

Each step's per-map status is read back asynchronously (ohm_map_status_async
into pinned host memory) behind the step.  A map whose step failed has its
status latched, which makes its later in-flight steps no-ops (the batch
kernels skip a map whose status is set); the loop then drains the pipeline,
repairs the map and integrates that map's in-flight scans again, in order.

Memory admission: each map's region pool is its share of the HBM cap (the
pools are allocated when the maps are made, so the cap is a pool size), and
an optional per-map budget evicts down to 3/4 of it every few steps.  A
scan that needs more regions than its map has free fails with
OHM_ERR_CAPACITY and changes nothing; the loop moves the least recently used
quarter of that map's regions to pinned host memory (ohm.Map.evict) and
integrates the scan again.  A scan that reaches regions evicted earlier fails
with OHM_ERR_EVICTED; the loop restores them (ohm.Map.restore_pending) and
integrates it again.

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
    capacity_faults: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": len(self.latencies_ms), "rays": self.rays, "steps": self.steps,
                "rays_per_s": self.rays / self.wall_s if self.wall_s else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "max": float(lat.max()), "mean": float(lat.mean())},
                "evicted_regions": self.evicted_regions, "restored_regions": self.restored_regions,
                "faults": self.faults, "capacity_faults": self.capacity_faults, "wall_s": self.wall_s}


class ServeLoop:
    def __init__(self, maps, stream=None, graph=True, depth=2, budget_regions=None, budget_every=8):
        """budget_regions: optionally also keep at most that many regions of
        each map resident, checked every `budget_every` steps (the check waits
        for the steps in flight); without it the maps' pools alone bound their
        residency."""
        self.budget = budget_regions
        self.budget_every = max(1, int(budget_every))
        self.maps = list(maps)
        self.batch = ohm.Batch(self.maps)
        self.stream = stream or torch.cuda.Stream()
        self.graph = graph
        self.depth = max(1, int(depth))
        self.queues = [collections.deque() for _ in self.maps]
        self.stats = ServeStats()
        self._visible = {}
        n = len(self.maps)
        self._status = torch.zeros((self.depth, n), dtype=torch.int32).pin_memory()
        self._done = [torch.cuda.Event() for _ in range(self.depth)]
        self._inflight = collections.deque()   # (slot, heads)
        self._slot = 0

    def _enqueue(self) -> bool:
        """Launch one batched step with the oldest waiting scan of each map."""
        if len(self._inflight) >= self.depth:
            return False
        heads = [q.popleft() if q else None for q in self.queues]
        if all(h is None for h in heads):
            return False
        slot = self._slot
        self._slot = (slot + 1) % self.depth
        with torch.cuda.stream(self.stream):
            self.batch.integrate([h.rays if h is not None else None for h in heads], graph=self.graph)
            for i, h in enumerate(heads):
                if h is not None:
                    self.maps[i].status_async(self._status[slot, i:i + 1], stream=self.stream)
        self._done[slot].record(self.stream)
        self._inflight.append((slot, heads))
        return True

    def _repair(self, i, err):
        """Map i failed (error code `err`, already cleared) on its scan of
        the oldest in-flight step; its scans in later in-flight steps were
        no-ops.  Free or restore regions and integrate all of them again, in
        order; returns the requests integrated."""
        m = self.maps[i]
        msg = ""
        todo = [h[i] for _, h in self._inflight if h[i] is not None]
        for r in todo:
            # a repeat either restores what it reached or frees room; a later
            # no-op step of the map cleared the failed call's restore list, so
            # it may take a repeat to ask for those regions again
            n_capacity, emptied = 0, False
            for _ in range(16):
                if err == ohm.ERR_EVICTED:
                    self.stats.faults += 1
                    self.stats.restored_regions += m.restore_pending(self.stream)
                elif err == ohm.ERR_CAPACITY:
                    # make room, then bring back what the failed call asked for:
                    # a call can run out of slots and reach evicted regions at
                    # once (the status reports the capacity failure).  Evict
                    # the least recently used quarter; after three such
                    # faults move every region out, so that the repeats bring
                    # back only what this scan touches.  A capacity fault on
                    # a pool holding nothing else means the scan alone does
                    # not fit.
                    self.stats.capacity_faults += 1
                    n_capacity += 1
                    if emptied:
                        raise ohm.OhmError(err, "served scan alone needs more regions than map %d's pool (%s)"
                                           % (i, msg))
                    resident, _ = m.residency(self.stream)
                    keep = resident * 3 // 4 if n_capacity < 3 else 0
                    emptied = keep == 0
                    self.stats.evicted_regions += m.evict(keep, self.stream)
                    self.stats.restored_regions += m.restore_pending(self.stream)
                elif err is not None:
                    raise ohm.OhmError(err, "served scan failed (%s)" % msg)
                try:
                    with torch.cuda.stream(self.stream):
                        m.integrate(*r.rays, stream=self.stream, sync=False)
                    m.sync(self.stream)
                    err = None
                    break
                except ohm.OhmError as e:
                    err, msg = e.code, str(e)
            else:
                raise ohm.OhmError(err, "served scan could not be integrated (%s)" % msg)
        return todo

    def _complete(self, r, now):
        r.done = now
        self.stats.latencies_ms.append(1e3 * (r.done - self._visible.get(id(r), r.arrival)))
        self.stats.rays += r.n

    def _retire(self, t0):
        """Wait for the oldest in-flight step and complete its scans."""
        slot, heads = self._inflight[0]
        self._done[slot].synchronize()
        st = self._status[slot].tolist()
        failed = [i for i, h in enumerate(heads) if h is not None and st[i] != 0]
        early = []
        if failed:
            self.stream.synchronize()  # drain: the later in-flight steps have run
            for i in failed:
                code = None
                try:
                    self.maps[i].sync(self.stream)
                except ohm.OhmError as e:
                    code = e.code
                done = self._repair(i, code)
                early += done[1:]
                # those scans are integrated now: later steps must not count them
                for _, hs in list(self._inflight)[1:]:
                    hs[i] = None
        self._inflight.popleft()
        now = time.perf_counter() - t0
        for r in heads:
            if r is not None:
                self._complete(r, now)
        for r in early:
            self._complete(r, now)
        self.stats.steps += 1
        if self.budget is not None and self.stats.steps % self.budget_every == 0:
            for m in self.maps:
                resident, _ = m.residency(self.stream)  # waits for the steps in flight
                if resident > self.budget:
                    self.stats.evicted_regions += m.evict(int(self.budget * 0.75), self.stream)

    def run(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival).  realtime: requests become
        visible at their arrival times on the wall clock; otherwise all are
        visible at once (arrival 0) and the loop runs as fast as it can."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        visible = [r.arrival if realtime else 0.0 for r in reqs]
        t0 = time.perf_counter()
        k = 0
        while k < len(reqs) or any(self.queues) or self._inflight:
            now = time.perf_counter() - t0
            while k < len(reqs) and visible[k] <= now:
                self._visible[id(reqs[k])] = visible[k]
                self.queues[reqs[k].map_index].append(reqs[k])
                k += 1
            if self._enqueue():
                continue
            if self._inflight:
                self._retire(t0)
            elif k < len(reqs):
                time.sleep(max(0.0, min(0.0005, visible[k] - now)))
        self.stats.wall_s = time.perf_counter() - t0
        return self.stats


def poisson_times(rate_hz: float, duration_s: float, rng) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate on [0, duration)."""
    n = rng.poisson(rate_hz * duration_s * 1.2 + 10)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    return t[t < duration_s]
