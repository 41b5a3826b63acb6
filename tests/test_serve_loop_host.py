"""Host logic of the serving loop (ServeLoop), no GPU.

The loop's queues, its two steps in flight, the read-back of each step's
per-map status and the drain-repair-repeat path run against fake maps that
keep the library's failure contract: a call that fails changes nothing and
latches the map's status; while the status is latched every later call of
that map is a no-op; Map.sync reports the latched error and clears it.
Each scripted fault fails one attempt of one scan.  The check is the
served-stream property: each map ends
with exactly its own scans, each applied once, in arrival order, whatever
failed on the way.
"""
import contextlib

import numpy as np
import pytest
import torch

from paper_2206_06079_gb300 import ohm, serve


class FakeStream:
    def synchronize(self):
        pass


class FakeEvent:
    def record(self, stream=None):
        pass

    def synchronize(self):
        pass


class FakeMap:
    """failures: {scan id: [error codes of its first attempts]}: attempt k of
    that scan fails with the k-th code (whatever the loop did in between),
    later attempts succeed."""

    def __init__(self, failures=None):
        self.failures = {k: list(v) for k, v in (failures or {}).items()}
        self.applied = []
        self.status = 0
        self.resident = 100

    def _call(self, scan):
        if self.status:
            return  # latched: a no-op, like the kernels of a failed map
        codes = self.failures.get(scan)
        if codes:
            self.status = codes.pop(0)
            return
        self.applied.append(scan)

    def integrate(self, origins, endpoints, flags=None, stream=None, sync=True):
        self._call(origins)
        if sync:
            self.sync(stream)

    def sync(self, stream=None):
        if self.status:
            code, self.status = self.status, 0
            raise ohm.OhmError(code, "fake failure")

    def status_async(self, out, stream=None):
        out[0] = self.status

    def residency(self, stream=None):
        return self.resident, 0

    def evict(self, keep, stream=None):
        moved = max(0, self.resident - keep)
        self.resident -= moved
        return moved

    def restore_pending(self, stream=None):
        return 1


class FakeBatch:
    def __init__(self, maps):
        self.maps = maps

    def integrate(self, raysets, stream=None, graph=True):
        for m, r in zip(self.maps, raysets):
            if r is not None:
                m._call(r[0])


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(ohm, "Batch", FakeBatch)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s=None: contextlib.nullcontext())
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)


def _requests(n_maps, per_map, rng):
    reqs = []
    for i in range(n_maps):
        t = np.sort(rng.uniform(0.0, 1.0, per_map))
        for j in range(per_map):
            reqs.append(serve.Request(i, float(t[j]), ("m%d-s%d" % (i, j), np.zeros((3, 3)), None)))
    return reqs


def _check_served(maps, reqs, stats):
    for i, m in enumerate(maps):
        want = [r.rays[0] for r in sorted(reqs, key=lambda r: r.arrival) if r.map_index == i]
        assert m.applied == want, i
    assert len(stats.latencies_ms) == len(reqs)
    assert all(np.isfinite(r.done) for r in reqs)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_every_map_gets_its_scans_once_in_arrival_order(fake_gpu, depth):
    rng = np.random.default_rng(depth)
    maps = [FakeMap() for _ in range(5)]
    reqs = _requests(5, 12, rng)
    loop = serve.ServeLoop(maps, stream=FakeStream(), depth=depth)
    stats = loop.run(reqs, realtime=False)
    _check_served(maps, reqs, stats)
    assert stats.faults == 0 and stats.capacity_faults == 0


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_failed_steps_are_repaired_and_repeated_in_order(fake_gpu, depth):
    rng = np.random.default_rng(10 + depth)
    E, C = ohm.ERR_EVICTED, ohm.ERR_CAPACITY
    maps = [
        FakeMap({"m0-s3": [C]}),                       # one capacity fault
        FakeMap({"m1-s0": [E], "m1-s7": [E, E]}),      # evicted regions, once and twice in a row
        FakeMap({"m2-s5": [C, E, C]}),                 # mixed faults on one scan
        FakeMap(),                                     # never fails: untouched by the others' repairs
        FakeMap({"m4-s11": [C]}),                      # the map's last scan
    ]
    reqs = _requests(5, 12, rng)
    loop = serve.ServeLoop(maps, stream=FakeStream(), depth=depth)
    stats = loop.run(reqs, realtime=False)
    _check_served(maps, reqs, stats)
    assert stats.capacity_faults == 4 and stats.faults == 4   # every failed attempt is counted once
    assert stats.evicted_regions > 0 and stats.restored_regions >= 4


def test_a_scan_that_never_fits_is_reported(fake_gpu):
    """Capacity faults that eviction cannot cure end the run with an error
    naming the map, instead of looping."""
    rng = np.random.default_rng(3)
    maps = [FakeMap({"m0-s2": [ohm.ERR_CAPACITY] * 50}), FakeMap()]
    loop = serve.ServeLoop(maps, stream=FakeStream(), depth=2)
    with pytest.raises(ohm.OhmError, match="map 0"):
        loop.run(_requests(2, 4, rng), realtime=False)
