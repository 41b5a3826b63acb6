"""Region cache: least recently used regions move to pinned host memory and
come back on demand (Sec. III-A GPU cache); a map that went through evictions
is bit-identical to one that never did."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_06079_gb300 import ohm, synth, workloads as W

from .parity import assert_maps_identical, compare_dense, compare_ndt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _params(**kw):
    p = dict(layers=W.OCC | W.NDT | W.COUNTS | W.DECAY | W.MEAN, max_rays=32768, max_range=20.0, max_regions=8192,
             max_ndt_regions=2048)
    p.update(kw)
    return W.tunnel_params(**p)


def _scan(i):
    r = synth.tunnel_scan(i, beams=32, azimuths=1024, max_range=20.0, step=2.0)
    return r.origins.cuda(), r.endpoints.cuda(), r.flags.cuda()


def test_evict_then_restore_all_is_identical():
    a, b = ohm.Map(**_params()), ohm.Map(**_params())
    for i in range(4):
        s = _scan(i)
        a.integrate(*s)
        b.integrate(*s)
    resident, _ = a.residency()
    moved = a.evict(100)
    assert moved == resident - 100 and a.residency() == (100, moved)
    assert a.restore_all() == moved
    assert a.residency() == (resident, 0)
    assert_maps_identical(a, b)


def test_integrating_into_evicted_regions_restores_them():
    p = _params()
    a, b = ohm.Map(**p), ohm.Map(**p)
    om = oracle.OracleMap(**W.oracle_params(p))
    for i in range(6):
        s = _scan(i)
        if i >= 2:
            a.evict(50)            # most of what the next scan needs is on the host
        a.integrate(*s)            # synchronous: restores what it touches and repeats
        b.integrate(*s)
        om.integrate(*[t.cpu().numpy() for t in s])
    a.restore_all()
    assert_maps_identical(a, b)
    compare_dense(b, om, path=True, mean=True)
    compare_ndt(b, om)


def test_async_call_reports_eviction_and_changes_nothing():
    a, b = ohm.Map(**_params()), ohm.Map(**_params())
    s0, s1 = _scan(0), _scan(1)
    for m in (a, b):
        m.integrate(*s0)
    a.evict(0)
    a.integrate(*s1, sync=False)
    with pytest.raises(ohm.OhmError) as ei:
        a.sync()
    assert ei.value.code == ohm.ERR_EVICTED
    assert a.restore_pending() > 0
    a.integrate(*s1, sync=False)
    a.sync()
    b.integrate(*s1)
    a.restore_all()
    assert_maps_identical(a, b)


def test_small_pool_under_lru_pressure():
    """Resident set kept at ~400 regions while the trajectory touches about
    four times that: every call restores what it needs from host memory."""
    a, b = ohm.Map(**_params(max_regions=3000, max_ndt_regions=3000)), ohm.Map(**_params())
    for i in range(10):
        a.evict(400)
        s = _scan(i)
        a.integrate(*s)
        b.integrate(*s)
    res, host = a.residency()
    assert host > 0
    a.restore_all()
    assert_maps_identical(a, b)


def test_full_pool_evicts_when_allowed():
    """evict_when_full: a synchronous call that finds the pool full evicts the
    least recently used regions and is repeated; the result equals a map with
    a large pool once everything is back."""
    probe = ohm.Map(**_params())
    probe.integrate(*_scan(0))
    pool = int(probe.region_count() * 1.15)  # one scan fits, three do not
    probe.close()
    small = _params(max_regions=pool, max_ndt_regions=pool, evict_when_full=1)
    a, b = ohm.Map(**small), ohm.Map(**_params())
    for i in range(3):
        s = _scan(2 * i)
        a.integrate(*s)
        b.integrate(*s)
    res, host = a.residency()
    assert b.region_count() > pool
    assert host > 0 and res <= pool
    # compare the resident part now ...
    pts = torch.cat([_scan(2 * i)[1] for i in range(3)])
    qa, qb = a.query(pts, ndt=True, counts=True), b.query(pts, ndt=True, counts=True)
    k = qa["known"] == 1
    assert int(k.sum()) > 0
    assert torch.equal(qa["occupancy"][k].view(torch.int32), qb["occupancy"][k].view(torch.int32))
    assert torch.equal(qa["counts"][k], qb["counts"][k])
    # ... then push everything out and integrate the first scan again: its
    # regions come back from host memory (others are evicted to make room)
    a.evict(0)
    assert a.residency()[0] == 0
    s0 = _scan(0)
    a.integrate(*s0)
    b.integrate(*s0)
    qa, qb = a.query(s0[1], ndt=True, counts=True), b.query(s0[1], ndt=True, counts=True)
    assert torch.equal(qa["known"], qb["known"]) and int(qa["known"].sum()) > 1000
    k = qa["known"] == 1
    assert torch.equal(qa["occupancy"][k].view(torch.int32), qb["occupancy"][k].view(torch.int32))
    assert torch.equal(qa["counts"], qb["counts"])
    assert torch.equal(qa["ndt"], qb["ndt"])


def test_without_eviction_a_full_pool_is_an_error():
    a = ohm.Map(**_params(max_regions=300, max_ndt_regions=300))
    with pytest.raises(ohm.OhmError) as ei:
        a.integrate(*_scan(0))
    assert ei.value.code == ohm.ERR_CAPACITY
    assert a.residency() == (0, 0)


def test_occupancy_ndt_map_through_repeated_eviction():
    """An occupancy + NDT map evicted down to 40 regions before each of five
    scans ends identical to one never evicted, and to the oracle."""
    p = _params(layers=W.OCC | W.NDT)
    a, b = ohm.Map(**p), ohm.Map(**p)
    om = oracle.OracleMap(**W.oracle_params(p))
    for i in range(8):
        s = _scan(i // 2)
        if i >= 3:
            a.evict(40)
        a.integrate(*s)
        b.integrate(*s)
        om.integrate(*[t.cpu().numpy() for t in s])
    a.restore_all()
    assert_maps_identical(a, b)
    compare_dense(a, om, counts=False)

