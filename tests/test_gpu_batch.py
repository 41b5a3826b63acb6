"""Batched multi-map integration (one launch per stage for all maps, CUDA graph
replay) gives, map for map, exactly what the single-map path gives."""
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


def _map_specs():
    return [
        W.tunnel_params(layers=W.OCC | W.NDT, max_rays=32768, max_regions=8192, max_ndt_regions=512, max_range=20.0),
        W.tunnel_params(layers=W.OCC | W.COUNTS | W.DECAY, voxel_size=0.05, max_rays=32768, max_regions=8192,
                        max_range=20.0),
        W.room_params(layers=W.DECAY, max_rays=32768),
        W.tsdf_params(layers=W.TSDF, max_rays=160 * 120),
        W.room_params(layers=W.OCC | W.COUNTS | W.NDT | W.MEAN, max_rays=32768, voxel_size=0.05, max_regions=4096),
        W.tsdf_params(layers=W.TSDF | W.OCC, max_rays=160 * 120),
    ]


def _rays_for(spec_index, step):
    k = spec_index
    if k in (0, 1):
        return synth.tunnel_scan(step * 3 + k, beams=32, azimuths=1024, max_range=20.0)
    if k in (2, 4):
        return synth.room_scan(seed=500 + 10 * k + step, n=20000 + 3000 * step)
    return W.tsdf_rays(step * 5 + k, width=160, height=120)


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single_map_path(graph):
    specs = _map_specs()
    batched = [ohm.Map(**p) for p in specs]
    single = [ohm.Map(**p) for p in specs]
    batch = ohm.Batch(batched)
    stream = torch.cuda.Stream()
    for step in range(4):
        sets = []
        for k in range(len(specs)):
            if (step + k) % 4 == 3:
                sets.append(None)  # this map gets no rays this step
                continue
            r = _rays_for(k, step).to("cuda")
            sets.append((r.origins, r.endpoints, r.flags))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            batch.integrate(sets, graph=graph)
        batch.sync(stream)
        for m, rs in zip(single, sets):
            if rs is not None:
                m.integrate(*rs)
    torch.cuda.synchronize()
    for a, b in zip(batched, single):
        assert_maps_identical(a, b)
    st = batch.stats()
    assert st["graph_launches"] == (4 if graph else 0)


def test_batch_tuning_keeps_results_and_matches_oracle():
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT, max_rays=8192)
    maps = [ohm.Map(**p) for _ in range(3)]
    refs = [oracle.OracleMap(**W.oracle_params(p)) for _ in range(3)]
    batch = ohm.Batch(maps)
    stream = torch.cuda.Stream()
    for step, (S, blocks) in enumerate([(0, 0), (1, 1), (13, 2), (4, 0)]):
        batch.tune(S, blocks)
        sets = []
        for k in range(3):
            r = synth.fuzz_rays(900 + 10 * step + k, 6000)
            refs[k].integrate(*r.numpy())
            r = r.to("cuda")
            sets.append((r.origins, r.endpoints, r.flags))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            batch.integrate(sets, graph=True)
        batch.sync(stream)
    for gm, om in zip(maps, refs):
        compare_dense(gm, om)
        compare_ndt(gm, om)


def test_batch_failure_is_isolated_to_its_map():
    ok_p = W.room_params(layers=W.OCC | W.COUNTS, max_rays=32768)
    small_p = W.room_params(layers=W.OCC | W.COUNTS, max_rays=32768, max_regions=8)
    good, bad = ohm.Map(**ok_p), ohm.Map(**small_p)
    ref = ohm.Map(**ok_p)
    batch = ohm.Batch([good, bad])
    r = W.room_rays(3).to("cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        batch.integrate([(r.origins, r.endpoints, r.flags), (r.origins, r.endpoints, r.flags)], graph=True)
    with pytest.raises(ohm.OhmError) as ei:
        batch.sync(stream)
    assert ei.value.code == ohm.ERR_CAPACITY
    assert bad.region_count() == 0
    ref.integrate(r.origins, r.endpoints, r.flags)
    assert_maps_identical(good, ref)
