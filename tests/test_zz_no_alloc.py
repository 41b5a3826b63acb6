"""The allocation-free entry point, ohm_count_rays_noalloc, against the
allocating path.

Callers that cannot allocate device memory when they integrate rays (code
inside CUDA-graph stream capture, real-time loops that must not wait on the
allocator, plug-ins whose host owns all device memory) count rays into their
own dense grids through this entry point; its working memory is a static
array inside the library.  Here its counts must equal, voxel for voxel, the
hit/miss counts ohm_integrate_rays keeps in a map's counts layer, after each
of two calls in a row (the second call reuses the static array the first one
left behind).  This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2206_06079_gb300 import ohm, synth, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _grid_points(grid):
    dx, dy, dz = grid["dims"]
    z, y, x = torch.meshgrid(torch.arange(dz), torch.arange(dy), torch.arange(dx), indexing="ij")
    v = torch.stack([x, y, z], -1).reshape(-1, 3).double() + torch.tensor(grid["corner"]).double() + 0.5
    return (v * grid["voxel_size"] + torch.tensor(grid["map_origin"]).double()).float().cuda()


def test_noalloc_counts_equal_the_counts_layer_on_two_calls():
    vs = 0.1
    grid = dict(voxel_size=vs, map_origin=(0.0, 0.0, 0.0), frac_bits=16, segment_steps=0, max_range=20.0,
                corner=(-56, -45, -6), dims=(112, 90, 52))
    n_cells = int(np.prod(grid["dims"]))
    hits = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    misses = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    gm = ohm.Map(**W.room_params(layers=W.COUNTS, max_rays=32768))
    pts = _grid_points(grid)
    scans = [synth.room_scan(seed=71, n=30000), synth.fuzz_rays(72, 20000, extent=4.0)]
    for k, rays in enumerate(scans):
        o, e, f = rays.origins.cuda(), rays.endpoints.cuda(), rays.flags.cuda()
        ohm.count_rays_noalloc(grid, o, e, f, hits, misses)
        gm.integrate(o, e, f)
        torch.cuda.synchronize()
        ref = gm.query(pts, counts=True)["counts"]  # (hits, misses) per grid cell
        assert torch.equal(hits, ref[:, 0]), "hit counts differ after call %d" % (k + 1)
        assert torch.equal(misses, ref[:, 1]), "miss counts differ after call %d" % (k + 1)
        assert int(misses.sum()) > 0 and int(hits.sum()) > 0


def test_noalloc_rejects_what_it_cannot_hold():
    grid = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16, segment_steps=0, max_range=20.0,
                corner=(0, 0, 0), dims=(8, 8, 8))
    h = torch.zeros(512, dtype=torch.int32, device="cuda")
    m = torch.zeros(512, dtype=torch.int32, device="cuda")
    big = torch.zeros((ohm.NOALLOC_MAX_RAYS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ohm.OhmError) as ei:
        ohm.count_rays_noalloc(grid, big[:1], big, None, h, m)
    assert ei.value.code == ohm.ERR_INVALID and "OHM_NOALLOC_MAX_RAYS" in str(ei.value)
    with pytest.raises(ohm.OhmError):  # host buffers: the call would need staging memory
        ohm.count_rays_noalloc(grid, np.zeros((1, 3), np.float32), np.ones((4, 3), np.float32), None, h, m)
    far = dict(grid, max_range=60.0)   # 32768 rays x 10 segments would not fit the static table
    e = torch.zeros((ohm.NOALLOC_MAX_RAYS, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ohm.OhmError):
        ohm.count_rays_noalloc(far, e[:1], e, None, h, m)


def test_noalloc_wrapper_checks_caller_buffers():
    """The C entry point cannot see the sizes of caller buffers; the binding
    rejects short, strided or wrongly typed outputs and short flags before
    anything is enqueued."""
    grid = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16, segment_steps=0, max_range=20.0,
                corner=(0, 0, 0), dims=(8, 8, 8))
    rays = synth.room_scan(seed=5, n=64)
    o, e = rays.origins.cuda(), rays.endpoints.cuda()
    ok = torch.zeros(512, dtype=torch.int32, device="cuda")
    bad_outputs = [torch.zeros(511, dtype=torch.int32, device="cuda"),            # short
                   torch.zeros(1024, dtype=torch.int32, device="cuda")[::2],       # strided
                   torch.zeros(512, dtype=torch.int64, device="cuda"),             # 64-bit
                   torch.zeros(512, dtype=torch.int32)]                            # host
    for bad in bad_outputs:
        for args in ((bad, ok), (ok, bad)):
            with pytest.raises(ohm.OhmError) as ei:
                ohm.count_rays_noalloc(grid, o, e, None, *args)
            assert ei.value.code == ohm.ERR_INVALID
    with pytest.raises(ohm.OhmError) as ei:
        ohm.count_rays_noalloc(grid, o, e, torch.zeros(63, dtype=torch.uint8, device="cuda"), ok, ok.clone())
    assert ei.value.code == ohm.ERR_INVALID and "flags" in str(ei.value)
    assert int(ok.abs().sum()) == 0  # nothing ran
