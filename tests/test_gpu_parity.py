"""GPU path (through the C ABI) against the oracle on seeded inputs.

Bar: voxel traversal bit-exact (region sets, per-voxel hit/miss counts, NDT
integer moments), log-odds bit-exact (both sides apply the same FP32 clamped
updates in the same per-call order), NDT mean/covariance within 1e-4
relative, TSDF distance within 1e-5 m absolute and weights exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_06079_gb300 import ohm, synth, workloads as W

from .parity import assert_maps_identical, compare_dense, compare_ndt, compare_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _pair(params):
    gm = ohm.Map(**params)
    om = oracle.OracleMap(**W.oracle_params(params))
    return gm, om


def _integrate_both(gm, om, rays, device_inputs=True):
    o, e, f = rays.numpy()
    if device_inputs:
        gm.integrate(rays.origins.cuda(), rays.endpoints.cuda(), rays.flags.cuda())
    else:
        gm.integrate(o, e, f)
    return om.integrate(o, e, f)


def _sample_points(rays, k=20000, seed=0):
    o, e, f = rays.numpy()
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(e), size=min(k, len(e)))
    t = rng.uniform(0, 1.05, size=(len(idx), 1))
    oo = o[0] if len(o) == 1 else o[idx]
    return np.concatenate([e[idx], oo + t * (e[idx] - oo)]).astype(np.float32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fuzz_rays_all_layers(seed):
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT, max_regions=4096, max_rays=4096, max_range=2.5)
    gm, om = _pair(p)
    for scan in range(3):
        rays = synth.fuzz_rays(seed * 100 + scan, 3000)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om)
    compare_ndt(gm, om)
    compare_query(gm, om, _sample_points(rays), ndt=True)


@pytest.mark.parametrize("steps", [1, 3, 17, 64, 100000])
def test_segment_split_never_changes_the_walk(steps):
    """Segments (Sec. III-B) are a scheduling device: every split reproduces
    the unsplit walk exactly."""
    p = W.tunnel_params(layers=W.OCC | W.COUNTS, segment_steps=steps, max_rays=16384, max_regions=16384)
    gm, om = _pair(p)
    for i in range(2):
        rays = synth.tunnel_scan(i, beams=16, azimuths=1024)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om)


def test_room_scan_full_size():
    p = W.room_params(layers=W.OCC | W.COUNTS)
    gm, om = _pair(p)
    rays = W.room_rays(0)
    visits = _integrate_both(gm, om, rays)
    assert gm.stats()["visits"] == visits
    compare_dense(gm, om)
    compare_query(gm, om, _sample_points(rays))


def test_tunnel_scans_full_size_occupancy_ndt():
    """The tunnel workload's map parameters and launch configuration, three
    full 131,072-ray scans, every layer compared."""
    p = W.tunnel_params(layers=W.OCC | W.NDT | W.COUNTS)
    gm, om = _pair(p)
    for i in range(3):
        rays = W.tunnel_rays(i)
        visits = _integrate_both(gm, om, rays)
        st = gm.stats()
        assert st["visits"] == visits and st["rays"] == rays.n
    compare_dense(gm, om, batch=512)
    nsamp, _ = compare_ndt(gm, om)
    assert nsamp > 10000
    compare_query(gm, om, _sample_points(rays), ndt=True)


def test_tunnel_bench_layers_query_parity():
    """Bench layers (occupancy + NDT, no counts): sampled outputs via query."""
    p = W.tunnel_params()
    gm, om = _pair(p)
    for i in range(2):
        rays = W.tunnel_rays(10 + i)
        _integrate_both(gm, om, rays)
    assert gm.region_count() == om.region_count()
    compare_query(gm, om, _sample_points(rays, k=50000), ndt=True)
    compare_ndt(gm, om)


@pytest.mark.parametrize("size", [(160, 120), (640, 480)])
def test_tsdf_frames(size):
    w, h = size
    p = W.tsdf_params(max_rays=w * h)
    gm, om = _pair(p)
    scene = synth.depth_scene()
    for i in range(3):
        rays = W.tsdf_rays(i * 7, width=w, height=h, scene=scene)
        visits = _integrate_both(gm, om, rays)
        assert gm.stats()["visits"] == visits
    n = compare_dense(gm, om, occupancy=False, counts=False, tsdf=True, tsdf_atol=1e-5)
    assert n > 0


def test_occupancy_and_tsdf_in_one_map():
    p = W.tsdf_params(layers=W.OCC | W.TSDF | W.COUNTS, max_rays=160 * 120)
    gm, om = _pair(p)
    rays = W.tsdf_rays(3, width=160, height=120)
    _integrate_both(gm, om, rays)
    compare_dense(gm, om, occupancy=True, counts=True, tsdf=True)


def test_host_inputs_match_device_inputs():
    p = W.room_params(layers=W.OCC | W.COUNTS)
    a = ohm.Map(**p)
    b = ohm.Map(**p)
    rays = W.room_rays(1)
    o, e, f = rays.numpy()
    a.integrate(o, e, f)
    b.integrate(rays.origins.cuda(), rays.endpoints.cuda(), rays.flags.cuda())
    ea, eb = a.export(counts=True), b.export(counts=True)
    ka, kb = ea["keys"].cpu().numpy(), eb["keys"].cpu().numpy()
    oa, ob = np.lexsort(ka.T[::-1]), np.lexsort(kb.T[::-1])
    assert np.array_equal(ka[oa], kb[ob])
    assert torch.equal(ea["occupancy"][torch.from_numpy(oa).cuda()].view(torch.int32),
                       eb["occupancy"][torch.from_numpy(ob).cuda()].view(torch.int32))


def test_repeat_runs_are_bit_identical():
    p = W.tunnel_params(layers=W.OCC | W.COUNTS | W.NDT, max_rays=32768)
    outs = []
    for _ in range(2):
        gm = ohm.Map(**p)
        for i in range(2):
            r = synth.tunnel_scan(i, beams=32, azimuths=1024)
            gm.integrate(r.origins.cuda(), r.endpoints.cuda(), r.flags.cuda())
        ex = gm.export(counts=True, ndt=False)
        k = ex["keys"].cpu().numpy()
        o = torch.from_numpy(np.lexsort(k.T[::-1])).cuda()
        outs.append((k[o.cpu().numpy()], ex["occupancy"][o].view(torch.int32).cpu(), ex["counts"][o].cpu()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1]) and torch.equal(outs[0][2], outs[1][2])


def test_per_ray_origins_and_async_sync():
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT, max_rays=8192)
    gm, om = _pair(p)
    rng = np.random.default_rng(5)
    o = rng.uniform(-1, 1, size=(8000, 3)).astype(np.float32)
    e = (o + rng.normal(size=(8000, 3)) * 3).astype(np.float32)
    f = (rng.uniform(size=8000) < 0.1).astype(np.uint8)
    gm.integrate(torch.from_numpy(o).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda(), sync=False)
    gm.integrate(torch.from_numpy(e).cuda(), torch.from_numpy(o).cuda(), None, sync=False)
    gm.sync()
    om.integrate(o, e, f)
    om.integrate(e, o, None)
    compare_dense(gm, om)
    compare_ndt(gm, om)


def test_edge_cases():
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT | W.DECAY | W.MEAN, max_rays=64)
    gm, om = _pair(p)
    gm.integrate(np.zeros((1, 3), np.float32), np.zeros((0, 3), np.float32))  # empty ray set
    assert gm.region_count() == 0
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    e = np.array([[0.05, 0.05, 0.05],            # zero length
                  [np.nan, 0, 0],                 # skipped
                  [1e30, 0, 0],                   # beyond fixed-point range: skipped
                  [0.1, 0.1, 0.1],                # corner of the origin voxel
                  [-0.1, 0.0, 0.0],               # on faces, negative direction
                  [30.0, 0.0, 0.0],               # truncated to 20 m
                  [0.3, -0.3, 0.3]], np.float32)  # exact diagonal
    f = np.array([0, 0, 0, 0, 0, 0, 1], np.uint8)
    _integrate_both(gm, om, synth.RaySet(torch.from_numpy(o), torch.from_numpy(e), torch.from_numpy(f)))
    compare_dense(gm, om, path=True, mean=True)
    compare_ndt(gm, om)
    # all rays skipped
    bad = np.full((5, 3), np.inf, np.float32)
    gm.integrate(o, bad)
    om.integrate(o, bad)
    compare_dense(gm, om, path=True, mean=True)
    with pytest.raises(ohm.OhmError):
        gm.integrate(o, np.zeros((65, 3), np.float32))  # more than max_rays


def test_region_pool_exhaustion_leaves_map_unchanged():
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT, max_regions=40, max_ndt_regions=40)
    gm, om = _pair(p)
    small = synth.room_scan(n=2000, room_min=(-1, -1, 0), room_max=(1, 1, 2))
    _integrate_both(gm, om, small)
    before = gm.export(counts=True)
    n_before = gm.region_count()
    with pytest.raises(ohm.OhmError) as ei:
        gm.integrate(*W.room_rays(0).numpy())  # needs 48 regions
    assert ei.value.code == ohm.ERR_CAPACITY
    assert gm.region_count() == n_before
    after = gm.export(counts=True)
    assert torch.equal(before["occupancy"].view(torch.int32), after["occupancy"].view(torch.int32))
    assert torch.equal(before["counts"], after["counts"])
    # the map keeps working and still matches the oracle that never saw the failed call
    _integrate_both(gm, om, synth.room_scan(seed=9, n=2000, room_min=(-1, -1, 0), room_max=(1, 1, 2)))
    compare_dense(gm, om)
    compare_ndt(gm, om)


def test_ndt_pool_exhaustion_leaves_map_unchanged():
    p = W.room_params(layers=W.OCC | W.NDT, max_regions=1024, max_ndt_regions=4)
    gm, om = _pair(p)
    with pytest.raises(ohm.OhmError) as ei:
        gm.integrate(*W.room_rays(0).numpy())
    assert ei.value.code == ohm.ERR_CAPACITY
    assert gm.region_count() == 0
    st = gm.stats()
    assert st["ndt_regions"] == 0
    tiny = synth.room_scan(n=500, room_min=(-0.5, -0.5, 0.5), room_max=(0.5, 0.5, 1.5))
    _integrate_both(gm, om, tiny)
    compare_dense(gm, om, counts=False)
    compare_ndt(gm, om)


def test_hash_probe_limit_leaves_map_unchanged():
    """A tiny probe bound (max_probe = 1: every region key must sit in its
    home bucket) makes the bounded insertion give up as soon as two of a
    call's region keys share a bucket.  The call returns OHM_ERR_PROBE_LIMIT,
    changes nothing, and the map keeps matching the oracle that never saw it."""
    p = W.room_params(layers=W.OCC | W.COUNTS, max_regions=4096, max_probe=1)
    gm, om = _pair(p)
    tiny = synth.room_scan(n=500, room_min=(-0.5, -0.5, 0.5), room_max=(0.5, 0.5, 1.5))
    _integrate_both(gm, om, tiny)
    before = gm.export(counts=True)
    n_before = gm.region_count()
    # rays to the walls of a 40 x 40 x 10 m box pass through a few hundred of
    # the 8192 buckets' keys: a shared bucket is all but certain
    big = synth.room_scan(seed=3, n=32768, room_min=(-20, -20, -5), room_max=(20, 20, 5))
    with pytest.raises(ohm.OhmError) as ei:
        gm.integrate(*big.numpy())
    assert ei.value.code == ohm.ERR_PROBE_LIMIT
    assert gm.region_count() == n_before
    after = gm.export(counts=True)
    assert torch.equal(before["occupancy"].view(torch.int32), after["occupancy"].view(torch.int32))
    assert torch.equal(before["counts"], after["counts"])
    _integrate_both(gm, om, tiny)
    compare_dense(gm, om)


@pytest.mark.parametrize("thr", [-1.0, 0.5])
def test_ndt_sample_clearing_matches_oracle(thr):
    p = W.tunnel_params(layers=W.OCC | W.NDT | W.COUNTS, ndt_clear_below=thr, max_rays=32768, max_range=20.0,
                        max_regions=8192)
    gm, om = _pair(p)
    for i in range(4):
        rays = synth.tunnel_scan(3 * i, beams=32, azimuths=1024, max_range=20.0)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om)
    compare_ndt(gm, om)


@pytest.mark.parametrize("seed", [4, 5])
def test_decay_layer_matches_oracle(seed):
    """Decay rate (Sec. II-E): per-voxel summed path lengths bit-exact, with
    occupancy and counts (H_i) in the same map."""
    p = W.room_params(layers=W.OCC | W.COUNTS | W.DECAY, max_regions=4096, max_rays=4096, max_range=2.5)
    gm, om = _pair(p)
    for scan in range(3):
        rays = synth.fuzz_rays(seed * 100 + scan, 3000)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om, path=True)
    compare_query(gm, om, _sample_points(rays), path=True)


@pytest.mark.parametrize("steps", [1, 3, 100000])
def test_decay_layer_segment_splits(steps):
    """A segment that starts mid-ray takes its entry distance from the
    dominant axis' crossing: every split gives the unsplit sums."""
    p = W.tunnel_params(layers=W.DECAY | W.COUNTS, segment_steps=steps, max_rays=16384, max_regions=16384)
    gm, om = _pair(p)
    for i in range(2):
        rays = synth.tunnel_scan(i + 20, beams=16, azimuths=1024)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om, occupancy=False, path=True)


def test_decay_layer_tunnel_full_size():
    """The tunnel workload (131,072 rays, 50 m truncation) with the decay
    layer: sampled voxels through query, every ray's total via the export."""
    p = W.tunnel_params(layers=W.OCC | W.NDT | W.COUNTS | W.DECAY)
    gm, om = _pair(p)
    rays = W.tunnel_rays(30)
    _integrate_both(gm, om, rays)
    compare_query(gm, om, _sample_points(rays, k=50000), ndt=True, path=True)
    compare_dense(gm, om, batch=512, path=True)


@pytest.mark.parametrize("layers", ["occ_mean", "mean_only"])
def test_voxel_mean_layer_matches_oracle(layers):
    """Voxel mean (Sec. III-C): packed 10-bit means and counts bit-exact
    over several calls (the per-call update makes them order-independent)."""
    L = W.OCC | W.COUNTS | W.MEAN if layers == "occ_mean" else W.MEAN
    p = W.room_params(layers=L, max_regions=4096, max_rays=8192, max_range=2.5)
    gm, om = _pair(p)
    for scan in range(4):
        rays = synth.fuzz_rays(700 + scan, 6000)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om, occupancy=bool(L & W.OCC), counts=bool(L & W.COUNTS), mean=True)
    compare_query(gm, om, _sample_points(rays), mean=True)


def test_voxel_mean_tunnel_with_every_layer():
    p = W.tunnel_params(layers=W.OCC | W.NDT | W.COUNTS | W.DECAY | W.MEAN)
    gm, om = _pair(p)
    for i in range(2):
        rays = W.tunnel_rays(40 + i)
        _integrate_both(gm, om, rays)
    compare_query(gm, om, _sample_points(rays, k=50000), ndt=True, path=True, mean=True)
    compare_dense(gm, om, batch=512, path=True, mean=True)



def _shared_end_rays(seed, n_origins_per_ray):
    """Rays whose samples pile into a few voxels: groups of 1, 2, 31, 32, 33,
    200 and 1000 rays end inside the same voxel (jittered within it), in an
    interleaved order so that warps see groups of every size, plus rays that
    pass through those voxels to end beyond them."""
    rng = np.random.default_rng(seed)
    centres = np.array([[1.05, 0.35, 0.25], [1.15, 0.35, 0.25], [-0.85, 1.45, 0.65], [0.45, -1.25, -0.35],
                        [1.65, 1.65, 0.05], [-1.35, -0.55, 1.15], [0.05, 0.05, 1.95]])
    sizes = [1, 2, 31, 32, 33, 200, 1000]
    ends = []
    for c, k in zip(centres, sizes):
        ends.append(c + rng.uniform(-0.045, 0.045, size=(k, 3)))
        ends.append(c * 1.4 + rng.uniform(-0.02, 0.02, size=(k // 3 + 1, 3)))  # through the voxel, beyond it
    e = np.concatenate(ends)
    e = e[rng.permutation(len(e))].astype(np.float32)
    if n_origins_per_ray:
        o = rng.uniform(-0.04, 0.04, size=e.shape).astype(np.float32)
    else:
        o = np.array([[0.01, 0.02, 0.03]], np.float32)
    f = np.zeros(len(e), np.uint8)
    f[rng.uniform(size=len(e)) < 0.05] = synth.FLAG_NO_RETURN
    return synth.RaySet(torch.from_numpy(o), torch.from_numpy(e), torch.from_numpy(f))


@pytest.mark.parametrize("layers", ["occ_counts_ndt", "occ_mean"])
@pytest.mark.parametrize("per_ray_origins", [False, True])
def test_many_samples_in_one_voxel(layers, per_ray_origins):
    """Samples of many rays in one voxel: the hit kernel applies a warp's hits
    on a voxel as one n-step clamped update (saturating at l_max after a few
    hits), and the counts, NDT moments and voxel-mean sums of every sample.
    Bit-identical to the oracle's one-sample-at-a-time updates."""
    L = W.OCC | W.COUNTS | W.NDT if layers == "occ_counts_ndt" else W.OCC | W.MEAN
    p = W.room_params(layers=L, max_regions=1024, max_ndt_regions=1024, max_rays=4096, max_range=3.0)
    gm, om = _pair(p)
    for scan in range(3):
        _integrate_both(gm, om, _shared_end_rays(10 * scan + 1, per_ray_origins))
    compare_dense(gm, om, counts=layers == "occ_counts_ndt", mean=layers == "occ_mean")
    if layers == "occ_counts_ndt":
        compare_ndt(gm, om)


@pytest.mark.parametrize("steps", [1, 4, 100000])
def test_many_scans_over_saturated_space(steps):
    """Ten scans over the same stretch of tunnel drive most free voxels to the
    clamp l_min (misses then change nothing, hits still do); occupancy + NDT
    stay bit-identical to the oracle at every segment split."""
    p = W.tunnel_params(layers=W.OCC | W.NDT, segment_steps=steps, max_rays=32768, max_range=20.0,
                        max_regions=8192, max_ndt_regions=2048)
    gm, om = _pair(p)
    for i in range(10):
        rays = synth.tunnel_scan(i // 2, beams=32, azimuths=1024, max_range=20.0)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om, counts=False)
    compare_ndt(gm, om)


def test_repeated_room_scans_from_moving_origins():
    """Repeated room scans from moving origins: free voxels reach l_min, then
    samples land on some of them again; occupancy only."""
    p = W.room_params(layers=W.OCC, max_rays=32768)
    gm, om = _pair(p)
    rng = np.random.default_rng(11)
    for i in range(12):
        rays = synth.room_scan(seed=900 + i, n=20000)
        o, e, f = rays.numpy()
        shift = rng.uniform(-0.5, 0.5, size=3).astype(np.float32)
        _integrate_both(gm, om, synth.RaySet(torch.from_numpy(o + shift), torch.from_numpy(e), torch.from_numpy(f)))
    compare_dense(gm, om, counts=False)


def test_status_async_reports_each_step_without_waiting():
    p = W.room_params(layers=W.OCC | W.COUNTS, max_regions=40, max_ndt_regions=40)
    gm, om = _pair(p)
    st = torch.full((3,), -7, dtype=torch.int32).pin_memory()
    small = synth.room_scan(n=2000, room_min=(-1, -1, 0), room_max=(1, 1, 2))
    gm.integrate(small.origins.cuda(), small.endpoints.cuda(), small.flags.cuda(), sync=False)
    gm.status_async(st[0:1])
    big = W.room_rays(0)  # needs 48 regions: the call fails and changes nothing
    gm.integrate(big.origins.cuda(), big.endpoints.cuda(), big.flags.cuda(), sync=False)
    gm.status_async(st[1:2])
    torch.cuda.synchronize()
    assert int(st[0]) == 0 and int(st[1]) != 0
    with pytest.raises(ohm.OhmError) as ei:
        gm.sync()
    assert ei.value.code == ohm.ERR_CAPACITY
    gm.status_async(st[2:3])
    torch.cuda.synchronize()
    assert int(st[2]) == 0  # cleared by the sync
    om.integrate(*small.numpy())
    compare_dense(gm, om)


def test_sampled_stage_timing_changes_nothing():
    """Stage events in every third call only (ohm_map_profile_every): the
    sampled calls are the ones counted, and the map equals one built without
    any events, bit for bit."""
    p = W.room_params(layers=W.OCC | W.NDT | W.COUNTS)
    a, b = ohm.Map(**p), ohm.Map(**p)
    a.profile(["walk", "hits"], every=3)
    for i in range(10):
        r = W.room_rays(i, n=4096)
        a.integrate(r.origins.cuda(), r.endpoints.cuda(), r.flags.cuda(), sync=False)
        b.integrate(r.origins.cuda(), r.endpoints.cuda(), r.flags.cuda(), sync=False)
    a.sync()
    b.sync()
    ms, n = a.profile_read("walk")
    assert n == 4 and ms > 0.0  # calls 1, 4, 7 and 10
    assert a.profile_read("hits")[1] == 4 and a.profile_read("prepare")[1] == 0
    assert_maps_identical(a, b)


def test_async_host_inputs_back_to_back():
    """Scans submitted from pinned host memory without waiting (two staging
    slots filled on the map's copy stream) give the map built from device
    inputs, bit for bit; pageable inputs too."""
    p = W.tunnel_params(layers=W.OCC | W.NDT | W.COUNTS, max_rays=32768, max_range=20.0, max_regions=8192,
                        max_ndt_regions=2048)
    a, b = ohm.Map(**p), ohm.Map(**p)
    scans = [synth.tunnel_scan(i, beams=32, azimuths=1024, max_range=20.0) for i in range(6)]
    stream = torch.cuda.Stream()
    held = []  # inputs must stay valid until the stream has passed their call
    for i, r in enumerate(scans):
        o, e, f = r.origins, r.endpoints, r.flags
        if i % 3 != 2:
            o, e, f = o.pin_memory(), e.pin_memory(), f.pin_memory()
        held.append((o, e, f))
        with torch.cuda.stream(stream):
            a.integrate(o, e, f, stream=stream, sync=False)
    a.sync(stream)
    for r in scans:
        b.integrate(r.origins.cuda(), r.endpoints.cuda(), r.flags.cuda())
    assert_maps_identical(a, b)



@pytest.mark.parametrize("vs, F, origin", [(0.05, 8, (0.0, 0.0, 0.0)), (0.37, 12, (-3.1, 2.7, 0.55)),
                                           (0.1, 20, (101.3, -57.9, 12.01)), (0.2, 16, (0.013, -0.007, 0.0))])
def test_grid_parameters_and_map_origin(vs, F, origin):
    """Other voxel sizes, fixed-point fractions and map origins (rays placed
    around the origin, with face/edge/corner hits at the voxel pitch): every
    layer bit-exact, NDT and query values within tolerance."""
    p = W.room_params(layers=W.OCC | W.COUNTS | W.NDT | W.DECAY | W.MEAN, voxel_size=vs, frac_bits=F,
                      map_origin=origin, max_regions=512, max_ndt_regions=512, max_rays=4096,
                      max_range=30.0 * vs)
    gm, om = _pair(p)
    shift = torch.tensor(origin, dtype=torch.float32)
    for scan in range(3):
        r = synth.fuzz_rays(900 + scan + int(F), 3000, voxel=vs, extent=12 * vs)
        rays = synth.RaySet(r.origins + shift, r.endpoints + shift, r.flags)
        _integrate_both(gm, om, rays)
    compare_dense(gm, om, path=True, mean=True)
    compare_ndt(gm, om)
    compare_query(gm, om, _sample_points(rays), ndt=True, path=True, mean=True)


def test_cas_count_and_probe():
    """The walk reports the log-odds CAS operations it issued: at least one
    per voxel whose value a call changed, none for a repeated saturated ray;
    the CAS-rate probe returns a positive rate."""
    p = W.room_params(layers=W.OCC | W.COUNTS, max_rays=64)
    gm = ohm.Map(**p)
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    e = np.array([[0.95, 0.05, 0.05]], np.float32)
    gm.integrate(o, e)
    assert gm.stats()["atomics"] >= 9  # nine voxels take their first miss
    for _ in range(6):
        gm.integrate(o, e)
    assert gm.stats()["atomics"] == 0  # misses now leave l_min unchanged: no CAS
    assert ohm.probe_cas_rate(0, words=1 << 20, ops=1 << 20) > 0

