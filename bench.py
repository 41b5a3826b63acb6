#!/usr/bin/env python
"""Benchmark of ray integration on the tunnel lidar trajectory.

Workload: a spinning lidar (128 beams x 1024 azimuths = 131,072 rays per scan,
+-22.5 deg) moving 0.5 m per scan along a 200 m sinusoidal tunnel of radius
3 m; 10 % of returns missing (miss-only rays to 50 m); occupancy + NDT-OM on
0.1 m voxels in 32^3 regions.  One step = one scan integrated through the
C ABI (quantise, region allocation, segmented voxel walk with miss updates,
sample updates with NDT moments).  Scan i of the run is trajectory scan
i mod 100.

Prints one JSON line.  `--impl reference` times the sequential CPU oracle on
a bounded sample of the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s and voxel-updates/s at 0.1 m voxels on 1 GB300; p99 per-scan latency"
UNIT = "rays/s"
WORKLOAD = ("tunnel lidar trajectory: 128x1024 = 131072 rays/scan, 100-scan sinusoidal tunnel (r = 3 m, 200 m), "
            "10% missing returns to 50 m, occupancy + NDT-OM, 0.1 m voxels, 32^3 regions")
SCANS = 100
WALK_PROFILE = os.path.join(ROOT, "profiles", "walk_miss_tunnel_traffic.json")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None, period_ms=50):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=timestamp," + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", str(period_ms)]
        if bus_id:
            cmd += ["-i", bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if not self.proc:
            return []
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append(parts)
        return rows

    @staticmethod
    def summarise(rows):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, name in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(name)
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _walk_source_hash():
    h = hashlib.sha256()
    for f in ("ohm_integrate.cu", "ohm_kernels.cuh", "ohm_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2206_06079_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_per_launch(rays_per_scan):
    """DRAM bytes per walk launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    try:
        prof = json.load(open(WALK_PROFILE))
    except (OSError, ValueError):
        return None
    if prof.get("source_hash") != _walk_source_hash():
        return None
    per_ray = prof["dram_bytes_per_launch"] / float(prof["rays_per_launch"])
    return per_ray * rays_per_scan


def _reduce_over_ranks(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce_over_ranks(x, ws, dist.ReduceOp.MAX)


def _sum_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce_over_ranks(x, ws, dist.ReduceOp.SUM)


def whole_job(units, elapsed_ms, ws):
    """Whole-job throughput of replicas: the units every rank processed over
    the slowest rank's time.  Returns (total units, max ms, units per second)."""
    max_ms = _max_over_ranks(elapsed_ms, ws)
    total = _sum_over_ranks(float(units), ws)
    return total, max_ms, total / (max_ms / 1e3)


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_run(scans_host, max_seconds=25.0, stride=1):
    """Integrate host scans with the oracle until max_seconds pass; returns
    (rays, seconds, scans used)."""
    import oracle
    from paper_2206_06079_gb300 import workloads as W
    om = oracle.OracleMap(**W.oracle_params(W.tunnel_params()))
    rays = 0
    t0 = time.perf_counter()
    used = 0
    for o, e, f in scans_host:
        om.integrate(o, e[::stride], f[::stride])
        rays += len(e[::stride])
        used += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    return rays, time.perf_counter() - t0, used


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    _barrier(ws)
    __graft_entry__.build()
    from paper_2206_06079_gb300 import ohm, workloads as W

    dev = torch.device("cuda", local)
    n_steps = args.warmup + args.steps
    n_unique = min(SCANS, n_steps)
    scans = [W.tunnel_rays(i % SCANS, device=dev) for i in range(n_unique)]
    torch.cuda.synchronize()
    rays_per_scan = scans[0].n

    pools = dict(max_regions=12288, max_ndt_regions=512) if args.profile_case else {}
    if args.segment_steps:
        pools["segment_steps"] = args.segment_steps
    gm = ohm.Map(**W.tunnel_params(device=local, **pools))
    stream = torch.cuda.current_stream()

    def scan(i):
        return scans[i % n_unique]

    for i in range(args.warmup):
        s = scan(i)
        gm.integrate(s.origins, s.endpoints, s.flags, sync=False)
    gm.sync()
    st0 = gm.stats()
    # the walk's launch duration (roofline) is taken with events around it in
    # every 10th timed step: an event between two kernels ends the
    # programmatic-launch overlap there, so the other steps run without them
    gm.profile(["walk"], every=10)
    props = torch.cuda.get_device_properties(dev)
    bus = None
    if hasattr(props, "pci_bus_id"):
        bus = "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id, props.pci_device_id)
    sampler = ClockSampler(bus)
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        s = scan(args.warmup + k)
        ev[k][0].record(stream)
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    rows = sampler.stop()
    gm.sync()
    st1 = gm.stats()
    walk_ms, walk_launches = gm.profile_read("walk")
    gm.profile([])
    elapsed_ms = t_start.elapsed_time(t_end)
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    visits = st1["total_visits"] - st0["total_visits"]
    launches = st1["launches"] - st0["launches"]

    # per-stage device time (separate, untimed pass with events around every kernel)
    stage_ms = {}
    if not args.profile_case:
        gm.profile(ohm.STAGES)
        for k in range(min(args.steps, 50)):
            s = scan(args.warmup + k)
            gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
        gm.sync()
        for name in ohm.STAGES:
            ms, nl = gm.profile_read(name)
            if nl:
                stage_ms[name] = ms / nl
        gm.profile([])

    total_rays, max_ms, value = whole_job(rays_per_scan * args.steps, elapsed_ms, ws)
    total_visits = _sum_over_ranks(float(visits), ws)

    if args.profile_case:
        if rank == 0:
            print(json.dumps({"profile_case": True, "rays_per_scan": rays_per_scan, "steps": args.steps,
                              "visits_per_scan": visits / args.steps, "walk_avg_ms": walk_ms / max(walk_launches, 1),
                              "segments_last_scan": st1["segments"], "regions": st1["regions"]}), flush=True)
        return
    # ---- end to end: host (pinned) inputs copied inside each call, status read back
    host = []
    for i in range(n_unique):
        o = scans[i].origins.cpu().pin_memory()
        e = scans[i].endpoints.cpu().pin_memory()
        f = scans[i].flags.cpu().pin_memory()
        host.append((o, e, f))
    gm2 = ohm.Map(**W.tunnel_params(device=local))
    for i in range(args.warmup):
        o, e, f = host[i % n_unique]
        gm2.integrate(o, e, f)
    # each step: H2D copies of the scan from pinned memory, the kernels, and a
    # D2H read of the map's status word into a pinned slot of its own; the
    # host submits scans back to back and checks every step's status at the end
    status = torch.zeros(args.steps, dtype=torch.int32).pin_memory()
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        o, e, f = host[(args.warmup + k) % n_unique]
        gm2.integrate(o, e, f, stream=stream, sync=False)
        gm2.status_async(status[k:k + 1], stream=stream)
    gm2.sync(stream)
    e2e_s = time.perf_counter() - t0
    if int(status.abs().sum()) != 0:
        raise RuntimeError("e2e: a step reported a failure")
    _barrier(ws)
    e2e_s = _max_over_ranks(e2e_s, ws)
    e2e_value = total_rays / e2e_s
    h2d = int(host[0][0].numel() * 4 + host[0][1].numel() * 4 + host[0][2].numel())
    gm2.close()

    # ---- roofline of the dominant kernel (the voxel walk)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if not hbm:
        hbm, peak_src = 6800.0, "fallback 6.8 TB/s (of fallback)"
    walk_avg_s = (walk_ms / max(walk_launches, 1)) / 1e3
    visits_per_scan = visits / args.steps
    segs_per_scan = st1["segments"]
    algo_bytes = 8.0 * visits_per_scan + 64.0 * rays_per_scan + 8.0 * segs_per_scan
    achieved = algo_bytes / walk_avg_s / 1e9
    traffic = _traffic_per_launch(rays_per_scan)
    # the walk's second ceiling: L2 compare-and-swap throughput on random words
    # (measured here with the library's probe, outside the timed region)
    cas_per_scan = float(st1["atomics"])
    cas_peak = ohm.probe_cas_rate(local, words=1 << 28, ops=1 << 26)
    cas_achieved = cas_per_scan / walk_avg_s

    # ---- CPU baseline: the oracle, single thread, on a bounded sample of scans
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        host_np = [(h[0].numpy(), h[1].numpy(), h[2].numpy()) for h in host]
        rays_c, secs, used = cpu_oracle_run(host_np, max_seconds=args.cpu_seconds)
        cpu = {"value": rays_c / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d scans of the trajectory (%d rays), fresh map, single thread, %.1f s"
                         % (used, rays_c, secs)}

    if rank == 0:
        clocks = ClockSampler.summarise(rows)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 log-odds, i64 fixed-point walk",
            "data": "synthetic (seeded tunnel lidar scans generated on the device)",
            "config": {"workload": WORKLOAD, "rays_per_scan": rays_per_scan, "scans": SCANS,
                       "layers": "occupancy+ndt", "voxel_size_m": 0.1, "max_range_m": 50.0,
                       "segment_target_voxel_steps": args.segment_steps or 24, "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "map working set per scan (~7.7k 128 KB regions) exceeds the 129 MB L2; "
                             "each step integrates a different scan"},
            "voxel_updates_per_s": total_visits / (max_ms / 1e3),
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                           "max": lat[-1]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4},
            "gpu_launches": int(launches),
            "stages_ms": stage_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "kernel": "k_walk_miss",
                         "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": walk_avg_s * 1e3,
                         "peak_source": peak_src,
                         "atomics": {"achieved": cas_achieved, "peak": cas_peak, "unit": "CAS/s",
                                     "frac": cas_achieved / cas_peak, "per_launch": cas_per_scan,
                                     "peak_source": "ohm_probe_cas_rate: load + CAS of random 4-byte words of a "
                                                    "1 GiB buffer, 4 in flight per thread, measured in this run"}},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


MULTIMAP_KINDS = ("lidar16x1800", "lidar64x1024", "lidar128x2048", "depth424x240")


def multimap_specs(n_maps=16):
    """16 maps: tunnel / room scenes alternating, 0.1 m and 0.05 m voxels
    alternating in pairs, occupancy, 20 m range (the paper's truncation)."""
    from paper_2206_06079_gb300 import workloads as W
    specs = []
    for i in range(n_maps):
        scene = "tunnel" if i % 2 == 0 else "room"
        vs = 0.1 if (i // 2) % 2 == 0 else 0.05
        specs.append((scene, W.tunnel_params(layers=W.OCC, voxel_size=vs, max_range=20.0, max_rays=262144,
                                             max_regions=8192 if vs == 0.1 else 32768, max_ndt_regions=1)))
    return specs


def run_multimap(args):
    """Batched multi-map workload: per step every map receives one scan drawn
    uniformly from four sensor types; the single-scan path (one integrate call
    per map) against the batched path (one launch per stage for all maps,
    replayed from a CUDA graph, autotuned tiles)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_06079_gb300 import ohm, synth, tuning

    dev = torch.device("cuda", 0)
    specs = multimap_specs()
    pool = {}
    for scene in ("tunnel", "room"):
        for kind in MULTIMAP_KINDS:
            pool[(scene, kind)] = [synth.mixed_scan(scene, kind, 1000 + 17 * j + 101 * len(pool), device=dev)
                                   for j in range(3)]
    rng = np.random.default_rng(0x0A15)
    n_steps = args.warmup + args.steps
    plans = [[pool[(sc, MULTIMAP_KINDS[rng.integers(4)])][rng.integers(3)] for sc, _ in specs] for _ in range(n_steps)]
    torch.cuda.synchronize()
    steps = [[(r.origins, r.endpoints, r.flags) for r in plan] for plan in plans]
    rays = [sum(r.n for r in plan) for plan in plans]
    stream = torch.cuda.Stream()
    params = [p for _, p in specs]

    # single-scan path
    maps_a = [ohm.Map(**p) for p in params]
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            for m, rs in zip(maps_a, steps[k]):
                m.integrate(*rs, stream=stream, sync=False)
    torch.cuda.synchronize()
    launches0 = sum(m.stats()["launches"] for m in maps_a)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for k in range(args.warmup, n_steps):
            for m, rs in zip(maps_a, steps[k]):
                m.integrate(*rs, stream=stream, sync=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_a = ev0.elapsed_time(ev1)
    launches_a = sum(m.stats()["launches"] for m in maps_a) - launches0
    for m in maps_a:
        m.sync(stream)

    # batched path: tune on scratch maps, then measure
    (best_s, best_b), table = tuning.autotune_batch(params, steps[:4], stream=stream)
    maps_b = [ohm.Map(**p) for p in params]
    batch = ohm.Batch(maps_b)
    batch.tune(best_s, best_b)
    for k in range(args.warmup):
        with torch.cuda.stream(stream):
            batch.integrate(steps[k], graph=True)
    batch.sync(stream)
    st0 = batch.stats()
    ev0.record(stream)
    for k in range(args.warmup, n_steps):
        with torch.cuda.stream(stream):
            batch.integrate(steps[k], graph=True)
    ev1.record(stream)
    batch.sync(stream)
    ms_b = ev0.elapsed_time(ev1)
    st1 = batch.stats()
    same = all(a.region_count() == b.region_count() for a, b in zip(maps_a, maps_b))
    total_rays = float(sum(rays[args.warmup:]))
    out = {"metric": METRIC, "workload": "multimap", "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "value": total_rays / (ms_b / 1e3), "single_scan_value": total_rays / (ms_a / 1e3),
           "speedup_vs_single_scan": ms_a / ms_b, "ms_per_step": ms_b / args.steps,
           "single_scan_ms_per_step": ms_a / args.steps, "higher_is_better": True,
           "config": {"workload": "16 maps (tunnel/room, 0.1/0.05 m voxels), per step each map gets one scan drawn "
                                  "uniformly from 16x1800, 64x1024, 128x2048 lidar and 424x240 depth",
                      "rays_per_step_mean": total_rays / args.steps,
                      "tuned": {"segment_steps": best_s, "walk_blocks_per_sm": best_b},
                      "tuning_ms_per_step": {"%d/%d" % k: v for k, v in sorted(table.items())}},
           "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
           "graph_launches": int(st1["graph_launches"] - st0["graph_launches"]),
           "single_scan_gpu_launches": int(launches_a), "region_counts_equal": same}
    print(json.dumps(out), flush=True)


def run_tsdf(args):
    """Depth-camera TSDF workload: 640 x 480 frames (fx = fy = 525, 0.3-6 m)
    around a room with 20 boxes and 10 spheres, 0.05 m voxels, tau = 0.2 m.
    Times the forward integration (ohm_integrate_depth) per frame and, on
    the same frames, forward + adjoint (ohm_tsdf_backward against 20,000
    query voxels)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_06079_gb300 import ohm, synth, workloads as W

    dev = torch.device("cuda", 0)
    scene = synth.depth_scene()
    w, h = 640, 480
    K = (525.0, 525.0, 319.5, 239.5)
    n_frames = min(64, args.warmup + args.steps)
    frames = []
    for i in range(n_frames):
        depth, pos, R = synth.depth_frame(scene, i, width=w, height=h, device=dev)
        frames.append((depth.contiguous(), np.concatenate([R.numpy(), pos.numpy()[:, None]], 1)))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    gm = ohm.Map(**W.tsdf_params(device=0))
    for k in range(args.warmup):
        d, P = frames[k % n_frames]
        gm.integrate_depth(d, K, P, sync=False)
    gm.sync()
    st0 = gm.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        d, P = frames[(args.warmup + k) % n_frames]
        gm.integrate_depth(d, K, P, sync=False)
    e1.record(stream)
    gm.sync()
    fwd_ms = e0.elapsed_time(e1) / args.steps
    st1 = gm.stats()
    visits = (st1["total_visits"] - st0["total_visits"]) / args.steps
    # forward + adjoint
    rng = np.random.default_rng(5)
    q = torch.from_numpy(rng.uniform([-3, -3, 0], [3, 3, 3], size=(20000, 3)).astype(np.float32)).to(dev)
    gq = torch.from_numpy(rng.normal(size=20000).astype(np.float32)).to(dev)
    gm2 = ohm.Map(**W.tsdf_params(device=0))
    for k in range(args.warmup):
        d, P = frames[k % n_frames]
        gm2.integrate_depth(d, K, P, sync=False)
        gm2.tsdf_backward(d, K, P, q, gq)
    gm2.sync()
    e0.record(stream)
    for k in range(args.steps):
        d, P = frames[(args.warmup + k) % n_frames]
        gm2.integrate_depth(d, K, P, sync=False)
        gm2.tsdf_backward(d, K, P, q, gq)
    e1.record(stream)
    gm2.sync()
    fb_ms = e0.elapsed_time(e1) / args.steps
    rays = w * h
    out = {"metric": METRIC, "workload": "tsdf", "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "value": rays / (fwd_ms / 1e3), "ms_per_step": fwd_ms,
           "voxel_updates_per_s": visits / (fwd_ms / 1e3), "higher_is_better": True,
           "forward_backward_ms_per_frame": fb_ms, "backward_ms_per_frame": fb_ms - fwd_ms,
           "config": {"workload": "640x480 depth frames, 0.05 m voxels, tau 0.2 m, TSDF layer", "frames": n_frames,
                      "band_visits_per_frame": visits, "adjoint_query_voxels": 20000}}
    print(json.dumps(out), flush=True)


def run_served(args):
    """Served stream: 8 robots in a 200 x 200 m world, each with a 128 x 1024
    lidar at 10 Hz and two 424 x 240 depth cameras at 30 Hz (Poisson
    arrivals), one resident occupancy + NDT map per robot at 0.1 m, pools sized
    to a 60 GB HBM cap with least-recently-used eviction to pinned host memory;
    real-time arrivals over --duration seconds; p50 / p99 scan latency and
    sustained rays/s."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_06079_gb300 import ohm, serve, synth, workloads as W

    n_robots, duration = 8, float(args.duration)
    cap = 60e9
    per_region = 4 * 32768 + 8 * 10 * 32768          # occupancy + an NDT block
    budget = int(cap / n_robots / per_region)          # regions each map may keep resident
    pool = int(budget * 1.1)
    params = W.tunnel_params(layers=W.OCC | W.NDT, max_range=30.0, max_rays=131072, max_regions=pool,
                             max_ndt_regions=pool, evict_when_full=1)
    world = synth.world_scene()
    # scan pool: each robot's sensors sampled every 0.5 s of its path
    step_s = 0.5
    n_pose = int(duration / step_s) + 1
    pool_scans = {}
    for rb in range(n_robots):
        for j in range(n_pose):
            t = j * step_s
            for kind, cam in (("lidar128x1024", 0), ("depth424x240", 0), ("depth424x240", 1)):
                r = synth.world_scan(world, rb, t, kind, camera=cam, device="cuda", max_range=30.0, seed=rb * 7919 + j)
                pool_scans[(rb, j, kind, cam)] = (r.origins, r.endpoints, r.flags)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0x0A17)
    reqs = []
    for rb in range(n_robots):
        for kind, cam, rate in (("lidar128x1024", 0, 10.0), ("depth424x240", 0, 30.0), ("depth424x240", 1, 30.0)):
            for t in serve.poisson_times(rate, duration, rng):
                j = min(int(t / step_s), n_pose - 1)
                reqs.append(serve.Request(rb, float(t), pool_scans[(rb, j, kind, cam)], kind))
    maps = [ohm.Map(**params) for _ in range(n_robots)]
    # warm the graph and the maps with a second of traffic, untimed
    warm = serve.ServeLoop(maps, budget_regions=budget)
    warm.run([serve.Request(r.map_index, 0.0, r.rays, r.kind) for r in reqs[:: max(1, len(reqs) // 200)]],
             realtime=False)
    loop = serve.ServeLoop(maps, budget_regions=budget)
    stats = loop.run(reqs, realtime=True).summary()
    resident = sum(m.residency()[0] for m in maps)
    host = sum(m.residency()[1] for m in maps)
    offered = sum(r.n for r in reqs) / duration
    out = {"metric": METRIC, "workload": "served", "unit": UNIT, "n_gpus": 1, "value": stats["rays_per_s"],
           "offered_rays_per_s": offered, "higher_is_better": True, "latency_ms": stats["latency_ms"],
           "requests": stats["requests"], "steps": stats["steps"], "duration_s": duration,
           "evicted_regions": stats["evicted_regions"], "restored_regions": stats["restored_regions"],
           "faults": stats["faults"], "resident_regions_end": resident, "host_regions_end": host,
           "config": {"workload": "8 robots x (128x1024 lidar @10 Hz + 2 x 424x240 depth @30 Hz), Poisson arrivals, "
                                  "200 x 200 m world, occupancy + NDT at 0.1 m, 60 GB cap with LRU eviction",
                      "budget_regions_per_map": budget, "pool_regions_per_map": pool}}
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The oracle as the reference arm: rank 0 only, host cores."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import numpy as np
    import torch
    from paper_2206_06079_gb300 import workloads as W
    import oracle  # noqa: F401  (builds the oracle)

    n_steps = args.warmup + args.steps
    n_unique = min(SCANS, n_steps)
    dev = torch.device("cuda", local) if torch.cuda.is_available() else torch.device("cpu")
    full = 131072
    # keep the whole run to about a minute of oracle time (~1e5 rays/s)
    per_step = int(min(full, max(4096, 6.0e6 / n_steps)))
    stride = max(1, full // per_step)
    scans = []
    for i in range(n_unique):
        s = W.tunnel_rays(i % SCANS, device=dev)
        o, e, f = s.numpy()
        scans.append((o, e[::stride].copy(), f[::stride].copy()))
    import oracle as orc
    om = orc.OracleMap(**W.oracle_params(W.tunnel_params()))
    for i in range(args.warmup):
        o, e, f = scans[i % n_unique]
        om.integrate(o, e, f)
    t0 = time.perf_counter()
    rays = 0
    for k in range(args.steps):
        o, e, f = scans[(args.warmup + k) % n_unique]
        om.integrate(o, e, f)
        rays += len(e)
    secs = time.perf_counter() - t0
    value = rays / secs
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 log-odds, i64 fixed-point walk (CPU)",
           "data": "synthetic (seeded tunnel lidar scans)",
           "config": {"workload": WORKLOAD, "rays_per_scan": full, "scans": SCANS, "layers": "occupancy+ndt",
                      "voxel_size_m": 0.1, "max_range_m": 50.0},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "every %d-th ray of each scan (%d rays/step), single thread" % (stride, len(scans[0][1]))},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--segment-steps", type=int, default=0, help="ray segment length (0 = library default)")
    ap.add_argument("--workload", default="tunnel", choices=["tunnel", "multimap", "tsdf", "served"],
                    help="tunnel: the single-map headline; multimap: 16 maps, single-scan vs batched path; "
                         "tsdf: depth frames, forward and adjoint; served: request loop")
    ap.add_argument("--duration", type=float, default=60.0, help="served workload: seconds of arrivals")
    ap.add_argument("--profile-case", action="store_true",
                    help="small pools (a few GB on the device), no e2e or CPU leg: the case ncu captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "multimap":
        run_multimap(args)
    elif args.workload == "tsdf":
        run_tsdf(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
