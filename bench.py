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
WALK_PROFILE = os.path.join(ROOT, "profiles", "walk_fast_tunnel_traffic.json")


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


def _stage_pass(gm, seq, warmup, stream):
    """Integrate the scans of `seq` into the fresh map `gm` with CUDA events
    around every kernel of the last len(seq) - warmup calls (on the call's
    stream).  Returns per-stage mean device ms and the mean miss-walk
    atomics of those calls."""
    from paper_2206_06079_gb300 import ohm
    for s in seq[:warmup]:
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    gm.sync(stream)
    gm.profile(ohm.STAGES)
    atomics = []
    for s in seq[warmup:]:
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
        atomics.append(gm.stats(stream)["atomics"])
    gm.sync(stream)
    stage_ms = {}
    for name in ohm.STAGES:
        ms, nl = gm.profile_read(name)
        if nl:
            stage_ms[name] = ms / nl
    gm.profile([])
    return stage_ms, sum(atomics) / max(1, len(atomics))


def _latency_pass(gm, scans, warmup, n, stream):
    """Per-call device latency (ms) of n calls after `warmup` untimed ones:
    CUDA events on the stream right before and after each call, no events
    inside a call."""
    import torch
    for k in range(warmup):
        s = scans[k % len(scans)]
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        s = scans[(warmup + k) % len(scans)]
        ev[k][0].record(stream)
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
        ev[k][1].record(stream)
    gm.sync(stream)
    return sorted(a.elapsed_time(b) for a, b in ev)


def _percentiles(lat):
    return {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
            "max": lat[-1], "samples": len(lat)}


LATENCY_WARMUP, LATENCY_SCANS = 10, 100


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
    # the latency pass needs LATENCY_WARMUP + LATENCY_SCANS distinct scans (the
    # trajectory has 100; later ones wrap around)
    n_unique = SCANS if not args.profile_case else min(SCANS, n_steps)
    scans = [W.tunnel_rays(i % SCANS, device=dev) for i in range(n_unique)]
    torch.cuda.synchronize()
    rays_per_scan = scans[0].n
    seq = [scans[i % n_unique] for i in range(n_steps)]

    pools = dict(max_regions=12288, max_ndt_regions=512) if args.profile_case else {}
    if args.segment_steps:
        pools["segment_steps"] = args.segment_steps
    params = W.tunnel_params(device=local, **pools)
    gm = ohm.Map(**params)
    stream = torch.cuda.current_stream()

    for s in seq[:args.warmup]:
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    gm.sync()
    st0 = gm.stats()
    props = torch.cuda.get_device_properties(dev)
    bus = None
    if hasattr(props, "pci_bus_id"):
        bus = "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id, props.pci_device_id)
    sampler = ClockSampler(bus)
    time.sleep(0.3)
    # ---- timed region: K scans back to back, events only around the whole run
    _barrier(ws)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in seq[args.warmup:]:
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    rows = sampler.stop()
    gm.sync()
    st1 = gm.stats()
    elapsed_ms = t_start.elapsed_time(t_end)
    visits = st1["total_visits"] - st0["total_visits"]
    launches = st1["launches"] - st0["launches"]
    total_rays, max_ms, value = whole_job(rays_per_scan * args.steps, elapsed_ms, ws)
    total_visits = _sum_over_ranks(float(visits), ws)
    gm.close()

    # ---- roofline pass: the same scan sequence into a fresh map, with events
    # around every kernel of the timed calls, so that every call meets the map
    # in the state it had in the timed region
    gr = ohm.Map(**params)
    stage_ms, atomics_per_scan = _stage_pass(gr, seq, args.warmup, stream)
    gr.close()
    walk_avg_s = stage_ms["walk"] / 1e3

    if args.profile_case:
        if rank == 0:
            print(json.dumps({"profile_case": True, "rays_per_scan": rays_per_scan, "steps": args.steps,
                              "visits_per_scan": visits / args.steps, "walk_avg_ms": walk_avg_s * 1e3,
                              "segments_last_scan": st1["segments"], "regions": st1["regions"]}), flush=True)
        return

    # ---- per-scan latency: its own pass of LATENCY_SCANS scans after LATENCY_WARMUP
    gl = ohm.Map(**params)
    lat = _latency_pass(gl, scans, LATENCY_WARMUP, LATENCY_SCANS, stream)
    gl.close()

    # ---- end to end: host (pinned) inputs copied inside each call, status read back
    host = []
    for s in scans[:min(n_unique, n_steps)]:
        host.append((s.origins.cpu().pin_memory(), s.endpoints.cpu().pin_memory(), s.flags.cpu().pin_memory()))
    gm2 = ohm.Map(**params)
    for i in range(args.warmup):
        o, e, f = host[i % len(host)]
        gm2.integrate(o, e, f)
    # each step: H2D copies of the scan from pinned memory, the kernels, and a
    # D2H read of the map's status word into a pinned slot of its own; the
    # host submits scans back to back and checks every step's status at the end
    status = torch.zeros(args.steps, dtype=torch.int32).pin_memory()
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        o, e, f = host[(args.warmup + k) % len(host)]
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
    visits_per_scan = visits / args.steps
    # the method's work per scan: 12 B endpoint + 1 B flag per ray, and per
    # voxel visit a 4-byte log-odds read and write
    algo_bytes = 8.0 * visits_per_scan + 13.0 * rays_per_scan
    achieved = algo_bytes / walk_avg_s / 1e9
    traffic = _traffic_per_launch(rays_per_scan)
    # measured ceilings of the walk's memory work (library probe kernels)
    l2_add = ohm.probe_rate(ohm.PROBE_L2_ADD, 1 << 22, device=local)
    sector = ohm.probe_rate(ohm.PROBE_SECTOR_RMW, 1 << 27, device=local)
    sector_gbs = sector * 64 / 1e9

    # ---- CPU baseline: the oracle, single thread, on a bounded sample of scans
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        host_np = [(h[0].numpy(), h[1].numpy(), h[2].numpy()) for h in host]
        rays_c, secs, used = cpu_oracle_run(host_np, max_seconds=args.cpu_seconds)
        cpu = {"value": rays_c / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d scans of the trajectory (%d rays), fresh map, single thread, %.1f s"
                         % (used, rays_c, secs)}

    extras = {}
    if ws == 1 and not args.no_extras:
        extras["room"] = room_leg(dev)
        extras["tsdf"] = tsdf_leg(dev, frames=16, warmup=3)
        extras["ndt_adjoint"] = ndt_adjoint_leg(dev)
        extras["multimap"] = multimap_leg(dev, steps=20, warmup=3)
        extras["served"] = served_leg(dev, duration=8.0, pool_regions=1150)
        # offered load far above what one GPU serves: rays/s over the wall
        # time until the backlog is drained is the sustained maximum
        extras["served_saturation"] = served_leg(dev, duration=3.0, rate_scale=40.0, pool_regions=1600)

    if rank == 0:
        clocks = ClockSampler.summarise(rows)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 log-odds, i64 fixed-point walk",
            "data": "synthetic (seeded tunnel lidar scans generated on the device)",
            "config": {"workload": WORKLOAD, "rays_per_scan": rays_per_scan, "scans": SCANS,
                       "layers": "occupancy+ndt", "voxel_size_m": 0.1, "max_range_m": 50.0,
                       "segment_target_voxels": args.segment_steps or 24,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "warmup_scans": args.warmup,
                       "l2": "map working set per scan (~7.7k 128 KB regions) exceeds the 129 MB L2; "
                             "each step integrates a different scan"},
            "voxel_updates_per_s": total_visits / (max_ms / 1e3),
            "latency_ms": _percentiles(lat),
            "latency_pass": "%d scans after %d warm-up scans on a fresh map, events around each call"
                            % (LATENCY_SCANS, LATENCY_WARMUP),
            "atomics_per_scan": atomics_per_scan,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4},
            "gpu_launches": int(launches),
            "stages_ms": stage_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "kernel": "k_walk_fast<1, 0, 0>",
                         "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": walk_avg_s * 1e3,
                         "peak_source": peak_src,
                         "duration_source": "events around the walk in a replay of the timed scan sequence "
                                            "on a fresh map (same stream), right after the timed region",
                         "atomics": {"achieved": atomics_per_scan / walk_avg_s, "peak": l2_add,
                                     "unit": "atomic ops/s", "frac": atomics_per_scan / walk_avg_s / l2_add,
                                     "per_launch": atomics_per_scan,
                                     "peak_source": "ohm_probe_rate OHM_PROBE_L2_ADD: float atomic adds to "
                                                    "random distinct words of a 16 MB (L2-resident) buffer, "
                                                    "measured in this run"},
                         # the walk's measured DRAM traffic against copy bandwidth
                         "dram": {"achieved": (traffic / walk_avg_s / 1e9) if traffic else None,
                                  "peak": hbm, "unit": "GB/s",
                                  "frac": (traffic / walk_avg_s / 1e9 / hbm) if traffic else None,
                                  "peak_source": peak_src,
                                  "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one ncu "
                                                    "capture of this kernel, scaled to this scan's rays"},
                         # context, not a ceiling: a random 32-byte-sector access pattern; the walk's
                         # accesses are spatially coherent and move their DRAM traffic faster
                         "random_sector_rmw": {"rate_gbs": sector_gbs,
                                               "source": "ohm_probe_rate OHM_PROBE_SECTOR_RMW: load + store of "
                                                         "a word of random 32-byte sectors of a 4 GB buffer, 64 "
                                                         "DRAM bytes per operation, measured in this run"}},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        out.update(extras)
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def room_leg(dev, warmup=LATENCY_WARMUP, scans=LATENCY_SCANS):
    """Single room scans (32,768 rays from (0, 0, 1) in a 10 x 8 x 4 m room,
    occupancy, 0.1 m voxels, 20 m range), ten seeded scan patterns in turn:
    throughput over `scans` calls without per-call events, then per-call
    latency over another `scans` calls."""
    import torch
    from paper_2206_06079_gb300 import ohm, workloads as W
    pool = [W.room_rays(i, device=dev) for i in range(10)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    gm = ohm.Map(**W.room_params(device=dev.index))
    for k in range(warmup):
        s = pool[k % 10]
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    gm.sync(stream)
    v0 = gm.stats()["total_visits"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(scans):
        s = pool[k % 10]
        gm.integrate(s.origins, s.endpoints, s.flags, stream=stream, sync=False)
    e1.record(stream)
    gm.sync(stream)
    ms = e0.elapsed_time(e1)
    visits = gm.stats()["total_visits"] - v0
    lat = _latency_pass(gm, pool, 0, scans, stream)
    gm.close()
    n = pool[0].n
    return {"workload": "room scan: 32768 rays, occupancy, 0.1 m voxels, 20 m range", "rays_per_s": n * scans / (ms / 1e3),
            "voxel_updates_per_s": visits / (ms / 1e3), "ms_per_scan": ms / scans, "latency_ms": _percentiles(lat),
            "scans": scans, "warmup": warmup}


def tsdf_leg(dev, frames=16, warmup=3, n_query=20000):
    """Depth-camera TSDF frames (640 x 480, fx = fy = 525, 0.3-6 m, 0.05 m
    voxels, tau = 0.2 m): forward integration per frame and, on a second map,
    forward + adjoint (ohm_tsdf_backward against n_query query voxels)."""
    import numpy as np
    import torch
    from paper_2206_06079_gb300 import ohm, synth, workloads as W
    scene = synth.depth_scene()
    w, h = 640, 480
    K = (525.0, 525.0, 319.5, 239.5)
    n_frames = warmup + frames
    fr = []
    for i in range(n_frames):
        depth, pos, R = synth.depth_frame(scene, i % 64, width=w, height=h, device=dev)
        fr.append((depth.contiguous(), np.concatenate([R.numpy(), pos.numpy()[:, None]], 1)))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    gm = ohm.Map(**W.tsdf_params(device=dev.index))
    for d, P in fr[:warmup]:
        gm.integrate_depth(d, K, P, sync=False)
    gm.sync()
    v0 = gm.stats()["total_visits"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for d, P in fr[warmup:]:
        gm.integrate_depth(d, K, P, sync=False)
    e1.record(stream)
    gm.sync()
    fwd_ms = e0.elapsed_time(e1) / frames
    visits = (gm.stats()["total_visits"] - v0) / frames
    gm.close()
    # per-stage device times: the same frames on a fresh map, events around every kernel
    gs = ohm.Map(**W.tsdf_params(device=dev.index))
    for d, P in fr[:warmup]:
        gs.integrate_depth(d, K, P, sync=False)
    gs.sync()
    gs.profile(ohm.STAGES)
    for d, P in fr[warmup:]:
        gs.integrate_depth(d, K, P, sync=False)
    gs.sync()
    stages = {}
    for name in ohm.STAGES:
        ms, nl = gs.profile_read(name)
        if nl:
            stages[name] = ms / nl
    gs.close()
    rng = np.random.default_rng(5)
    q = torch.from_numpy(rng.uniform([-3, -3, 0], [3, 3, 3], size=(n_query, 3)).astype(np.float32)).to(dev)
    gq = torch.from_numpy(rng.normal(size=n_query).astype(np.float32)).to(dev)
    gm2 = ohm.Map(**W.tsdf_params(device=dev.index))
    for d, P in fr[:warmup]:
        gm2.integrate_depth(d, K, P, sync=False)
        gm2.tsdf_backward(d, K, P, q, gq)
    gm2.sync()
    e0.record(stream)
    for d, P in fr[warmup:]:
        gm2.integrate_depth(d, K, P, sync=False)
        gm2.tsdf_backward(d, K, P, q, gq)
    e1.record(stream)
    gm2.sync()
    fb_ms = e0.elapsed_time(e1) / frames
    gm2.close()
    return {"workload": "640x480 depth frames, 0.05 m voxels, tau 0.2 m, TSDF layer", "rays_per_s": w * h / (fwd_ms / 1e3),
            "ms_per_frame": fwd_ms, "voxel_updates_per_s": visits / (fwd_ms / 1e3),
            "forward_backward_ms_per_frame": fb_ms, "backward_ms_per_frame": fb_ms - fwd_ms,
            "stages_ms": stages, "frames": frames, "warmup": warmup, "adjoint_query_voxels": n_query}


def ndt_adjoint_leg(dev, scans=8, warmup=3, n_query=20000):
    """NDT-OM adjoint on tunnel scans: each scan is given in the sensor frame
    and integrated by ohm_integrate_posed, then ohm_ndt_backward gives the
    gradient of a loss on the mean and covariance of n_query voxels with
    respect to every endpoint and the pose twist.  Device ms per scan for the
    forward call and for forward + backward."""
    import numpy as np
    import torch
    from paper_2206_06079_gb300 import ohm, workloads as W
    rng = np.random.default_rng(9)
    frames = []
    for i in range(warmup + scans):
        s = W.tunnel_rays(i, device=dev)
        pose = np.concatenate([np.eye(3), rng.uniform(-0.2, 0.2, size=(3, 1))], 1)
        t = torch.from_numpy(pose[:, 3]).to(dev)
        frames.append((pose, (s.origins.double() - t).float(), (s.endpoints.double() - t).float(), s.flags))
    q = torch.from_numpy(rng.uniform([0, -6, -3], [20, 6, 3], size=(n_query, 3)).astype(np.float32)).to(dev)
    gmean = torch.from_numpy(rng.normal(size=(n_query, 3)).astype(np.float32)).to(dev)
    gcov = torch.from_numpy(rng.normal(size=(n_query, 6)).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    out = {}
    for with_backward in (False, True):
        gm = ohm.Map(**W.tunnel_params(device=dev.index))
        for pose, o, e, f in frames[:warmup]:
            gm.integrate_posed(pose, o, e, f, sync=False)
            if with_backward:
                gm.ndt_backward(pose, o, e, f, q, gmean, gcov)
        gm.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pose, o, e, f in frames[warmup:]:
            gm.integrate_posed(pose, o, e, f, sync=False)
            if with_backward:
                gm.ndt_backward(pose, o, e, f, q, gmean, gcov)
        e1.record(stream)
        gm.sync()
        out["forward_backward_ms_per_scan" if with_backward else "forward_ms_per_scan"] = e0.elapsed_time(e1) / scans
        gm.close()
    out["backward_ms_per_scan"] = out["forward_backward_ms_per_scan"] - out["forward_ms_per_scan"]
    out.update({"workload": "tunnel scans (131072 rays) in the sensor frame with a pose, occupancy + NDT-OM; "
                            "gradient of mean/covariance losses on %d query voxels" % n_query,
                "scans": scans, "warmup": warmup})
    return out


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


def multimap_leg(dev, steps=20, warmup=3, tune_segments=(16, 24, 32), tune_blocks=(0,)):
    """Batched multi-map workload: per step every one of 16 maps receives one
    scan drawn uniformly from four sensor types; the single-scan path (one
    integrate call per map) against the batched path (one launch per stage
    for all maps, replayed from a CUDA graph, autotuned tiles)."""
    import numpy as np
    import torch
    from paper_2206_06079_gb300 import ohm, synth, tuning

    specs = multimap_specs()
    pool = {}
    for scene in ("tunnel", "room"):
        for kind in MULTIMAP_KINDS:
            pool[(scene, kind)] = [synth.mixed_scan(scene, kind, 1000 + 17 * j + 101 * len(pool), device=dev)
                                   for j in range(3)]
    rng = np.random.default_rng(0x0A15)
    n_steps = warmup + steps
    plans = [[pool[(sc, MULTIMAP_KINDS[rng.integers(4)])][rng.integers(3)] for sc, _ in specs] for _ in range(n_steps)]
    torch.cuda.synchronize()
    step_sets = [[(r.origins, r.endpoints, r.flags) for r in plan] for plan in plans]
    rays = [sum(r.n for r in plan) for plan in plans]
    stream = torch.cuda.Stream(device=dev)
    params = [dict(p, device=dev.index) for _, p in specs]

    # single-scan path
    maps_a = [ohm.Map(**p) for p in params]
    with torch.cuda.stream(stream):
        for k in range(warmup):
            for m, rs in zip(maps_a, step_sets[k]):
                m.integrate(*rs, stream=stream, sync=False)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for k in range(warmup, n_steps):
            for m, rs in zip(maps_a, step_sets[k]):
                m.integrate(*rs, stream=stream, sync=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_a = ev0.elapsed_time(ev1)
    for m in maps_a:
        m.sync(stream)
    counts_a = [m.region_count() for m in maps_a]
    for m in maps_a:
        m.close()

    # batched path: tune on scratch maps, then measure
    (best_s, best_b), table = tuning.autotune_batch(params, step_sets[:4], segment_steps=tune_segments,
                                                    walk_blocks=tune_blocks, stream=stream)
    maps_b = [ohm.Map(**p) for p in params]
    batch = ohm.Batch(maps_b)
    batch.tune(best_s, best_b)
    for k in range(warmup):
        with torch.cuda.stream(stream):
            batch.integrate(step_sets[k], graph=True)
    batch.sync(stream)
    st0 = batch.stats()
    ev0.record(stream)
    for k in range(warmup, n_steps):
        with torch.cuda.stream(stream):
            batch.integrate(step_sets[k], graph=True)
    ev1.record(stream)
    batch.sync(stream)
    ms_b = ev0.elapsed_time(ev1)
    st1 = batch.stats()
    same = counts_a == [m.region_count() for m in maps_b]
    batch.close()
    for m in maps_b:
        m.close()
    total_rays = float(sum(rays[warmup:]))
    return {"workload": "16 maps (tunnel/room, 0.1/0.05 m voxels), per step each map gets one scan drawn uniformly "
                        "from 16x1800, 64x1024, 128x2048 lidar and 424x240 depth",
            "rays_per_s": total_rays / (ms_b / 1e3), "single_scan_rays_per_s": total_rays / (ms_a / 1e3),
            "speedup_vs_single_scan": ms_a / ms_b, "ms_per_step": ms_b / steps,
            "single_scan_ms_per_step": ms_a / steps, "steps": steps, "warmup": warmup,
            "rays_per_step_mean": total_rays / steps,
            "tuned": {"segment_steps": best_s, "walk_blocks_per_sm": best_b},
            "tuning_ms_per_step": {"%d/%d" % k: v for k, v in sorted(table.items())},
            "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
            "graph_launches": int(st1["graph_launches"] - st0["graph_launches"]), "region_counts_equal": same}


def served_leg(dev, duration=8.0, budget_frac=1.0, n_robots=8, realtime=True, rate_scale=1.0, pool_regions=None):
    """Served stream: 8 robots in a 200 x 200 m world, each with a 128 x 1024
    lidar at 10 Hz and two 424 x 240 depth cameras at 30 Hz (Poisson
    arrivals), one resident occupancy + NDT map per robot at 0.1 m, admission
    by a 60 GB HBM cap (times budget_frac: small values force least recently
    used regions out to pinned host memory), arrivals in real time over
    `duration` seconds (rate_scale multiplies the arrival rates: a
    saturation run offers more than the loop can serve).  p50 / p99 scan
    latency and sustained rays/s."""
    import numpy as np
    import torch
    from paper_2206_06079_gb300 import ohm, serve, synth, workloads as W

    per_region = 4 * 32768 + 8 * 10 * 32768          # occupancy + an NDT block
    # each map's region pool is its share of the cap: a scan that needs more
    # fails, the loop evicts least recently used regions and repeats it (one
    # 128 x 1024 lidar scan here touches up to about 1100 regions)
    if pool_regions is None:
        pool_regions = max(1150, int(60e9 * budget_frac / n_robots / per_region))
    cap = pool_regions * per_region * n_robots
    params = W.tunnel_params(layers=W.OCC | W.NDT, max_range=30.0, max_rays=131072, max_regions=pool_regions,
                             max_ndt_regions=pool_regions, evict_when_full=1, device=dev.index)
    world = synth.world_scene()
    step_s = 0.5
    n_pose = int(duration / step_s) + 1
    pool_scans = {}
    for rb in range(n_robots):
        for j in range(n_pose):
            t = j * step_s
            for kind, cam in (("lidar128x1024", 0), ("depth424x240", 0), ("depth424x240", 1)):
                r = synth.world_scan(world, rb, t, kind, camera=cam, device=dev, max_range=30.0, seed=rb * 7919 + j)
                pool_scans[(rb, j, kind, cam)] = (r.origins, r.endpoints, r.flags)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0x0A17)
    reqs = []
    for rb in range(n_robots):
        for kind, cam, rate in (("lidar128x1024", 0, 10.0), ("depth424x240", 0, 30.0), ("depth424x240", 1, 30.0)):
            for t in serve.poisson_times(rate * rate_scale, duration, rng):
                j = min(int(t / step_s), n_pose - 1)
                reqs.append(serve.Request(rb, float(t), pool_scans[(rb, j, kind, cam)], kind))
    maps = [ohm.Map(**params) for _ in range(n_robots)]
    # warm the graph and the maps with a sample of the traffic, untimed
    warm = serve.ServeLoop(maps)
    warm.run([serve.Request(r.map_index, 0.0, r.rays, r.kind) for r in reqs[:: max(1, len(reqs) // 200)]],
             realtime=False)
    loop = serve.ServeLoop(maps)
    stats = loop.run(reqs, realtime=realtime).summary()
    resident = sum(m.residency()[0] for m in maps)
    host = sum(m.residency()[1] for m in maps)
    offered = sum(r.n for r in reqs) / duration
    for m in maps:
        m.close()
    return {"workload": "8 robots x (128x1024 lidar @10 Hz + 2 x 424x240 depth @30 Hz) x %g, Poisson arrivals, "
                        "200 x 200 m world, occupancy + NDT at 0.1 m" % rate_scale,
            "rays_per_s": stats["rays_per_s"], "offered_rays_per_s": offered, "latency_ms": stats["latency_ms"],
            "requests": stats["requests"], "steps": stats["steps"], "duration_s": duration,
            "evicted_regions": stats["evicted_regions"], "restored_regions": stats["restored_regions"],
            "faults": stats["faults"], "capacity_faults": stats["capacity_faults"], "wall_s": stats["wall_s"],
            "saturated": offered > 1.02 * stats["rays_per_s"], "resident_regions_end": resident,
            "host_regions_end": host, "hbm_cap_gb": cap / 1e9, "pool_regions_per_map": pool_regions,
            "pipeline_depth": loop.depth}


def run_multimap(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    out = multimap_leg(torch.device("cuda", 0), steps=args.steps, warmup=args.warmup,
                       tune_segments=(6, 10, 16, 24, 32), tune_blocks=(0, 2, 3, 4))
    out.update({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "value": out["rays_per_s"], "higher_is_better": True})
    print(json.dumps(out), flush=True)


def run_tsdf(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    out = tsdf_leg(torch.device("cuda", 0), frames=args.steps, warmup=args.warmup)
    out.update({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "value": out["rays_per_s"], "higher_is_better": True})
    print(json.dumps(out), flush=True)


def run_served(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    out = served_leg(torch.device("cuda", 0), duration=args.duration, budget_frac=args.budget_frac,
                     rate_scale=args.rate_scale, pool_regions=args.pool_regions or None)
    out.update({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "value": out["rays_per_s"], "higher_is_better": True})
    print(json.dumps(out), flush=True)


def run_room(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    out = room_leg(torch.device("cuda", 0), warmup=max(args.warmup, LATENCY_WARMUP), scans=max(args.steps, LATENCY_SCANS))
    out.update({"metric": METRIC, "unit": UNIT, "n_gpus": 1, "value": out["rays_per_s"], "higher_is_better": True})
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
    ap.add_argument("--no-extras", action="store_true", help="tunnel headline only (no room/tsdf/multimap/served legs)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--segment-steps", type=int, default=0, help="ray segment length (0 = library default)")
    ap.add_argument("--workload", default="tunnel", choices=["tunnel", "room", "multimap", "tsdf", "served"],
                    help="tunnel: the single-map headline (plus compact sub-results of the other workloads); "
                         "room: single room scans; multimap: 16 maps, single-scan vs batched path; "
                         "tsdf: depth frames, forward and adjoint; served: request loop")
    ap.add_argument("--duration", type=float, default=60.0, help="served workload: seconds of arrivals")
    ap.add_argument("--budget-frac", type=float, default=1.0,
                    help="served workload: fraction of the 60 GB HBM cap the maps may keep resident")
    ap.add_argument("--pool-regions", type=int, default=0,
                    help="served workload: region pool per map (overrides --budget-frac; the cap follows)")
    ap.add_argument("--rate-scale", type=float, default=1.0, help="served workload: arrival rate multiplier")
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
    elif args.workload == "room":
        run_room(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
