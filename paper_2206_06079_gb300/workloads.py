"""The synthetic workloads: map parameters plus the ray sets that feed them.

Each stands in for one of the paper's measurement settings (Sec. IV-A:
0.1 m voxels, 32^3 regions, 20 m truncation, 10 m segments; VLP-16 class
lidar) with seeded synthetic scenes, since the recorded datasets are not
available.  Configuration only: no mapping arithmetic lives here.
"""
import math

import numpy as np

from . import synth

OCC, NDT, TSDF, COUNTS, DECAY, MEAN = 1, 2, 4, 8, 16, 32

HIT = float(np.float32(math.log(0.7 / 0.3)))    # p = 0.7 -> +0.847
MISS = float(np.float32(math.log(0.4 / 0.6)))   # p = 0.4 -> -0.405


def room_params(**kw):
    """Single room scan: 32,768 rays, occupancy, 0.1 m voxels, 20 m range."""
    p = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16, layers=OCC, hit=HIT, miss=MISS,
             l_min=-2.0, l_max=3.5, ndt_clear_below=float("-inf"), max_range=20.0, min_range=0.0, tsdf_trunc=0.2, tsdf_wmax=float(1 << 20),
             max_regions=1024, max_ndt_regions=1024, max_rays=32768, segment_steps=0, device=0, evict_when_full=0, max_probe=0)
    p.update(kw)
    return p


def room_rays(i=0, n=32768, device="cpu"):
    return synth.room_scan(seed=0x0A12 + i, n=n, device=device)


def tunnel_params(**kw):
    """Spinning-lidar tunnel trajectory: 131,072 rays per scan (128 beams x
    1024 azimuths), occupancy + NDT-OM, 0.1 m voxels, 50 m maximum range for
    missing returns."""
    p = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16, layers=OCC | NDT, hit=HIT, miss=MISS,
             l_min=-2.0, l_max=3.5, ndt_clear_below=float("-inf"), max_range=50.0, min_range=0.0, tsdf_trunc=0.2, tsdf_wmax=float(1 << 20),
             max_regions=24576, max_ndt_regions=4096, max_rays=131072, segment_steps=0, device=0, evict_when_full=0, max_probe=0)
    p.update(kw)
    return p


def tunnel_rays(i, device="cpu", beams=128, azimuths=1024):
    return synth.tunnel_scan(i, beams=beams, azimuths=azimuths, device=device)


TUNNEL_SCANS = 100


def tsdf_params(**kw):
    """Depth-camera TSDF: 640 x 480 frames, 0.05 m voxels, tau = 0.2 m."""
    p = dict(voxel_size=0.05, map_origin=(0.0, 0.0, 0.0), frac_bits=16, layers=TSDF, hit=HIT, miss=MISS,
             l_min=-2.0, l_max=3.5, ndt_clear_below=float("-inf"), max_range=10.0, min_range=0.0, tsdf_trunc=0.2, tsdf_wmax=float(1 << 20),
             max_regions=2048, max_ndt_regions=1, max_rays=640 * 480, segment_steps=0, device=0, evict_when_full=0, max_probe=0)
    p.update(kw)
    return p


def tsdf_rays(i, device="cpu", width=640, height=480, scene=None):
    scene = scene or synth.depth_scene()
    s = width / 640.0
    depth, pos, R = synth.depth_frame(scene, i, width=width, height=height, fx=525.0 * s, fy=525.0 * s,
                                      cx=(width - 1) / 2.0, cy=(height - 1) / 2.0, device=device)
    return synth.depth_to_rays(depth, pos, R, fx=525.0 * s, fy=525.0 * s, cx=(width - 1) / 2.0,
                               cy=(height - 1) / 2.0)


TSDF_FRAMES = 64


def oracle_params(p):
    """The oracle's parameter names for a map parameter dict."""
    keys = ("voxel_size", "map_origin", "frac_bits", "layers", "hit", "miss", "l_min", "l_max", "ndt_clear_below",
            "max_range", "min_range", "tsdf_trunc", "tsdf_wmax")
    return {k: p[k] for k in keys}
