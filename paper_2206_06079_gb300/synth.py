"""Seeded synthetic ray sets shaped like the paper's sensors and scenes.

The paper measures on five recorded VLP-16 datasets (Sec. IV) that are not
public; these generators stand in for them.  They produce world-frame rays:
a sensor origin (one per scan), an endpoint per ray and a flag byte per ray
(bit 0 = NO_RETURN: the beam saw nothing, the endpoint sits at maximum range and
the ray only carries pass-through evidence).

This module only builds inputs.  It holds none of the mapping arithmetic
(quantisation, line walk, log-odds, NDT or TSDF updates), so the CUDA path and
the CPU oracle can both consume its output.

Every random number is drawn on the CPU from a torch.Generator seeded by the
caller; geometry is evaluated in float64 on the requested device and rounded to
float32 at the end.
"""
import math
from dataclasses import dataclass

import torch

FLAG_NO_RETURN = 1


@dataclass
class RaySet:
    origins: torch.Tensor    # (1, 3) or (n, 3) float32
    endpoints: torch.Tensor  # (n, 3) float32
    flags: torch.Tensor      # (n,) uint8

    @property
    def n(self) -> int:
        return int(self.endpoints.shape[0])

    def to(self, device) -> "RaySet":
        return RaySet(self.origins.to(device), self.endpoints.to(device), self.flags.to(device))

    def numpy(self):
        return (self.origins.cpu().numpy(), self.endpoints.cpu().numpy(), self.flags.cpu().numpy())


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


# ---------------------------------------------------------------------------
# Room: one scan of rays uniform on the sphere inside an axis-aligned box room.
# ---------------------------------------------------------------------------
ROOM_MIN = (-5.0, -4.0, 0.0)
ROOM_MAX = (5.0, 4.0, 4.0)
ROOM_SENSOR = (0.0, 0.0, 1.0)


def room_scan(seed: int = 0x0A12, n: int = 32768, noise: float = 0.02, device="cpu",
              sensor=ROOM_SENSOR, room_min=ROOM_MIN, room_max=ROOM_MAX) -> RaySet:
    """n rays from `sensor`, directions uniform on the sphere (z ~ U[-1,1],
    azimuth ~ U[0, 2 pi)), each ending at the first wall + N(0, noise) along the
    ray.  Every ray is a return."""
    g = _gen(seed)
    z = torch.rand(n, generator=g, dtype=torch.float64) * 2.0 - 1.0
    phi = torch.rand(n, generator=g, dtype=torch.float64) * (2.0 * math.pi)
    eps = torch.randn(n, generator=g, dtype=torch.float64) * noise
    z, phi, eps = z.to(device), phi.to(device), eps.to(device)
    r = torch.sqrt(torch.clamp(1.0 - z * z, min=0.0))
    u = torch.stack([r * torch.cos(phi), r * torch.sin(phi), z], dim=1)
    o = torch.tensor(sensor, dtype=torch.float64, device=device)
    lo = torch.tensor(room_min, dtype=torch.float64, device=device)
    hi = torch.tensor(room_max, dtype=torch.float64, device=device)
    # Exit distance through the box from inside: per axis, the face the ray heads to.
    with torch.no_grad():
        bound = torch.where(u > 0, hi, lo)
        safe = torch.where(u == 0, torch.ones_like(u), u)
        t_axis = torch.where(u == 0, torch.full_like(u, float("inf")), (bound - o) / safe)
        t_wall = t_axis.min(dim=1).values
    t = t_wall + eps
    e = o + t[:, None] * u
    return RaySet(o[None].float(), e.float(), torch.zeros(n, dtype=torch.uint8, device=device))


# ---------------------------------------------------------------------------
# Tunnel: a spinning lidar moving along a sinusoidal tunnel.
# ---------------------------------------------------------------------------
TUNNEL_RADIUS = 3.0
TUNNEL_AMPLITUDE = 3.0
TUNNEL_WAVELENGTH = 50.0
TUNNEL_X_RANGE = (-75.0, 125.0)  # 200 m; every ray of every pose stays inside


def tunnel_centre_y(x):
    return TUNNEL_AMPLITUDE * torch.sin((2.0 * math.pi / TUNNEL_WAVELENGTH) * x)


def _tunnel_radial(p):
    """Distance from the tunnel's cross-section centre: sqrt((y - yc(x))^2 + z^2)."""
    dy = p[..., 1] - tunnel_centre_y(p[..., 0])
    return torch.sqrt(dy * dy + p[..., 2] * p[..., 2])


def tunnel_pose(i: int, step: float = 0.5, yaw_sigma_deg: float = 1.0, seed: int = 0x0A13):
    """Sensor position and yaw of scan i: x = step * i on the centreline, yaw =
    centreline heading + N(0, yaw_sigma)."""
    g = _gen(seed * 1000003 + i)
    noise = float(torch.randn(1, generator=g, dtype=torch.float64)[0]) * math.radians(yaw_sigma_deg)
    x = step * i
    y = TUNNEL_AMPLITUDE * math.sin(2.0 * math.pi * x / TUNNEL_WAVELENGTH)
    slope = TUNNEL_AMPLITUDE * (2.0 * math.pi / TUNNEL_WAVELENGTH) * math.cos(2.0 * math.pi * x / TUNNEL_WAVELENGTH)
    return (x, y, 0.0), math.atan(slope) + noise


def lidar_directions(beams: int, azimuths: int, fov_deg: float = 22.5, device="cpu", dtype=torch.float64):
    """Unit beam directions in the sensor frame: `beams` elevations evenly over
    [-fov, +fov] times `azimuths` evenly spaced azimuths, beam-major."""
    if beams > 1:
        el = torch.linspace(-math.radians(fov_deg), math.radians(fov_deg), beams, dtype=dtype, device=device)
    else:
        el = torch.zeros(1, dtype=dtype, device=device)
    az = torch.arange(azimuths, dtype=dtype, device=device) * (2.0 * math.pi / azimuths)
    ce, se = torch.cos(el)[:, None], torch.sin(el)[:, None]
    d = torch.stack([(ce * torch.cos(az)[None]).expand(beams, azimuths),
                     (ce * torch.sin(az)[None]).expand(beams, azimuths),
                     se.expand(beams, azimuths)], dim=-1)
    return d.reshape(-1, 3)


def march_tunnel(o, u, max_range: float):
    """Distance along unit rays u from o (inside the tunnel) to the wall, or
    >= max_range when none is met: sphere tracing on a conservative bound
    (|grad radial| <= sqrt(1 + (A k)^2)), a 1 cm step floor, then bisection."""
    k = 2.0 * math.pi / TUNNEL_WAVELENGTH
    lip = math.sqrt(1.0 + (TUNNEL_AMPLITUDE * k) ** 2)
    limit = max_range + 1.0
    n = u.shape[0]
    t = torch.zeros(n, dtype=torch.float64, device=u.device)
    prev = torch.zeros_like(t)
    for _ in range(1000):
        gap = TUNNEL_RADIUS - _tunnel_radial(o + t[:, None] * u)
        active = (gap > 0) & (t < limit)
        if not bool(active.any()):
            break
        prev = torch.where(active, t, prev)
        t = torch.where(active, torch.clamp(t + torch.clamp(gap / lip, min=0.01), max=limit), t)
    lo, hi = prev, t
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        inside = _tunnel_radial(o + mid[:, None] * u) < TUNNEL_RADIUS
        lo = torch.where(inside, mid, lo)
        hi = torch.where(inside, hi, mid)
    return 0.5 * (lo + hi)


def tunnel_scan(i: int, seed: int = 0x0A13, beams: int = 128, azimuths: int = 1024, max_range: float = 50.0,
                missing: float = 0.1, range_noise: float = 0.03, device="cpu", fov_deg: float = 22.5,
                step: float = 0.5) -> RaySet:
    """Scan i of the tunnel trajectory.  Each beam is marched to the tunnel wall
    (sphere tracing on a conservative distance bound, then bisection); a
    return gets N(0, range_noise) along the beam.  A Bernoulli(missing) beam, or
    one that meets no wall within max_range, becomes NO_RETURN at max_range."""
    g = _gen(seed * 7919 + i)
    n = beams * azimuths
    miss_draw = torch.rand(n, generator=g, dtype=torch.float64).to(device)
    noise = (torch.randn(n, generator=g, dtype=torch.float64) * range_noise).to(device)
    pos, yaw = tunnel_pose(i, step=step, seed=seed)
    o = torch.tensor(pos, dtype=torch.float64, device=device)
    d = lidar_directions(beams, azimuths, fov_deg, device=device)
    cy, sy = math.cos(yaw), math.sin(yaw)
    u = torch.stack([cy * d[:, 0] - sy * d[:, 1], sy * d[:, 0] + cy * d[:, 1], d[:, 2]], dim=1)
    # |grad radial| <= sqrt(1 + (A k)^2), so (R - radial) / L never oversteps the
    # wall; a floor of 1 cm per step bounds the iteration count near grazing.
    k = 2.0 * math.pi / TUNNEL_WAVELENGTH
    lip = math.sqrt(1.0 + (TUNNEL_AMPLITUDE * k) ** 2)
    limit = max_range + 1.0
    t = torch.zeros(n, dtype=torch.float64, device=device)
    prev = torch.zeros_like(t)
    for _ in range(1000):
        gap = TUNNEL_RADIUS - _tunnel_radial(o + t[:, None] * u)
        active = (gap > 0) & (t < limit)
        if not bool(active.any()):
            break
        prev = torch.where(active, t, prev)
        t = torch.where(active, torch.clamp(t + torch.clamp(gap / lip, min=0.01), max=limit), t)
    # Bracket [prev, t]: prev inside, t outside (or at the range limit).
    lo = prev
    hi = t
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        inside = _tunnel_radial(o + mid[:, None] * u) < TUNNEL_RADIUS
        lo = torch.where(inside, mid, lo)
        hi = torch.where(inside, hi, mid)
    t_wall = 0.5 * (lo + hi)
    rng = t_wall + noise
    no_return = (miss_draw < missing) | (t_wall >= max_range)
    rng = torch.where(no_return, torch.full_like(rng, max_range), rng)
    e = o + rng[:, None] * u
    flags = no_return.to(torch.uint8) * FLAG_NO_RETURN
    return RaySet(o[None].float(), e.float(), flags)


# ---------------------------------------------------------------------------
# Depth camera frames of a room with boxes and spheres.
# ---------------------------------------------------------------------------
@dataclass
class DepthScene:
    boxes_lo: torch.Tensor   # (nb, 3) float64
    boxes_hi: torch.Tensor   # (nb, 3)
    spheres_c: torch.Tensor  # (ns, 3)
    spheres_r: torch.Tensor  # (ns,)
    room_lo: tuple = (-3.0, -3.0, 0.0)
    room_hi: tuple = (3.0, 3.0, 3.0)


def depth_scene(seed: int = 0x0A14, n_boxes: int = 20, n_spheres: int = 10) -> DepthScene:
    """20 axis-aligned boxes (sides U[0.2, 1] m) and 10 spheres (radius
    U[0.1, 0.5] m) at seeded positions within 2 m of the room's vertical axis,
    inside a 6 x 6 x 3 m room."""
    g = _gen(seed)

    def centre_xy(k):
        r = torch.sqrt(torch.rand(k, generator=g, dtype=torch.float64)) * 1.8
        a = torch.rand(k, generator=g, dtype=torch.float64) * (2 * math.pi)
        return torch.stack([r * torch.cos(a), r * torch.sin(a)], 1)

    side = 0.2 + 0.8 * torch.rand(n_boxes, 3, generator=g, dtype=torch.float64)
    bxy = centre_xy(n_boxes)
    bz = side[:, 2] / 2 + torch.rand(n_boxes, generator=g, dtype=torch.float64) * 1.2
    bc = torch.cat([bxy, bz[:, None]], 1)
    rad = 0.1 + 0.4 * torch.rand(n_spheres, generator=g, dtype=torch.float64)
    sxy = centre_xy(n_spheres)
    sz = rad + torch.rand(n_spheres, generator=g, dtype=torch.float64) * 1.5
    sc = torch.cat([sxy, sz[:, None]], 1)
    return DepthScene(bc - side / 2, bc + side / 2, sc, rad)


def camera_pose(i: int, n_frames: int = 64, radius: float = 2.5, height: float = 1.5, seed: int = 0x0A14):
    """Camera i on a circle of `radius` at `height`, looking at (0, 0, 1) with
    seeded jitter.  Returns (position (3,), R (3, 3)) float64; R maps camera
    axes (x right, y down, z forward) to world axes."""
    g = _gen(seed * 104729 + i)
    jit = torch.randn(6, generator=g, dtype=torch.float64)
    a = 2 * math.pi * i / n_frames + 0.02 * float(jit[0])
    pos = torch.tensor([radius * math.cos(a) + 0.05 * float(jit[1]), radius * math.sin(a) + 0.05 * float(jit[2]),
                        height + 0.05 * float(jit[3])], dtype=torch.float64)
    target = torch.tensor([0.1 * float(jit[4]), 0.1 * float(jit[5]), 1.0], dtype=torch.float64)
    f = target - pos
    f = f / f.norm()
    up = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64)
    r = torch.linalg.cross(f, up)
    r = r / r.norm()
    dn = torch.linalg.cross(f, r)
    return pos, torch.stack([r, dn, f], dim=1)


def _ray_box_entry(o, u, lo, hi):
    """Smallest t > 0 at which rays (o + t u) enter each box; inf where they miss.
    o (3,), u (n, 3), lo/hi (m, 3) -> (n, m)."""
    inv = 1.0 / torch.where(u == 0, torch.full_like(u, 1e-300), u)
    t1 = (lo[None] - o[None, None]) * inv[:, None]
    t2 = (hi[None] - o[None, None]) * inv[:, None]
    tn = torch.minimum(t1, t2).max(dim=2).values
    tf = torch.maximum(t1, t2).min(dim=2).values
    hit = (tn <= tf) & (tn > 0)
    return torch.where(hit, tn, torch.full_like(tn, float("inf")))


def _ray_sphere(o, u, c, r):
    oc = o[None, None] - c[None]                      # (1, m, 3)
    b = (u[:, None] * oc).sum(-1)                    # (n, m)
    cc = (oc * oc).sum(-1) - (r * r)[None]
    disc = b * b - cc
    t = -b - torch.sqrt(torch.clamp(disc, min=0.0))
    ok = (disc >= 0) & (t > 0)
    return torch.where(ok, t, torch.full_like(t, float("inf")))


def depth_frame(scene: DepthScene, i: int, n_frames: int = 64, width: int = 640, height: int = 480,
                fx: float = 525.0, fy: float = 525.0, cx: float = 319.5, cy: float = 239.5,
                device="cpu"):
    """Noise-free z-depth image (height, width) float32 of frame i, and its pose."""
    pos, R = camera_pose(i, n_frames)
    vv, uu = torch.meshgrid(torch.arange(height, dtype=torch.float64), torch.arange(width, dtype=torch.float64),
                            indexing="ij")
    dc = torch.stack([(uu - cx) / fx, (vv - cy) / fy, torch.ones_like(uu)], -1).reshape(-1, 3).to(device)
    norm = dc.norm(dim=1)
    u = (dc / norm[:, None]) @ R.to(device).T
    o = pos.to(device)
    lo = torch.tensor(scene.room_lo, dtype=torch.float64, device=device)
    hi = torch.tensor(scene.room_hi, dtype=torch.float64, device=device)
    bound = torch.where(u > 0, hi, lo)
    safe = torch.where(u == 0, torch.ones_like(u), u)
    t = torch.where(u == 0, torch.full_like(u, float("inf")), (bound - o) / safe).min(dim=1).values
    t = torch.minimum(t, _ray_box_entry(o, u, scene.boxes_lo.to(device), scene.boxes_hi.to(device)).min(1).values)
    t = torch.minimum(t, _ray_sphere(o, u, scene.spheres_c.to(device), scene.spheres_r.to(device)).min(1).values)
    z = t / norm  # z-depth: distance along the optical axis
    return z.reshape(height, width).float(), pos, R


def depth_to_rays(depth, pos, R, fx=525.0, fy=525.0, cx=319.5, cy=239.5, z_min=0.3, z_max=6.0) -> RaySet:
    """Back-project a z-depth image into world rays; pixels outside
    (z_min, z_max] become NO_RETURN rays ending at z_max along their pixel."""
    h, w = depth.shape
    device = depth.device
    vv, uu = torch.meshgrid(torch.arange(h, dtype=torch.float64, device=device),
                            torch.arange(w, dtype=torch.float64, device=device), indexing="ij")
    z = depth.double()
    valid = (z > z_min) & (z <= z_max)
    zz = torch.where(valid, z, torch.full_like(z, z_max))
    pc = torch.stack([(uu - cx) / fx * zz, (vv - cy) / fy * zz, zz], -1).reshape(-1, 3)
    e = pos.to(device)[None] + pc @ R.to(device).T
    flags = (~valid).reshape(-1).to(torch.uint8) * FLAG_NO_RETURN
    return RaySet(pos.to(device)[None].float(), e.float(), flags)


def tsdf_frame(i: int, scene: DepthScene = None, n_frames: int = 64, width: int = 640, height: int = 480,
               device="cpu") -> RaySet:
    scene = scene or depth_scene()
    depth, pos, R = depth_frame(scene, i, n_frames, width, height, device=device)
    return depth_to_rays(depth, pos, R)


# ---------------------------------------------------------------------------
# Small fuzz cases: rays on voxel faces, edges and corners, zero length, etc.
# ---------------------------------------------------------------------------
def fuzz_rays(seed: int, n: int, voxel: float = 0.1, extent: float = 2.0, device="cpu") -> RaySet:
    """Rays whose coordinates are drawn to land exactly on voxel faces, edges
    and corners often, plus zero-length, axis-aligned and diagonal rays, with a
    few NO_RETURN flags."""
    g = _gen(seed)
    kind = torch.randint(0, 4, (n, 3), generator=g)
    cont = (torch.rand(n, 3, generator=g, dtype=torch.float64) * 2 - 1) * extent
    grid = torch.round(cont / voxel) * voxel
    half = grid + 0.5 * voxel
    pts_e = torch.where(kind == 0, cont, torch.where(kind == 1, grid, torch.where(kind == 2, half, cont)))
    o_kind = torch.randint(0, 3, (n, 3), generator=g)
    oc = (torch.rand(n, 3, generator=g, dtype=torch.float64) * 2 - 1) * extent * 0.5
    og = torch.round(oc / voxel) * voxel
    pts_o = torch.where(o_kind == 0, oc, torch.where(o_kind == 1, og, og + 0.5 * voxel))
    special = torch.randint(0, 10, (n,), generator=g)
    pts_e = torch.where((special == 0)[:, None], pts_o, pts_e)                           # zero length
    axis = torch.randint(0, 3, (n,), generator=g)
    aligned = pts_o.clone()
    aligned[torch.arange(n), axis] = pts_e[torch.arange(n), axis]
    pts_e = torch.where((special == 1)[:, None], aligned, pts_e)                        # axis aligned
    diag = pts_o + (pts_e[:, :1] - pts_o[:, :1])
    pts_e = torch.where((special == 2)[:, None], diag, pts_e)                           # exact diagonal
    flags = (torch.rand(n, generator=g) < 0.15).to(torch.uint8) * FLAG_NO_RETURN
    return RaySet(pts_o.float().to(device), pts_e.float().to(device), flags.to(device))


# ---------------------------------------------------------------------------
# Mixed sensors in either scene (the batched multi-map workload).
# ---------------------------------------------------------------------------
def pinhole_directions(width: int, height: int, R, fov_x_deg: float = None, fx: float = None, device="cpu"):
    """World-frame unit directions and z-scale of a pinhole camera (x right,
    y down, z forward; R maps camera to world axes), principal point at the
    image centre.  Returns (u (h*w, 3), cos_to_axis (h*w,))."""
    if fx is None:
        fx = 0.5 * width / math.tan(math.radians(fov_x_deg) / 2)
    vv, uu = torch.meshgrid(torch.arange(height, dtype=torch.float64), torch.arange(width, dtype=torch.float64),
                            indexing="ij")
    dc = torch.stack([(uu - (width - 1) / 2) / fx, (vv - (height - 1) / 2) / fx, torch.ones_like(uu)], -1).reshape(-1, 3)
    norm = dc.norm(dim=1)
    u = (dc / norm[:, None]) @ R.to(torch.float64).T
    return u.to(device), (1.0 / norm).to(device)


def mixed_scan(scene: str, kind: str, seed: int, device="cpu", max_range: float = 20.0) -> RaySet:
    """One scan of `kind` in `scene`.  kind: 'lidar16x1800', 'lidar64x1024',
    'lidar128x2048' (spinning lidar, +-22.5 deg, 2 % missing returns) or
    'depth424x240' (pinhole, fx = fy = 525 * 424 / 640, z in (0.3, 6] m).
    scene: 'tunnel' (sensor on the centreline at a seeded x) or 'room' (sensor
    at a seeded point of the 6 x 6 x 3 m room with boxes and spheres)."""
    g = _gen(seed)
    jit = torch.rand(4, generator=g, dtype=torch.float64)
    if scene == "tunnel":
        x = float(jit[0]) * 40.0
        o = torch.tensor([x, TUNNEL_AMPLITUDE * math.sin(2 * math.pi * x / TUNNEL_WAVELENGTH), 0.0],
                         dtype=torch.float64, device=device)
        yaw = math.atan(TUNNEL_AMPLITUDE * (2 * math.pi / TUNNEL_WAVELENGTH) * math.cos(2 * math.pi * x / TUNNEL_WAVELENGTH))
    else:
        o = torch.tensor([-1.0 + 2.0 * float(jit[0]), -2.5 + 0.4 * float(jit[1]), 1.0 + float(jit[2])],
                         dtype=torch.float64, device=device)
        yaw = 2 * math.pi * float(jit[3])
    cy, sy = math.cos(yaw), math.sin(yaw)
    if kind.startswith("lidar"):
        beams, az = (int(v) for v in kind[5:].split("x"))
        d = lidar_directions(beams, az, 22.5, device=device)
        u = torch.stack([cy * d[:, 0] - sy * d[:, 1], sy * d[:, 0] + cy * d[:, 1], d[:, 2]], dim=1)
        zscale = None
    else:
        w, h = (int(v) for v in kind[5:].split("x"))
        # camera looking along the heading, level
        f = torch.tensor([cy, sy, 0.0], dtype=torch.float64)
        r = torch.tensor([sy, -cy, 0.0], dtype=torch.float64)
        dn = torch.linalg.cross(f, r)
        R = torch.stack([r, dn, f], dim=1)
        u, zscale = pinhole_directions(w, h, R, fx=525.0 * w / 640.0, device=device)
    n = u.shape[0]
    miss_draw = torch.rand(n, generator=g, dtype=torch.float64).to(device)
    noise = (torch.randn(n, generator=g, dtype=torch.float64) * 0.02).to(device)
    if scene == "tunnel":
        t = march_tunnel(o, u, max_range)
    else:
        sc = depth_scene()
        lo = torch.tensor(sc.room_lo, dtype=torch.float64, device=device)
        hi = torch.tensor(sc.room_hi, dtype=torch.float64, device=device)
        bound = torch.where(u > 0, hi, lo)
        safe = torch.where(u == 0, torch.ones_like(u), u)
        t = torch.where(u == 0, torch.full_like(u, float("inf")), (bound - o) / safe).min(dim=1).values
        t = torch.minimum(t, _ray_box_entry(o, u, sc.boxes_lo.to(device), sc.boxes_hi.to(device)).min(1).values)
        t = torch.minimum(t, _ray_sphere(o, u, sc.spheres_c.to(device), sc.spheres_r.to(device)).min(1).values)
    if zscale is None:
        no_ret = (miss_draw < 0.02) | (t >= max_range)
        rng = torch.where(no_ret, torch.full_like(t, max_range), t + noise)
    else:
        z = t * zscale
        no_ret = (z <= 0.3) | (z > 6.0)
        rng = torch.where(no_ret, 6.0 / zscale, t)
    e = o[None] + rng[:, None] * u
    return RaySet(o[None].float(), e.float(), no_ret.to(torch.uint8) * FLAG_NO_RETURN)


# ---------------------------------------------------------------------------
# An outdoor world for the served stream: ground plane and box buildings.
# ---------------------------------------------------------------------------
@dataclass
class World:
    boxes_lo: torch.Tensor   # (nb, 3)
    boxes_hi: torch.Tensor
    half: float              # the world spans [-half, half]^2 in x, y


def world_scene(seed: int = 0x0A16, n_boxes: int = 160, half: float = 100.0) -> World:
    """Ground plane z = 0 and n_boxes axis-aligned buildings (footprint
    U[2, 12] m, height U[2, 25] m) scattered over [-half, half]^2."""
    g = _gen(seed)
    c = (torch.rand(n_boxes, 2, generator=g, dtype=torch.float64) * 2 - 1) * (half - 10)
    size = 2 + 10 * torch.rand(n_boxes, 2, generator=g, dtype=torch.float64)
    hgt = 2 + 23 * torch.rand(n_boxes, generator=g, dtype=torch.float64)
    lo = torch.cat([c - size / 2, torch.zeros(n_boxes, 1, dtype=torch.float64)], 1)
    hi = torch.cat([c + size / 2, hgt[:, None]], 1)
    return World(lo, hi, half)


def robot_pose(robot: int, t: float, half: float = 100.0):
    """Position and heading of robot `robot` at time t: a Lissajous path at
    about 1 m/s, 1 m above the ground, kept inside the world."""
    a = 0.8 * (half - 20)
    w1, w2 = 0.011 + 0.0013 * robot, 0.007 + 0.0017 * robot
    ph = 0.9 * robot
    x = a * math.sin(w1 * t + ph)
    y = a * math.sin(w2 * t + 2 * ph)
    dx, dy = a * w1 * math.cos(w1 * t + ph), a * w2 * math.cos(w2 * t + 2 * ph)
    return (x, y, 1.0), math.atan2(dy, dx)


def world_scan(world: World, robot: int, t: float, kind: str, camera: int = 0, device="cpu",
               max_range: float = 30.0, seed: int = 0) -> RaySet:
    """A lidar scan ('lidar128x1024') or a depth frame ('depth424x240',
    camera 0 looks ahead, camera 1 to the left) of robot `robot` at time t."""
    pos, yaw = robot_pose(robot, t, world.half)
    o = torch.tensor(pos, dtype=torch.float64, device=device)
    if kind.startswith("lidar"):
        beams, az = (int(v) for v in kind[5:].split("x"))
        d = lidar_directions(beams, az, 22.5, device=device)
        cy, sy = math.cos(yaw), math.sin(yaw)
        u = torch.stack([cy * d[:, 0] - sy * d[:, 1], sy * d[:, 0] + cy * d[:, 1], d[:, 2]], dim=1)
        zscale = None
    else:
        w, h = (int(v) for v in kind[5:].split("x"))
        heading = yaw + (math.pi / 2 if camera else 0.0)
        cy, sy = math.cos(heading), math.sin(heading)
        f = torch.tensor([cy, sy, -0.2], dtype=torch.float64)
        f = f / f.norm()
        r = torch.tensor([sy, -cy, 0.0], dtype=torch.float64)
        dn = torch.linalg.cross(f, r)
        u, zscale = pinhole_directions(w, h, torch.stack([r, dn, f], dim=1), fx=525.0 * w / 640.0, device=device)
    t_ground = torch.where(u[:, 2] < 0, -o[2] / torch.where(u[:, 2] < 0, u[:, 2], -torch.ones_like(u[:, 2])),
                           torch.full_like(u[:, 2], float("inf")))
    t_box = _ray_box_entry(o, u, world.boxes_lo.to(device), world.boxes_hi.to(device)).min(1).values
    t = torch.minimum(t_ground, t_box)
    g = _gen(seed)
    noise = (torch.randn(u.shape[0], generator=g, dtype=torch.float64) * 0.02).to(device)
    if zscale is None:
        no_ret = t >= max_range
        rng = torch.where(no_ret, torch.full_like(t, max_range), t + noise)
    else:
        z = t * zscale
        no_ret = (z <= 0.3) | (z > 6.0)
        rng = torch.where(no_ret, 6.0 / zscale, t)
    e = o[None] + rng[:, None] * u
    return RaySet(o[None].float(), e.float(), no_ret.to(torch.uint8) * FLAG_NO_RETURN)
