"""TSDF and NDT-OM adjoint references (TEST INFRASTRUCTURE ONLY): depth-image
and posed lidar rays, the chain rule from endpoint / origin gradients to
per-pixel depth and pose-twist gradients, in float64 numpy around the C++
oracle's frozen-voxel-set losses (oracle_tsdf_frame_eval,
oracle_ndt_frame_eval).

Depth back-projection (the same formula, operation for operation, as the CUDA
library's depth entry point): for pixel (u, v) with depth z,
    x = ((u - cx) / fx) * z,  y = ((v - cy) / fy) * z,
    e_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k   (double), stored as float32,
and the sensor origin is t (float32).  A pixel with z outside (z_min, z_max]
becomes a NO_RETURN ray at depth z_max.

Pose perturbation: a twist xi = (rho, phi) moves every world point p of the
frame to p + rho + phi x p (left perturbation), so dL/drho = sum_j (dL/de_j)
+ dL/do and dL/dphi = sum_j e_j x dL/de_j + o x dL/do.
"""
import ctypes

import numpy as np

from . import _load, _ptr

FLAG_NO_RETURN = 1


def depth_rays(depth, K, pose, z_min, z_max):
    """(origin (1, 3) float32, endpoints (h*w, 3) float32, flags, pixel
    directions p~ (h*w, 3) float64) of a z-depth image.  K = (fx, fy, cx, cy),
    pose = 3 x 4 camera-to-world [R | t]."""
    depth = np.asarray(depth, np.float32)
    h, w = depth.shape
    fx, fy, cx, cy = (float(k) for k in K)
    P = np.asarray(pose, np.float64)
    R, t = P[:, :3], P[:, 3]
    vv, uu = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    z = depth.astype(np.float64)
    valid = (z > z_min) & (z <= z_max)
    zz = np.where(valid, z, z_max)
    px = (uu - cx) / fx
    py = (vv - cy) / fy
    x = px * zz
    y = py * zz
    e = np.empty((h, w, 3), np.float64)
    for k in range(3):
        e[..., k] = ((R[k, 0] * x + R[k, 1] * y) + R[k, 2] * zz) + t[k]
    flags = (~valid).astype(np.uint8) * FLAG_NO_RETURN
    pt = np.stack([px, py, np.ones_like(px)], -1).reshape(-1, 3)
    return t.astype(np.float32)[None], e.reshape(-1, 3).astype(np.float32), flags.reshape(-1), pt


def frame_eval(omap, o_nom, e_nom, flags, o_eval, e_eval, qvox, g):
    """(L, dL/de (n, 3), dL/do (3,)) from the C++ oracle, float64."""
    o_nom = np.ascontiguousarray(o_nom, np.float32).reshape(3)
    e_nom = np.ascontiguousarray(e_nom, np.float32).reshape(-1, 3)
    f = np.ascontiguousarray(flags, np.uint8)
    o_eval = np.ascontiguousarray(o_eval, np.float64).reshape(3)
    e_eval = np.ascontiguousarray(e_eval, np.float64).reshape(-1, 3)
    qvox = np.ascontiguousarray(qvox, np.int64).reshape(-1, 3)
    g = np.ascontiguousarray(g, np.float64)
    n = e_nom.shape[0]
    loss = ctypes.c_double()
    ge = np.zeros((n, 3), np.float64)
    go = np.zeros(3, np.float64)
    lib = _load()
    lib.oracle_tsdf_frame_eval.restype = ctypes.c_int
    lib.oracle_tsdf_frame_eval.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 3 + [ctypes.c_int64] + \
        [ctypes.c_void_p] * 4 + [ctypes.c_int64] + [ctypes.c_void_p] * 3
    rc = lib.oracle_tsdf_frame_eval(omap._h, _ptr(o_nom), _ptr(e_nom), _ptr(f), n, _ptr(o_eval), _ptr(e_eval),
                                    _ptr(qvox), _ptr(g), len(g), ctypes.byref(loss), _ptr(ge), _ptr(go))
    if rc:
        raise ValueError("oracle_tsdf_frame_eval failed")
    return loss.value, ge, go


def posed_rays(origins, endpoints, pose):
    """Sensor-frame float rays moved to the world by a 3 x 4 camera-to-world
    pose [R | t], the same formula, operation for operation, as the CUDA
    library's posed entry point: p_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k in
    double, stored as float32.  Returns (origins, endpoints) float32 and the
    endpoints before rounding (float64)."""
    P = np.asarray(pose, np.float64).reshape(3, 4)

    def move(x):
        x = np.asarray(x, np.float32).reshape(-1, 3).astype(np.float64)
        out = np.empty_like(x)
        for k in range(3):
            out[:, k] = ((P[k, 0] * x[:, 0] + P[k, 1] * x[:, 1]) + P[k, 2] * x[:, 2]) + P[k, 3]
        return out
    o64, e64 = move(origins), move(endpoints)
    return o64.astype(np.float32), e64.astype(np.float32), e64


def ndt_frame_eval(omap, o_nom, e_nom, flags, e_eval, qvox, gm, gc):
    """(L, dL/de (n, 3)) of the NDT-OM frame loss from the C++ oracle
    (oracle_ndt_frame_eval), float64.  o_nom: one origin or one per ray."""
    o_nom = np.ascontiguousarray(o_nom, np.float32).reshape(-1, 3)
    e_nom = np.ascontiguousarray(e_nom, np.float32).reshape(-1, 3)
    n = e_nom.shape[0]
    f = np.ascontiguousarray(flags, np.uint8) if flags is not None else np.zeros(n, np.uint8)
    e_eval = np.ascontiguousarray(e_eval, np.float64).reshape(-1, 3)
    qvox = np.ascontiguousarray(qvox, np.int64).reshape(-1, 3)
    gm = np.ascontiguousarray(gm, np.float64).reshape(-1, 3)
    gc = np.ascontiguousarray(gc, np.float64).reshape(-1, 6)
    loss = ctypes.c_double()
    ge = np.zeros((n, 3), np.float64)
    lib = _load()
    lib.oracle_ndt_frame_eval.restype = ctypes.c_int
    lib.oracle_ndt_frame_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 2 + \
        [ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_int64] + [ctypes.c_void_p] * 2
    rc = lib.oracle_ndt_frame_eval(omap._h, _ptr(o_nom), o_nom.shape[0], _ptr(e_nom), _ptr(f), n, _ptr(e_eval),
                                   _ptr(qvox), _ptr(gm), _ptr(gc), qvox.shape[0], ctypes.byref(loss), _ptr(ge))
    if rc:
        raise ValueError("oracle_ndt_frame_eval failed")
    return loss.value, ge


def twist_from_point_gradients(points, grad):
    """Gradient with respect to a left twist (rho, phi) moving every point p
    to p + rho + phi x p, from per-point gradients: (sum g, sum p x g)."""
    points = np.asarray(points, np.float64).reshape(-1, 3)
    grad = np.asarray(grad, np.float64).reshape(-1, 3)
    return np.concatenate([grad.sum(0), np.cross(points, grad).sum(0)])


def band_margin(omap, o_nom, e_nom, flags, o_eval, e_eval):
    """Per ray, min over its frozen band voxels of | |s| - tau | at the
    continuous geometry (oracle_tsdf_band_margin); +inf without a band."""
    o_nom = np.ascontiguousarray(o_nom, np.float32).reshape(3)
    e_nom = np.ascontiguousarray(e_nom, np.float32).reshape(-1, 3)
    f = np.ascontiguousarray(flags, np.uint8)
    o_eval = np.ascontiguousarray(o_eval, np.float64).reshape(3)
    e_eval = np.ascontiguousarray(e_eval, np.float64).reshape(-1, 3)
    n = e_nom.shape[0]
    out = np.zeros(n, np.float64)
    lib = _load()
    lib.oracle_tsdf_band_margin.restype = ctypes.c_int
    lib.oracle_tsdf_band_margin.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64] + [ctypes.c_void_p] * 3
    if lib.oracle_tsdf_band_margin(omap._h, _ptr(o_nom), _ptr(e_nom), _ptr(f), n, _ptr(o_eval), _ptr(e_eval), _ptr(out)):
        raise ValueError("oracle_tsdf_band_margin failed")
    return out


def chain_to_depth_and_twist(ge, go, e_world, o_world, R, pt):
    """Per-pixel dL/dz = dL/de . (R p~) and the twist gradient (6,)."""
    de_dz = pt @ np.asarray(R, np.float64).T
    gz = (ge * de_dz).sum(1)
    rho = ge.sum(0) + go
    phi = np.cross(e_world, ge).sum(0) + np.cross(o_world, go)
    return gz, np.concatenate([rho, phi])


def twist_matrix(xi):
    """exp of a twist (rho, phi) as a 4 x 4 rigid transform (Rodrigues)."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = np.linalg.norm(phi)
    Kx = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        Rm, V = np.eye(3) + Kx, np.eye(3) + 0.5 * Kx
    else:
        Rm = np.eye(3) + np.sin(th) / th * Kx + (1 - np.cos(th)) / th ** 2 * Kx @ Kx
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * Kx + (th - np.sin(th)) / th ** 3 * Kx @ Kx
    T = np.eye(4)
    T[:3, :3] = Rm
    T[:3, 3] = V @ rho
    return T
