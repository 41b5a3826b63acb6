"""Pins of the oracle's TSDF adjoint: its analytic gradients with respect to
per-pixel depth and the pose twist equal float64 central finite differences
of its own frozen-voxel-set loss (the voxel sets held fixed, Sec. II-F TSDF
update)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint
from paper_2206_06079_gb300 import synth, workloads as W

W_, H_ = 48, 36
S_ = W_ / 640.0
K = (525.0 * S_, 525.0 * S_, (W_ - 1) / 2.0, (H_ - 1) / 2.0)


def _frame(i, scene):
    depth, pos, R = synth.depth_frame(scene, i, width=W_, height=H_, fx=K[0], fy=K[1], cx=K[2], cy=K[3])
    pose = np.concatenate([R.numpy(), pos.numpy()[:, None]], 1)
    return depth.numpy(), pose


def _setup():
    scene = synth.depth_scene()
    m = oracle.OracleMap(**W.oracle_params(W.tsdf_params()))
    d0, p0 = _frame(3, scene)
    o, e, f, _ = adjoint.depth_rays(d0, K, p0, 0.3, 6.0)
    m.integrate(o, e, f)                           # prior state: W, D nonzero
    depth, pose = _frame(5, scene)
    o, e, f, pt = adjoint.depth_rays(depth, K, pose, 0.3, 6.0)
    rng = np.random.default_rng(3)
    vs = 0.05
    # query voxels around the samples, along the rays
    sel = np.flatnonzero(f == 0)
    pick = rng.choice(sel, size=300, replace=False)
    u = e[pick] - o[0]
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    off = rng.uniform(-0.18, 0.18, size=(300, 1))
    qpts = e[pick] + off * u
    qvox = np.floor(qpts / vs).astype(np.int64)
    g = rng.normal(size=300)
    return m, depth, pose, o, e, f, pt, qvox, g


def _eval_geometry(depth, pose, z_override=None):
    """Continuous (float64) origin and endpoints of the frame."""
    fx, fy, cx, cy = K
    h, w = depth.shape
    vv, uu = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    z = depth.astype(np.float64).reshape(-1) if z_override is None else z_override
    z = np.where((z > 0.3) & (z <= 6.0), z, 6.0)
    pc = np.stack([(uu.reshape(-1) - cx) / fx * z, (vv.reshape(-1) - cy) / fy * z, z], 1)
    return pose[:, 3].astype(np.float64), pc @ pose[:, :3].T + pose[:, 3]


def test_depth_gradient_matches_finite_differences():
    m, depth, pose, o, e, f, pt, qvox, g = _setup()
    o64, e64 = _eval_geometry(depth, pose)
    L0, ge, go = adjoint.frame_eval(m, o[0], e, f, o64, e64, qvox, g)
    gz, _ = adjoint.chain_to_depth_and_twist(ge, go, e64, o64, pose[:, :3], pt)
    rng = np.random.default_rng(4)
    cand = np.flatnonzero((f == 0) & (np.abs(gz) > 1e-6))
    assert len(cand) > 40
    smooth = 0
    for j in rng.choice(cand, size=40, replace=False):
        fd = []
        for h in (1e-4, 5e-5):
            z = depth.astype(np.float64).reshape(-1).copy()
            z[j] += h
            Lp = adjoint.frame_eval(m, o[0], e, f, *_eval_geometry(depth, pose, z), qvox, g)[0]
            z[j] -= 2 * h
            Lm = adjoint.frame_eval(m, o[0], e, f, *_eval_geometry(depth, pose, z), qvox, g)[0]
            fd.append((Lp - Lm) / (2 * h))
        if abs(fd[0] - fd[1]) > 1e-7 * max(1.0, abs(fd[1])):
            continue  # a clamp kink lies within h: finite differences are not meaningful here
        smooth += 1
        assert abs(fd[0] - gz[j]) <= 1e-6 * max(abs(gz[j]), 1e-3), (j, fd[0], gz[j])
    assert smooth >= 32


def test_twist_gradient_matches_finite_differences():
    m, depth, pose, o, e, f, pt, qvox, g = _setup()
    o64, e64 = _eval_geometry(depth, pose)
    _, ge, go = adjoint.frame_eval(m, o[0], e, f, o64, e64, qvox, g)
    _, gxi = adjoint.chain_to_depth_and_twist(ge, go, e64, o64, pose[:, :3], pt)
    h = 1e-6
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Tp, Tm = adjoint.twist_matrix(xi), adjoint.twist_matrix(-xi)
        Lp = adjoint.frame_eval(m, o[0], e, f, Tp[:3, :3] @ o64 + Tp[:3, 3], e64 @ Tp[:3, :3].T + Tp[:3, 3], qvox, g)[0]
        Lm = adjoint.frame_eval(m, o[0], e, f, Tm[:3, :3] @ o64 + Tm[:3, 3], e64 @ Tm[:3, :3].T + Tm[:3, 3], qvox, g)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gxi[k]) <= 1e-5 * max(abs(gxi[k]), 1e-2), (k, fd, gxi[k])


def test_loss_with_no_rays_is_the_prior_state():
    m, depth, pose, o, e, f, pt, qvox, g = _setup()
    allbad = np.ones_like(f)
    L, ge, go = adjoint.frame_eval(m, o[0], e, allbad, *_eval_geometry(depth, pose), qvox, g)
    D = m.query((qvox + 0.5) * 0.05)["tsdf"][:, 0]
    assert abs(L - float((g * D).sum())) < 1e-12 and not ge.any() and not go.any()
