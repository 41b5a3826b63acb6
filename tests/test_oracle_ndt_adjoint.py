"""Pins of the oracle's NDT-OM adjoint (oracle_ndt_frame_eval): the loss is
the sample statistics of Sec. II-D / III-C (per voxel the mean and the
population covariance of its samples), and its analytic gradient with respect
to the frame's sample positions -- the voxel of every sample held fixed -- must
equal closed forms, an invariant of the covariance, and float64 central
finite differences of the oracle's own loss."""
import numpy as np

import oracle
from oracle import adjoint
from paper_2206_06079_gb300 import synth, workloads as W

VS = 0.1


def _map():
    return oracle.OracleMap(**W.oracle_params(W.tunnel_params(layers=W.OCC | W.NDT, max_range=20.0)))


def _one_voxel_frame(k=7, seed=0):
    """k samples inside voxel (12, 3, 5), rays from a common origin."""
    rng = np.random.default_rng(seed)
    v = np.array([12, 3, 5])
    e = ((v + rng.uniform(0.05, 0.95, size=(k, 3))) * VS).astype(np.float32)
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    return o, e, np.zeros(k, np.uint8), v


def test_mean_gradient_is_one_over_n():
    m = _map()
    o, e, f, v = _one_voxel_frame()
    gm = np.array([[0.3, -1.2, 2.0]])
    L, ge = adjoint.ndt_frame_eval(m, o, e, f, e.astype(np.float64), v[None], gm, np.zeros((1, 6)))
    assert np.allclose(L, gm[0] @ e.astype(np.float64).mean(0), rtol=1e-13)
    assert np.allclose(ge, np.broadcast_to(gm / len(e), ge.shape), rtol=1e-13, atol=0)


def test_covariance_is_the_population_covariance_and_its_gradients_sum_to_zero():
    m = _map()
    o, e, f, v = _one_voxel_frame(k=9, seed=1)
    rng = np.random.default_rng(2)
    gc = rng.normal(size=(1, 6))
    L, ge = adjoint.ndt_frame_eval(m, o, e, f, e.astype(np.float64), v[None], np.zeros((1, 3)), gc)
    C = np.cov(e.astype(np.float64).T, bias=True)
    packed = np.array([C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]])
    assert np.isclose(L, gc[0] @ packed, rtol=1e-10, atol=1e-18)
    # the covariance does not change when every sample moves together
    assert np.abs(ge.sum(0)).max() < 1e-12 * np.abs(ge).max()
    # closed form: dL/de_j = (1/n) (G + G^T)(e_j - mean)
    G = np.zeros((3, 3))
    G[np.triu_indices(3)] = gc[0]
    d = e.astype(np.float64) - e.astype(np.float64).mean(0)
    assert np.allclose(ge, d @ (G + G.T).T / len(e), rtol=1e-10, atol=1e-15)


def _frame_with_prior():
    """A tunnel lidar frame into a map that already holds an earlier scan's
    samples, query voxels at sampled voxels with random weights."""
    m = _map()
    prior = synth.tunnel_scan(0, beams=16, azimuths=256, max_range=20.0)
    m.integrate(*prior.numpy())
    rays = synth.tunnel_scan(1, beams=16, azimuths=256, max_range=20.0)
    o, e, f = rays.numpy()
    rng = np.random.default_rng(4)
    sel = np.flatnonzero(f == 0)
    pick = rng.choice(sel, size=200, replace=False)
    qvox = np.floor(e[pick].astype(np.float64) / VS).astype(np.int64)
    qvox = np.unique(qvox, axis=0)
    gm = rng.normal(size=(len(qvox), 3))
    gc = rng.normal(size=(len(qvox), 6)) * 50.0
    return m, o, e, f, qvox, gm, gc


def test_endpoint_gradient_matches_finite_differences():
    m, o, e, f, qvox, gm, gc = _frame_with_prior()
    e64 = e.astype(np.float64)
    L0, ge = adjoint.ndt_frame_eval(m, o, e, f, e64, qvox, gm, gc)
    cand = np.flatnonzero(np.abs(ge).sum(1) > 0)
    assert len(cand) > 20
    rng = np.random.default_rng(5)
    h = 1e-5
    for j in rng.choice(cand, size=20, replace=False):
        for k in range(3):
            ep, em = e64.copy(), e64.copy()
            ep[j, k] += h
            em[j, k] -= h
            fd = (adjoint.ndt_frame_eval(m, o, e, f, ep, qvox, gm, gc)[0] -
                  adjoint.ndt_frame_eval(m, o, e, f, em, qvox, gm, gc)[0]) / (2 * h)
            assert abs(fd - ge[j, k]) <= 1e-6 * max(1.0, abs(ge[j, k])), (j, k, fd, ge[j, k])


def test_twist_gradient_matches_finite_differences():
    m, o, e, f, qvox, gm, gc = _frame_with_prior()
    e64 = e.astype(np.float64)
    _, ge = adjoint.ndt_frame_eval(m, o, e, f, e64, qvox, gm, gc)
    gxi = adjoint.twist_from_point_gradients(e64, ge)
    h = 1e-6
    fd = np.zeros(6)
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Tp, Tm = adjoint.twist_matrix(xi), adjoint.twist_matrix(-xi)
        Lp = adjoint.ndt_frame_eval(m, o, e, f, e64 @ Tp[:3, :3].T + Tp[:3, 3], qvox, gm, gc)[0]
        Lm = adjoint.ndt_frame_eval(m, o, e, f, e64 @ Tm[:3, :3].T + Tm[:3, 3], qvox, gm, gc)[0]
        fd[k] = (Lp - Lm) / (2 * h)
    assert np.linalg.norm(gxi - fd) <= 1e-6 * np.linalg.norm(fd), (gxi, fd)


def test_loss_at_the_nominal_rays_matches_the_integrated_map():
    """Evaluated at the (float) nominal sample positions, the oracle's loss
    equals the loss formed from the statistics of the map after integrating
    the frame, up to the fixed-point quantisation of the samples."""
    m, o, e, f, qvox, gm, gc = _frame_with_prior()
    L, _ = adjoint.ndt_frame_eval(m, o, e, f, e.astype(np.float64), qvox, gm, gc)
    m.integrate(o, e, f)
    r = m.query(((qvox + 0.5) * VS).astype(np.float32))["ndt"]
    has = r[:, 0] > 0
    L_map = (gm[has] * r[has, 1:4]).sum() + (gc[has] * r[has, 4:10]).sum()
    assert abs(L - L_map) <= 1e-6 * max(1.0, abs(L)), (L, L_map)
