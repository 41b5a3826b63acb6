"""NDT-OM adjoint on the GPU (ohm_ndt_backward behind a torch.autograd.Function)
against the oracle's float64 analytic gradient and central finite
differences of its loss, the voxel of every sample held fixed; tolerance 1e-3
relative.  The posed forward pass (sensor-frame rays moved by a pose on the
device) is checked against the oracle first, moments bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint
from paper_2206_06079_gb300 import ohm, synth, workloads as W

from .parity import compare_ndt

pytestmark = pytest.mark.gpu

VS = 0.1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _params(**kw):
    return W.tunnel_params(layers=W.OCC | W.NDT, max_range=20.0, max_rays=32768, max_regions=8192,
                           max_ndt_regions=2048, **kw)


def _pose(seed):
    rng = np.random.default_rng(seed)
    R = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    return np.concatenate([R, rng.uniform(-2, 2, size=(3, 1))], 1)


def _setup(seed=0, beams=32, azimuths=512):
    """GPU map and oracle map holding a prior scan; the next scan as
    sensor-frame rays with a pose, query voxels and float32 weights."""
    gm = ohm.Map(**_params())
    om = oracle.OracleMap(**W.oracle_params(_params()))
    prior = synth.tunnel_scan(0, beams=beams, azimuths=azimuths, max_range=20.0)
    gm.integrate(prior.origins.cuda(), prior.endpoints.cuda(), prior.flags.cuda())
    om.integrate(*prior.numpy())
    frame = synth.tunnel_scan(1, beams=beams, azimuths=azimuths, max_range=20.0)
    o_w, e_w, f = frame.numpy()
    P = _pose(seed)
    R, t = P[:, :3], P[:, 3]
    # sensor-frame rays whose pose P brings them back near the scan's world rays
    o_s = ((o_w.astype(np.float64) - t) @ R).astype(np.float32)
    e_s = ((e_w.astype(np.float64) - t) @ R).astype(np.float32)
    o_p, e_p, e64 = adjoint.posed_rays(o_s, e_s, P)   # what the device computes, and before rounding
    rng = np.random.default_rng(seed + 1)
    sel = np.flatnonzero(f == 0)
    pick = rng.choice(sel, size=400, replace=False)
    qvox = np.unique(np.floor(e_p[pick].astype(np.float64) / VS).astype(np.int64), axis=0)
    gmean = rng.normal(size=(len(qvox), 3)).astype(np.float32)
    gcov = (rng.normal(size=(len(qvox), 6)) * 30.0).astype(np.float32)
    return gm, om, P, (o_s, e_s, f), (o_p, e_p, e64), qvox, gmean, gcov


def _gpu_backward(gm, P, rays_s, qvox, gmean, gcov):
    o_s, e_s, f = rays_s
    qpts = torch.from_numpy(((qvox + 0.5) * VS).astype(np.float32)).cuda()
    ge, gxi = gm.ndt_backward(P, torch.from_numpy(o_s).cuda(), torch.from_numpy(e_s).cuda(), torch.from_numpy(f).cuda(),
                              qpts, torch.from_numpy(gmean).cuda(), torch.from_numpy(gcov).cuda())
    return ge.cpu().numpy().astype(np.float64), gxi.cpu().numpy()


def _quantisation_bound(gm, e_p, samples, qvox, gcov):
    """Per sample, how far the GPU's gradient may sit from the oracle's
    because it forms d = p_j - S/n from the stored fixed-point positions: they
    differ from the continuous ones by at most DELTA = 4e-6 m per axis (half a
    2^-16-voxel unit, 7.6e-7 m, plus float32 rounding of world points within
    20 m, 1.2e-6 m, for p_j and for S/n), which moves (1/n)(G + G^T) d by at
    most |G + G^T|_F sqrt(3) DELTA / n."""
    DELTA = 4e-6
    vox = np.floor(e_p[samples].astype(np.float64) / VS).astype(np.int64)
    counts = gm.query(torch.from_numpy(e_p[samples]).cuda(), ndt=True)["ndt"][:, 0].cpu().numpy().astype(np.float64)
    row = {tuple(v): i for i, v in enumerate(qvox.tolist())}
    gsym = np.zeros(len(samples))
    for k, v in enumerate(vox.tolist()):
        G = np.zeros((3, 3))
        G[np.triu_indices(3)] = gcov[row[tuple(v)]]
        gsym[k] = np.linalg.norm(G + G.T)
    return gsym * np.sqrt(3) * DELTA / counts + 1e-9


def test_posed_forward_matches_oracle_and_adjoint_matches_analytic_gradient():
    gm, om, P, rays_s, (o_p, e_p, e64), qvox, gmean, gcov = _setup()
    o_s, e_s, f = rays_s
    # the oracle's analytic gradient at the continuous (double) world positions,
    # with the map state before the frame
    L, ge_w = adjoint.ndt_frame_eval(om, o_p, e_p, f, e64, qvox, gmean.astype(np.float64), gcov.astype(np.float64))
    ge_ref = ge_w @ P[:, :3]                      # R^T dL/dp per ray: sensor frame
    gxi_ref = adjoint.twist_from_point_gradients(e64, ge_w)
    # forward on both sides, moments bit for bit
    gm.integrate_posed(P, torch.from_numpy(o_s).cuda(), torch.from_numpy(e_s).cuda(), torch.from_numpy(f).cuda())
    ge, gxi = _gpu_backward(gm, P, rays_s, qvox, gmean, gcov)
    om.integrate(o_p, e_p, f)
    compare_ndt(gm, om)
    has = np.abs(ge_ref).sum(1) > 0
    assert has.sum() > 100
    assert np.array_equal(np.abs(ge).sum(1) > 0, has), "rays with a gradient differ"
    assert np.linalg.norm(ge - ge_ref) <= 1e-3 * np.linalg.norm(ge_ref)
    samples = np.flatnonzero(has)
    bound = 1e-3 * np.linalg.norm(ge_ref[samples], axis=1) + _quantisation_bound(gm, e_p, samples, qvox, gcov)
    err = np.linalg.norm(ge[samples] - ge_ref[samples], axis=1)
    assert (err <= bound).all(), (err.max(), int(np.argmax(err / bound)), float((err / bound).max()))
    assert np.linalg.norm(gxi - gxi_ref) <= 1e-3 * np.linalg.norm(gxi_ref), (gxi, gxi_ref)


def test_adjoint_against_finite_differences():
    """Central differences of the oracle's float64 loss (fixed voxel
    assignment) in the world positions of a few samples and in the pose twist."""
    gm, om, P, rays_s, (o_p, e_p, e64), qvox, gmean, gcov = _setup(seed=3, beams=16, azimuths=512)
    o_s, e_s, f = rays_s
    g64m, g64c = gmean.astype(np.float64), gcov.astype(np.float64)
    gm.integrate_posed(P, torch.from_numpy(o_s).cuda(), torch.from_numpy(e_s).cuda(), torch.from_numpy(f).cuda())
    ge, gxi = _gpu_backward(gm, P, rays_s, qvox, gmean, gcov)
    ge_w = ge @ P[:, :3].T                          # back to world: R dL/de_s
    rng = np.random.default_rng(7)
    cand = np.flatnonzero(np.abs(ge).sum(1) > 1e-3 * np.abs(ge).sum(1).max())
    pick = rng.choice(cand, size=min(15, len(cand)), replace=False)
    qb = _quantisation_bound(gm, e_p, pick, qvox, gcov)
    h = 1e-5
    for j, q in zip(pick, qb):
        fd = np.zeros(3)
        for k in range(3):
            ep, em = e64.copy(), e64.copy()
            ep[j, k] += h
            em[j, k] -= h
            fd[k] = (adjoint.ndt_frame_eval(om, o_p, e_p, f, ep, qvox, g64m, g64c)[0] -
                     adjoint.ndt_frame_eval(om, o_p, e_p, f, em, qvox, g64m, g64c)[0]) / (2 * h)
        assert np.linalg.norm(ge_w[j] - fd) <= 1e-3 * np.linalg.norm(fd) + q, (j, ge_w[j], fd)
    hx = 1e-6
    fdxi = np.zeros(6)
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = hx
        Tp, Tm = adjoint.twist_matrix(xi), adjoint.twist_matrix(-xi)
        Lp = adjoint.ndt_frame_eval(om, o_p, e_p, f, e64 @ Tp[:3, :3].T + Tp[:3, 3], qvox, g64m, g64c)[0]
        Lm = adjoint.ndt_frame_eval(om, o_p, e_p, f, e64 @ Tm[:3, :3].T + Tm[:3, 3], qvox, g64m, g64c)[0]
        fdxi[k] = (Lp - Lm) / (2 * hx)
    assert np.linalg.norm(gxi - fdxi) <= 1e-3 * np.linalg.norm(fdxi), (gxi, fdxi)


def test_autograd_function_wraps_the_kernel():
    gm, om, P, rays_s, _, qvox, gmean, gcov = _setup(seed=5, beams=16, azimuths=256)
    o_s, e_s, f = (torch.from_numpy(x).cuda() for x in rays_s)
    gm2 = ohm.Map(**_params())
    prior = synth.tunnel_scan(0, beams=16, azimuths=256, max_range=20.0)
    gm2.integrate(prior.origins.cuda(), prior.endpoints.cuda(), prior.flags.cuda())
    qpts = torch.from_numpy(((qvox + 0.5) * VS).astype(np.float32)).cuda()
    e = e_s.clone().requires_grad_(True)
    xi = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    mean, cov = ohm.NdtFrame.apply(e, xi, gm, P, o_s, f, qpts)
    gmt, gct = torch.from_numpy(gmean).cuda(), torch.from_numpy(gcov).cuda()
    ((mean * gmt).sum() + (cov * gct).sum()).backward()
    gm2.integrate_posed(ohm.twist_pose(np.zeros(6), P), o_s, e_s, f)
    ref_e, ref_xi = gm2.ndt_backward(ohm.twist_pose(np.zeros(6), P), o_s, e_s, f, qpts, gmt, gct)
    assert torch.equal(e.grad, ref_e)
    assert torch.allclose(xi.grad, ref_xi.cpu().to(xi.grad.dtype))
    assert float(ref_e.abs().sum()) > 0


def test_adjoint_refuses_maps_that_clear_samples():
    gm = ohm.Map(**_params(ndt_clear_below=0.0))
    z = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ohm.OhmError) as ei:
        gm.ndt_backward(np.eye(3, 4), z[:1], z, None, z, z, torch.zeros((4, 6), device="cuda"))
    assert ei.value.code == ohm.ERR_UNSUPPORTED
