"""Helpers comparing a GPU map (through the C ABI) with the oracle."""
import numpy as np
import torch

import oracle
from paper_2206_06079_gb300 import ohm


def gpu_region_order(gm: ohm.Map):
    """GPU region keys and the permutation sorting them like the oracle."""
    n = gm.region_count()
    keys = gm.export(occupancy=False, count=n)["keys"].cpu().numpy().astype(np.int64)
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    return keys, order


def compare_dense(gm: ohm.Map, om: oracle.OracleMap, occupancy=True, counts=True, tsdf=False,
                  tsdf_atol=1e-5, batch=1024, path=False, mean=False):
    """Region set equal; occupancy bit-exact; hit/miss counts exact; TSDF D
    within tsdf_atol and W exact; decay-rate path sums exact (both sides
    use the same integer definition); voxel-mean words exact.  Returns the
    number of regions compared."""
    keys, order = gpu_region_order(gm)
    n = len(order)
    assert n == om.region_count(), (n, om.region_count())
    for i0 in range(0, n, batch):
        i1 = min(n, i0 + batch)
        ref = om.export(first=i0, count=i1 - i0, occupancy=occupancy, counts=counts, ndt=False, tsdf=tsdf,
                        path=path, mean=mean)
        assert np.array_equal(keys[order[i0:i1]], ref["keys"]), "region keys differ"
        slots = torch.from_numpy(order[i0:i1]).cuda()
        for s0 in range(0, i1 - i0, 256):
            sl = slots[s0:s0 + 256]
            # export contiguous GPU slots covering this batch, then gather
            lo, hi = int(sl.min()), int(sl.max()) + 1
            ex = gm.export(occupancy=occupancy, counts=counts, tsdf=tsdf, path_sum=path, mean=mean, first=lo,
                           count=hi - lo)
            idx = sl - lo
            r = slice(s0, s0 + len(sl))
            if occupancy:
                g = ex["occupancy"][idx].cpu().numpy()
                o = ref["occupancy"][r]
                known = ~np.isnan(o)
                assert np.array_equal(~np.isnan(g), known), "known voxel sets differ"
                assert np.array_equal(g[known].view(np.uint32), o[known].view(np.uint32)), "occupancy differs"
            if counts:
                c = ex["counts"][idx].cpu().numpy().view(np.uint32)
                assert np.array_equal(c[..., 0], ref["hits"][r]), "hit counts differ"
                assert np.array_equal(c[..., 1], ref["misses"][r]), "miss counts differ"
            if path:
                ps = ex["path_sum"][idx].cpu().numpy().view(np.uint64)
                assert np.array_equal(ps, ref["path"][r]), "decay path sums differ"
            if mean:
                w = ex["mean"][idx].cpu().numpy().view(np.uint64)
                dec = np.stack([w >> 32, w & 1023, (w >> 10) & 1023, (w >> 20) & 1023], -1).astype(np.uint32)
                assert np.array_equal(dec, ref["mean"][r]), "voxel means differ"
                assert not ((w >> 30) & 3).any(), "unused bits of a voxel-mean word set"
            if tsdf:
                t = ex["tsdf"][idx].cpu().numpy().astype(np.float64)
                assert np.array_equal(t[..., 1], ref["tsdf"][r][..., 1]), "TSDF weights differ"
                err = np.abs(t[..., 0] - ref["tsdf"][r][..., 0]).max()
                assert err <= tsdf_atol, "TSDF distance differs by %g" % err
    return n


def gpu_ndt_sparse(gm: ohm.Map, batch=64):
    """(voxels, moments) of every GPU voxel holding a sample, in oracle order."""
    keys, order = gpu_region_order(gm)
    vox_all, mom_all = [], []
    n = len(keys)
    lin = torch.arange(ohm.REGION_VOXELS, device="cuda")
    local = torch.stack([lin % 32, (lin // 32) % 32, lin // 1024], 1)
    for s0 in range(0, n, batch):
        cnt = min(batch, n - s0)
        ex = gm.export(occupancy=False, ndt=True, first=s0, count=cnt)
        nd = ex["ndt"]
        hit = nd[..., 0] > 0
        r, v = torch.nonzero(hit, as_tuple=True)
        k = ex["keys"].long()[r] * 32 + local[v]
        vox_all.append(k.cpu().numpy())
        mom_all.append(nd[r, v].cpu().numpy())
    vox = np.concatenate(vox_all) if vox_all else np.zeros((0, 3), np.int64)
    mom = np.concatenate(mom_all) if mom_all else np.zeros((0, 10), np.int64)
    return vox, mom


def compare_ndt(gm: ohm.Map, om: oracle.OracleMap):
    """Exact equality of every sample voxel's integer moments."""
    gv, gmom = gpu_ndt_sparse(gm)
    ov, omom = om.ndt_sparse()
    assert len(gv) == len(ov), (len(gv), len(ov))
    og = np.lexsort((gv[:, 0], gv[:, 1], gv[:, 2]))
    oo = np.lexsort((ov[:, 0], ov[:, 1], ov[:, 2]))
    assert np.array_equal(gv[og], ov[oo]), "NDT voxel sets differ"
    assert np.array_equal(gmom[og], omom[oo]), "NDT moments differ"
    return len(gv), ov


def compare_query(gm: ohm.Map, om: oracle.OracleMap, pts: np.ndarray, ndt=False, tsdf=False, ndt_rtol=1e-4,
                  tsdf_atol=1e-5, path=False, mean=False):
    g = gm.query(torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda(), ndt=ndt, tsdf=tsdf,
                 path_sum=path, mean=mean)
    r = om.query(pts)
    if mean:
        gm4 = g["mean"].cpu().numpy().astype(np.float64)
        assert np.array_equal(gm4[:, 3], r["mean"][:, 3]), "voxel-mean counts differ"
        assert np.allclose(gm4[:, :3], r["mean"][:, :3], rtol=1e-6, atol=1e-6, equal_nan=True), "voxel means differ"
    if path:
        assert np.array_equal(g["path_sum"].cpu().numpy().view(np.uint64), r["path"]), "decay path sums differ"
    assert np.array_equal(g["known"].cpu().numpy(), r["known"]), "known flags differ"
    k = r["known"] == 1
    go = g["occupancy"].cpu().numpy()
    assert np.array_equal(go[k].view(np.uint32), r["occupancy"][k].view(np.uint32)), "occupancy differs"
    assert np.isnan(go[~k]).all()
    if ndt:
        gn = g["ndt"].cpu().numpy().astype(np.float64)
        rn = r["ndt"]
        assert np.array_equal(gn[:, 0], rn[:, 0]), "NDT counts differ"
        s = rn[:, 0] > 0
        assert np.allclose(gn[s, 1:4], rn[s, 1:4], rtol=ndt_rtol, atol=0), "NDT means differ"
        # covariance: relative to the voxel's squared size (entries can be ~0)
        vs2 = gm.params["voxel_size"] ** 2
        assert np.allclose(gn[s, 4:], rn[s, 4:], rtol=ndt_rtol, atol=ndt_rtol * vs2), "NDT covariances differ"
    if tsdf:
        gt = g["tsdf"].cpu().numpy().astype(np.float64)
        assert np.array_equal(gt[:, 1], r["tsdf"][:, 1])
        assert np.abs(gt[:, 0] - r["tsdf"][:, 0]).max(initial=0) <= tsdf_atol
    return int(k.sum())


def export_sorted(gm: ohm.Map):
    """Every layer of every region, regions sorted by key (CPU tensors)."""
    L = gm.params["layers"]
    ex = gm.export(occupancy=bool(L & ohm.LAYER_OCCUPANCY), counts=bool(L & ohm.LAYER_COUNTS),
                   ndt=bool(L & ohm.LAYER_NDT), tsdf=bool(L & ohm.LAYER_TSDF), path_sum=bool(L & ohm.LAYER_DECAY),
                   mean=bool(L & ohm.LAYER_MEAN))
    keys = ex["keys"].cpu().numpy()
    order = torch.from_numpy(np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))).to(ex["keys"].device)
    out = {}
    for k, v in ex.items():
        v = v[order]
        if v.dtype == torch.float32:
            v = v.view(torch.int32)  # bitwise comparison (NaN = unknown)
        out[k] = v.cpu()
    return out


def assert_maps_identical(a: ohm.Map, b: ohm.Map):
    ea, eb = export_sorted(a), export_sorted(b)
    assert ea.keys() == eb.keys()
    for k in ea:
        assert torch.equal(ea[k], eb[k]), "layer %s differs" % k


def compare_resident_with_oracle(gm: ohm.Map, om: oracle.OracleMap):
    """For a map whose pool evicted regions to host memory: every region live
    on the device (a pool slot with an observed voxel; released slots read as
    unobserved) equals the oracle's region of the same key, occupancy bit for
    bit and NDT moments exactly.  Returns the number of regions compared."""
    n = gm.region_count()
    L = gm.params["layers"]
    ndt = bool(L & ohm.LAYER_NDT)
    ex = gm.export(occupancy=True, ndt=ndt, count=n)
    keys = ex["keys"].cpu().numpy().astype(np.int64)
    occ = ex["occupancy"].cpu().numpy()
    live = np.flatnonzero(~np.isnan(occ).all(1))
    ref = om.export(occupancy=True, counts=False, ndt=ndt, tsdf=False, path=False, mean=False)
    index = {tuple(k): i for i, k in enumerate(ref["keys"].tolist())}
    for s in live:
        j = index.get(tuple(keys[s].tolist()))
        assert j is not None, "a live region is unknown to the oracle"
        o = ref["occupancy"][j]
        known = ~np.isnan(o)
        assert np.array_equal(~np.isnan(occ[s]), known), "known voxel sets differ"
        assert np.array_equal(occ[s][known].view(np.uint32), o[known].view(np.uint32)), "occupancy differs"
        if ndt:
            g = ex["ndt"][s].cpu().numpy()
            assert np.array_equal(g, ref["ndt"][j]), "NDT moments differ"
    return len(live)
