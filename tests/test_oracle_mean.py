"""Pins of the oracle's voxel-mean layer (Sec. III-C: a 10-bit-per-axis
sub-voxel mean packed in 32 bits plus a 32-bit sample count) against hand
values, exact rational means and the exact NDT mean of the same samples."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import LAYER_COUNTS, LAYER_MEAN, LAYER_NDT, LAYER_OCCUPANCY

U = 1 << 16
VS = 0.1


def _map(**kw):
    p = dict(voxel_size=VS, layers=LAYER_OCCUPANCY | LAYER_COUNTS | LAYER_MEAN | LAYER_NDT, max_range=1e6)
    p.update(kw)
    return oracle.OracleMap(**p)


def _mean_word(m, voxel):
    """(count, mx, my, mz) of one voxel from the export."""
    ex = m.export(occupancy=False, ndt=False, tsdf=False)
    key = np.array([c // 32 for c in voxel])
    r = int(np.nonzero((ex["keys"] == key).all(1))[0][0])
    lx, ly, lz = (c % 32 for c in voxel)
    return tuple(int(x) for x in ex["mean"][r, lx + 32 * (ly + 32 * lz)]), int(ex["hits"][r, lx + 32 * (ly + 32 * lz)])


def _points_in_voxel(offsets_1024):
    """World points in voxel (0, 0, 0) whose positions inside it are the given
    multiples of 1/1024 voxel (exactly representable: 0.1 m / 1024 steps are
    not, so the fixed-point offsets are checked by the caller)."""
    return (np.asarray(offsets_1024, np.float64) + 0.25) / 1024.0 * VS


def test_hand_values_two_calls():
    """One sample at 100/1024 then one at 101/1024 (x): after two calls the
    mean is round-half-up(201 / 2) = 101; y, z the same way."""
    m = _map()
    o = np.array([[-1.0, -1.0, -1.0]], np.float32)
    for k in (100, 101):
        e = np.float32(_points_in_voxel([[k, 2 * k, 5]]))
        prep = m.prepare(o, e)
        assert [int(q) * 1024 // U for q in prep["qe"][0]] == [k, 2 * k, 5]
        m.integrate(o, e)
    (n, mx, my, mz), hits = _mean_word(m, (0, 0, 0))
    assert (n, mx, my, mz) == (2, 101, 201, 5) and hits == 2


def test_one_call_is_the_rounded_exact_mean():
    rng = np.random.default_rng(0)
    m = _map()
    pts = rng.uniform(0.0, VS, size=(37, 3)).astype(np.float32)
    o = np.array([[-2.0, 0.03, 0.07]], np.float32)
    m.integrate(o, pts)
    q = m.prepare(o, pts)["qe"]
    (n, *mm), hits = _mean_word(m, (0, 0, 0))
    assert n == hits == 37
    for a in range(3):
        p10 = [int(q[i, a]) * 1024 // U for i in range(37)]
        exact = Fraction(sum(p10), 37)
        assert mm[a] == int(exact + Fraction(1, 2))  # round half up


def test_order_of_samples_within_a_call_does_not_matter():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.3, 0.3, size=(500, 3)).astype(np.float32)
    o = np.array([[0.0, 0.0, 1.0]], np.float32)
    a, b = _map(), _map()
    a.integrate(o, pts)
    b.integrate(o, pts[rng.permutation(500)])
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["mean"], eb["mean"])


@pytest.mark.parametrize("calls", [1, 6])
def test_mean_tracks_the_exact_ndt_mean(calls):
    """Against the exact NDT mean of the same samples: quantising each sample
    down to 1/1024 voxel and reconstructing at +1/2 costs at most 1/2048 of a
    voxel, and every call's rounding at most another 1/2048."""
    rng = np.random.default_rng(2 + calls)
    m = _map()
    o = np.array([[0.0, 0.0, 0.0]], np.float32)
    for c in range(calls):
        centre = np.array([0.45, -0.25, 0.15])
        pts = (centre + rng.normal(size=(400, 3)) * 0.08).astype(np.float32)
        m.integrate(o, pts)
    vox, mom = m.ndt_sparse()
    pts_w = (vox.astype(np.float64) + 0.5) * VS
    q = m.query(pts_w)
    nd = q["ndt"]
    assert np.array_equal(q["mean"][:, 3], nd[:, 0])
    bound = (0.5 + 0.5 * calls) / 1024.0 * VS + 1e-12
    err = np.abs(q["mean"][:, :3] - nd[:, 1:4]).max()
    assert err <= bound, (err, bound)


def test_empty_voxel_has_no_mean():
    m = _map()
    m.integrate(np.array([[0.0, 0.0, 0.0]], np.float32), np.array([[0.95, 0.05, 0.05]], np.float32))
    q = m.query(np.array([[0.55, 0.05, 0.05]], np.float32))  # passed through, no sample
    assert q["mean"][0, 3] == 0 and np.isnan(q["mean"][0, :3]).all()


def test_mean_only_map_sees_its_samples():
    m = _map(layers=LAYER_MEAN)
    m.integrate(np.array([[-1.0, 0.05, 0.05]], np.float32), np.array([[0.05, 0.05, 0.05]], np.float32))
    assert m.region_count() == 2  # the ray passes through region -1 and ends in region 0
    q = m.query(np.array([[0.05, 0.05, 0.05]], np.float32))
    assert q["mean"][0, 3] == 1
    assert np.allclose(q["mean"][0, :3], 0.05, atol=VS / 1024)
