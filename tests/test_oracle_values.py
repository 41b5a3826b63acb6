"""Pins of the oracle's quantiser, truncation, log-odds, hit/miss counts, NDT
statistics and TSDF values against exact arithmetic and closed forms."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import FLAG_NO_RETURN, LAYER_COUNTS, LAYER_NDT, LAYER_OCCUPANCY, LAYER_TSDF

U = 1 << 16
HIT = float(np.float32(oracle.logit(0.7)))
MISS = float(np.float32(oracle.logit(0.4)))


def test_logit_constants():
    # Eq. 3 with P(z|occ)/P(z|emp) = 0.7/0.3 and 0.4/0.6; the workload quotes
    # them rounded as +0.847 and -0.405.
    assert abs(HIT - 0.847) < 5e-4 and abs(MISS + 0.405) < 5e-4


def test_quantisation_matches_exact_rounding():
    """q = rint((x - o) * 2^F / vs): the double evaluation differs from exact
    rational rounding by at most one unit, and only next to a half-unit tie."""
    rng = np.random.default_rng(1)
    vs = 0.1
    origin = (0.3, -1.7, 2.25)
    m = oracle.OracleMap(voxel_size=vs, map_origin=origin, max_range=1e6)
    pts = rng.uniform(-60, 60, size=(5000, 3)).astype(np.float32)
    prep = m.prepare(pts[:1], pts)
    q = prep["qe"]
    scale = Fraction(U) / Fraction(vs)
    for i in range(0, 5000, 7):
        for k in range(3):
            exact = (Fraction(float(pts[i, k])) - Fraction(origin[k])) * scale
            assert abs(q[i, k] - exact) <= Fraction(1, 2) + Fraction(1, 10 ** 6)
            # the voxel index is floor((x - o) / vs) away from faces
            v = q[i, k] >> 16
            frac = exact / U - math.floor(exact / U)
            if Fraction(1, 1000) < frac < Fraction(999, 1000):
                assert v == math.floor(exact / U)


def test_truncation_to_max_range():
    rng = np.random.default_rng(2)
    m = oracle.OracleMap(max_range=20.0)
    o = np.array([[0.37, -0.21, 1.05]], np.float32)
    u = rng.normal(size=(400, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    length = rng.uniform(1, 60, size=400)
    e = (o + u * length[:, None]).astype(np.float32)
    flags = (rng.uniform(size=400) < 0.2).astype(np.uint8)
    prep = m.prepare(o, e, flags)
    scale = U / 0.1
    d_in = prep["qe"] - prep["qo"]
    got_len = np.linalg.norm(d_in.astype(np.float64), axis=1) / scale
    long_ = length > 20.0 + 1e-3
    short = length < 20.0 - 1e-3
    assert np.all(np.abs(got_len[long_] - 20.0) < 2.0 / scale)            # within 1 unit per axis
    assert np.all(np.abs(got_len[short] - length[short]) < 1e-5)
    # direction is kept
    cosang = (d_in[long_] * u[long_]).sum(1) / np.linalg.norm(d_in[long_].astype(np.float64), axis=1)
    assert np.all(cosang > 1 - 1e-9)
    # a truncated ray, or a NO_RETURN ray, carries no sample
    assert not prep["has_sample"][long_].any()
    assert np.array_equal(prep["has_sample"][short], flags[short] == 0)


def test_nonfinite_rays_are_skipped():
    m = oracle.OracleMap()
    o = np.array([[0.0, 0.0, 0.0]], np.float32)
    e = np.array([[1.0, 0.0, 0.0], [np.nan, 0, 0], [np.inf, 1, 1]], np.float32)
    prep = m.prepare(o, e)
    assert prep["valid"].tolist() == [True, False, False]


def _closed_form(l0, k, mm, hit, miss, lmin, lmax):
    """Eq. 2-3 with the clamp of Sec. II-B, misses first then samples (Sec.
    III-C), in exact arithmetic: min(max(l0 + k miss, lmin) + m hit, lmax)."""
    l = 0.0 if l0 is None else l0
    if k:
        l = max(l + k * miss, lmin)
    if mm:
        l = min(l + mm * hit, lmax)
    return l


def _single_voxel_scan(k, mm):
    """Rays for one scan in which voxel (5, 0, 0) sees k pass-throughs and mm
    samples: k rays along +x through it and mm rays ending in it."""
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    ends = []
    for i in range(k):
        ends.append([1.55, 0.05 + 0.0001 * i, 0.05])       # passes x = 0.5..0.6
    for i in range(mm):
        ends.append([0.55 + 0.001 * i, 0.05, 0.05])        # sample inside voxel 5
    return o, np.array(ends, np.float32).reshape(-1, 3)


def test_log_odds_closed_form_multi_scan():
    rng = np.random.default_rng(3)
    for trial in range(20):
        m = oracle.OracleMap(l_min=-2.0, l_max=3.5)
        expect = None
        for scan in range(6):
            k = int(rng.integers(0, 12))
            mm = int(rng.integers(0, 10))
            if k + mm == 0:
                continue
            o, e = _single_voxel_scan(k, mm)
            m.integrate(o, e)
            expect = _closed_form(expect, k, mm, HIT, MISS, -2.0, 3.5)
            got = m.query(np.array([[0.55, 0.05, 0.05]], np.float32))
            assert got["known"][0] == 1
            assert abs(float(got["occupancy"][0]) - expect) < 1e-5, (trial, scan, k, mm)


def test_misses_precede_samples_within_a_scan():
    # 10 misses and 1 sample from unknown: misses first gives -2 + 0.847; the
    # other order would give max(0.847 - 10 * 0.405, -2) = -2.
    m = oracle.OracleMap()
    o, e = _single_voxel_scan(10, 1)
    m.integrate(o, e)
    got = float(m.query(np.array([[0.55, 0.05, 0.05]], np.float32))["occupancy"][0])
    assert abs(got - (-2.0 + HIT)) < 1e-6


def test_saturation_at_both_clamps():
    m = oracle.OracleMap()
    o, e = _single_voxel_scan(0, 50)
    m.integrate(o, e)
    assert float(m.query(np.array([[0.55, 0.05, 0.05]], np.float32))["occupancy"][0]) == np.float32(3.5)
    o, e = _single_voxel_scan(50, 0)
    m.integrate(o, e)
    assert float(m.query(np.array([[0.55, 0.05, 0.05]], np.float32))["occupancy"][0]) == np.float32(-2.0)


def test_hit_and_miss_counts_axis_rays():
    """Counts H_i, M_i for rays along +x from the centre of voxel 0: voxel j
    gets one miss from every ray that ends beyond it and one hit from every ray
    that ends in it."""
    rng = np.random.default_rng(4)
    m = oracle.OracleMap(layers=LAYER_OCCUPANCY | LAYER_COUNTS)
    ends_v = rng.integers(0, 40, size=300)
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    e = np.stack([ends_v * 0.1 + 0.05, np.full(300, 0.05), np.full(300, 0.05)], 1).astype(np.float32)
    m.integrate(o, e)
    ex = m.export()
    assert ex["keys"].tolist() == [[0, 0, 0], [1, 0, 0]]
    hits = ex["hits"].reshape(2, 32, 32, 32)   # (region, z, y, x)
    misses = ex["misses"].reshape(2, 32, 32, 32)
    for j in range(45):
        r, x = divmod(j, 32)
        assert hits[r, 0, 0, x] == np.sum(ends_v == j)
        assert misses[r, 0, 0, x] == np.sum(ends_v > j)
    assert hits.sum() == 300 and misses.sum() == int(ends_v.sum())


def test_region_set_is_regions_of_visited_voxels():
    rng = np.random.default_rng(5)
    m = oracle.OracleMap(layers=LAYER_OCCUPANCY, max_range=30.0)
    o = np.array([[0.11, -0.23, 0.4]], np.float32)
    e = (o + rng.normal(size=(200, 3)) * 6).astype(np.float32)
    m.integrate(o, e)
    prep = m.prepare(o, e)
    want = set()
    for qo, qe in zip(prep["qo"], prep["qe"]):
        for v in oracle.walk(qo, qe):
            want.add(tuple(int(c) for c in np.floor_divide(v, 32)))
    got = set(tuple(k) for k in m.export()["keys"].tolist())
    assert got == want


def test_ndt_mean_covariance_equal_sample_statistics():
    """Sec. II-D / III-C: a voxel's NDT mean and covariance are the statistics
    of the samples that fell in it (population covariance)."""
    rng = np.random.default_rng(6)
    vs = 0.1
    m = oracle.OracleMap(layers=LAYER_OCCUPANCY | LAYER_NDT, voxel_size=vs, map_origin=(0.0, 0.0, 0.0))
    o = np.array([[-1.0, -1.0, -1.0]], np.float32)
    centre = np.array([0.25, 0.35, 0.15])
    pts = (centre + rng.uniform(-0.049, 0.049, size=(400, 3))).astype(np.float32)
    for chunk in np.array_split(pts, 4):  # over several scans
        m.integrate(o, chunk)
    prep = m.prepare(o, pts)
    qpts = prep["qe"].astype(np.float64) * (vs / U)
    q = m.query(centre[None].astype(np.float32))["ndt"][0]
    assert q[0] == 400
    assert np.allclose(q[1:4], qpts.mean(0), rtol=0, atol=1e-12)
    cov = np.cov(qpts.T, ddof=0)
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    assert np.allclose(q[4:], [cov[i, j] for i, j in iu], rtol=1e-9, atol=1e-15)
    # against the unquantised points: within the quantisation step
    assert np.allclose(q[1:4], pts.astype(np.float64).mean(0), atol=vs / U)
    # invariants: mean inside the voxel, covariance positive semi-definite
    assert np.all(np.floor(q[1:4] / vs) == np.floor(centre / vs))
    c = np.array([[q[4], q[5], q[6]], [q[5], q[7], q[8]], [q[6], q[8], q[9]]])
    assert np.linalg.eigvalsh(c).min() > -1e-15


def test_ndt_export_moments_integer_sums():
    m = oracle.OracleMap(layers=LAYER_NDT)
    o = np.array([[0.0, 0.0, 0.0]], np.float32)
    e = np.array([[0.55, 0.05, 0.05], [0.56, 0.07, 0.01]], np.float32)
    m.integrate(o, e)
    prep = m.prepare(o, e)
    ex = m.export()
    p = prep["qe"] - (prep["qe"] // U) * U
    idx = 5  # voxel (5, 0, 0)
    s = ex["ndt"][0, idx]
    assert s[0] == 2
    assert s[1:4].tolist() == p.sum(0).tolist()
    assert s[4] == int((p[:, 0] * p[:, 0]).sum()) and s[9] == int((p[:, 2] * p[:, 2]).sum())


def test_tsdf_single_frontal_ray():
    """One ray along +x from a voxel centre: band voxels j get
    s = clamp(d - j vs, -tau, tau) and weight 1 (Sec. II-F, projective SDF)."""
    vs, tau = 0.05, 0.2
    m = oracle.OracleMap(layers=LAYER_TSDF, voxel_size=vs, tsdf_trunc=tau, max_range=10.0)
    o = np.array([[0.025, 0.025, 0.025]], np.float32)
    d = 1.2371
    e = np.array([[0.025 + d, 0.025, 0.025]], np.float32)
    m.integrate(o, e)
    prep = m.prepare(o, e)
    d_q = float(prep["qe"][0, 0] - prep["qo"][0, 0]) * vs / U   # the quantised range
    ox = float(prep["qo"][0, 0]) * vs / U
    xs = (np.arange(0, 40) + 0.5) * vs
    q = m.query(np.stack([xs, np.full(40, 0.025), np.full(40, 0.025)], 1).astype(np.float32))["tsdf"]
    for j in range(40):
        lo, hi = j * vs, (j + 1) * vs
        in_band = hi > ox + d_q - tau and lo <= ox + d_q + tau
        if in_band:
            s = min(max(d_q - (xs[j] - ox), -tau), tau)
            assert q[j, 1] == 1 and abs(q[j, 0] - s) < 1e-12, j
        else:
            assert q[j, 1] == 0, j


def test_tsdf_repeated_scans_keep_value_and_count_weight():
    vs, tau = 0.05, 0.2
    m = oracle.OracleMap(layers=LAYER_TSDF, voxel_size=vs, tsdf_trunc=tau, max_range=10.0)
    rng = np.random.default_rng(9)
    o = np.array([[0.01, 0.02, 0.03]], np.float32)
    e = (o + rng.normal(size=(50, 3))).astype(np.float32)
    m.integrate(o, e)
    first = m.export()["tsdf"].copy()
    for _ in range(4):
        m.integrate(o, e)
    last = m.export()["tsdf"]
    w1 = first[..., 1]
    assert np.array_equal(last[..., 1], 5 * w1)
    sel = w1 > 0
    assert np.allclose(last[..., 0][sel], first[..., 0][sel], atol=1e-12)


def test_tsdf_skips_no_return_and_out_of_range():
    m = oracle.OracleMap(layers=LAYER_TSDF, voxel_size=0.05, min_range=0.3, max_range=6.0)
    o = np.array([[0.0, 0.0, 0.0]], np.float32)
    e = np.array([[1.0, 0.0, 0.0], [0.0, 0.2, 0.0], [0.0, 0.0, 7.0], [0.0, -1.0, 0.0]], np.float32)
    f = np.array([0, 0, 0, FLAG_NO_RETURN], np.uint8)
    m.integrate(o, e, f)
    q = m.query(np.array([[1.0, 0, 0], [0, 0.2, 0], [0, 0, 7.0], [0, -1.0, 0]], np.float32))["tsdf"]
    assert q[0, 1] == 1 and q[1, 1] == 0 and q[2, 1] == 0 and q[3, 1] == 0


def test_ndt_samples_cleared_when_occupancy_falls_below_threshold():
    """Sec. II-D: sample data is cleared when the voxel's occupancy falls below
    a threshold.  Voxel (5, 0, 0) gets 3 samples (l = 3 * 0.847 = 2.54), then
    scans of k misses each; with threshold 0.5 the samples survive while
    l >= 0.5 and vanish on the miss that takes l below it; new samples then
    start a fresh mean."""
    thr = 0.5
    m = oracle.OracleMap(layers=LAYER_OCCUPANCY | LAYER_NDT, ndt_clear_below=thr)
    probe = np.array([[0.55, 0.05, 0.05]], np.float32)
    o, e = _single_voxel_scan(0, 3)
    m.integrate(o, e)
    assert m.query(probe)["ndt"][0, 0] == 3
    l = float(m.query(probe)["occupancy"][0])
    for k in (2, 2, 2):
        o, e = _single_voxel_scan(k, 0)
        m.integrate(o, e)
        for _ in range(k):
            l = max(l + MISS, -2.0)
        n = m.query(probe)["ndt"][0, 0]
        assert n == (3 if l >= thr else 0), (l, n)
    assert n == 0
    o, e = _single_voxel_scan(0, 2)
    m.integrate(o, e)
    assert m.query(probe)["ndt"][0, 0] == 2


def test_ndt_clearing_off_by_default():
    m = oracle.OracleMap(layers=LAYER_OCCUPANCY | LAYER_NDT)
    o, e = _single_voxel_scan(0, 3)
    m.integrate(o, e)
    o, e = _single_voxel_scan(40, 0)
    m.integrate(o, e)
    assert m.query(np.array([[0.55, 0.05, 0.05]], np.float32))["ndt"][0, 0] == 3
