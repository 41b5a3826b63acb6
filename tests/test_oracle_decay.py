"""Pins of the oracle's decay-rate layer (Sec. II-E: lambda_i = H_i / sum_j
d_i(j), with d_i(j) the distance ray j travels inside voxel i) against closed
forms and a brute-force clip of each ray against every voxel box in exact
rational arithmetic."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import LAYER_COUNTS, LAYER_DECAY, LAYER_OCCUPANCY

U = 1 << 16
VS = 0.1
PER_M = oracle.PATH_UNITS_PER_METRE


def _map(**kw):
    p = dict(voxel_size=VS, layers=LAYER_OCCUPANCY | LAYER_COUNTS | LAYER_DECAY, max_range=1e6)
    p.update(kw)
    return oracle.OracleMap(**p)


def _voxel_values(m):
    """{voxel: (path units, hits)} of every voxel with a nonzero path sum or hit."""
    ex = m.export(occupancy=False, ndt=False, tsdf=False)
    out = {}
    lin = np.arange(32 ** 3)
    local = np.stack([lin % 32, (lin // 32) % 32, lin // 1024], 1)
    hits = ex["hits"] if ex["hits"] is not None else np.zeros_like(ex["path"], np.uint32)
    for r, key in enumerate(ex["keys"]):
        nz = np.nonzero((ex["path"][r] > 0) | (hits[r] > 0))[0]
        for i in nz:
            v = tuple(int(x) for x in key * 32 + local[i])
            out[v] = (int(ex["path"][r][i]), int(hits[r][i]))
    return out


def _exact_clip(qa, qb):
    """{voxel: exact length in metres} of the segment qa -> qb (fixed point)
    inside each voxel box it meets with positive length, by clipping the
    segment against every box in its bounding box (rational t)."""
    delta = [qb[k] - qa[k] for k in range(3)]
    length = math.sqrt(sum(float(d) ** 2 for d in delta)) * VS / U
    lo = [min(qa[k], qb[k]) >> 16 for k in range(3)]
    hi = [max(qa[k], qb[k]) >> 16 for k in range(3)]
    out = {}
    for x in range(lo[0], hi[0] + 1):
        for y in range(lo[1], hi[1] + 1):
            for z in range(lo[2], hi[2] + 1):
                t0, t1 = Fraction(0), Fraction(1)
                for k, v in enumerate((x, y, z)):
                    b0, b1 = v * U, (v + 1) * U
                    if delta[k] == 0:
                        if not (b0 <= qa[k] < b1):
                            t0, t1 = Fraction(1), Fraction(0)
                        continue
                    e0 = Fraction(b0 - qa[k], delta[k])
                    e1 = Fraction(b1 - qa[k], delta[k])
                    t0, t1 = max(t0, min(e0, e1)), min(t1, max(e0, e1))
                if t1 > t0:
                    out[(x, y, z)] = float(t1 - t0) * length
    return out


def test_axis_aligned_ray_closed_form():
    """A ray along x from 0.05 m to 0.95 m crosses ten 0.1 m voxels: 0.05 m in
    the first and last, 0.1 m in the eight between."""
    m = _map()
    m.integrate(np.array([[0.05, 0.05, 0.05]], np.float32), np.array([[0.95, 0.05, 0.05]], np.float32))
    got = _voxel_values(m)
    assert sorted(got) == [(i, 0, 0) for i in range(10)]
    for i in range(10):
        want = (0.05 if i in (0, 9) else 0.1) * PER_M
        assert abs(got[(i, 0, 0)][0] - want) <= 1.0, (i, got[(i, 0, 0)][0], want)
    assert got[(9, 0, 0)][1] == 1  # the sample
    assert sum(v[0] for v in got.values()) == round(0.9 * PER_M)


def test_decay_rate_of_a_voxel_closed_form():
    """Rays that end in one voxel after entering it through its -x face each
    travel 0.05 m inside it: lambda = H / sum d = 1 / 0.05 m = 20 per metre."""
    m = _map()
    n = 7
    o = np.array([[-1.0 - 0.3 * i, 0.05, 0.05] for i in range(n)], np.float32)
    e = np.tile(np.array([[0.05, 0.05, 0.05]], np.float32), (n, 1))
    m.integrate(o, e)
    path, hits = _voxel_values(m)[(0, 0, 0)]
    assert hits == n
    lam = hits / (path / PER_M)
    assert abs(lam - 20.0) < 20.0 * 1e-5


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_clip(seed):
    """Every voxel's path sum against the exact segment/box clip, summed over
    the rays: the integer rounding costs at most 2 units of 2^-20 m per visit."""
    rng = np.random.default_rng(seed)
    m = _map(layers=LAYER_DECAY)
    n = 40
    o = rng.uniform(-0.35, 0.35, size=(n, 3)).astype(np.float32)
    e = (o + rng.normal(size=(n, 3)) * 0.25).astype(np.float32)
    # exact ties: some rays along face and edge diagonals from voxel corners
    o[:6] = np.float32(0.1) * rng.integers(-2, 2, size=(6, 3)).astype(np.float32)
    e[:6] = o[:6] + np.float32(0.1) * np.array([[1, 1, 1], [2, 2, 0], [0, 3, 3], [-2, 2, 2], [1, -1, 0], [3, 3, 3]],
                                               np.float32)
    m.integrate(o, e)
    prep = m.prepare(o, e)
    want, visits = {}, {}
    for i in range(n):
        qa, qb = [int(x) for x in prep["qo"][i]], [int(x) for x in prep["qe"][i]]
        for v, d in _exact_clip(qa, qb).items():
            want[v] = want.get(v, 0.0) + d * PER_M
            visits[v] = visits.get(v, 0) + 1
    got = {v: p for v, (p, _) in _voxel_values(m).items() if p > 0}
    for v in set(got) | set(want):
        g, w = got.get(v, 0), want.get(v, 0.0)
        assert abs(g - w) <= 2.0 * max(1, visits.get(v, 1)), (v, g, w)


def test_one_ray_adds_up_to_its_length():
    """The distances of one ray sum to its length rounded to 2^-20 m."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        m = _map(layers=LAYER_DECAY)
        o = rng.uniform(-3, 3, size=(1, 3)).astype(np.float32)
        e = (o + rng.normal(size=(1, 3)) * 2).astype(np.float32)
        m.integrate(o, e)
        prep = m.prepare(o, e)
        d = [Fraction(int(prep["qe"][0][k]) - int(prep["qo"][0][k])) for k in range(3)]
        exact = math.sqrt(float(sum(x * x for x in d))) * VS / U * PER_M
        total = sum(p for p, _ in _voxel_values(m).values())
        assert abs(total - exact) <= 0.5 + 1e-6 * exact


def test_truncated_ray_counts_only_the_walked_length():
    m = _map(layers=LAYER_DECAY, max_range=1.0)
    o = np.array([[0.05, 0.05, 0.05]], np.float32)
    e = np.array([[3.05, 0.05, 0.05]], np.float32)
    m.integrate(o, e)
    total = sum(p for p, _ in _voxel_values(m).values())
    assert abs(total - PER_M) <= 1.0


def test_degenerate_rays():
    m = _map()
    # zero length: the voxel gets the sample and no distance
    m.integrate(np.array([[0.05, 0.05, 0.05]], np.float32), np.array([[0.05, 0.05, 0.05]], np.float32))
    assert _voxel_values(m) == {(0, 0, 0): (0, 1)}
    # inside one voxel: all of the length goes to it
    m = _map()
    m.integrate(np.array([[0.01, 0.02, 0.03]], np.float32), np.array([[0.07, 0.06, 0.05]], np.float32))
    p, h = _voxel_values(m)[(0, 0, 0)]
    assert h == 1 and abs(p - math.sqrt(0.06 ** 2 + 0.04 ** 2 + 0.02 ** 2) * PER_M) <= 1.0


def test_timed_walk_matches_walk():
    rng = np.random.default_rng(3)
    for _ in range(200):
        a = rng.integers(-5 * U, 5 * U, size=3)
        b = a + rng.integers(-8 * U, 8 * U, size=3)
        vox, t = oracle.walk_timed(a, b)
        assert np.array_equal(vox, oracle.walk(a, b))
        assert t[0, 0] == 0 and t[-1, 1] == 1 << 32
        assert np.array_equal(t[1:, 0], t[:-1, 1])
        assert (t[:, 1] >= t[:, 0]).all()
