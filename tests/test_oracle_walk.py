"""Pins of the oracle's voxel walk (Sec. III-B, Amanatides & Woo) against
hand-derived cases, closed forms and exact rational brute force."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

U = 1 << 16
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "walk_ties.json")


def test_golden_walks():
    spec = json.load(open(GOLDEN))
    for case in spec["cases"]:
        got = oracle.walk(case["a"], case["b"], spec["frac_bits"]).tolist()
        assert got == case["visits"], case["name"]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_axis_aligned_visits_interval(axis, sign):
    rng = np.random.default_rng(100 + axis * 2 + (sign > 0))
    for _ in range(200):
        a = rng.integers(-40 * U, 40 * U, size=3)
        b = a.copy()
        b[axis] = a[axis] + sign * int(rng.integers(0, 30 * U))
        got = oracle.walk(a, b)
        va, vb = a // U, b // U  # numpy floor division
        lo, hi = sorted((va[axis], vb[axis]))
        expect = np.repeat(va[None], hi - lo + 1, axis=0)
        expect[:, axis] = np.arange(va[axis], vb[axis] + sign, sign) if hi > lo else va[axis]
        assert np.array_equal(got, expect)


def test_visit_count_and_steps():
    """1 + |dv|_1 voxels; consecutive voxels differ by one unit step along one
    axis, in the direction of the ray; first/last are the voxels of a and b."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        a = rng.integers(-200 * U, 200 * U, size=3)
        b = a + rng.integers(-60 * U, 60 * U, size=3)
        got = oracle.walk(a, b)
        va, vb = a // U, b // U
        assert len(got) == 1 + int(np.abs(vb - va).sum())
        assert np.array_equal(got[0], va) and np.array_equal(got[-1], vb)
        d = np.diff(got, axis=0)
        assert np.all(np.abs(d).sum(axis=1) == 1)
        sgn = np.sign(b - a)
        assert np.all((d == 0) | (d == sgn[None]))


def _box_meets_segment(v, a, b, open_box):
    """Exact test whether voxel v's box (open interior or closed) meets the
    segment a + t (b - a), t in [0, 1].  a, b are Fractions in voxel units."""
    lo, hi = Fraction(0), Fraction(1)
    strict_lo = strict_hi = False
    for k in range(3):
        d = b[k] - a[k]
        if d == 0:
            inside = (v[k] < a[k] < v[k] + 1) if open_box else (v[k] <= a[k] <= v[k] + 1)
            if not inside:
                return False
            continue
        t1 = (v[k] - a[k]) / d
        t2 = (v[k] + 1 - a[k]) / d
        l, h = min(t1, t2), max(t1, t2)
        if l > lo or (l == lo and open_box):
            lo, strict_lo = l, open_box
        if h < hi or (h == hi and open_box):
            hi, strict_hi = h, open_box
    if strict_lo or strict_hi:
        return lo < hi
    return lo <= hi


def _brute_force_case(a, b):
    af = [Fraction(int(x), U) for x in a]
    bf = [Fraction(int(x), U) for x in b]
    got = [tuple(v) for v in oracle.walk(a, b).tolist()]
    lo = np.minimum(a, b) // U - 1
    hi = np.maximum(a, b) // U + 1
    interior, closed = set(), set()
    for x in range(lo[0], hi[0] + 1):
        for y in range(lo[1], hi[1] + 1):
            for z in range(lo[2], hi[2] + 1):
                if _box_meets_segment((x, y, z), af, bf, True):
                    interior.add((x, y, z))
                if _box_meets_segment((x, y, z), af, bf, False):
                    closed.add((x, y, z))
    s = set(got)
    assert len(s) == len(got), "a voxel was visited twice"
    assert interior <= s, "a voxel whose interior the ray crosses was skipped"
    assert s <= closed, "a visited voxel does not touch the ray"


def test_brute_force_random_rays():
    rng = np.random.default_rng(11)
    for _ in range(300):
        a = rng.integers(-4 * U, 4 * U, size=3)
        b = rng.integers(-4 * U, 4 * U, size=3)
        _brute_force_case(a, b)


def test_brute_force_lattice_rays():
    """End points on a quarter-voxel lattice, so faces, edges, corners and ties
    occur often."""
    rng = np.random.default_rng(12)
    q = U // 4
    for _ in range(400):
        a = rng.integers(-12, 12, size=3) * q
        b = rng.integers(-12, 12, size=3) * q
        _brute_force_case(a, b)


def test_reverse_walk_visits_same_set_without_ties():
    """Walking b -> a visits the same voxels as a -> b when no two axes cross
    at the same t and neither end lies on a face (reverse ray tracing, Table 3
    caption)."""
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(400):
        a = rng.integers(-50 * U, 50 * U, size=3) | 1  # odd: never on a face
        b = rng.integers(-50 * U, 50 * U, size=3) | 1
        fwd = oracle.walk(a, b)
        rev = oracle.walk(b, a)
        if len(fwd) != len(rev):
            continue
        assert np.array_equal(fwd, rev[::-1])
        checked += 1
    assert checked > 350
