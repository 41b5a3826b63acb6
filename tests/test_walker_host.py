"""The CUDA library's walker, compiled for the host, against the oracle's
walk: identical voxel sequences for every segment length (Sec. III-B ray
segments must not change the walk), on tie-heavy and random rays."""
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
U = 1 << 16


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("walker") / "walker_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-x", "cu", os.path.join(HERE, "host", "walker_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def _run(exe, rays, F=16, S=64, inv=False):
    lines = ["%d %d %d" % (F, S, len(rays))] + ["%d %d %d %d %d %d" % tuple(int(v) for v in (*a, *b)) for a, b in rays]
    args = [exe, "inv"] if inv else [exe]
    out = subprocess.run(args, input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert out.returncode == 0, "walker check exited %d (Morton mismatch = 2)" % out.returncode
    tok = out.stdout.split()
    res, i = [], 0
    for _ in rays:
        c = int(tok[i]); i += 1
        res.append(np.array(tok[i:i + 3 * c], dtype=np.int64).reshape(c, 3)); i += 3 * c
    return res


def _rays(seed, n, lattice):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        if lattice:
            q = U // 4
            a = rng.integers(-40, 40, size=3) * q
            b = a + rng.integers(-200, 200, size=3) * q
        else:
            a = rng.integers(-100 * U, 100 * U, size=3)
            b = a + rng.integers(-300 * U, 300 * U, size=3)
        if rng.uniform() < 0.1:
            b[rng.integers(0, 3)] = a[rng.integers(0, 3)]
        if rng.uniform() < 0.05:
            b = a.copy()
        out.append((a, b))
    return out


@pytest.mark.parametrize("S", [1, 2, 5, 8, 64, 1 << 20])
@pytest.mark.parametrize("lattice", [False, True])
@pytest.mark.parametrize("inv", [False, True])
def test_device_walker_matches_oracle(checker, S, lattice, inv):
    rays = _rays(100 + S + lattice, 150, lattice)
    got = _run(checker, rays, S=S, inv=inv)
    for (a, b), g in zip(rays, got):
        assert np.array_equal(g, oracle.walk(a, b)), (a, b)


def test_golden_ties_through_device_walker(checker):
    import json
    spec = json.load(open(os.path.join(HERE, "golden", "walk_ties.json")))
    rays = [(np.array(c["a"]), np.array(c["b"])) for c in spec["cases"]]
    for S, inv in ((1, False), (1, True), (64, True)):
        for c, g in zip(spec["cases"], _run(checker, rays, S=S, inv=inv)):
            assert g.tolist() == c["visits"], c["name"]


def test_region_resolution_walk_covers_voxel_regions(checker):
    """The region pass walks the same line with 2^(F+5) units; it must visit
    exactly the regions of the voxels the voxel walk visits."""
    rays = _rays(7, 200, True) + _rays(8, 200, False)
    reg = _run(checker, rays, F=16 + 5, S=1 << 20)
    for (a, b), r in zip(rays, reg):
        v = oracle.walk(a, b)
        want = []
        for x in np.floor_divide(v, 32).tolist():
            if not want or want[-1] != x:
                want.append(x)
        assert r.tolist() == want
