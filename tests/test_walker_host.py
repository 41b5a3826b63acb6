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


_EXIT = {2: "Morton mismatch", 3: "bad ray record", 4: "region tracking mismatch", 5: "segment end / visit count mismatch"}


def _run(exe, rays, F=16, S=64, mode="plain", stats=None):
    lines = ["%d %d %d" % (F, S, len(rays))] + ["%d %d %d %d %d %d" % tuple(int(v) for v in (*a, *b)) for a, b in rays]
    out = subprocess.run([exe, mode], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert out.returncode == 0, "walker check exited %d (%s)" % (out.returncode, _EXIT.get(out.returncode, "?"))
    if stats is not None:
        stats["exact"] = int(out.stderr.split()[1])
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


@pytest.mark.parametrize("S", [1, 2, 5, 8, 24, 64, 1 << 20])
@pytest.mark.parametrize("lattice", [False, True])
@pytest.mark.parametrize("mode", ["plain", "rec", "fast"])
def test_device_walker_matches_oracle(checker, S, lattice, mode):
    rays = _rays(100 + S + lattice, 150, lattice)
    stats = {}
    got = _run(checker, rays, S=S, mode=mode, stats=stats)
    for (a, b), g in zip(rays, got):
        assert np.array_equal(g, oracle.walk(a, b)), (a, b)
    if mode == "fast" and lattice:
        # lattice rays are full of exact ties: the exact fallback must have run
        assert stats["exact"] > 0


def test_fast_walk_near_ties(checker):
    """Rays whose crossings along two axes come within a few fixed-point units
    of each other (end points one unit off exact diagonals and lattice
    points): the FP32 filter must hand these to the exact rule."""
    rng = np.random.default_rng(11)
    rays = []
    for _ in range(400):
        a = rng.integers(-20, 20, size=3) * U + rng.integers(0, U, size=3)
        d = rng.integers(-150, 150) * U
        b = a + np.array([d, d, rng.integers(-150, 150) * U]) + rng.integers(-2, 3, size=3)
        rays.append((a, b))
    stats = {}
    for S in (3, 24):
        for (a, b), g in zip(rays, _run(checker, rays, S=S, mode="fast", stats=stats)):
            assert np.array_equal(g, oracle.walk(a, b)), (a, b)
    assert stats["exact"] > 0


def test_golden_ties_through_device_walker(checker):
    import json
    spec = json.load(open(os.path.join(HERE, "golden", "walk_ties.json")))
    rays = [(np.array(c["a"]), np.array(c["b"])) for c in spec["cases"]]
    for S, mode in ((1, "plain"), (1, "rec"), (64, "rec"), (1, "fast"), (3, "fast"), (64, "fast")):
        for c, g in zip(spec["cases"], _run(checker, rays, S=S, mode=mode)):
            assert g.tolist() == c["visits"], (c["name"], mode, S)


def test_region_resolution_walk_covers_voxel_regions(checker):
    """The region pass walks the same line with 2^(F+5) units; it must visit
    exactly the regions of the voxels the voxel walk visits."""
    rays = _rays(7, 200, True) + _rays(8, 200, False)
    reg = _run(checker, rays, F=16 + 5, S=1 << 20, mode="plain")
    for (a, b), r in zip(rays, reg):
        v = oracle.walk(a, b)
        want = []
        for x in np.floor_divide(v, 32).tolist():
            if not want or want[-1] != x:
                want.append(x)
        assert r.tolist() == want


def test_tsdf_band_reciprocal_equals_divisions(tmp_path):
    """The TSDF band end points and direction formed through one reciprocal
    (tsdf_band, compiled for the host) equal the direct double divisions on
    random rays and on rays built to land on half-integers and float rounding
    midpoints, where it falls back to the divisions."""
    exe = str(tmp_path / "band_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-x", "cu",
                    os.path.join(HERE, "host", "band_check.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr[-500:])
    tok = out.stdout.split()
    cases, fallback = int(tok[1]), int(tok[3])
    assert cases > 600000 and 0 < fallback < cases


def test_tsdf_band_float_float_equals_double(tmp_path):
    """The TSDF range test and band settled in float-float arithmetic
    (tsdf_band_ff, compiled for the host) equal the double evaluation on every
    case they settle: random rays (of which they must settle nearly all), rays
    built to land an end point on a half-integer, lengths at the range limits
    and at tau, where they must decline.  Float ops are compiled without
    contraction, as the device code writes every rounding explicitly."""
    exe = str(tmp_path / "band_ff_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-Xcompiler",
                    "-ffp-contract=off", "-x", "cu", os.path.join(HERE, "host", "band_ff_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr[-500:])
    tok = out.stdout.split()
    cases, settled, rnd, rnd_settled = int(tok[1]), int(tok[3]), int(tok[5]), int(tok[7])
    assert cases > 1500000 and rnd > 590000
    assert rnd_settled > 0.999 * rnd      # the float-float path decides nearly every ordinary ray
    assert settled < 0.5 * cases          # and declines the built near-ties
