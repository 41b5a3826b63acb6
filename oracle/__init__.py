"""Sequential CPU oracle for OHM ray integration: TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check in __graft_entry__.py and the CPU-baseline leg of
bench.py may import this package.  The product path (the CUDA library and its
binding) never calls it.  See ohm_oracle.cpp for what each function computes
and which section or equation of the paper it follows.

This module is argument marshalling over ctypes; the arithmetic is in C++.
"""
import ctypes
import math

import numpy as np

from . import build as _build

REGION_DIM = 32
REGION_VOXELS = REGION_DIM ** 3

LAYER_OCCUPANCY = 1
LAYER_NDT = 2
LAYER_TSDF = 4
LAYER_COUNTS = 8
LAYER_DECAY = 16
LAYER_MEAN = 32
PATH_UNITS_PER_METRE = float(1 << 20)

FLAG_NO_RETURN = 1


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("voxel_size", ctypes.c_double),
        ("map_origin", ctypes.c_double * 3),
        ("frac_bits", ctypes.c_int32),
        ("layers", ctypes.c_int32),
        ("hit", ctypes.c_float),
        ("miss", ctypes.c_float),
        ("l_min", ctypes.c_float),
        ("l_max", ctypes.c_float),
        ("ndt_clear_below", ctypes.c_float),
        ("max_range", ctypes.c_double),
        ("min_range", ctypes.c_double),
        ("tsdf_trunc", ctypes.c_double),
        ("tsdf_wmax", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        vp, i64, p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_create.restype = vp
        lib.oracle_create.argtypes = [ctypes.POINTER(OracleParams)]
        lib.oracle_destroy.argtypes = [vp]
        lib.oracle_integrate.restype = i64
        lib.oracle_integrate.argtypes = [vp, p, i64, p, p, i64]
        lib.oracle_region_count.restype = i64
        lib.oracle_region_count.argtypes = [vp]
        lib.oracle_export.restype = ctypes.c_int
        lib.oracle_export.argtypes = [vp, i64, i64, p, p, p, p, p, p, p, p]
        lib.oracle_ndt_region_count.restype = i64
        lib.oracle_ndt_region_count.argtypes = [vp]
        lib.oracle_ndt_sparse.restype = i64
        lib.oracle_ndt_sparse.argtypes = [vp, i64, p, p]
        lib.oracle_query.argtypes = [vp, p, i64, p, p, p, p, p, p]
        lib.oracle_walk.restype = i64
        lib.oracle_walk.argtypes = [p, p, ctypes.c_int32, p, i64]
        lib.oracle_walk_timed.restype = i64
        lib.oracle_walk_timed.argtypes = [p, p, ctypes.c_int32, p, p, i64]
        lib.oracle_prepare.argtypes = [vp, p, i64, p, p, i64, p, p, p, p]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def logit(p: float) -> float:
    """Log-odds of a probability, Eq. 3: log(P(z|occ) / P(z|emp))."""
    return math.log(p / (1.0 - p))


def default_params(**kw) -> dict:
    """Parameters of the room and tunnel occupancy workloads (0.1 m voxels)."""
    p = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16,
             layers=LAYER_OCCUPANCY | LAYER_COUNTS,
             hit=float(np.float32(logit(0.7))), miss=float(np.float32(logit(0.4))),
             l_min=-2.0, l_max=3.5, ndt_clear_below=float("-inf"), max_range=20.0, min_range=0.0,
             tsdf_trunc=0.2, tsdf_wmax=float(1 << 20))
    p.update(kw)
    return p


class OracleMap:
    """One sequential oracle map."""

    def __init__(self, **params):
        self.params = default_params(**params)
        lib = _load()
        cp = OracleParams()
        for k, v in self.params.items():
            if k == "map_origin":
                for i in range(3):
                    cp.map_origin[i] = float(v[i])
            else:
                setattr(cp, k, v)
        self._h = lib.oracle_create(ctypes.byref(cp))

    def close(self):
        if self._h:
            _load().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, origins, endpoints, flags=None) -> int:
        """Integrate one ray set; returns the number of voxel visits."""
        o = np.ascontiguousarray(origins, dtype=np.float32).reshape(-1, 3)
        e = np.ascontiguousarray(endpoints, dtype=np.float32).reshape(-1, 3)
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        n = e.shape[0]
        r = _load().oracle_integrate(self._h, _ptr(o), o.shape[0], _ptr(e), _ptr(f), n)
        if r < 0:
            raise ValueError("oracle_integrate: bad arguments")
        return int(r)

    def region_count(self) -> int:
        return int(_load().oracle_region_count(self._h))

    def ndt_region_count(self) -> int:
        return int(_load().oracle_ndt_region_count(self._h))

    def export(self, first=0, count=None, occupancy=True, counts=True, ndt=True, tsdf=True, path=True, mean=True):
        """Regions [first, first + count) in (rx, ry, rz) order: a dict of numpy
        arrays (a layer the map lacks, or one not asked for, is None)."""
        total = self.region_count()
        if count is None:
            count = total - first
        n = max(0, min(count, total - first))
        L = self.params["layers"]
        keys = np.zeros((n, 3), np.int64)
        occ = np.full((n, REGION_VOXELS), np.nan, np.float32) if (L & LAYER_OCCUPANCY and occupancy) else None
        hits = np.zeros((n, REGION_VOXELS), np.uint32) if (L & LAYER_COUNTS and counts) else None
        misses = np.zeros((n, REGION_VOXELS), np.uint32) if (L & LAYER_COUNTS and counts) else None
        nd = np.zeros((n, REGION_VOXELS, 10), np.int64) if (L & LAYER_NDT and ndt) else None
        ts = np.zeros((n, REGION_VOXELS, 2), np.float64) if (L & LAYER_TSDF and tsdf) else None
        ps = np.zeros((n, REGION_VOXELS), np.uint64) if (L & LAYER_DECAY and path) else None
        mn = np.zeros((n, REGION_VOXELS, 4), np.uint32) if (L & LAYER_MEAN and mean) else None
        rc = _load().oracle_export(self._h, first, n, _ptr(keys), _ptr(occ), _ptr(hits), _ptr(misses), _ptr(nd),
                                   _ptr(ts), _ptr(ps), _ptr(mn))
        if rc:
            raise OverflowError("NDT moment sum exceeds int64")
        return dict(keys=keys, occupancy=occ, hits=hits, misses=misses, ndt=nd, tsdf=ts, path=ps, mean=mn)

    def ndt_sparse(self):
        """(voxels (k, 3) int64, moments (k, 10) int64) of every voxel holding
        a sample: n, Sx, Sy, Sz, Sxx, Sxy, Sxz, Syy, Syz, Szz."""
        lib = _load()
        k = int(lib.oracle_ndt_sparse(self._h, 0, None, None))
        vox = np.zeros((k, 3), np.int64)
        mom = np.zeros((k, 10), np.int64)
        lib.oracle_ndt_sparse(self._h, k, _ptr(vox), _ptr(mom))
        return vox, mom

    def query(self, points):
        pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
        n = pts.shape[0]
        occ = np.zeros(n, np.float32)
        known = np.zeros(n, np.uint8)
        ndt = np.zeros((n, 10), np.float64)
        tsdf = np.zeros((n, 2), np.float64)
        path = np.zeros(n, np.uint64)
        mean = np.zeros((n, 4), np.float64)
        _load().oracle_query(self._h, _ptr(pts), n, _ptr(occ), _ptr(known), _ptr(ndt), _ptr(tsdf), _ptr(path),
                             _ptr(mean))
        return dict(occupancy=occ, known=known, ndt=ndt, tsdf=tsdf, path=path, mean=mean)

    def prepare(self, origins, endpoints, flags=None):
        o = np.ascontiguousarray(origins, dtype=np.float32).reshape(-1, 3)
        e = np.ascontiguousarray(endpoints, dtype=np.float32).reshape(-1, 3)
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        n = e.shape[0]
        qo = np.zeros((n, 3), np.int64)
        qe = np.zeros((n, 3), np.int64)
        hs = np.zeros(n, np.uint8)
        ok = np.zeros(n, np.uint8)
        _load().oracle_prepare(self._h, _ptr(o), o.shape[0], _ptr(e), _ptr(f), n, _ptr(qo), _ptr(qe), _ptr(hs), _ptr(ok))
        return dict(qo=qo, qe=qe, has_sample=hs.astype(bool), valid=ok.astype(bool))


def walk(a, b, frac_bits: int = 16):
    """Voxels visited walking from fixed-point point a to fixed-point point b."""
    a = np.ascontiguousarray(a, dtype=np.int64).reshape(3)
    b = np.ascontiguousarray(b, dtype=np.int64).reshape(3)
    lib = _load()
    n = lib.oracle_walk(_ptr(a), _ptr(b), frac_bits, None, 0)
    out = np.zeros((max(n, 1), 3), np.int64)
    lib.oracle_walk(_ptr(a), _ptr(b), frac_bits, _ptr(out), n)
    return out[:n]


def walk_timed(a, b, frac_bits: int = 16):
    """walk() plus each voxel's (t_in, t_out) ray parameters as uint64
    fractions of 2^32, the decay-rate layer's distance bookkeeping (Sec. II-E)."""
    a = np.ascontiguousarray(a, dtype=np.int64).reshape(3)
    b = np.ascontiguousarray(b, dtype=np.int64).reshape(3)
    lib = _load()
    n = lib.oracle_walk_timed(_ptr(a), _ptr(b), frac_bits, None, None, 0)
    out = np.zeros((max(n, 1), 3), np.int64)
    t = np.zeros((max(n, 1), 2), np.uint64)
    lib.oracle_walk_timed(_ptr(a), _ptr(b), frac_bits, _ptr(out), _ptr(t), n)
    return out[:n], t[:n]
