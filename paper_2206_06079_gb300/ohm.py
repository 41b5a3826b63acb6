"""Python binding of the GB300 ray-integration library (include/ohm_gb.h).

Argument marshalling only: every step of ray integration, query and export
runs in the CUDA library.  PyTorch supplies device memory and streams.  If the
library has not been built, or no CUDA device is present, calls raise; there
is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# OHM_GB_LIB may point at a build of the same sources with other compile-time
# tile parameters (used when tuning); by default the in-tree build is loaded.
LIB_PATH = os.environ.get("OHM_GB_LIB") or os.path.join(_HERE, "_lib", "libohm_gb.so")

OK, ERR_INVALID, ERR_CAPACITY, ERR_CUDA, ERR_PROBE_LIMIT, ERR_UNSUPPORTED, ERR_EVICTED = range(7)
LAYER_OCCUPANCY, LAYER_NDT, LAYER_TSDF, LAYER_COUNTS, LAYER_DECAY, LAYER_MEAN = 1, 2, 4, 8, 16, 32
DECAY_UNITS = float(1 << 20)   # path_sum units per metre
FLAG_NO_RETURN = 1
REGION_VOXELS = 32768

_STATUS_NAMES = {ERR_INVALID: "invalid argument", ERR_CAPACITY: "capacity", ERR_CUDA: "CUDA error",
                 ERR_PROBE_LIMIT: "hash probe limit", ERR_UNSUPPORTED: "unsupported", ERR_EVICTED: "evicted"}

# Every symbol include/ohm_gb.h declares.
EXPORTED = ["ohm_map_create", "ohm_map_destroy", "ohm_integrate_rays", "ohm_integrate_rays_async", "ohm_map_sync", "ohm_map_status_async", "ohm_probe_cas_rate",
            "ohm_query_voxels", "ohm_map_region_count", "ohm_map_export", "ohm_map_stats", "ohm_map_profile", "ohm_map_profile_every", "ohm_probe_rate",
            "ohm_map_profile_read", "ohm_last_error", "ohm_count_rays_noalloc", "ohm_batch_create",
            "ohm_batch_destroy", "ohm_batch_tune", "ohm_batch_integrate", "ohm_batch_sync", "ohm_batch_stats",
            "ohm_integrate_depth", "ohm_tsdf_backward", "ohm_twist_pose", "ohm_integrate_posed", "ohm_ndt_backward", "ohm_map_evict", "ohm_map_restore_pending",
            "ohm_map_restore_all", "ohm_map_residency"]

BATCH_MAX_MAPS = 32

NOALLOC_MAX_RAYS = 32768

# Kernel stages of an integrate call (ohm_stage).
STAGES = ["begin", "prepare", "ndt_alloc", "prepare_tsdf", "walk", "hits", "tsdf_walk", "tsdf_apply", "end",
          "mean_apply"]


class OhmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


class MapParams(ctypes.Structure):
    _fields_ = [
        ("voxel_size", ctypes.c_double),
        ("map_origin", ctypes.c_double * 3),
        ("frac_bits", ctypes.c_int32),
        ("layers", ctypes.c_uint32),
        ("hit", ctypes.c_float),
        ("miss", ctypes.c_float),
        ("l_min", ctypes.c_float),
        ("l_max", ctypes.c_float),
        ("ndt_clear_below", ctypes.c_float),
        ("max_range", ctypes.c_double),
        ("min_range", ctypes.c_double),
        ("tsdf_trunc", ctypes.c_double),
        ("tsdf_wmax", ctypes.c_double),
        ("max_regions", ctypes.c_int64),
        ("max_ndt_regions", ctypes.c_int64),
        ("max_rays", ctypes.c_int64),
        ("segment_steps", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("evict_when_full", ctypes.c_int32),
        ("max_probe", ctypes.c_int32),
    ]


class CallStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("rays", "segments", "visits", "regions", "ndt_regions", "touched",
                                              "total_visits", "launches", "atomics")]


class CountGrid(ctypes.Structure):
    """ohm_count_grid: a dense voxel box for ohm_count_rays_noalloc."""
    _fields_ = [
        ("voxel_size", ctypes.c_double),
        ("map_origin", ctypes.c_double * 3),
        ("frac_bits", ctypes.c_int32),
        ("segment_steps", ctypes.c_int32),
        ("max_range", ctypes.c_double),
        ("corner", ctypes.c_int64 * 3),
        ("dims", ctypes.c_int64 * 3),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the shared library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i64, p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
    st = ctypes.c_int
    lib.ohm_map_create.restype = st
    lib.ohm_map_create.argtypes = [ctypes.POINTER(MapParams), ctypes.POINTER(vp)]
    lib.ohm_map_destroy.restype = None
    lib.ohm_map_destroy.argtypes = [vp]
    for name in ("ohm_integrate_rays", "ohm_integrate_rays_async"):
        f = getattr(lib, name)
        f.restype = st
        f.argtypes = [vp, p, i64, p, p, i64, vp]
    lib.ohm_map_sync.restype = st
    lib.ohm_map_sync.argtypes = [vp, vp]
    lib.ohm_map_status_async.restype = st
    lib.ohm_map_status_async.argtypes = [vp, p, vp]
    lib.ohm_probe_cas_rate.restype = st
    lib.ohm_probe_cas_rate.argtypes = [ctypes.c_int32, i64, i64, ctypes.POINTER(ctypes.c_double)]
    lib.ohm_probe_rate.restype = st
    lib.ohm_probe_rate.argtypes = [ctypes.c_int32, ctypes.c_int32, i64, i64, ctypes.POINTER(ctypes.c_double)]
    lib.ohm_query_voxels.restype = st
    lib.ohm_query_voxels.argtypes = [vp, p, i64, p, p, p, p, p, p, p, vp]
    lib.ohm_map_region_count.restype = st
    lib.ohm_map_region_count.argtypes = [vp, ctypes.POINTER(i64), vp]
    lib.ohm_map_export.restype = st
    lib.ohm_map_export.argtypes = [vp, i64, i64, p, p, p, p, p, p, p, vp]
    lib.ohm_map_stats.restype = st
    lib.ohm_map_stats.argtypes = [vp, ctypes.POINTER(CallStats), vp]
    lib.ohm_map_profile.restype = st
    lib.ohm_map_profile.argtypes = [vp, ctypes.c_uint32]
    lib.ohm_map_profile_every.restype = st
    lib.ohm_map_profile_every.argtypes = [vp, ctypes.c_uint32, ctypes.c_int32]
    lib.ohm_map_profile_read.restype = st
    lib.ohm_map_profile_read.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.ohm_count_rays_noalloc.restype = st
    lib.ohm_count_rays_noalloc.argtypes = [ctypes.POINTER(CountGrid), p, i64, p, p, i64, p, p, vp]
    lib.ohm_batch_create.restype = st
    lib.ohm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(vp)]
    lib.ohm_batch_destroy.restype = None
    lib.ohm_batch_destroy.argtypes = [vp]
    lib.ohm_batch_tune.restype = st
    lib.ohm_batch_tune.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.ohm_batch_integrate.restype = st
    lib.ohm_batch_integrate.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.c_int32, vp]
    lib.ohm_batch_sync.restype = st
    lib.ohm_batch_sync.argtypes = [vp, vp]
    lib.ohm_batch_stats.restype = st
    lib.ohm_batch_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.ohm_integrate_depth.restype = st
    lib.ohm_integrate_depth.argtypes = [vp, p, ctypes.c_int32, ctypes.c_int32, dp, dp, ctypes.c_double,
                                        ctypes.c_double, vp]
    lib.ohm_tsdf_backward.restype = st
    lib.ohm_tsdf_backward.argtypes = [vp, p, ctypes.c_int32, ctypes.c_int32, dp, dp, ctypes.c_double, ctypes.c_double,
                                      p, p, i64, p, p, vp]
    lib.ohm_integrate_posed.restype = st
    lib.ohm_integrate_posed.argtypes = [vp, dp, p, i64, p, p, i64, vp]
    lib.ohm_ndt_backward.restype = st
    lib.ohm_ndt_backward.argtypes = [vp, dp, p, i64, p, p, i64, p, p, p, i64, p, p, vp]
    lib.ohm_twist_pose.restype = st
    lib.ohm_twist_pose.argtypes = [dp, dp, dp]
    for name in ("ohm_map_evict",):
        f = getattr(lib, name)
        f.restype = st
        f.argtypes = [vp, i64, ctypes.POINTER(i64), vp]
    for name in ("ohm_map_restore_pending", "ohm_map_restore_all"):
        f = getattr(lib, name)
        f.restype = st
        f.argtypes = [vp, ctypes.POINTER(i64), vp]
    lib.ohm_map_residency.restype = st
    lib.ohm_map_residency.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    lib.ohm_last_error.restype = ctypes.c_char_p
    lib.ohm_last_error.argtypes = []
    _lib = lib
    return lib


def _check(code):
    if code != OK:
        raise OhmError(code, load_library().ohm_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(x):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


_COUNT_DTYPES = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())


def _keep_for_stream(stream, *pairs):
    """Copies made by _as_points / _as_flags (for contiguity or dtype) go back
    to torch's caching allocator when the call returns, tied to the current
    stream; when the work runs on another stream, record that stream on them
    so their memory is not reused before that work has read it."""
    if stream is None:
        return
    s = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(int(stream))
    if s == torch.cuda.current_stream():
        return
    for orig, t in pairs:
        if isinstance(t, torch.Tensor) and t.is_cuda and t is not orig:
            t.record_stream(s)


def _as_points(x, name):
    if isinstance(x, torch.Tensor):
        t = x.contiguous()
        if t.dtype != torch.float32:
            raise TypeError("%s must be float32" % name)
        return t.reshape(-1, 3)
    a = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    return a


def _as_flags(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.uint8:
            raise TypeError("flags must be uint8")
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=np.uint8)


def default_params(**kw) -> dict:
    """Room / tunnel occupancy workload parameters (0.1 m voxels)."""
    import math
    p = dict(voxel_size=0.1, map_origin=(0.0, 0.0, 0.0), frac_bits=16, layers=LAYER_OCCUPANCY,
             hit=float(np.float32(math.log(0.7 / 0.3))), miss=float(np.float32(math.log(0.4 / 0.6))),
             l_min=-2.0, l_max=3.5, ndt_clear_below=float("-inf"), max_range=20.0, min_range=0.0, tsdf_trunc=0.2,
             tsdf_wmax=float(1 << 20), max_regions=4096, max_ndt_regions=1024, max_rays=1 << 18, segment_steps=0, device=0,
             evict_when_full=0, max_probe=0)
    p.update(kw)
    return p


class Map:
    """A voxel map living on one CUDA device."""

    def __init__(self, **params):
        lib = load_library()
        self.params = default_params(**params)
        cp = MapParams()
        for k, v in self.params.items():
            if k == "map_origin":
                for i in range(3):
                    cp.map_origin[i] = float(v[i])
            else:
                setattr(cp, k, v)
        h = ctypes.c_void_p()
        _check(lib.ohm_map_create(ctypes.byref(cp), ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", int(self.params["device"]))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load_library().ohm_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def integrate(self, origins, endpoints, flags=None, stream=None, sync=True):
        """Integrate one ray set.  Inputs may be CUDA tensors or host arrays."""
        o = _as_points(origins, "origins")
        e = _as_points(endpoints, "endpoints")
        f = _as_flags(flags)
        _keep_for_stream(stream, (origins, o), (endpoints, e), (flags, f))
        lib = load_library()
        fn = lib.ohm_integrate_rays if sync else lib.ohm_integrate_rays_async
        _check(fn(self._h, _ptr(o), int(o.shape[0]), _ptr(e), _ptr(f), int(e.shape[0]), _stream_handle(stream)))

    def sync(self, stream=None):
        _check(load_library().ohm_map_sync(self._h, _stream_handle(stream)))

    def status_async(self, out, stream=None):
        """Enqueue a copy of the latched status bits into `out` (an int32 CPU
        tensor element, pinned for an asynchronous copy); nonzero after the
        stream passes it means an earlier call failed (see sync)."""
        if out.device.type != "cpu" or out.dtype != torch.int32:
            raise ValueError("status_async: out must be an int32 CPU tensor")
        _check(load_library().ohm_map_status_async(self._h, _ptr(out), _stream_handle(stream)))

    @staticmethod
    def _frame_args(K, pose):
        k = (ctypes.c_double * 4)(*[float(v) for v in K])
        P = np.asarray(pose, np.float64).reshape(3, 4)
        p = (ctypes.c_double * 12)(*[float(v) for v in P.reshape(-1)])
        return k, p

    def integrate_depth(self, depth, K, pose, z_min=0.3, z_max=6.0, stream=None, sync=True):
        """Integrate a z-depth image (CUDA float32 tensor, height x width) seen
        from pose (3 x 4 camera-to-world) with intrinsics K = (fx, fy, cx, cy)."""
        d = depth.contiguous()
        if d.dtype != torch.float32 or not d.is_cuda:
            raise TypeError("depth must be a CUDA float32 tensor")
        _keep_for_stream(stream, (depth, d))
        k, p = self._frame_args(K, pose)
        h, w = d.shape
        _check(load_library().ohm_integrate_depth(self._h, _ptr(d), int(w), int(h), k, p, float(z_min), float(z_max),
                                                  _stream_handle(stream)))
        if sync:
            self.sync(stream)

    def tsdf_backward(self, depth, K, pose, query_points, grad_query, z_min=0.3, z_max=6.0, stream=None):
        """(dL/d depth (height x width), dL/d twist (6,)) for
        L = sum_q grad_query[q] * D(query_points[q]) right after
        integrate_depth of the same frame (voxel sets held fixed)."""
        d = depth.contiguous()
        q = _as_points(query_points, "query_points")
        g = grad_query.contiguous().float()
        gd = torch.empty_like(d)
        gt = torch.empty(6, dtype=torch.float64, device=d.device)
        k, p = self._frame_args(K, pose)
        h, w = d.shape
        _check(load_library().ohm_tsdf_backward(self._h, _ptr(d), int(w), int(h), k, p, float(z_min), float(z_max),
                                                _ptr(q), _ptr(g), int(q.shape[0]), _ptr(gd), _ptr(gt),
                                                _stream_handle(stream)))
        return gd, gt

    @staticmethod
    def _pose_arg(pose):
        P = np.asarray(pose, np.float64).reshape(3, 4)
        return (ctypes.c_double * 12)(*[float(v) for v in P.reshape(-1)])

    def integrate_posed(self, pose, origins, endpoints, flags=None, stream=None, sync=True):
        """Integrate sensor-frame rays (CUDA tensors) moved to the world by a
        3 x 4 camera-to-world pose."""
        o = _as_points(origins, "origins")
        e = _as_points(endpoints, "endpoints")
        f = _as_flags(flags)
        _keep_for_stream(stream, (origins, o), (endpoints, e), (flags, f))
        _check(load_library().ohm_integrate_posed(self._h, self._pose_arg(pose), _ptr(o), int(o.shape[0]), _ptr(e),
                                                  _ptr(f), int(e.shape[0]), _stream_handle(stream)))
        if sync:
            self.sync(stream)

    def ndt_backward(self, pose, origins, endpoints, flags, query_points, grad_mean, grad_cov, stream=None):
        """(dL/d endpoints (n x 3, sensor frame), dL/d twist (6,)) for
        L = sum_q grad_mean[q] . mean(q) + grad_cov[q] . cov(q) of the NDT
        statistics right after integrate_posed of the same rays (the voxel of
        every sample held fixed)."""
        o = _as_points(origins, "origins")
        e = _as_points(endpoints, "endpoints")
        f = _as_flags(flags)
        q = _as_points(query_points, "query_points")
        gmean = grad_mean.contiguous().float()
        gcov = grad_cov.contiguous().float()
        ge = torch.empty((e.shape[0], 3), dtype=torch.float32, device=e.device)
        gt = torch.empty(6, dtype=torch.float64, device=e.device)
        _keep_for_stream(stream, (origins, o), (endpoints, e), (flags, f), (query_points, q), (grad_mean, gmean),
                         (grad_cov, gcov))
        _check(load_library().ohm_ndt_backward(self._h, self._pose_arg(pose), _ptr(o), int(o.shape[0]), _ptr(e),
                                               _ptr(f), int(e.shape[0]), _ptr(q), _ptr(gmean), _ptr(gcov),
                                               int(q.shape[0]), _ptr(ge), _ptr(gt), _stream_handle(stream)))
        return ge, gt

    def query(self, points, stream=None, ndt=False, tsdf=False, counts=False, path_sum=False, mean=False):
        """Look up world points; returns a dict of CUDA tensors (path_sum:
        int64 summed path length in 2^-20 m units, the decay layer; mean:
        (n, 4) float32 voxel-mean position x y z and sample count)."""
        p = _as_points(points, "points")
        _keep_for_stream(stream, (points, p))
        n = int(p.shape[0])
        dev = self.device
        out = dict(occupancy=torch.empty(n, dtype=torch.float32, device=dev),
                   known=torch.empty(n, dtype=torch.uint8, device=dev))
        if ndt:
            out["ndt"] = torch.empty((n, 10), dtype=torch.float32, device=dev)
        if tsdf:
            out["tsdf"] = torch.empty((n, 2), dtype=torch.float32, device=dev)
        if counts:
            out["counts"] = torch.empty((n, 2), dtype=torch.int32, device=dev)
        if path_sum:
            out["path_sum"] = torch.empty(n, dtype=torch.int64, device=dev)
        if mean:
            out["mean"] = torch.empty((n, 4), dtype=torch.float32, device=dev)
        _check(load_library().ohm_query_voxels(self._h, _ptr(p), n, _ptr(out["occupancy"]), _ptr(out["known"]),
                                               _ptr(out.get("ndt")), _ptr(out.get("tsdf")), _ptr(out.get("counts")),
                                               _ptr(out.get("path_sum")), _ptr(out.get("mean")),
                                               _stream_handle(stream)))
        return out

    def evict(self, keep_regions: int, stream=None) -> int:
        """Move least recently used regions to host memory until at most
        keep_regions stay resident; returns how many moved."""
        n = ctypes.c_int64()
        _check(load_library().ohm_map_evict(self._h, int(keep_regions), ctypes.byref(n), _stream_handle(stream)))
        return int(n.value)

    def restore_pending(self, stream=None) -> int:
        n = ctypes.c_int64()
        _check(load_library().ohm_map_restore_pending(self._h, ctypes.byref(n), _stream_handle(stream)))
        return int(n.value)

    def restore_all(self, stream=None) -> int:
        n = ctypes.c_int64()
        _check(load_library().ohm_map_restore_all(self._h, ctypes.byref(n), _stream_handle(stream)))
        return int(n.value)

    def residency(self, stream=None):
        """(regions resident on the device, regions held in host memory)"""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().ohm_map_residency(self._h, ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)))
        return int(a.value), int(b.value)

    def region_count(self, stream=None) -> int:
        c = ctypes.c_int64()
        _check(load_library().ohm_map_region_count(self._h, ctypes.byref(c), _stream_handle(stream)))
        return int(c.value)

    def stats(self, stream=None) -> dict:
        s = CallStats()
        _check(load_library().ohm_map_stats(self._h, ctypes.byref(s), _stream_handle(stream)))
        return {k: int(getattr(s, k)) for k, _ in CallStats._fields_}

    def profile(self, stages=(), every=1):
        """Time the kernels of the named stages (see STAGES) in later calls;
        with every > 1 only in every every-th call (the others run without
        events, keeping the programmatic-launch overlap of their kernels)."""
        mask = 0
        for name in stages:
            mask |= 1 << STAGES.index(name)
        if every == 1:
            _check(load_library().ohm_map_profile(self._h, mask))
        else:
            _check(load_library().ohm_map_profile_every(self._h, mask, int(every)))

    def profile_read(self, stage: str):
        """(total device ms, launches) of a profiled stage; waits for them."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(load_library().ohm_map_profile_read(self._h, STAGES.index(stage), ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def export(self, occupancy=True, counts=False, ndt=False, tsdf=False, path_sum=False, mean=False, first=0,
               count=None, stream=None):
        """Regions [first, first + count) in allocation order as CUDA tensors;
        voxels x fastest inside a region."""
        if count is None:
            count = self.region_count(stream) - first
        dev = self.device
        out = dict(keys=torch.empty((count, 3), dtype=torch.int32, device=dev))
        if occupancy:
            out["occupancy"] = torch.empty((count, REGION_VOXELS), dtype=torch.float32, device=dev)
        if counts:
            out["counts"] = torch.empty((count, REGION_VOXELS, 2), dtype=torch.int32, device=dev)
        if ndt:
            out["ndt"] = torch.empty((count, REGION_VOXELS, 10), dtype=torch.int64, device=dev)
        if tsdf:
            out["tsdf"] = torch.empty((count, REGION_VOXELS, 2), dtype=torch.float32, device=dev)
        if path_sum:
            out["path_sum"] = torch.empty((count, REGION_VOXELS), dtype=torch.int64, device=dev)
        if mean:
            out["mean"] = torch.empty((count, REGION_VOXELS), dtype=torch.int64, device=dev)
        _check(load_library().ohm_map_export(self._h, first, count, _ptr(out["keys"]), _ptr(out.get("occupancy")),
                                             _ptr(out.get("counts")), _ptr(out.get("ndt")), _ptr(out.get("tsdf")),
                                             _ptr(out.get("path_sum")), _ptr(out.get("mean")),
                                             _stream_handle(stream)))
        return out


def probe_cas_rate(device=0, words=1 << 28, ops=1 << 26) -> float:
    """Random-word compare-and-swap operations per second on `device` (the
    miss walk's access pattern; see ohm_probe_cas_rate)."""
    r = ctypes.c_double()
    _check(load_library().ohm_probe_cas_rate(int(device), int(words), int(ops), ctypes.byref(r)))
    return float(r.value)


PROBE_L2_ADD, PROBE_L2_CAS, PROBE_SECTOR_RMW = 0, 1, 2


def probe_rate(kind, units, ops=1 << 28, device=0) -> float:
    """Operations per second of one of the library's ceiling probes (see
    ohm_probe_rate): PROBE_L2_ADD, PROBE_L2_CAS or PROBE_SECTOR_RMW."""
    r = ctypes.c_double()
    _check(load_library().ohm_probe_rate(int(device), int(kind), int(units), int(ops), ctypes.byref(r)))
    return float(r.value)


def count_rays_noalloc(grid: dict, origins, endpoints, flags, hits, misses, stream=None):
    """Add each ray's per-voxel hit and miss counts into the caller's dense
    uint32 grids `hits` and `misses` (CUDA tensors of dims[0]*dims[1]*dims[2]
    elements, x fastest) without any device allocation by the library.  All
    inputs must be CUDA tensors.  `grid` holds voxel_size, map_origin,
    frac_bits, segment_steps, max_range, corner and dims (see ohm_count_grid).

    The C entry point writes to whatever the pointers address, so the sizes
    are checked here: hits and misses contiguous 32-bit CUDA tensors on the
    current device with at least prod(dims) elements, flags at least one byte
    per ray; anything else raises OhmError(ERR_INVALID) before the call."""
    dev = torch.device("cuda", torch.cuda.current_device())
    n_cells = 1
    for d in grid["dims"]:
        n_cells *= int(d)
    for name, t in (("hits", hits), ("misses", misses)):
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise OhmError(ERR_INVALID, "count_rays_noalloc: %s must be a CUDA tensor on the current device" % name)
        if t.dtype not in _COUNT_DTYPES or not t.is_contiguous():
            raise OhmError(ERR_INVALID, "count_rays_noalloc: %s must be a contiguous 32-bit integer tensor" % name)
        if t.numel() < n_cells:
            raise OhmError(ERR_INVALID, "count_rays_noalloc: %s holds %d elements, the grid has %d voxels"
                           % (name, t.numel(), n_cells))
    for name, t in (("origins", origins), ("endpoints", endpoints), ("flags", flags)):
        if t is not None and (not isinstance(t, torch.Tensor) or t.device != dev):
            raise OhmError(ERR_INVALID, "count_rays_noalloc: %s must be a CUDA tensor on the current device" % name)
    n_rays = int(endpoints.numel()) // 3
    if flags is not None and int(flags.numel()) < n_rays:
        raise OhmError(ERR_INVALID, "count_rays_noalloc: flags holds %d bytes for %d rays" % (flags.numel(), n_rays))
    g = CountGrid()
    g.voxel_size = float(grid["voxel_size"])
    for i in range(3):
        g.map_origin[i] = float(grid.get("map_origin", (0.0, 0.0, 0.0))[i])
        g.corner[i] = int(grid["corner"][i])
        g.dims[i] = int(grid["dims"][i])
    g.frac_bits = int(grid.get("frac_bits", 16))
    g.segment_steps = int(grid.get("segment_steps", 0))
    g.max_range = float(grid["max_range"])
    o = _as_points(origins, "origins")
    e = _as_points(endpoints, "endpoints")
    f = _as_flags(flags)
    _keep_for_stream(stream, (origins, o), (endpoints, e), (flags, f))
    _check(load_library().ohm_count_rays_noalloc(ctypes.byref(g), _ptr(o), int(o.shape[0]), _ptr(e), _ptr(f),
                                                 int(e.shape[0]), _ptr(hits), _ptr(misses), _stream_handle(stream)))


class Batch:
    """Up to 32 maps integrated together, one launch per kernel stage for all
    of them, optionally replayed from a captured CUDA graph."""

    def __init__(self, maps):
        lib = load_library()
        self.maps = list(maps)
        n = len(self.maps)
        arr = (ctypes.c_void_p * n)(*[m.handle.value for m in self.maps])
        h = ctypes.c_void_p()
        _check(lib.ohm_batch_create(arr, n, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load_library().ohm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, segment_steps=0, walk_blocks_per_sm=0):
        _check(load_library().ohm_batch_tune(self._h, int(segment_steps), int(walk_blocks_per_sm)))

    def integrate(self, raysets, stream=None, graph=True):
        """raysets[i] = (origins, endpoints, flags) CUDA tensors for map i, or
        None for no rays this step."""
        n = len(self.maps)
        P = ctypes.c_void_p * n
        I = ctypes.c_int64 * n
        o, e, f = P(), P(), P()
        no, nn = I(), I()
        self._keep = []
        for i, rs in enumerate(raysets):
            if rs is None:
                no[i], nn[i] = 1, 0
                continue
            oo = _as_points(rs[0], "origins")
            ee = _as_points(rs[1], "endpoints")
            ff = _as_flags(rs[2]) if len(rs) > 2 else None
            self._keep += [oo, ee, ff]
            o[i], e[i] = oo.data_ptr(), ee.data_ptr()
            f[i] = ff.data_ptr() if ff is not None else None
            no[i], nn[i] = int(oo.shape[0]), int(ee.shape[0])
        _check(load_library().ohm_batch_integrate(self._h, o, no, e, f, nn, 1 if graph else 0, _stream_handle(stream)))

    def sync(self, stream=None):
        _check(load_library().ohm_batch_sync(self._h, _stream_handle(stream)))

    def stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().ohm_batch_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"kernel_launches": int(a.value), "graph_launches": int(b.value)}


def twist_pose(xi, pose0):
    """exp(xi) applied on the left of a 3 x 4 camera-to-world pose, computed
    by the library (ohm_twist_pose); float64 numpy (3, 4)."""
    x = (ctypes.c_double * 6)(*[float(v) for v in np.asarray(xi, np.float64).reshape(6)])
    p0 = (ctypes.c_double * 12)(*[float(v) for v in np.asarray(pose0, np.float64).reshape(12)])
    out = (ctypes.c_double * 12)()
    _check(load_library().ohm_twist_pose(x, p0, out))
    return np.array(out[:], np.float64).reshape(3, 4)


class TsdfFrame(torch.autograd.Function):
    """D at query points after integrating one depth frame, differentiable in
    the per-pixel depth and in a pose twist xi applied on the left of pose0.

    forward(depth, xi, gmap, K, pose0, query_points, z_min, z_max) integrates
    the frame into gmap (a side effect: calling it twice integrates twice) and
    returns D at the query points.  backward gives dL/d depth and the
    tangent-space pose gradient at the evaluated pose (the derivative with
    respect to xi at xi = 0), with the walk's voxel sets held fixed."""

    @staticmethod
    def forward(ctx, depth, xi, gmap, K, pose0, query_points, z_min=0.3, z_max=6.0):
        pose = twist_pose(xi.detach().cpu().numpy(), pose0)
        gmap.integrate_depth(depth.detach(), K, pose, z_min, z_max)
        out = gmap.query(query_points, tsdf=True)["tsdf"][:, 0]
        ctx.gmap, ctx.K, ctx.pose, ctx.z = gmap, K, pose, (z_min, z_max)
        ctx.xi_like = (xi.dtype, xi.device)
        ctx.save_for_backward(depth.detach(), query_points)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        depth, q = ctx.saved_tensors
        gd, gt = ctx.gmap.tsdf_backward(depth, ctx.K, ctx.pose, q, grad_out, *ctx.z)
        return gd, gt.to(dtype=ctx.xi_like[0], device=ctx.xi_like[1]), None, None, None, None, None, None


class NdtFrame(torch.autograd.Function):
    """NDT-OM mean (q x 3) and covariance (q x 6, packed xx xy xz yy yz zz)
    at query points after integrating one ray set given in a sensor frame,
    differentiable in the sensor-frame endpoints and in a pose twist xi
    applied on the left of pose0.

    forward(endpoints, xi, gmap, pose0, origins, flags, query_points)
    integrates the rays seen from exp(xi) pose0 into gmap (a side effect) and
    returns (mean, cov) of the query voxels (zeros where a voxel holds no
    sample).  backward gives dL/d endpoints and the tangent-space pose gradient
    at the evaluated pose (the derivative with respect to xi at xi = 0), with
    the voxel of every sample held fixed (ohm_ndt_backward)."""

    @staticmethod
    def forward(ctx, endpoints, xi, gmap, pose0, origins, flags, query_points):
        pose = twist_pose(xi.detach().cpu().numpy(), pose0)
        gmap.integrate_posed(pose, origins, endpoints.detach(), flags)
        r = gmap.query(query_points, ndt=True)["ndt"]
        ctx.gmap, ctx.pose = gmap, pose
        ctx.xi_like = (xi.dtype, xi.device)
        ctx.save_for_backward(endpoints.detach(), origins, flags if flags is not None else torch.empty(0),
                              query_points)
        return r[:, 1:4].contiguous(), r[:, 4:10].contiguous()

    @staticmethod
    def backward(ctx, grad_mean, grad_cov):
        e, o, f, q = ctx.saved_tensors
        ge, gt = ctx.gmap.ndt_backward(ctx.pose, o, e, f if f.numel() else None, q, grad_mean, grad_cov)
        return ge, gt.to(dtype=ctx.xi_like[0], device=ctx.xi_like[1]), None, None, None, None, None
