"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/ohm_gb.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2206_06079_gb300 import build_lib, ohm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ohm_gb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ohm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ohm_map_create", "ohm_integrate_rays", "ohm_query_voxels", "ohm_map_destroy"):
        assert required in names
    assert set(names) == set(ohm.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build_lib.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_rejects_a_missing_library(tmp_path):
    import pytest
    saved = ohm._lib
    ohm._lib = None
    try:
        with pytest.raises(RuntimeError):
            ohm.load_library(str(tmp_path / "missing.so"))
    finally:
        ohm._lib = saved


def _c_layout(struct, fields, tmp_path):
    """Field offsets and size of a header struct, as gcc lays it out."""
    import subprocess
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ohm_gb.h"', 'int main(void) {']
    for f in fields:
        lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f))
    lines.append('  printf("%%zu\\n", sizeof(%s));' % struct)
    lines.append('  return 0; }')
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return [int(x) for x in out]


def test_param_structs_match_the_header(tmp_path):
    for cls, name in ((ohm.MapParams, "ohm_map_params"), (ohm.CallStats, "ohm_call_stats"),
                      (ohm.CountGrid, "ohm_count_grid")):
        fields = [f for f, _ in cls._fields_]
        got = _c_layout(name, fields, tmp_path)
        assert got[:-1] == [getattr(cls, f).offset for f in fields], name
        assert got[-1] == ctypes.sizeof(cls), name


def test_create_rejects_bad_parameters_before_touching_a_device():
    """Parameter validation is host logic: every rejection below returns
    OHM_ERR_INVALID with a message and needs no GPU."""
    import pytest
    from paper_2206_06079_gb300 import workloads as W
    build_lib.build()
    cases = [
        (dict(layers=0), "layer mask"),
        (dict(layers=64), "layer mask"),
        (dict(frac_bits=7), "frac_bits"),
        (dict(frac_bits=21), "frac_bits"),
        (dict(max_regions=(1 << 16) + 1), "max_regions"),
        (dict(layers=W.OCC | W.MEAN, max_rays=(1 << 22) + 1), "mean layer"),
        (dict(max_range=1e5), "2^30"),
        (dict(l_min=1.0, l_max=0.0), "l_min"),
        (dict(miss=-1e-35), "2^-100"),
        (dict(ndt_clear_below=float("nan")), "NaN"),
        (dict(layers=W.NDT, max_ndt_regions=0), "max_ndt_regions"),
    ]
    for kw, msg in cases:
        with pytest.raises(ohm.OhmError) as ei:
            ohm.Map(**W.room_params(**kw))
        assert ei.value.code == ohm.ERR_INVALID, kw
        assert msg in str(ei.value), (kw, str(ei.value))


def test_sampled_profiling_rejects_bad_arguments_without_a_device():
    build_lib.build()
    lib = ohm.load_library()
    assert lib.ohm_map_profile_every(None, 0, 2) == ohm.ERR_INVALID
    assert b"NULL" in lib.ohm_last_error()


def _doc_before(name):
    """The comment block right before a declaration in the header."""
    text = open(HEADER).read()
    i = re.search(r"\n[a-z][^\n]*[ *]%s\(" % name, text).start()  # the declaration line
    head = text[:i]
    j = head.rindex("/*")
    k = head.rindex("*/")
    assert k > j and text[k + 2:i].count(";") == 0, name
    return head[j:k]


def test_boundary_declarations_cite_the_paper():
    """Every entry point of the method's boundary (create, integrate, query,
    export, destroy, error report) names the passage that defines it."""
    for name in ("ohm_map_create", "ohm_integrate_rays", "ohm_query_voxels", "ohm_map_export",
                 "ohm_map_destroy", "ohm_last_error"):
        assert "Sec." in _doc_before(name), name


def test_twist_pose_is_the_rigid_motion_of_the_twist():
    """ohm_twist_pose (library host code) against the oracle's exponential of
    the twist, from zero rotation through small angles to large ones, and the
    result's rotation is orthonormal."""
    import numpy as np
    from oracle import adjoint
    build_lib.build()
    rng = np.random.default_rng(0)
    for s in (0.0, 1e-13, 1e-6, 1e-3, 0.7, 2.5, 3.1):
        xi = rng.normal(size=6)
        xi[3:] *= (s / np.linalg.norm(xi[3:])) if s else 0.0
        P0 = np.concatenate([np.linalg.qr(rng.normal(size=(3, 3)))[0], rng.normal(size=(3, 1))], 1)
        T = adjoint.twist_matrix(xi)
        ref = np.concatenate([T[:3, :3] @ P0[:, :3], (T[:3, :3] @ P0[:, 3] + T[:3, 3])[:, None]], 1)
        got = ohm.twist_pose(xi, P0)
        assert np.abs(got - ref).max() < 1e-12, s
        if s > 1e-6:
            R = got[:, :3]
            assert np.abs(R @ R.T - np.eye(3)).max() < 1e-12
