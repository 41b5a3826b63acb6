"""Build the CUDA library in-tree: paper_2206_06079_gb300/_lib/libohm_gb.so.

Each translation unit is compiled by nvcc for sm_103a only (in parallel), then
linked into one shared library with the C ABI of include/ohm_gb.h.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libohm_gb.so")
SOURCES = ["ohm_integrate.cu", "ohm_capi.cu", "ohm_noalloc.cu", "ohm_batch.cu", "ohm_adjoint.cu", "ohm_cache.cu"]
HEADERS = ["ohm_device.cuh", "ohm_kernels.cuh", "ohm_host.h", os.path.join("..", "..", "include", "ohm_gb.h")]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    objs = []
    cmds = []
    for s in SOURCES:
        obj = os.path.join(OUT, s.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([NVCC] + FLAGS + ["-c", os.path.join(CSRC, s), "-o", obj])
    with concurrent.futures.ThreadPoolExecutor(len(cmds)) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
    for c, r in zip(cmds, results):
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(c))
    tmp = LIB + ".tmp.%d" % os.getpid()
    r = subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs,
                       capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
