"""Build libgc.so (the CUDA colouring library) in-tree with nvcc for sm_103a.

Translation units compile in parallel into ``_build/`` and link into
``libgc.so`` next to this file.  The library links the shared CUDA runtime so
that, inside a PyTorch process, it binds to the runtime PyTorch already
loaded (device pointers and streams are then interchangeable).
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgc.so")
SOURCES = ["gc_kernels.cu", "gc_api.cu", "gc_noalloc.cu", "gc_server.cu", "gc_tune.cu", "gc_classes.cu", "gc_d2.cu",
           "gc_diag.cu", "gc_host.cpp"]
HEADERS = [os.path.join(CSRC, "gc_internal.h"), os.path.join(CSRC, "gc_device.cuh"), os.path.join(CSRC, "gc_ctx.h"),
           os.path.join(CSRC, "gc_nvtx.h"),
           os.path.join(INCLUDE, "gc.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (cand == "nvcc" or os.path.exists(cand)):
            return cand
    return "nvcc"


def _cuda_lib_dir() -> str:
    nv = _nvcc()
    if os.path.isabs(nv):
        return os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")
    return "/usr/local/cuda/lib64"


_OPENMP = None


def _openmp_flags() -> list:
    """["-Xcompiler", "-fopenmp"] if the host compiler builds and links an
    OpenMP program, else [] (gc_host_color then runs on one thread)."""
    global _OPENMP
    if _OPENMP is None:
        import tempfile
        with tempfile.TemporaryDirectory() as d:
            src = os.path.join(d, "t.cpp")
            with open(src, "w") as f:
                f.write("#include <omp.h>\nint main() { return omp_get_max_threads() > 0 ? 0 : 1; }\n")
            ok = subprocess.run(["g++", "-fopenmp", src, "-o", os.path.join(d, "t")],
                                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL).returncode == 0
        _OPENMP = ["-Xcompiler", "-fopenmp"] if ok else []
    return _OPENMP


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libgc.so."""
    lib = LIB
    bdir = BUILD
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I", INCLUDE, "-I", CSRC]
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            extra = _openmp_flags() if src.endswith(".cpp") else []
            cmd = [nvcc] + common + extra + ["-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd), o))
    failed = False
    for p, o in procs:
        if p.wait() != 0:
            failed = True
        else:
            os.replace(o + ".tmp", o)
    if failed:
        raise RuntimeError("nvcc failed while building libgc")
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + _openmp_flags() + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", f"-rpath,{_cuda_lib_dir()}"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
