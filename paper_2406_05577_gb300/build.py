"""In-tree build of libfftb.so for sm_103a (nvcc + g++, no cmake).

Compiles the CUDA translation units and the host C++ in parallel into
``_build/`` and links ``libfftb.so`` next to this file. Objects are rebuilt
when their source or any header is newer. ``FFTB_NVCC_FLAGS`` (environment)
adds nvcc flags, e.g. ``-DFFTB_PLANE_NW=12`` to try a kernel tuning knob; it
forces a rebuild. ``build(check=True)`` makes the checked library
``libfftb_check.so`` in ``_build_check/`` instead: the kernels compiled with
``-DFFTB_CHECK`` test every index against its buffer before the access.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfftb.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libfftb_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["k_f32.cu", "k_f32_pf.cu", "k_f32_alt.cu", "k_f32_bg.cu", "k_scale.cu", "k_f64.cu", "k_tc.cu", "k_tc5.cu", "noalloc.cu", "k_generic.cu", "k_cluster.cu", "k_f32_zq.cu"]
CPP_SOURCES = ["geometry.cpp", "fftb_api.cpp"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _stale(obj: str, src: str, deps) -> bool:
    if not os.path.exists(obj) or os.environ.get("FFTB_NVCC_FLAGS"):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *deps])


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, flush=True)


def build(verbose: bool = False, ptxas_verbose: bool = False, check: bool = False) -> str:
    """Builds (if needed) and returns the path of libfftb.so, or with check
    the path of libfftb_check.so (device bounds checks compiled in)."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    BUILD = BUILD_CHECK if check else globals()["BUILD"]
    LIB = LIB_CHECK if check else globals()["LIB"]
    os.makedirs(BUILD, exist_ok=True)
    deps = _headers()
    jobs = []
    for s in CU_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        if _stale(obj, src, deps) or ptxas_verbose:
            cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", *ARCH, "-lineinfo",
                   "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", CSRC, "-I", INCLUDE]
            if ptxas_verbose:
                cmd += ["-Xptxas", "-v"]
            if check:
                cmd += ["-DFFTB_CHECK"]
            cmd += os.environ.get("FFTB_NVCC_FLAGS", "").split()
            jobs.append(cmd)
    for s in CPP_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        if _stale(obj, src, deps):
            jobs.append(["g++", "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC",
                         "-fvisibility=hidden", "-ffp-contract=off", "-Wall",
                         "-I", os.path.join(cuda, "include"), "-I", CSRC, "-I", INCLUDE])
    if jobs:
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            list(ex.map(lambda c: _run(c, verbose or ptxas_verbose), jobs))
    objs = [os.path.join(BUILD, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        _run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static",
              "-Xlinker", "--no-undefined"], verbose)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv))
