"""Build libfewsum.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel (one -gencode, -O3, -lineinfo) and linked into
paper_2104_04582_gb300/_lib/libfewsum.so with the static CUDA runtime.  A stamp of the source
hashes and flags skips rebuilds when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
from typing import List

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libfewsum.so")
PROBE_LIB = os.path.join(LIBDIR, "libfewprobe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}"]
SOURCES = ["api.cpp", "spline.cu", "fold.cu", "sum.cu", "anchor.cu", "selftest.cu", "noalloc.cu",
           "select.cu", "direct.cu", "rb.cu"]
HEADERS = ["fewsum_internal.h", "phase_eval.cuh", "harmonics.cuh", "convert.cuh", "async.cuh"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfewsum.so")
    return p


def _stamp(files: List[str], extra: List[str]) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()


def _compile(src: str, obj: str, extra: List[str]) -> None:
    cmd = [nvcc()] + ARCH + CFLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")


def _link(lib: str, objs: List[str]) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static",
                                                           "-Xlinker", "-z,defs"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def _build_one(lib: str, sources: List[str], headers: List[str], extra: List[str],
               force: bool, jobs: int) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in sources]
    deps = srcs + [os.path.join(CSRC, h) for h in headers] + [os.path.join(ROOT, "include",
                                                                           "fewsum.h")]
    stamp = _stamp(deps, ARCH + CFLAGS + extra)
    stamp_file = lib + ".stamp"
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return lib
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.splitext(os.path.basename(s))[0] + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=max(1, jobs)) as ex:
        futs = [ex.submit(_compile, s, o, extra) for s, o in zip(srcs, objs)]
        for f in futs:
            f.result()
    _link(lib, objs)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return lib


def build(force: bool = False, jobs: int = 0) -> str:
    """Compile libfewsum.so (and the pipe-peak probe library); returns the library path."""
    jobs = jobs or min(8, os.cpu_count() or 4)
    _build_one(LIB, SOURCES, HEADERS, [], force, jobs)
    if os.path.exists(os.path.join(CSRC, "probe.cu")):
        _build_one(PROBE_LIB, ["probe.cu"], [], [], force, jobs)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
