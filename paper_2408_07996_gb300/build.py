"""Builds the CUDA library libmcev.so in-tree (paper_2408_07996_gb300/_build/).

Every translation unit is compiled for sm_103a only, in parallel, then
linked with nvcc.  No CMake; takes well under a minute."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmcev.so")
SOURCES = ["kernels.cu", "quality.cu", "api.cpp", "bvh.cpp", "bvh8.cpp", "tdist.cpp"]
HEADERS = ["layout.h", "device.cuh", "kernels.h", "quality.h", "bvh.h", "tdist.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# kernels.cu is compiled without implicit multiply-add contraction: its
# traversal code is instantiated several times (single frame or batched jobs,
# two BVH layouts, different register caps), and the compiler may fuse a
# different product of the same expression in each, so the same ray could
# round differently in two instantiations.  The fused multiply-adds that the
# hot loops want are written out as fmaf().
PER_SOURCE = {"kernels.cu": ["-fmad=false"]}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "mcev.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *common, *PER_SOURCE.get(src, []), *(extra or [])]
        if src.endswith(".cu"):
            cmd += [*ARCH, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3"]
        cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
