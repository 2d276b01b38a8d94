"""The compressed 8-wide BVH builder on the host (no GPU): the builder's own
invariants, containment of every triangle in the dequantized boxes of its
slot and all ancestors, and closest hits through the node format's traversal
rules equal to brute force (tests/bvh8_check.cpp, compiled with g++ against
the library's host sources)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_07996_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("bvh8") / "bvh8_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", inc,
                    os.path.join(ROOT, "tests", "bvh8_check.cpp"), os.path.join(CSRC, "bvh.cpp"),
                    os.path.join(CSRC, "bvh8.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("kind,n,seed", [(0, 1, 1), (0, 5, 2), (0, 3000, 3), (1, 20000, 4), (2, 2000, 5),
                                         (2, 7, 6)])
def test_wide_bvh_builder(checker, kind, n, seed):
    out = subprocess.run([checker, str(kind), str(n), str(seed)], capture_output=True, text=True, timeout=120)
    print(out.stdout.strip())
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
