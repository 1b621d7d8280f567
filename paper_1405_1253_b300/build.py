"""Build the CUDA library csrc/liblbm.so in-tree for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(CSRC, "liblbm.so")
# the same library with every population load and store index-checked (LBM_BOUNDS_CHECK):
# an out-of-range index is counted and redirected to element 0 instead of being used
LIB_CHECKED = os.path.join(CSRC, "liblbm_checked.so")
SOURCES = [os.path.join(CSRC, "lbm.cu")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "lbm.h"))
    return max(os.path.getmtime(p) for p in paths)


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile liblbm.so (or, checked=True, liblbm_checked.so) if it is missing or older
    than its sources."""
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
           *(["-DLBM_BOUNDS_CHECK"] if checked else []),
           "-Xcompiler", "-fPIC", "-shared", "-o", lib + ".tmp", *SOURCES, "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
