"""Build the C-ABI shared library ``_lib/libbse.so`` for sm_103a (in-tree).

Every translation unit is compiled in parallel (nvcc for .cu, g++ for the host
planner, which is built with -ffp-contract=off so its sphere keys are
bit-exact), then linked against the shared CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libbse.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["pair.cu", "build.cu", "haydock.cu", "adjoint.cu", "tc.cu", "screen.cu", "coupled.cu", "gcorr.cu", "ritz.cu", "sym.cu", "scan.cu", "tddft.cu", "eig.cu", "tcpair.cu", "tcgram.cu"]
CPP_SOURCES = ["plan.cpp"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _compile(src, verbose):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "--expt-relaxed-constexpr", *inc, "-c", path, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *inc, "-I",
               os.path.join(CUDA, "include"), "-c", path, "-o", obj]
    return obj, _run(cmd)


def _stale(objs):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "bse.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; returns the library path.  Rebuilds only when a source is newer."""
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale(None):
        return LIB
    srcs = CU_SOURCES + CPP_SOURCES
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            sys.stdout.write(log)
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
          "-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")])
    shutil.move(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
