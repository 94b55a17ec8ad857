"""Builds the in-tree CUDA library libtc.so for sm_103a (nvcc, no cmake).

The pipeline specialisations (precision x FFT box size) are compiled as
separate objects in parallel from csrc/tc_inst.cu with -DTC_REAL/-DTC_N.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                  "-I" + os.path.join(HERE, "..", "include")]
SIZES = (9, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 48)
REALS = ("float", "double")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(verbose=False, jobs=None, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    steps = []
    steps.append(["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(SRC, "tc_setup.cpp"),
                  "-o", os.path.join(BUILD, "tc_setup.o")])
    steps.append([nvcc] + NVFLAGS + extra + ["-c", os.path.join(SRC, "tc_api.cu"), "-o", os.path.join(BUILD, "tc_api.o")])
    for name in ("tc_noalloc", "tc_batch", "tc_davidson", "tc_symmetry", "tc_peak"):
        steps.append([nvcc] + NVFLAGS + extra + ["-c", os.path.join(SRC, name + ".cu"),
                                                 "-o", os.path.join(BUILD, name + ".o")])
    for real in REALS:
        for n in SIZES:
            obj = os.path.join(BUILD, "tc_inst_%s_%d.o" % (real, n))
            steps.append([nvcc] + NVFLAGS + extra + ["-DTC_REAL=%s" % real, "-DTC_N=%d" % n, "-c",
                                                     os.path.join(SRC, "tc_inst.cu"), "-o", obj])
    objs = [s[s.index("-o") + 1] for s in steps]
    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        logs = list(ex.map(_run, steps))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
