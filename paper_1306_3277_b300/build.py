"""Build the CUDA library paper_1306_3277_b300/libpf_b300.so for sm_103a.

nvcc, -gencode arch=compute_103a,code=sm_103a, and -fmad=false so that the
only fused multiply-adds are the explicit fma()/fmaf() calls (results are
reproducible bit for bit); IEEE division and square root.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libpf_b300.so")
LIB_CHECKED = os.path.join(HERE, "libpf_b300_checked.so")  # PF_CHECKED=1 (invariant counters)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
         "-ftz=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps += glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=(), checked=False):
    """The library's path, compiled first if a source is newer; checked=True
    gives the PF_CHECKED=1 build (invariant counters, pf_debug_check_counts)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + FLAGS + list(extra) + (["-DPF_CHECKED=1"] if checked else [])
    cmd += ["-I", INCLUDE, "-I", CSRC, "-shared", "-o", tmp]
    cmd += sources() + ["-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v, extra=extra, checked="--checked" in sys.argv))
