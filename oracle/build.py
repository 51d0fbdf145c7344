"""Build the CPU oracle (test infrastructure) as oracle/liboracle.so.

Plain gcc, -O2, no SIMD intrinsics, -ffp-contract=off so that only the
explicit fma() calls in pf_oracle.c fuse; OpenMP only parallelises the
independent per-particle loop (results do not depend on the thread count).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRCS = [os.path.join(HERE, "pf_oracle.c"), os.path.join(HERE, "pf_smc.c")]


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max([os.path.getmtime(f) for f in SRCS] +
                                             [os.path.getmtime(os.path.join(HERE, "pf_oracle.h"))])):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-D_GNU_SOURCE", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
           *SRCS, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
