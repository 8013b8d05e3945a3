"""Compile the FP64 CPU oracle into ``oracle/_build/liboracle.so`` with g++.

Test infrastructure only: the oracle is a plain restatement of the paper's
equations used to check the GPU library.  Plain C++17, no x86-specific flags,
so the same sources build on the x86 development host and the Arm GPU host.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["fft.cpp", "cp.cpp", "rve.cpp"]
OUT = os.path.join(HERE, "_build", "liboracle.so")


def build(force=False, verbose=False):
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "oracle_internal.hpp")]
    if not force and os.path.exists(OUT):
        t_out = os.path.getmtime(OUT)
        if all(os.path.getmtime(d) <= t_out for d in deps):
            return OUT
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", *srcs, "-o", OUT + ".tmp"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
