"""Compile the FP64 CPU oracle (test infrastructure) into a shared library.

Plain C99, -O2, -ffp-contract=off (no fused multiply-add contraction, so x86
and aarch64 round identically), no fast-math, OpenMP over the per-node loops
(results do not depend on the thread count). The library is written next to
this file and is git-ignored.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tlv_oracle.c")
LIB = os.path.join(HERE, "libtlv_oracle.so")


def build(force: bool = False) -> str:
    """Build libtlv_oracle.so if it is missing or older than its sources."""
    deps = [SRC, os.path.join(HERE, "tlv_oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB) and all(
        os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps
    ):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [
        "gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
        "-Wall", "-shared", "-o", tmp, SRC, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
