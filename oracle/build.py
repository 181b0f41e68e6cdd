"""Compile the FP64 CPU oracle (plain C) into oracle/liboracle.so with gcc.

Test infrastructure: the CUDA library never links or loads this file's output.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "oracle.c"), os.path.join(HERE, "amg.c")]


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "oracle.h")
    newest = max(os.path.getmtime(p) for p in SRC + [hdr])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    # -ffp-contract=off: products and sums are rounded exactly as written (no FMA fusion),
    # so the oracle's arithmetic is the same on x86 and Arm hosts.
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp] + SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
