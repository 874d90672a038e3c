"""Builds the FP64 CPU oracle (test infrastructure) into oracle/liborhgs.so.

The oracle is compiled as ISO C11 with -ffp-contract=off so that its
canonical FP32 binning arithmetic is one IEEE binary32 operation per source
operation, without fused multiply-adds.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hgs_oracle.c")
LIB = os.path.join(HERE, "liborhgs.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
