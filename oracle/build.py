"""Build the FP64 CPU oracle shared library (test infrastructure only).

Compiles ``gsvr_oracle.c`` and ``cnn_oracle.c`` with gcc and OpenMP into ``liboracle.so`` next to
this file.  Building the checker is not using it: only the tests, the smoke
check and the CPU baseline of the benchmark load the library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "gsvr_oracle.c"), os.path.join(HERE, "cnn_oracle.c")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-Wno-unused-function",
           *SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
